// Cluster-resident sampler and Wiener filter for 256 x 256 and 512 x 512 images (Alg. 1 of the paper with
// A = I, and its G -> 0 form with lambda-cooling, §2.2).
//
// A 256^2 field's packed half spectrum (256 KB) does not fit one SM, but it fits the distributed shared
// memory of a thread-block cluster. One field (one chain) is a cluster of P = N / M CTAs of N / 2 threads
// (M = 64 rows per CTA at 256^2, 32 at 512^2); CTA b keeps the global rows y = P a + b (a < M), each row
// as N / 2 float2 slots, for all sweeps.
//
// Row transforms (length L = N / 2 complex, real-to-complex packing) stay inside a CTA: the R = L / M
// threads of a row (lanes of one warp) each run an M-point register FFT over every R-th slot, then
// radix-R butterflies across them, with the real-transform pre/post pass of the mode pairs (K, L - K)
// fused into the butterflies. The half spectrum of a row is kept in digit-reversed slot order, X[K] at
// slot R (K mod M) + K / M, which the column pass simply follows.
//
// Column transforms (length N) are split over the cluster by decimation in time over the CTA rank:
// each CTA runs an M-point register FFT down every column of its rows (twiddled by W_N^(b k')), then one
// radix-P stage combines the P partial transforms through distributed shared memory; the s-draw happens
// right there, on the complete column spectrum, followed by the inverse radix-P stage, the inverse twiddle
// and the local inverse FFTs. Two cluster barriers per sweep (hardware barriers, no spin waits).
// Draws follow the Philox counter layout of the on-chip sampler, so the chain is the same Markov chain
// draw for draw. The Wiener-filter form (k_cpipe: level norms, cooled solve, then samples from s_W, one
// image per cluster) replaces the draw by the level-lambda update and sums its FP64 residual per CTA and
// then across the cluster in rank order, so every thread takes the same schedule decisions.
#pragma once

#include <cooperative_groups.h>

#include "wf_gbatch.cuh"

namespace wf {

// rows per CTA (the local transform length), by default: 64 at 256^2 (clusters of 4 CTAs, 3 per SM); 32 at
// 512^2 (clusters of 16 CTAs of 66 KB, 2 per SM). 512^2 is also built with 64 rows (clusters of 8 CTAs of
// 130 KB, 1 per SM), which the batch autotuner can choose.
__host__ __device__ constexpr int cluster_rows(int N) { return N == 512 ? 32 : 64; }

template <int N_, int M_>
struct CGeo {
  static constexpr int N = N_, H = N_, W = N_;
  static constexpr int M = M_;  // rows per CTA = local transform length
  static constexpr int A = M;
  static constexpr int P = N / M;             // CTAs per cluster
  static constexpr int L = N / 2;             // complex length of a row transform = threads per CTA
  static constexpr int R = L / M;             // threads per row in the row passes
  // float2 stride of a row: with the row-major lane map below (the R threads of a row are lanes
  // a, a + 32/R, ...), a half-warp reads slots R i + h of 32/R rows a for R/2 values of h; a stride of
  // R/2 modulo 16 float2 puts those 16 reads in 16 distinct bank pairs (measured at 512^2, R = 8: 7.5%
  // faster sampling than the stride log2 R, which left two-way conflicts)
  static constexpr int SP = L + R / 2;
  static constexpr int ROWS_BYTES = A * SP * 8;
  static constexpr int SMEM = ROWS_BYTES + N * 8 + (33 + 16 + kMaxLevels) * 8;  // rows, twiddles, FP64 sums, level norms
  static constexpr int WH = W / 2 + 1;
  static_assert(M * P == N && R * M == L && R >= 2 && 32 % R == 0, "cluster geometry");
  static_assert(P <= 16, "at most 16 CTAs per cluster (the non-portable maximum)");
  static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
  static_assert(ROWS_BYTES % 8 == 0, "FP64 sums after the rows stay 8-byte aligned");
};

// Mode tables of the cluster kernels (the s-draw coefficients fg and the spectrum P) are stored in the
// column slot order of the packed half spectrum, so that the threads of a column unit (consecutive slots
// t) read consecutive addresses: entry (ky, kx) with kx < W/2 at ky L + t, t = (kx mod M) R + kx / M (the
// slot holding kx), and the Nyquist column kx = W/2 (packed with kx = 0 in slot 0) at H L + ky.
template <int N, int MR>
__host__ __device__ inline int cslot_of(int kx) {
  using G = CGeo<N, MR>;
  return (kx % G::M) * G::R + kx / G::M;
}
template <int N, int MR>
__host__ __device__ inline int ctab_index(int ky, int kx) {
  using G = CGeo<N, MR>;
  return kx < G::W / 2 ? ky * G::L + cslot_of<N, MR>(kx) : G::H * G::L + ky;
}

// Loads of the per-call tables marked evict-last in L2: the tables are re-read every sweep (in a batch
// each image has its own), while the samples stream out with evict-first stores (crows_store)
__device__ __forceinline__ uint64_t l2_keep() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ float2 ldk(const float2* a, uint64_t pol) {
  float2 v;
  asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ float ldk(const float* a, uint64_t pol) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
  return v;
}

// Physical position of slot s of a staged row. With R = 8 threads per row (512^2, 32 rows per CTA) the R
// slots of each butterfly unit u (slots R u .. R u + R - 1) are stored XOR-swizzled by u mod 4, so that a
// half-warp's reads of one slot of four units of four rows fall in 16 distinct bank pairs both in the
// radix-R butterflies and in the strided M-point pass (without it the butterflies were 4-way conflicted);
// every access to the row buffers goes through this map.
template <int N, int MR>
__host__ __device__ inline int cphys(int s) {
  constexpr int R = CGeo<N, MR>::R;
  if constexpr (R == 8) return s ^ ((s >> 3) & 3);
  return s;
}

// ---------------------------------------------------------------------------------------------
// row passes (R threads per row, h = the thread's index within its row)
// ---------------------------------------------------------------------------------------------
// local row a and index h of thread tid: a warp holds 32/R rows, thread h of each in lanes 32h/R ..
template <int N, int MR>
WF_HD void crow_of(int tid, int& a, int& h) {
  constexpr int per = 32 / CGeo<N, MR>::R;
  const int lane = tid % 32;
  a = (tid / 32) * per + lane % per;
  h = lane / per;
}

// real-transform post pass of the mode pair (K, L - K) (forward): c[K] and c[L - K] of the packed-complex
// FFT -> R[K] and R[L - K], with W = exp(-2 pi i K / N)
WF_HD void c_r2c_pair(float2& a, float2& b, float2 w) {
  const float2 bc = b;
  const float2 E = cscale(cadd_conj(a, bc), 0.5f);
  const float2 O = cmul_mi(cscale(csub_conj(a, bc), 0.5f));
  const float2 WO = cmul(O, w);
  a = cadd(E, WO);
  b = cconj(csub(E, WO));
}
// inverse pre pass of the pair: R[K], R[L - K] -> C'[K], C'[L - K] with W = exp(-2 pi i K / N)
WF_HD void c_c2r_pair(float2& a, float2& b, float2 w) {
  const float2 bc = b;
  const float2 E = cadd_conj(a, bc);
  const float2 O = cmul(csub_conj(a, bc), cconj(w));
  a = cadd(E, cmul_i(O));
  b = cadd(cconj(E), cmul_i(cconj(O)));
}

// forward: staged real row (slot i = (s[2i], s[2i+1])) -> packed half spectrum in digit-reversed slots
template <int N, int MR>
__device__ __forceinline__ void crow_fwd(float2* row, int h, const float2* tw) {
  using G = CGeo<N, MR>;
  constexpr int R = G::R;
  {
    float2 x[G::M];
#pragma unroll
    for (int i = 0; i < G::M; ++i) x[i] = row[cphys<N, MR>(R * i + h)];
    fft<G::M, false>(x);
#pragma unroll
    for (int k = 0; k < G::M; ++k) row[cphys<N, MR>(R * k + h)] = k == 0 ? x[0] : cmul(x[k], tw[2 * h * k]);  // W_L^(h k)
  }
  __syncwarp();
  for (int u = h; u <= G::M / 2; u += R) {  // butterfly unit k' = u with its mirror v = M - u
    const int v = G::M - u;
    const bool two = u != 0 && u != G::M / 2;
    float2 p[R], q[R];
#pragma unroll
    for (int j = 0; j < R; ++j) p[j] = row[cphys<N, MR>(R * u + j)];
    fft<R, false>(p);  // p[m] = C[u + M m]
    if (two) {
#pragma unroll
      for (int j = 0; j < R; ++j) q[j] = row[cphys<N, MR>(R * v + j)];
      fft<R, false>(q);  // q[m] = C[v + M m]
    }
    if (u == 0) {
      p[0] = make_float2(p[0].x + p[0].y, p[0].x - p[0].y);  // (R[0], R[L])
#pragma unroll
      for (int m = 1; m < R; ++m) {
        if (2 * m == R) p[m] = cconj(p[m]);
        else if (m < R - m) c_r2c_pair(p[m], p[R - m], tw[G::M * m]);
      }
    } else if (u == G::M / 2) {
#pragma unroll
      for (int m = 0; m < R / 2; ++m) c_r2c_pair(p[m], p[R - 1 - m], tw[G::M / 2 + G::M * m]);
    } else {
#pragma unroll
      for (int m = 0; m < R; ++m) c_r2c_pair(p[m], q[R - 1 - m], tw[u + G::M * m]);
    }
#pragma unroll
    for (int m = 0; m < R; ++m) row[cphys<N, MR>(R * u + m)] = p[m];
    if (two) {
#pragma unroll
      for (int m = 0; m < R; ++m) row[cphys<N, MR>(R * v + m)] = q[m];
    }
  }
}

// inverse: packed half spectrum (digit-reversed slots) -> real row in natural slots (unnormalised)
template <int N, int MR>
__device__ __forceinline__ void crow_inv(float2* row, int h, const float2* tw) {
  using G = CGeo<N, MR>;
  constexpr int R = G::R;
  for (int u = h; u <= G::M / 2; u += R) {
    const int v = G::M - u;
    const bool two = u != 0 && u != G::M / 2;
    float2 p[R], q[R];
#pragma unroll
    for (int m = 0; m < R; ++m) p[m] = row[cphys<N, MR>(R * u + m)];
    if (two) {
#pragma unroll
      for (int m = 0; m < R; ++m) q[m] = row[cphys<N, MR>(R * v + m)];
    }
    if (u == 0) {
      p[0] = make_float2(p[0].x + p[0].y, p[0].x - p[0].y);
#pragma unroll
      for (int m = 1; m < R; ++m) {
        if (2 * m == R) p[m] = cscale(cconj(p[m]), 2.0f);
        else if (m < R - m) c_c2r_pair(p[m], p[R - m], tw[G::M * m]);
      }
    } else if (u == G::M / 2) {
#pragma unroll
      for (int m = 0; m < R / 2; ++m) c_c2r_pair(p[m], p[R - 1 - m], tw[G::M / 2 + G::M * m]);
    } else {
#pragma unroll
      for (int m = 0; m < R; ++m) c_c2r_pair(p[m], q[R - 1 - m], tw[u + G::M * m]);
    }
    fft<R, true>(p);  // p[j] = sum_m exp(+2 pi i j m / R) C'[u + M m]
#pragma unroll
    for (int j = 0; j < R; ++j) row[cphys<N, MR>(R * u + j)] = j == 0 ? p[0] : cmul(p[j], cconj(tw[2 * j * u]));
    if (two) {
      fft<R, true>(q);
#pragma unroll
      for (int j = 0; j < R; ++j) row[cphys<N, MR>(R * v + j)] = j == 0 ? q[0] : cmul(q[j], cconj(tw[2 * j * v]));
    }
  }
  __syncwarp();
  float2 x[G::M];
#pragma unroll
  for (int k = 0; k < G::M; ++k) x[k] = row[cphys<N, MR>(R * k + h)];
  fft<G::M, true>(x);
#pragma unroll
  for (int i = 0; i < G::M; ++i) row[cphys<N, MR>(R * i + h)] = x[i];
}

// t-draw of global row y on its staged row: t = a + q (q s + sqrt(tau) xi), table aq[x*H + ty] =
// ((1 - w) d, sqrt(w)) with the CTA-contiguous row index ty = b*M + a; Philox stream ts (0; 8 for the
// second shear component), group y*W/4 + q feeds pixels 4q .. 4q+3 (q = h, h + R, ...)
template <int N, int MR>
__device__ __forceinline__ void ct_draw(float2* row, int y, int ty, int h, const float2* __restrict__ aq,
                                        float sqrt_tau, uint32_t step, uint32_t chain, uint32_t k0, uint32_t k1,
                                        uint32_t ts = 0u) {
  using G = CGeo<N, MR>;
  const uint64_t pol = l2_keep();
#pragma unroll 2
  for (int q = h; q < G::W / 4; q += G::R) {
    float z[4];
    normals4(uint32_t(y * (G::W / 4) + q), step, chain, ts, k0, k1, z);
    float2 p0 = row[cphys<N, MR>(2 * q)], p1 = row[cphys<N, MR>(2 * q + 1)];
    const float2 c0 = ldk(aq + (4 * q) * G::H + ty, pol), c1 = ldk(aq + (4 * q + 1) * G::H + ty, pol);
    const float2 c2 = ldk(aq + (4 * q + 2) * G::H + ty, pol), c3 = ldk(aq + (4 * q + 3) * G::H + ty, pol);
    p0.x = fmaf(c0.y, fmaf(c0.y, p0.x, sqrt_tau * z[0]), c0.x);
    p0.y = fmaf(c1.y, fmaf(c1.y, p0.y, sqrt_tau * z[1]), c1.x);
    p1.x = fmaf(c2.y, fmaf(c2.y, p1.x, sqrt_tau * z[2]), c2.x);
    p1.y = fmaf(c3.y, fmaf(c3.y, p1.y, sqrt_tau * z[3]), c3.x);
    row[cphys<N, MR>(2 * q)] = p0;
    row[cphys<N, MR>(2 * q + 1)] = p1;
  }
}

// ---------------------------------------------------------------------------------------------
// column passes
// ---------------------------------------------------------------------------------------------
// local forward: M-point FFT down slot t of this CTA's rows, output k' twiddled by W_N^(b k')
template <int N, int MR>
__device__ __forceinline__ void ccol_fwd(float2* rows, int t, int b, const float2* tw) {
  using G = CGeo<N, MR>;
  float2 x[G::M];
  const int pt = cphys<N, MR>(t);
#pragma unroll
  for (int a = 0; a < G::M; ++a) x[a] = rows[a * G::SP + pt];
  fft<G::M, false>(x);
#pragma unroll
  for (int k = 0; k < G::M; ++k) rows[k * G::SP + pt] = k == 0 ? x[0] : cmul(x[k], tw[b * k]);
}
// local inverse: untwiddle by W_N^(-b k'), inverse M-point FFT back to the rows
template <int N, int MR>
__device__ __forceinline__ void ccol_inv(float2* rows, int t, int b, const float2* tw) {
  using G = CGeo<N, MR>;
  float2 x[G::M];
  const int pt = cphys<N, MR>(t);
#pragma unroll
  for (int k = 0; k < G::M; ++k) {
    const float2 v = rows[k * G::SP + pt];
    x[k] = k == 0 ? v : cmul(v, cconj(tw[b * k]));
  }
  fft<G::M, true>(x);
#pragma unroll
  for (int a = 0; a < G::M; ++a) rows[a * G::SP + pt] = x[a];
}

// Mode coefficients of the cluster s-draw, looked up by the slot-order index i = ctab_index(ky, kx).
// CTabCoef reads the per-call table fg = (f / n, g / sqrt(2 n)). CBandCoef (the hierarchical sampler)
// takes them from the per-band table cb = band_coef(P_b) of the mode's bin (bmap[i].x >= 0; -1: the
// table's coefficients) and stores the band statistics of each new mode, (n |s_hat|^2 weighted by the
// mirror modes it stands for, the squares of its stream-6 normals), to its own position bmap[i].y of the
// chain's bin-ordered buffer (< 0: not summed), so that the band sums need no atomics.
struct CTabCoef {
  static constexpr bool kBand = false;
  const float2* __restrict__ fg;
  __device__ __forceinline__ float2 m(int i) const { return ldk(fg + i, l2_keep()); }
  __device__ __forceinline__ void add2(int, float, float, int, float, float) const {}
};
struct CBandCoef {
  static constexpr bool kBand = true;
  const float2* __restrict__ fg;
  const int2* __restrict__ bmap;  // slot order: (bin, position in the bin-ordered buffer)
  const float2* cb;               // shared [n_bins]: band_coef of each band power
  float2* buf;                    // this chain's statistics, bin-ordered (global, L2)
  float n;
  __device__ __forceinline__ float2 m(int i) const {
    const int b = WF_LDG(bmap + i).x;
    return b < 0 ? WF_LDG(fg + i) : cb[b];
  }
  __device__ __forceinline__ void put(int i, float s2, float x2) const {
    if (i < 0) return;
    const int pos = WF_LDG(bmap + i).y;
    if (pos >= 0) __stcg(buf + pos, make_float2(s2 * n, x2));
  }
  __device__ __forceinline__ void add2(int i0, float s0, float x0, int i1, float s1, float x1) const {
    put(i0, s0, x0);
    put(i1, s1, x1);
  }
};

// One mode pair (ky1, ky2 = N - ky1, or N/2 when ky1 = 0) of packed column slot t (kx = K) with the
// s-draw s_hat = f t_hat + g zeta, coefficients from cf. Interior columns: Philox stream 1 group
// K*H/2 + ky1, variates 0, 1 for ky1 and 2, 3 for ky2. Packed edge column (K = 0: kx = 0 as A and
// kx = W/2 as B in Y = A + i B): group ky1 draws (ky1, 0) from variates 0, 1 and (ky1, W/2) from 2, 3,
// the conjugates filling ky2; group 0 holds the four real modes (0,0), (H/2,0), (0,W/2), (H/2,W/2).
// With band statistics the stream-6 normals of the same group enter X_b in the same pattern.
template <int N, int MR, class C>
__device__ __forceinline__ void cdraw_pair(float2& y1, float2& y2, int K, int t, int ky1, int ky2, const C& cf,
                                           uint32_t step, uint32_t chain, uint32_t k0, uint32_t k1) {
  using G = CGeo<N, MR>;
  const uint32_t grp = uint32_t(K * (G::H / 2) + ky1);
  float z[4], zb[4];
  normals4(grp, step, chain, 1u, k0, k1, z);
  if constexpr (C::kBand) normals4(grp, step, chain, 6u, k0, k1, zb);
  auto sq = [](float2 v) { return fmaf(v.x, v.x, v.y * v.y); };
  // band statistics of the new modes: (index, weighted |s_hat|^2, sum of squared stream-6 normals), two
  // entries per pair; the edge lane's real modes (H/2, 0), (H/2, W/2) of group 0 come after
  int ia = -1, ib = -1;
  float sa = 0.f, xa = 0.f, sb = 0.f, xb = 0.f;
  if (K != 0) {
    const int i1 = ky1 * G::L + t, i2 = ky2 * G::L + t;
    const float2 m1 = cf.m(i1), m2 = cf.m(i2);
    y1 = make_float2(fmaf(m1.x, y1.x, m1.y * z[0]), fmaf(m1.x, y1.y, m1.y * z[1]));
    y2 = make_float2(fmaf(m2.x, y2.x, m2.y * z[2]), fmaf(m2.x, y2.y, m2.y * z[3]));
    if constexpr (C::kBand) {  // both modes have their mirror in the other half plane: weight 2
      ia = i1, sa = 2.0f * sq(y1), xa = fmaf(zb[0], zb[0], zb[1] * zb[1]);
      ib = i2, sb = 2.0f * sq(y2), xb = fmaf(zb[2], zb[2], zb[3] * zb[3]);
    }
  } else {
    const int ia1 = ky1 * G::L, ib1 = G::H * G::L + ky1;
    const float2 a1 = cf.m(ia1), b1 = cf.m(ib1);
    if (ky1 == 0) {
      const float2 a2 = cf.m(ky2 * G::L), b2 = cf.m(G::H * G::L + ky2);
      constexpr float R2 = 1.41421356237309505f;
      y1 = make_float2(fmaf(a1.x, y1.x, R2 * a1.y * z[0]), fmaf(b1.x, y1.y, R2 * b1.y * z[2]));
      y2 = make_float2(fmaf(a2.x, y2.x, R2 * a2.y * z[1]), fmaf(b2.x, y2.y, R2 * b2.y * z[3]));
      if constexpr (C::kBand) {  // one real degree of freedom each
        ia = ia1, sa = y1.x * y1.x, xa = zb[0] * zb[0];
        ib = ib1, sb = y1.y * y1.y, xb = zb[2] * zb[2];
      }
    } else {
      const float2 y2c = cconj(y2);
      const float2 Am = cscale(cadd(y1, y2c), 0.5f);
      const float2 Bm = cmul_mi(cscale(csub(y1, y2c), 0.5f));
      const float2 Ap = make_float2(fmaf(a1.x, Am.x, a1.y * z[0]), fmaf(a1.x, Am.y, a1.y * z[1]));
      const float2 Bp = make_float2(fmaf(b1.x, Bm.x, b1.y * z[2]), fmaf(b1.x, Bm.y, b1.y * z[3]));
      y1 = cadd(Ap, cmul_i(Bp));
      y2 = cadd(cconj(Ap), cmul_i(cconj(Bp)));
      if constexpr (C::kBand) {  // (ky1, 0) and (ky1, W/2) with their mirrors at H - ky1: weight 2
        ia = ia1, sa = 2.0f * sq(Ap), xa = fmaf(zb[0], zb[0], zb[1] * zb[1]);
        ib = ib1, sb = 2.0f * sq(Bp), xb = fmaf(zb[2], zb[2], zb[3] * zb[3]);
      }
    }
  }
  if constexpr (C::kBand) {
    cf.add2(ia, sa, xa, ib, sb, xb);
    if (K == 0 && ky1 == 0)  // the edge lane's real modes (H/2, 0) and (H/2, W/2)
      cf.add2(ky2 * G::L, y2.x * y2.x, zb[1] * zb[1], G::H * G::L + ky2, y2.y * y2.y, zb[3] * zb[3]);
  }
}

// Cross-cluster radix-P stage. Work unit (slot t, k' = u with its mirror v = M - u; u = 0 is paired with
// u = M/2, the two half-size units): gathers Y_j[u] (and Y_j[v]) from every CTA j, forms the column spectrum
// t_hat[u + M m], hands every mode pair (ky1 < N/2, ky2 = N - ky1, or N/2 when ky1 = 0) of column K to
// fn(K, t, y1, y2, ky1, ky2), and with WRITE scatters the inverse stage back. g = the thread's index in the
// cluster. Every mode of the half spectrum is in exactly one pair of one unit, and there are L M / 2 units
// of equal size, a whole number per thread of the cluster (one each at 512^2, eight at 256^2).
template <int N, int MR, bool WRITE, class F>
__device__ __forceinline__ void ccol_units(cooperative_groups::cluster_group& cl, float2* rows, int g, F&& fn) {
  using G = CGeo<N, MR>;
  constexpr int P = G::P, L = G::L, R = G::R;
  constexpr int M = G::M;
  constexpr int PAIRS = L * (M / 2);
  static_assert(PAIRS % (P * L) == 0, "equal work units per thread");
  if constexpr (PAIRS == P * L) {
    // One unit pair per thread (512^2, 16 CTAs of 32 rows): each thread takes one unit of a pair in turn
    // (two units), its partner lane (lane ^ 16, same slot t) the other, so a thread holds P values instead of
    // 2 P. For u != 0 each lane leads, at step m, the pair whose first mode is its own y[m] (ky1 = uu + M m):
    // it fetches the second mode from its partner's y[P-1-m] by a shuffle, runs fn on both, and hands the new
    // second value back (the led and the handed indices are disjoint). The units u = 0 and M/2 hold their
    // pairs themselves. Same pairs, roles and draws as the two-unit form below.
    static_assert(L % 16 == 0, "a half-warp of consecutive slots shares one unit");
    const int lane = int(threadIdx.x) % 32, half = lane / 16;
    const int w0 = (g / 32) * 16 + lane % 16;
#pragma unroll 1
    for (int rep = 0; rep < 2; ++rep) {
      const int w = w0 + rep * (PAIRS / 2);
      const int t = w % L, u = w / L;
      const int uu = half == 0 ? u : (u == 0 ? M / 2 : M - u);  // this lane's unit
      const int K = (t % R) * M + t / R;                         // kx held by slot t
      float2 y[P];
#pragma unroll
      for (int j = 0; j < P; ++j) y[j] = cl.map_shared_rank(rows, j)[uu * G::SP + cphys<N, MR>(t)];
      fft<P, false>(y);  // y[m] = t_hat[uu + M m]
      if (u == 0) {      // the same in every lane of the warp
        if (half == 0) {
          fn(K, t, y[0], y[P / 2], 0, N / 2);
#pragma unroll
          for (int m = 1; m < P / 2; ++m) fn(K, t, y[m], y[P - m], M * m, N - M * m);
        } else {
#pragma unroll
          for (int m = 0; m < P / 2; ++m) fn(K, t, y[m], y[P - 1 - m], M / 2 + M * m, N - M / 2 - M * m);
        }
      } else {
#pragma unroll
        for (int m = 0; m < P / 2; ++m) {
          float2 y2 = make_float2(__shfl_xor_sync(0xffffffffu, y[P - 1 - m].x, 16),
                                  __shfl_xor_sync(0xffffffffu, y[P - 1 - m].y, 16));
          fn(K, t, y[m], y2, uu + M * m, N - uu - M * m);
          y[P - 1 - m] = make_float2(__shfl_xor_sync(0xffffffffu, y2.x, 16), __shfl_xor_sync(0xffffffffu, y2.y, 16));
        }
      }
      if (WRITE) {
        fft<P, true>(y);
#pragma unroll
        for (int j = 0; j < P; ++j) cl.map_shared_rank(rows, j)[uu * G::SP + cphys<N, MR>(t)] = y[j];
      }
    }
    return;
  }
  for (int w = g; w < L * (M / 2); w += P * L) {
    const int t = w % L, u = w / L, v = u == 0 ? M / 2 : M - u;
    const int K = (t % R) * M + t / R;  // kx held by slot t
    float2 p[P], q[P];
#pragma unroll
    for (int j = 0; j < P; ++j) p[j] = cl.map_shared_rank(rows, j)[u * G::SP + cphys<N, MR>(t)];
#pragma unroll
    for (int j = 0; j < P; ++j) q[j] = cl.map_shared_rank(rows, j)[v * G::SP + cphys<N, MR>(t)];
    fft<P, false>(p);  // p[m] = t_hat[u + M m]
    fft<P, false>(q);  // q[m] = t_hat[v + M m]
    if (u == 0) {
      fn(K, t, p[0], p[P / 2], 0, N / 2);
#pragma unroll
      for (int m = 1; m < P / 2; ++m) fn(K, t, p[m], p[P - m], M * m, N - M * m);
#pragma unroll
      for (int m = 0; m < P / 2; ++m) fn(K, t, q[m], q[P - 1 - m], M / 2 + M * m, N - M / 2 - M * m);
    } else {
#pragma unroll
      for (int m = 0; m < P / 2; ++m) {
        fn(K, t, p[m], q[P - 1 - m], u + M * m, N - u - M * m);
        fn(K, t, q[m], p[P - 1 - m], v + M * m, N - v - M * m);
      }
    }
    if (WRITE) {
      fft<P, true>(q);
#pragma unroll
      for (int j = 0; j < P; ++j) cl.map_shared_rank(rows, j)[v * G::SP + cphys<N, MR>(t)] = q[j];
      fft<P, true>(p);
#pragma unroll
      for (int j = 0; j < P; ++j) cl.map_shared_rank(rows, j)[u * G::SP + cphys<N, MR>(t)] = p[j];
    }
  }
}

// the s-draw of Alg. 1 on every mode
template <int N, int MR, class C>
__device__ __forceinline__ void ccol_draw(cooperative_groups::cluster_group& cl, float2* rows, int g, const C& cf,
                                          uint32_t step, uint32_t chain, uint32_t k0, uint32_t k1) {
  ccol_units<N, MR, true>(cl, rows, g, [&](int K, int t, float2& y1, float2& y2, int ky1, int ky2) {
    cdraw_pair<N, MR>(y1, y2, K, t, ky1, ky2, cf, step, chain, k0, k1);
  });
}

// Wiener-filter update at level lambda (G -> 0): s_hat = f t_hat with f = P / (P + lambda tau) (scaled by
// 1/n). With CMP the residual of the previous iterate, |s_hat_new - s_hat_old|^2 (1 + P / (lambda tau))^2,
// is summed over the full spectrum (the mirror modes counted; returned as this thread's share, summed in
// FP32 over its units); with STORE
// the new modes go to prev[ky * W/2 + t] (slot order; packed edge column as stored). Pk in slot order
// (ctab_index).
template <int N, int MR>
__device__ __forceinline__ double ccol_wf(cooperative_groups::cluster_group& cl, float2* rows, int g,
                                          const float* __restrict__ Pk, float lt_, float2* __restrict__ prev,
                                          bool cmp, bool store) {
  using G = CGeo<N, MR>;
  constexpr int LR = G::L;
  constexpr float INV_N = 1.0f / float(G::H * G::W);
  const float inv_lt = 1.0f / lt_;
  auto wres = [&](float P, float dre, float dim) -> float {
    const float q = fmaf(P, inv_lt, 1.0f);
    return fmaf(dre, dre, dim * dim) * (q * q);
  };
  auto fcoef = [&](float P) { return wf_fdiv(P, P + lt_) * INV_N; };
  float acc = 0.0f;  // this thread's units in FP32; the cluster sum is FP64
  const uint64_t pol = l2_keep();
  ccol_units<N, MR, true>(cl, rows, g, [&](int K, int t, float2& y1, float2& y2, int ky1, int ky2) {
    if (K != 0) {
      const float P1 = ldk(Pk + ky1 * LR + t, pol), P2 = ldk(Pk + ky2 * LR + t, pol);
      const float2 n1 = cscale(y1, fcoef(P1)), n2 = cscale(y2, fcoef(P2));
      if (cmp) {
        const float2 o1 = prev[ky1 * LR + t], o2 = prev[ky2 * LR + t];
        acc += 2.0f * (wres(P1, n1.x - o1.x, n1.y - o1.y) + wres(P2, n2.x - o2.x, n2.y - o2.y));
      }
      y1 = n1;
      y2 = n2;
    } else {
      const float Pa1 = WF_LDG(Pk + ky1 * LR), Pb1 = WF_LDG(Pk + G::H * LR + ky1);
      const float fa1 = fcoef(Pa1), fb1 = fcoef(Pb1);
      if (ky1 == 0) {
        const float Pa2 = WF_LDG(Pk + ky2 * LR), Pb2 = WF_LDG(Pk + G::H * LR + ky2);
        const float2 n1 = make_float2(fa1 * y1.x, fb1 * y1.y);
        const float2 n2 = make_float2(fcoef(Pa2) * y2.x, fcoef(Pb2) * y2.y);
        if (cmp) {
          const float2 o1 = prev[ky1 * LR], o2 = prev[ky2 * LR];
          acc += wres(Pa1, n1.x - o1.x, 0.f) + wres(Pb1, n1.y - o1.y, 0.f) + wres(Pa2, n2.x - o2.x, 0.f) +
                 wres(Pb2, n2.y - o2.y, 0.f);
        }
        y1 = n1;
        y2 = n2;
      } else {
        const float2 y2c = cconj(y2);
        const float2 A = cscale(cscale(cadd(y1, y2c), 0.5f), fa1);
        const float2 B = cscale(cmul_mi(cscale(csub(y1, y2c), 0.5f)), fb1);
        if (cmp) {
          const float2 o1 = prev[ky1 * LR], o2c = cconj(prev[ky2 * LR]);
          const float2 oA = cscale(cadd(o1, o2c), 0.5f);
          const float2 oB = cmul_mi(cscale(csub(o1, o2c), 0.5f));
          acc += 2.0f * (wres(Pa1, A.x - oA.x, A.y - oA.y) + wres(Pb1, B.x - oB.x, B.y - oB.y));
        }
        y1 = cadd(A, cmul_i(B));
        y2 = cadd(cconj(A), cmul_i(cconj(B)));
      }
    }
    if (store) {
      prev[ky1 * LR + t] = y1;
      prev[ky2 * LR + t] = y2;
    }
  });
  return double(acc);
}

// sum over the full spectrum of P^2 |V|^2 for the forward transform V (level norms); this thread's share
template <int N, int MR>
__device__ __forceinline__ double ccol_p2(cooperative_groups::cluster_group& cl, float2* rows, int g,
                                          const float* __restrict__ Pk) {
  using G = CGeo<N, MR>;
  constexpr int WH = G::WH;
  auto p2 = [](float P, float re, float im) -> float { return P * P * fmaf(re, re, im * im); };
  float acc = 0.0f;
  ccol_units<N, MR, false>(cl, rows, g, [&](int K, int t, float2& y1, float2& y2, int ky1, int ky2) {
    if (K != 0) {
      acc += 2.0f * (p2(WF_LDG(Pk + ky1 * G::L + t), y1.x, y1.y) + p2(WF_LDG(Pk + ky2 * G::L + t), y2.x, y2.y));
    } else if (ky1 == 0) {
      acc += p2(WF_LDG(Pk + ky1 * G::L), y1.x, 0.f) + p2(WF_LDG(Pk + G::H * G::L + ky1), y1.y, 0.f) +
             p2(WF_LDG(Pk + ky2 * G::L), y2.x, 0.f) + p2(WF_LDG(Pk + G::H * G::L + ky2), y2.y, 0.f);
    } else {
      const float2 y2c = cconj(y2);
      const float2 A = cscale(cadd(y1, y2c), 0.5f);
      const float2 B = cmul_mi(cscale(csub(y1, y2c), 0.5f));
      acc += 2.0f * (p2(WF_LDG(Pk + ky1 * G::L), A.x, A.y) + p2(WF_LDG(Pk + G::H * G::L + ky1), B.x, B.y));
    }
  });
  return double(acc);
}

// Wiener-filter pixel update of a row at level lambda: t = d + w (s - d), w = 1 / (1 + lambda tau / N_bar),
// table dn[x*H + y] = (d, 1/N_bar) ((0, 0) on missing pixels: t = s), y the CTA-contiguous table row b*M + a
template <int N, int MR>
__device__ __forceinline__ void ct_update_wf(float2* row, int y, int h, const float2* __restrict__ dn, float lt_) {
  using G = CGeo<N, MR>;
  const uint64_t pol = l2_keep();
  for (int x2 = h; x2 < G::W / 2; x2 += G::R) {
    float2 v = row[cphys<N, MR>(x2)];
    const float2 c0 = ldk(dn + (2 * x2) * G::H + y, pol), c1 = ldk(dn + (2 * x2 + 1) * G::H + y, pol);
    const float w0 = wf_rcp(fmaf(lt_, c0.y, 1.0f)), w1 = wf_rcp(fmaf(lt_, c1.y, 1.0f));
    v.x = fmaf(w0, v.x - c0.x, c0.x);
    v.y = fmaf(w1, v.y - c1.x, c1.x);
    row[cphys<N, MR>(x2)] = v;
  }
}

// right-hand side N_lambda^-1 d = d / (N_bar + lambda tau) of one staged row (0 on missing pixels), by the
// row's R threads over the same slots as the pixel updates (x2 = h, h + R, ...), table row ty (CTA-
// contiguous, so the row threads' loads coalesce); each thread writes only slots it reads next
template <int N, int MR>
__device__ __forceinline__ void crhs_row(float2* row, int ty, int h, const float2* __restrict__ dn, float lt_) {
  using G = CGeo<N, MR>;
  for (int x2 = h; x2 < G::W / 2; x2 += G::R) {
    const float2 c0 = WF_LDG(dn + (2 * x2) * G::H + ty), c1 = WF_LDG(dn + (2 * x2 + 1) * G::H + ty);
    const float nb0 = c0.y > 0.0f ? wf_rcp(c0.y) : wf_inf(), nb1 = c1.y > 0.0f ? wf_rcp(c1.y) : wf_inf();
    row[cphys<N, MR>(x2)] = make_float2(c0.x / (nb0 + lt_), c1.x / (nb1 + lt_));
  }
}

// Cluster-wide sum of one double per thread, the same in every thread: block sums, then the P CTA sums
// collected in CTA 0's shared slots part[0..P) and added in rank order. red: >= 33 doubles.
template <int N, int MR>
__device__ __forceinline__ double cluster_sum(cooperative_groups::cluster_group& cl, double v, double* red,
                                              double* part) {
  using G = CGeo<N, MR>;
  const double s = block_sum(v, red);
  if (threadIdx.x == 0) cl.map_shared_rank(part, 0)[cl.block_rank()] = s;
  cl.sync();
  const double* p0 = cl.map_shared_rank(part, 0);
  double tot = 0.0;
#pragma unroll
  for (int j = 0; j < G::P; ++j) tot += p0[j];
  return tot;
}

// ---------------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------------
template <int N, int MR>
constexpr int csample_min_ctas() { return CGeo<N, MR>::L <= 128 ? 3 : (CGeo<N, MR>::M <= 32 ? 2 : 1); }

// twiddles exp(-2 pi i j / N) (FP64, rounded once) into shared memory
template <int N, int MR>
__device__ __forceinline__ void ctw_init(float2* tw) {
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * double(j) / double(N), &sn, &cs);
    tw[j] = make_float2(float(cs), float(sn));
  }
}

// this CTA's rows of a row-major [H][W] image into the staged rows (nullptr: zero), by the L threads
// lt = 0 .. L-1
template <int N, int MR>
__device__ __forceinline__ void crows_load(float2* rows, int b, const float* src, int lt = threadIdx.x) {
  using G = CGeo<N, MR>;
  for (int e = lt; e < G::A * G::L; e += G::L) {
    const int ar = e / G::L, i = e % G::L;
    float2 v = make_float2(0.f, 0.f);
    if (src != nullptr) v = WF_LDG(reinterpret_cast<const float2*>(src + (long long)(G::P * ar + b) * G::W) + i);
    rows[ar * G::SP + cphys<N, MR>(i)] = v;
  }
}

// the staged rows to this CTA's rows of an image of element type t, by the L threads lt = 0 .. L-1
template <int N, int MR>
__device__ __forceinline__ void crows_store(const float2* rows, int b, void* dst, int t, int lt = threadIdx.x) {
  using G = CGeo<N, MR>;
  for (int e = lt; e < G::A * G::L; e += G::L) {
    const int r2 = e / G::L, i = e % G::L;
    const long long at = (long long)(G::P * r2 + b) * G::L + i;
    const float2 v = rows[r2 * G::SP + cphys<N, MR>(i)];
    if (t == kOutF32) {
      __stcs(reinterpret_cast<float2*>(dst) + at, v);  // evict-first: the samples are not read again
    } else {
      store_pair(dst, at, v, t);
    }
  }
}

// Sampler sweeps (Alg. 1) of one chain by its cluster from the staged rows (the current s) of NC fields
// (NC = 2: the two shear components, field c's rows at rows + c A SP, its pixel table at aq + c H W, its
// t-draw from Philox stream 8 c). With SPLIT (NC = 2, 2 L threads) threads c L .. c L + L - 1 run field
// c's row and column passes; otherwise each of the L threads runs them for every field in turn. Per sweep
// (done = the sweeps before it in this call, step = step0 + done): t-draws and forward transforms, then
// col(step, done) between the two cluster barriers (the column spectra complete: the s-draw),
// post(step, done) right after the second (every CTA's column work done), the inverse transforms. Sample
// m (the state after sweep burn_in + (m + 1) thin) goes to out + (m NC + c) H W elements of type out_dtype.
template <int N, int MR, int NC, bool SPLIT, class Col, class Post>
__device__ __forceinline__ void csweeps(cooperative_groups::cluster_group& cl, float2* rows, const float2* tw,
                                        const float2* __restrict__ aq, float sqrt_tau, void* out_v, int out_dtype,
                                        int n_sweeps, int burn_in, int thin, uint32_t step0, uint32_t chain,
                                        uint32_t k0, uint32_t k1, Col&& col, Post&& post) {
  using G = CGeo<N, MR>;
  static_assert(!SPLIT || NC == 2, "split threads: one field per half of the CTA");
  constexpr int CS = G::A * G::SP;
  constexpr int C0N = SPLIT ? 1 : NC;  // fields per thread
  constexpr long long NPIX = (long long)G::H * G::W;
  const int lt = SPLIT ? int(threadIdx.x) % G::L : int(threadIdx.x), b = int(cl.block_rank());
  const int cf = SPLIT ? int(threadIdx.x) / G::L : 0;  // the thread's first field
  int ar, h;
  crow_of<N, MR>(lt, ar, h);
  const int y = G::P * ar + b;
  const int eb = out_elem_bytes(out_dtype);
  char* out = reinterpret_cast<char*>(out_v);
  for (int done = 0;;) {
    const uint32_t step = step0 + uint32_t(done);
#pragma unroll
    for (int k = 0; k < C0N; ++k) {
      const int c = cf + k;
      float2* row = rows + c * CS + ar * G::SP;
      ct_draw<N, MR>(row, y, b * G::M + ar, h, aq + c * NPIX, sqrt_tau, step, chain, k0, k1, 8u * uint32_t(c));
      __syncwarp();
      crow_fwd<N, MR>(row, h, tw);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < C0N; ++k) ccol_fwd<N, MR>(rows + (cf + k) * CS, lt, b, tw);
    cl.sync();  // every CTA's partial column transforms are in place
    col(step, done);
    cl.sync();  // every unit's inverse stage has landed
    post(step, done);
#pragma unroll
    for (int k = 0; k < C0N; ++k) ccol_inv<N, MR>(rows + (cf + k) * CS, lt, b, tw);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < C0N; ++k) crow_inv<N, MR>(rows + (cf + k) * CS + ar * G::SP, h, tw);
    ++done;
    if (done > burn_in && (done - burn_in) % thin == 0) {
      const long long m = (done - burn_in) / thin - 1;
      __syncthreads();
#pragma unroll
      for (int k = 0; k < C0N; ++k)
        crows_store<N, MR>(rows + (cf + k) * CS, b, out + (m * NC + cf + k) * NPIX * eb, out_dtype, lt);
      __syncthreads();
    }
    if (done == n_sweeps) break;
    __syncwarp();
  }
}

// the scalar sampler's sweeps (table coefficients fg in slot order)
template <int N, int MR>
__device__ __forceinline__ void csample_loop(cooperative_groups::cluster_group& cl, float2* rows, const float2* tw,
                                             const float2* __restrict__ aq, const float2* __restrict__ fg,
                                             float sqrt_tau, void* out_v, int out_dtype, int n_sweeps, int burn_in,
                                             int thin, uint32_t step0, uint32_t chain, uint32_t k0, uint32_t k1) {
  using G = CGeo<N, MR>;
  const int g = int(cl.block_rank()) * G::L + int(threadIdx.x);
  csweeps<N, MR, 1, false>(
      cl, rows, tw, aq, sqrt_tau, out_v, out_dtype, n_sweeps, burn_in, thin, step0, chain, k0, k1,
      [&](uint32_t step, int) { ccol_draw<N, MR>(cl, rows, g, CTabCoef{fg}, step, chain, k0, k1); },
      [](uint32_t, int) {});
}

// The cooled G -> 0 iteration (Alg. 1 without draws, lambda-cooling) of one image by its cluster from
// s = 0, with the per-level norms ||S N_lambda^-1 d||^2 computed first. Leaves s_W in the staged rows and
// returns the wf_status (0 converged, 5 not converged, 6 non-finite); it and rho receive the sweeps and
// the last measured residual. red: 33 doubles, part: P doubles, bn: kMaxLevels doubles (shared).
template <int N, int MR>
__device__ __forceinline__ int csolve_loop(cooperative_groups::cluster_group& cl, float2* rows, const float2* tw,
                                           double* red, double* part, double* bn, const float2* __restrict__ dn,
                                           const float* __restrict__ Pk, const Scalars& sc, float2* prev, double tol,
                                           double eta, double level_tol, int max_iter, int level_max, int check,
                                           int& it, double& rho) {
  using G = CGeo<N, MR>;
  const int tid = threadIdx.x, b = int(cl.block_rank()), g = b * G::L + tid;
  int ar, h;
  crow_of<N, MR>(tid, ar, h);
  const int y = G::P * ar + b;
  float2* row = rows + ar * G::SP;
  constexpr double NPIX = double(G::H) * double(G::W);
  for (int lev = 0; lev < sc.n_levels; ++lev) {  // level norms
    crhs_row<N, MR>(row, b * G::M + ar, h, dn, float(level_lambda(sc, lev, eta) * sc.tau));
    __syncwarp();
    crow_fwd<N, MR>(row, h, tw);
    __syncthreads();
    ccol_fwd<N, MR>(rows, tid, b, tw);
    cl.sync();
    const double tot = cluster_sum<N, MR>(cl, ccol_p2<N, MR>(cl, rows, g, Pk), red, part);
    if (tid == 0) bn[lev] = tot / NPIX;
    cl.sync();  // every CTA has read the partial sums and finished its remote reads of the rows
  }
  crows_load<N, MR>(rows, b, nullptr);
  __syncthreads();
  const double tau = sc.tau;
  int lev = 0, k = 0, status = 1;
  double lam = sc.lam0;
  float ltau = float(lam * tau);
  const int last_level = sc.n_levels - 1;
  it = 0;
  rho = -1.0;
  while (true) {
    ++k;
    ++it;
    const bool cmp = (k % check == 0) && k >= 2;
    const bool store = ((k + 1) % check == 0);
    ct_update_wf<N, MR>(row, b * G::M + ar, h, dn, ltau);
    __syncwarp();
    crow_fwd<N, MR>(row, h, tw);
    __syncthreads();
    ccol_fwd<N, MR>(rows, tid, b, tw);
    cl.sync();
    const double acc = ccol_wf<N, MR>(cl, rows, g, Pk, ltau, prev, cmp, store);
    cl.sync();
    if (cmp) {
      const double tot = cluster_sum<N, MR>(cl, acc, red, part) * NPIX;
      const double bnl = bn[lev];
      const double r2 = bnl > 0.0 ? tot / bnl : tot;
      rho = sqrt(r2);
      if (!(r2 == r2) || r2 > 1e300) {
        status = 6;  // non-finite residual
      } else if (lev < last_level) {
        if (rho < level_tol || k >= level_max) {
          ++lev;
          lam = level_lambda(sc, lev, eta);
          ltau = float(lam * tau);
          k = 0;
        }
      } else if (rho < tol) {
        status = 0;
      }
    }
    if (status == 1 && it >= max_iter) status = 5;  // not converged
    ccol_inv<N, MR>(rows, tid, b, tw);
    __syncthreads();
    crow_inv<N, MR>(row, h, tw);
    if (status != 1) break;
    __syncwarp();
  }
  __syncthreads();
  return status;
}

// one problem, grid = n_chains clusters of P CTAs (chain = cluster index)
template <int N, int MR>
__global__ void __launch_bounds__(N / 2, csample_min_ctas<N, MR>()) k_csample(SampleArgs a) {
  using G = CGeo<N, MR>;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* rows = reinterpret_cast<float2*>(smem_raw);
  float2* tw = reinterpret_cast<float2*>(smem_raw + G::ROWS_BYTES);
  if (a.sc->status != 0) return;  // uniform over the grid
  const long long ci = blockIdx.x / G::P;
  const int eb = out_elem_bytes(a.out_dtype);
  ctw_init<N, MR>(tw);
  crows_load<N, MR>(rows, int(cl.block_rank()), a.init_s ? a.init_s + ci * a.init_stride : nullptr);
  __syncthreads();
  csample_loop<N, MR>(cl, rows, tw, a.aq, a.fg, a.sc->sqrt_tau,
                  reinterpret_cast<char*>(a.out) + ci * a.n_samples * (long long)(G::H * G::W) * eb, a.out_dtype,
                  a.n_sweeps, a.burn_in, a.thin, a.step0, a.chain0 + uint32_t(ci), a.key0, a.key1);
  cl.sync();  // no CTA leaves while another may still address its shared memory
}

// Whole pipeline of a batch of large images, one cluster per image: level norms, the cooled Wiener solve
// from s = 0 (result to fields[f].out_wf when given, status to res[fields[f].item]), then n_samples
// sampler sweeps from s_W with step words 0, 1, ... and the image's chain and key into
// fields[f].out_samples. Images whose set-up failed only report their status.
struct CBArgs {
  const GBField* fields;
  const Scalars* sc;
  BatchResult* res;
  int F;
  double tol, eta, level_tol;
  int max_iter, level_max, check, n_samples;
};
template <int N, int MR>
__global__ void __launch_bounds__(N / 2, csample_min_ctas<N, MR>()) k_cpipe(CBArgs a) {
  using G = CGeo<N, MR>;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* rows = reinterpret_cast<float2*>(smem_raw);
  float2* tw = reinterpret_cast<float2*>(smem_raw + G::ROWS_BYTES);
  double* red = reinterpret_cast<double*>(smem_raw + G::ROWS_BYTES + N * 8);
  double* part = red + 33;
  double* bn = part + 16;
  const int f = blockIdx.x / G::P;
  const GBField fd = a.fields[f];
  const Scalars sc = a.sc[f];
  const bool lead = cl.block_rank() == 0 && threadIdx.x == 0;
  if (sc.status != 0) {  // uniform over the cluster
    if (lead) a.res[fd.item] = BatchResult{-1.0, 0, sc.status};
    return;
  }
  ctw_init<N, MR>(tw);
  __syncthreads();
  int it = 0;
  double rho = -1.0;
  const int status = csolve_loop<N, MR>(cl, rows, tw, red, part, bn, fd.dn, fd.Pk, sc, fd.prev, a.tol, a.eta,
                                    a.level_tol, a.max_iter, a.level_max, a.check, it, rho);
  if (fd.out_wf) crows_store<N, MR>(rows, int(cl.block_rank()), fd.out_wf, kOutF32);
  if (lead) a.res[fd.item] = BatchResult{rho, it, status};
  __syncthreads();
  if (a.n_samples > 0 && fd.out_samples)
    csample_loop<N, MR>(cl, rows, tw, fd.aq, fd.fg, sc.sqrt_tau, fd.out_samples, kOutF32, a.n_samples, 0, 1, 0u,
                    fd.chain, fd.key0, fd.key1);
  cl.sync();  // no CTA leaves while another may still address its shared memory
}

}  // namespace wf
