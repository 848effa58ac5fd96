// Messenger-field sweeps for images too large to keep a field in one SM (N in {256, 512, 1024}).
//
// The packed half spectrum Z[H][W/2] of every field (kx = 0 and W/2 packed as re/im of column 0) lives in
// global memory (L2-resident when the working set allows). One persistent cooperative kernel runs every
// sweep as two phases separated by a bounded grid barrier:
//   row phase    (CTA = RB rows of one field): Z rows -> C2R -> s -> [sample write] -> t-draw -> R2C -> Z
//   column phase (CTA = CB columns of one field): Z columns -> FFT -> s-draw -> inverse FFT -> Z
// (Alg. 1 of the paper with A = I). Each 1D transform of length L = R * S (S = 64, or 32 at 1024^2) runs
// in shared memory as R-point register DFTs on the S strided subsequences with twiddles W_L^(q n), then
// S-point register FFTs (decimation in frequency), with 1 float2 of padding per 64 to keep the strided accesses
// conflict-free. Every CTA uses 128 threads and 66,560 bytes of shared memory.
#pragma once

#include "wf_gibbs.cuh"

namespace wf {

// Length S of the register sub-transforms. A shorter S means fewer rows and columns per CTA and more work
// items per phase, so a single field keeps more CTAs busy: with S = 16 a 1024^2 field has 256 row and 256
// column items per phase (64 with S = 64). Measured on GB300 (one image): 1024^2 precision solve 3.27 s
// (S = 64) -> 2.14 s (32) -> 1.84 s (16); 256^2 solve of 184 sweeps 15.0 -> 7.2 -> 4.4 ms.
// Row and column sub-transform lengths measured on GB300 (one image, after the split of large step-A
// DFTs), microseconds per Wiener-filter sweep at 256^2 / 512^2 / 1024^2 (and ms for 4 chains x 50 samples
// at 256^2 / 512^2): rows 16, columns 16: 23.0 / 25.1 / 42.6 (0.97 / 1.56); rows 16, columns 32: 27.7 /
// 28.3 / 42.5; rows 32, columns 16: 34.1 / 48.7 / 65.3; rows 8, columns 16: 18.0 / 20.9 / 52.7 (0.80 /
// 2.14). So rows of 8-point sub-transforms at 256^2 and 16 elsewhere, columns 16.
template <int N_>
struct GGeo {
  static constexpr int N = N_, H = N_, W = N_;
  static constexpr int SR = N_ == 256 ? 8 : 16;  // sub-transform length of the row transforms
  static constexpr int SC = 16;                  // ... and of the column transforms
  static constexpr int LR = W / 2;          // complex length of a row transform
  static constexpr int RR = LR / SR;        // row radix
  static constexpr int RC = H / SC;         // column radix
  static constexpr int RB = 128 / RR;       // rows per CTA
  static constexpr int CB = 128 / RC;       // columns per CTA
  // float2 stride between vectors in shared memory: each vector carries 1 float2 of padding per 64 and
  // room for the skewed blocks between the two steps of fft_smem (R blocks of S + 1), and the stride is odd
  // (2 x odd when only 8 vectors share a half-warp) so that a half-warp reading the same element of
  // consecutive vectors hits distinct banks
  static constexpr int vstride(int len, int nv, int r) {
    const int v0 = len + len / 64, v = v0 > len + r ? v0 : len + r;
    return nv >= 16 ? (v % 2 == 1 ? v : v + 1) : (v % 16 == 2 ? v : v + ((18 - v % 16) % 16));
  }
  static constexpr int VROW = vstride(LR, 128 / RR, RR);
  static constexpr int VCOL = vstride(H, 128 / RC, RC);
  static constexpr int SMEM = (RB * VROW > CB * VCOL ? RB * VROW : CB * VCOL) * 8;
  static constexpr int ROW_ITEMS = H / RB;  // row-phase work items per field
  static constexpr int COL_ITEMS = LR / CB; // column-phase work items per field
  static constexpr int WH = W / 2 + 1;
};

WF_HD int padi(int i) { return i + (i >> 6); }

// Forward DFT of length L = R*S of the padded vectors v_j = buf + j*V (j < NV), natural order in and out.
// tw[j] = exp(-2 pi i j / L). INV: inverse via conjugation on the way in and out. 128 threads = NV * R.
//   step A: for each n < S, the R-point DFT A[q] = sum_m x[n + S m] w_R^(q m), twiddled by W_L^(q n),
//           stored at n + S q (block q);
//   step C: for each q < R, the S-point FFT of block q; output k goes to q + R k (decimation in
//           frequency: X[q + R k] = sum_n W_L^(q n) w_S^(n k) A_n[q]).
// When NV * S < 128 (one or two warps would carry step A alone) the R-point DFTs are themselves split,
// R = R1 R2 with m = m2 + R2 m1 and q = q1 + R1 q2:
//   A1: for each (n, m2), B[q1] = sum_m1 x[n + S (m2 + R2 m1)] w_R1^(q1 m1), twiddled by w_R^(m2 q1),
//       stored back at n + S (m2 + R2 q1);
//   A2: for each (n, q1), A[q1 + R1 q2] = sum_m2 B'[m2][q1] w_R2^(q2 m2), twiddled by W_L^(q n) and
//       stored in block q,
// so every pass has NV S R2 or NV S R1 small DFTs spread over all 128 threads, consecutive threads on
// consecutive n (contiguous addresses). A2 holds its inputs in registers across a CTA barrier anyway, so
// it writes the blocks skewed by one float2 each (block q at q (S + 1), not padded): the threads of a warp,
// each reading its own block in step C, then hit distinct banks.
template <int R>
__host__ __device__ constexpr int fft_smem_r1() { return R > 16 ? 8 : R; }

template <int R, int NV, int V, bool INV, int S = 64>
__device__ __forceinline__ void fft_smem(float2* buf, const float2* __restrict__ tw) {
  static_assert(NV * R == 128, "one sub-transform per thread in step C");
  constexpr int L = R * S;
  constexpr bool SPLIT = !(NV * S >= 128 || R <= 16);
  static_assert(!SPLIT || R * (S + 1) <= V, "room for the skewed blocks");
  const int tid = threadIdx.x;
  if constexpr (!SPLIT) {
    // step A: R-point DFT across the S strided subsequences, twiddled by W_L^(q n), in place
    for (int task = tid; task < NV * S; task += 128) {
      const int j = task / S, n = task % S;
      float2* v = buf + j * V;
      float2 a[R];
#pragma unroll
      for (int m = 0; m < R; ++m) {
        a[m] = v[padi(n + S * m)];
        if (INV) a[m].y = -a[m].y;
      }
      fft<R, false>(a);
#pragma unroll
      for (int q = 0; q < R; ++q) v[padi(n + S * q)] = q == 0 ? a[0] : cmul(a[q], __ldg(tw + q * n));
    }
  } else {
    constexpr int R1 = fft_smem_r1<R>(), R2 = R / R1;
    static_assert(R1 * R2 == R && (NV * S * R2) % 128 == 0 && (NV * S * R1) % 128 == 0, "split step A");
    // A1: R1-point DFTs over m1, twiddle w_R^(m2 q1) = W_L^((L/R) m2 q1), in place
    for (int task = tid; task < NV * S * R2; task += 128) {
      const int n = task % S, m2 = (task / S) % R2, j = task / (S * R2);
      float2* v = buf + j * V;
      float2 a[R1];
#pragma unroll
      for (int m1 = 0; m1 < R1; ++m1) {
        a[m1] = v[padi(n + S * (m2 + R2 * m1))];
        if (INV) a[m1].y = -a[m1].y;
      }
      fft<R1, false>(a);
#pragma unroll
      for (int q1 = 0; q1 < R1; ++q1)
        v[padi(n + S * (m2 + R2 * q1))] = q1 == 0 ? a[0] : cmul(a[q1], __ldg(tw + (L / R) * m2 * q1));
    }
    __syncthreads();
    // A2: R2-point DFTs over m2, twiddle W_L^(q n), q = q1 + R1 q2, to block q
    constexpr int T2 = NV * S * R1 / 128;  // tasks per thread
    float2 b[T2][R2];
#pragma unroll
    for (int t = 0; t < T2; ++t) {
      const int task = tid + 128 * t;
      const int n = task % S, q1 = (task / S) % R1, j = task / (S * R1);
      const float2* v = buf + j * V;
#pragma unroll
      for (int m2 = 0; m2 < R2; ++m2) b[t][m2] = v[padi(n + S * (m2 + R2 * q1))];
      fft<R2, false>(b[t]);
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < T2; ++t) {
      const int task = tid + 128 * t;
      const int n = task % S, q1 = (task / S) % R1, j = task / (S * R1);
      float2* v = buf + j * V;
#pragma unroll
      for (int q2 = 0; q2 < R2; ++q2) {
        const int q = q1 + R1 * q2;
        v[q * (S + 1) + n] = q == 0 ? b[t][q2] : cmul(b[t][q2], __ldg(tw + q * n));
      }
    }
  }
  __syncthreads();
  // step C: S-point FFT of each twiddled subsequence q (block q); output k goes to position q + R k
  // (consecutive threads take consecutive vectors)
  const int j = tid % NV, q = tid / NV;
  float2* v = buf + j * V;
  float2 u[S];
#pragma unroll
  for (int n = 0; n < S; ++n) u[n] = SPLIT ? v[q * (S + 1) + n] : v[padi(S * q + n)];
  __syncthreads();
  fft<S, false>(u);
#pragma unroll
  for (int k = 0; k < S; ++k) {
    float2 o = u[k];
    if (INV) o.y = -o.y;
    v[padi(q + R * k)] = o;
  }
  __syncthreads();
}

// Bounded grid barrier for a cooperative launch: arrive on count, the last arrival bumps gen.
// Gives up after 2^22 polls (a few seconds) and raises WF_ERR_TIMEOUT in *err; callers then leave.
struct GridBar {
  unsigned int count;
  unsigned int gen;
  int err;
  int pad;
};

__device__ __forceinline__ bool grid_barrier(GridBar* gb, unsigned int nblocks) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int g = atomicAdd(&gb->gen, 0u);
    if (atomicAdd(&gb->count, 1u) == nblocks - 1) {
      atomicExch(&gb->count, 0u);
      __threadfence();
      atomicAdd(&gb->gen, 1u);
      s_ok = 1;
    } else {
      int ok = 0;
      for (long it = 0; it < (1L << 22); ++it) {
        if (*reinterpret_cast<volatile unsigned int*>(&gb->gen) != g) { ok = 1; break; }
        if (*reinterpret_cast<volatile int*>(&gb->err) != 0) break;
        __nanosleep(64);
      }
      if (!ok) atomicExch(&gb->err, 7);  // WF_ERR_TIMEOUT
      s_ok = ok;
    }
    __threadfence();
  }
  __syncthreads();
  return s_ok != 0;
}

struct GlobalArgs {
  float2* Z;               // [n_fields][H][W/2] packed half spectra (state)
  const float2* tw_row;    // exp(-2 pi i j / (W/2)), j < W/2
  const float2* tw_col;    // exp(-2 pi i j / H), j < H
  const float2* tw_real;   // exp(-2 pi i k / W), k < W/2
  const float2* aq;        // sampler pixel table [W][H] (a, q)
  const float2* fg;        // sampler mode table [H][W/2+1]
  const float2* dn;        // Wiener-filter pixel table [W][H] (d, 1/N_bar)
  const float* Pk;         // [H][W/2+1]
  const Scalars* sc;
  GridBar* bar;
  // sampler
  const float* init_s;
  long long init_stride;
  float* out;
  long long n_samples;
  int n_fields;
  int n_sweeps;
  int burn_in;
  int thin;
  uint32_t chain0;
  uint32_t step0;
  uint32_t key0, key1;
  // Wiener filter (n_fields == 1)
  const double* bnorm2;
  double* acc;             // [2] residual accumulators (alternating)
  float2* prev;            // [H][W/2]
  SolveStatus* st;
  double tol, eta, level_tol;
  int max_iter, level_max, check;
  int rhs_mode;            // mode 1: dn holds (r, 1/N_bar), t = lambda tau r + w s (refinement correction)
  int mode;                // 0 sampler, 1 Wiener filter, 2 level norms (fields = levels), 3 weighted power
  double* bnorm_out;       // mode 2: [n_fields]
  // mode 3: fields v_f = va_f + vsign * vb_f, tables wts[nw][H][W/2+1], sums into wout[f*nw + j]
  const float* va;
  const float* vb;
  float vsign;
  const float* wts;
  int nw;
  double* wout;
  int grid_pct;            // host side: percent of the co-resident grid to launch (0 or >= 100: all of it)
  int out_dtype;           // mode 0: OutType of the samples
};

// R2C post-processing / C2R pre-processing of one padded row vector (pairs k <-> LR - k), all threads of
// the CTA over all rows in it. Same arithmetic as r2c_post_pair / c2r_pre_pair with run-time twiddles.
template <int N, bool POST>
__device__ __forceinline__ void real_pass(float2* buf, int nrows, const float2* __restrict__ tw_real) {
  using G = GGeo<N>;
  constexpr int L = G::LR;
  for (int task = threadIdx.x; task < nrows * (L / 2 + 1); task += 128) {
    const int j = task / (L / 2 + 1), k = task % (L / 2 + 1);
    float2* v = buf + j * G::VROW;
    if (k == 0) {
      const float2 c0 = v[0];
      v[0] = make_float2(c0.x + c0.y, c0.x - c0.y);
    } else if (2 * k == L) {
      const float2 c = v[padi(k)];
      v[padi(k)] = POST ? cconj(c) : cscale(cconj(c), 2.0f);
    } else if (k < L / 2) {
      const float2 w = __ldg(tw_real + k);  // exp(-2 pi i k / W)
      float2 a = v[padi(k)], b = cconj(v[padi(L - k)]);
      if (POST) {
        const float2 E = cscale(cadd(a, b), 0.5f);
        const float2 O = cmul_mi(cscale(csub(a, b), 0.5f));
        const float2 WO = cmul(O, w);
        v[padi(k)] = cadd(E, WO);
        v[padi(L - k)] = cconj(csub(E, WO));
      } else {
        const float2 E = cadd(a, b);
        const float2 O = cmul(csub(a, b), cconj(w));
        v[padi(k)] = cadd(E, cmul_i(O));
        v[padi(L - k)] = cadd(cconj(E), cmul_i(cconj(O)));
      }
    }
  }
  __syncthreads();
}

// Row-phase pixel update of rows y0 .. y0+RB-1 held in buf as (s[2m], s[2m+1]) pairs (then a CTA barrier):
//   mode 0: sampler t-draw t = (1 - w) d + sqrt(w) (sqrt(w) s + sqrt(tau) xi) with the (a, q) table, Philox
//           counter (pixel group (y W + x) / 4, step, chain, stream 0);
//   mode 1: Wiener-filter t-update t = w (s - d) + d, w = 1 / (1 + lambda tau / N_bar) from the (d, 1/N_bar)
//           table (rhs_mode: t = w s + lambda tau r with r in place of d);
//   mode 2: the level right-hand side N_lambda^-1 d with N_lambda = N_bar + lt2 (s ignored).
template <int N>
__device__ __forceinline__ void pixel_update(int mode, float2* buf, int y0, const float2* __restrict__ aq,
                                             const float2* __restrict__ dn, uint32_t step, uint32_t chain,
                                             uint32_t key0, uint32_t key1, float sqrt_tau, float ltau, int rhs_mode,
                                             float lt2) {
  using G = GGeo<N>;
  for (int task = threadIdx.x; task < G::RB * (G::W / 4); task += 128) {
    const int j = task / (G::W / 4), q = task % (G::W / 4);
    const int y = y0 + j;
    float2* v = buf + j * G::VROW;
    float2 p0 = v[padi(2 * q)], p1 = v[padi(2 * q + 1)];
    float s4[4] = {p0.x, p0.y, p1.x, p1.y};
    if (mode == 0) {
      float z[4];
      normals4(uint32_t(y * (G::W / 4) + q), step, chain, 0u, key0, key1, z);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 co = __ldg(aq + (4 * q + e) * G::H + y);
        s4[e] = fmaf(co.y, fmaf(co.y, s4[e], sqrt_tau * z[e]), co.x);
      }
    } else if (mode == 1) {
      const float g = rhs_mode ? 0.0f : 1.0f, h = rhs_mode ? ltau : 1.0f;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 co = __ldg(dn + (4 * q + e) * G::H + y);
        const float w = wf_rcp(fmaf(ltau, co.y, 1.0f));
        s4[e] = fmaf(w, fmaf(-g, co.x, s4[e]), h * co.x);
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 co = __ldg(dn + (4 * q + e) * G::H + y);
        const float nbar = co.y > 0.0f ? wf_rcp(co.y) : wf_inf();
        s4[e] = co.x / (nbar + lt2);
      }
    }
    v[padi(2 * q)] = make_float2(s4[0], s4[1]);
    v[padi(2 * q + 1)] = make_float2(s4[2], s4[3]);
  }
  __syncthreads();
}

// Row phase on one work item: rows y0 .. y0+RB-1 of field f. first: start from the real state s0.
template <int N>
__device__ void row_item(const GlobalArgs& a, float2* buf, int f, int y0, int done, bool first, bool emit_only,
                         float ltau, const Scalars& sc) {
  using G = GGeo<N>;
  constexpr int L = G::LR;
  float2* Zf = a.Z + (long long)f * G::H * L;
  const int nthr = 128;
  if (first) {
    for (int e = threadIdx.x; e < G::RB * L; e += nthr) {
      const int j = e / L, m = e % L;
      float2 v = make_float2(0.f, 0.f);
      if (a.mode == 0 && a.init_s != nullptr)
        v = reinterpret_cast<const float2*>(a.init_s + f * a.init_stride + (long long)(y0 + j) * G::W)[m];
      if (a.mode == 3) {
        const long long o = (long long)f * G::H * G::W + (long long)(y0 + j) * G::W;
        v = reinterpret_cast<const float2*>(a.va + o)[m];
        if (a.vb) {
          const float2 u = reinterpret_cast<const float2*>(a.vb + o)[m];
          v = make_float2(fmaf(a.vsign, u.x, v.x), fmaf(a.vsign, u.y, v.y));
        }
      }
      buf[j * G::VROW + padi(m)] = v;
    }
    __syncthreads();
  } else {
    for (int e = threadIdx.x; e < G::RB * L; e += nthr) {
      const int j = e / L, m = e % L;
      buf[j * G::VROW + padi(m)] = __ldcg(Zf + (long long)(y0 + j) * L + m);
    }
    __syncthreads();
    real_pass<N, false>(buf, G::RB, a.tw_real);
    fft_smem<G::RR, G::RB, G::VROW, true, G::SR>(buf, a.tw_row);
  }
  // buf rows hold (s[2m], s[2m+1]) (scaled as the fused kernels: unnormalised transforms, the 1/n and
  // 1/sqrt(2n) factors are in the Fourier-space tables)
  if (a.mode == 0 && !first) {
    const int d1 = done;  // sweeps completed
    if (d1 > a.burn_in && (d1 - a.burn_in) % a.thin == 0 && f < a.n_fields) {
      const long long ms = (d1 - a.burn_in) / a.thin - 1;
      const long long base = ((long long)f * a.n_samples + ms) * (long long)(G::H * G::W) / 2;  // pairs
      for (int e = threadIdx.x; e < G::RB * L; e += nthr) {
        const int j = e / L, m = e % L;
        store_pair(a.out, base + (long long)(y0 + j) * (G::W / 2) + m, buf[j * G::VROW + padi(m)], a.out_dtype);
      }
    }
    __syncthreads();  // the pixel update below maps threads to other elements of buf
  }
  if (emit_only) {
    if (a.mode == 1) {  // Wiener filter: final state to out
      for (int e = threadIdx.x; e < G::RB * L; e += nthr) {
        const int j = e / L, m = e % L;
        reinterpret_cast<float2*>(a.out + (long long)(y0 + j) * G::W)[m] = buf[j * G::VROW + padi(m)];
      }
    }
    __syncthreads();
    return;
  }
  // pixel-space update on 4-pixel groups (Philox group (y W + x)/4 in the sampler); mode 3 transforms
  // the field as loaded
  if (a.mode != 3)
    pixel_update<N>(a.mode, buf, y0, a.aq, a.dn, a.step0 + uint32_t(done), a.chain0 + uint32_t(f), a.key0, a.key1,
                    sc.sqrt_tau, ltau, a.rhs_mode, a.mode == 2 ? float(level_lambda(sc, f, a.eta) * sc.tau) : 0.f);
  else
    __syncthreads();
  fft_smem<G::RR, G::RB, G::VROW, false, G::SR>(buf, a.tw_row);
  real_pass<N, true>(buf, G::RB, a.tw_real);
  for (int e = threadIdx.x; e < G::RB * L; e += nthr) {
    const int j = e / L, m = e % L;
    __stcg(Zf + (long long)(y0 + j) * L + m, buf[j * G::VROW + padi(m)]);
  }
  __syncthreads();
}

// Column-phase spectral update of columns c0 .. c0+CB-1 held in buf (after the forward column FFT), over
// the mode pairs (j, H - j) of each column (j = 0 pairs ky = 0 with ky = H/2), then a CTA barrier:
//   mode 0: sampler s-draw s_hat = f t_hat + g zeta with the (f/n, g/sqrt(2n)) table and Philox counter
//           (column pair group col H/2 + j, step, chain, stream 1; edge column shared as in the on-chip kernel);
//   mode 1: Wiener-filter update s_hat = P/(P + lambda tau) t_hat / n; with cmp, returns this CTA's part of
//           sum_k |s_hat - prev|^2 ((P + lambda tau)/(lambda tau))^2 (the residual from consecutive
//           iterates); with store, keeps s_hat in prev;
//   mode 2: returns sum_k P^2 |t_hat|^2 of the level right-hand side (buf unchanged).
template <int N>
__device__ __forceinline__ double col_update(int mode, float2* buf, int c0, const float2* __restrict__ fg,
                                             const float* __restrict__ Pk, float2* prev, uint32_t step,
                                             uint32_t chain, uint32_t key0, uint32_t key1, float ltau, bool cmp,
                                             bool store) {
  using G = GGeo<N>;
  constexpr int L = G::LR, H = G::H, WH = G::WH;
  constexpr float INV_N = 1.0f / float(G::H * G::W);
  float acc = 0.0f;  // this thread's tasks in FP32; the CTA and grid sums are FP64
  // mode pairs (j, H - j) of each column, j in [0, H/2); j = 0 pairs ky = 0 with ky = H/2
  for (int task = threadIdx.x; task < G::CB * (H / 2); task += 128) {
    const int jc = task / (H / 2), j = task % (H / 2);
    const int col = c0 + jc;
    const int ky1 = j, ky2 = j == 0 ? H / 2 : H - j;
    float2* v = buf + jc * G::VCOL;
    float2 y1 = v[padi(ky1)], y2 = v[padi(ky2)];
    if (mode == 0) {
      float z[4];
      normals4(uint32_t(col * (H / 2) + j), step, chain, 1u, key0, key1, z);
      if (col != 0) {
        const float2 m1 = __ldg(fg + ky1 * WH + col), m2 = __ldg(fg + ky2 * WH + col);
        y1 = make_float2(fmaf(m1.x, y1.x, m1.y * z[0]), fmaf(m1.x, y1.y, m1.y * z[1]));
        y2 = make_float2(fmaf(m2.x, y2.x, m2.y * z[2]), fmaf(m2.x, y2.y, m2.y * z[3]));
      } else {
        const float2 a1 = __ldg(fg + ky1 * WH), b1 = __ldg(fg + ky1 * WH + G::W / 2);
        if (j == 0) {
          const float2 a2 = __ldg(fg + ky2 * WH), b2 = __ldg(fg + ky2 * WH + G::W / 2);
          constexpr float R2 = 1.41421356237309505f;
          y1 = make_float2(fmaf(a1.x, y1.x, R2 * a1.y * z[0]), fmaf(b1.x, y1.y, R2 * b1.y * z[2]));
          y2 = make_float2(fmaf(a2.x, y2.x, R2 * a2.y * z[1]), fmaf(b2.x, y2.y, R2 * b2.y * z[3]));
        } else {
          const float2 y2c = cconj(y2);
          const float2 A = cscale(cadd(y1, y2c), 0.5f);
          const float2 B = cmul_mi(cscale(csub(y1, y2c), 0.5f));
          const float2 Ap = make_float2(fmaf(a1.x, A.x, a1.y * z[0]), fmaf(a1.x, A.y, a1.y * z[1]));
          const float2 Bp = make_float2(fmaf(b1.x, B.x, b1.y * z[2]), fmaf(b1.x, B.y, b1.y * z[3]));
          y1 = cadd(Ap, cmul_i(Bp));
          y2 = cadd(cconj(Ap), cmul_i(cconj(Bp)));
        }
      }
    } else if (mode == 1) {
      // per-mode residual terms and the thread's partial sum in FP32, CTA and grid sums in FP64 (as
      // s_update_wf_parked)
      const float inv_lt = 1.0f / ltau;
      auto wres = [&](float P, float dre, float dim) -> float {
        const float g = fmaf(P, inv_lt, 1.0f);
        return fmaf(dre, dre, dim * dim) * (g * g);
      };
      if (col != 0) {
        const float P1 = __ldg(Pk + ky1 * WH + col), P2 = __ldg(Pk + ky2 * WH + col);
        const float2 n1 = cscale(y1, wf_fdiv(P1, P1 + ltau) * INV_N), n2 = cscale(y2, wf_fdiv(P2, P2 + ltau) * INV_N);
        if (cmp) {
          const float2 o1 = prev[ky1 * L + col], o2 = prev[ky2 * L + col];
          acc += 2.0f * (wres(P1, n1.x - o1.x, n1.y - o1.y) + wres(P2, n2.x - o2.x, n2.y - o2.y));
        }
        y1 = n1;
        y2 = n2;
      } else {
        const float Pa1 = __ldg(Pk + ky1 * WH), Pb1 = __ldg(Pk + ky1 * WH + G::W / 2);
        const float Pa2 = __ldg(Pk + ky2 * WH), Pb2 = __ldg(Pk + ky2 * WH + G::W / 2);
        const float fa1 = wf_fdiv(Pa1, Pa1 + ltau) * INV_N, fb1 = wf_fdiv(Pb1, Pb1 + ltau) * INV_N;
        const float fa2 = wf_fdiv(Pa2, Pa2 + ltau) * INV_N, fb2 = wf_fdiv(Pb2, Pb2 + ltau) * INV_N;
        if (j == 0) {
          const float2 n1 = make_float2(fa1 * y1.x, fb1 * y1.y), n2 = make_float2(fa2 * y2.x, fb2 * y2.y);
          if (cmp) {
            const float2 o1 = prev[ky1 * L], o2 = prev[ky2 * L];
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
            const float2 o1 = prev[ky1 * L], o2c = cconj(prev[ky2 * L]);
            const float2 oA = cscale(cadd(o1, o2c), 0.5f);
            const float2 oB = cmul_mi(cscale(csub(o1, o2c), 0.5f));
            acc += 2.0f * (wres(Pa1, A.x - oA.x, A.y - oA.y) + wres(Pb1, B.x - oB.x, B.y - oB.y));
          }
          y1 = cadd(A, cmul_i(B));
          y2 = cadd(cconj(A), cmul_i(cconj(B)));
        }
      }
      if (store) {
        prev[ky1 * L + col] = y1;
        prev[ky2 * L + col] = y2;
      }
    } else {
      auto p2 = [](float P, float re, float im) -> float { return P * P * fmaf(re, re, im * im); };
      if (col != 0) {
        acc += 2.0f * (p2(__ldg(Pk + ky1 * WH + col), y1.x, y1.y) + p2(__ldg(Pk + ky2 * WH + col), y2.x, y2.y));
      } else if (j == 0) {
        acc += p2(__ldg(Pk + ky1 * WH), y1.x, 0.f) + p2(__ldg(Pk + ky1 * WH + G::W / 2), y1.y, 0.f) +
               p2(__ldg(Pk + ky2 * WH), y2.x, 0.f) + p2(__ldg(Pk + ky2 * WH + G::W / 2), y2.y, 0.f);
      } else {
        const float2 y2c = cconj(y2);
        const float2 A = cscale(cadd(y1, y2c), 0.5f);
        const float2 B = cmul_mi(cscale(csub(y1, y2c), 0.5f));
        acc += 2.0f * (p2(__ldg(Pk + ky1 * WH), A.x, A.y) + p2(__ldg(Pk + ky1 * WH + G::W / 2), B.x, B.y));
      }
    }
    v[padi(ky1)] = y1;
    v[padi(ky2)] = y2;
  }
  __syncthreads();
  return double(acc);
}

// Column phase on one work item: columns c0 .. c0+CB-1 of field f.
// mode 0: s-draw; mode 1: s_hat = f_lambda t_hat with residual bookkeeping (returns this CTA's partial
// sum when cmp); mode 2: P^2 |V|^2 power of the level right-hand side (no write-back).
template <int N>
__device__ double col_item(const GlobalArgs& a, float2* buf, int f, int c0, int done, float ltau, bool cmp,
                           bool store) {
  using G = GGeo<N>;
  constexpr int L = G::LR, H = G::H;
  float2* Zf = a.Z + (long long)f * H * L;
  for (int e = threadIdx.x; e < G::CB * H; e += 128) {
    const int j = e % G::CB, y = e / G::CB;  // consecutive threads: consecutive columns of a row
    buf[j * G::VCOL + padi(y)] = __ldcg(Zf + (long long)y * L + c0 + j);
  }
  __syncthreads();
  fft_smem<G::RC, G::CB, G::VCOL, false, G::SC>(buf, a.tw_col);
  const double acc = col_update<N>(a.mode, buf, c0, a.fg, a.Pk, a.prev, a.step0 + uint32_t(done),
                                   a.chain0 + uint32_t(f), a.key0, a.key1, ltau, cmp, store);
  if (a.mode == 2) return acc;
  fft_smem<G::RC, G::CB, G::VCOL, true, G::SC>(buf, a.tw_col);
  for (int e = threadIdx.x; e < G::CB * H; e += 128) {
    const int j = e % G::CB, y = e / G::CB;
    __stcg(Zf + (long long)y * L + c0 + j, buf[j * G::VCOL + padi(y)]);
  }
  __syncthreads();
  return acc;
}

// mode 3: weighted power sums of CB columns of field f into acc[j], j < nw
template <int N>
__device__ void col_wpower(const GlobalArgs& a, float2* buf, int f, int c0, double (&acc)[4]) {
  using G = GGeo<N>;
  constexpr int L = G::LR, H = G::H, WH = G::WH, TS = G::H * G::WH;
  const float2* Zf = a.Z + (long long)f * H * L;
  for (int e = threadIdx.x; e < G::CB * H; e += 128) {
    const int j = e % G::CB, y = e / G::CB;
    buf[j * G::VCOL + padi(y)] = __ldcg(Zf + (long long)y * L + c0 + j);
  }
  __syncthreads();
  fft_smem<G::RC, G::CB, G::VCOL, false, G::SC>(buf, a.tw_col);
  auto sq = [](float p, float q) -> double { return double(p) * p + double(q) * q; };
  for (int task = threadIdx.x; task < G::CB * (H / 2); task += 128) {
    const int jc = task / (H / 2), j = task % (H / 2);
    const int col = c0 + jc;
    const int ky1 = j, ky2 = j == 0 ? H / 2 : H - j;
    const float2* v = buf + jc * G::VCOL;
    const float2 y1 = v[padi(ky1)], y2 = v[padi(ky2)];
    for (int t = 0; t < a.nw; ++t) {
      const float* wt = a.wts + t * TS;
      double s;
      if (col != 0) {
        s = 2.0 * (__ldg(wt + ky1 * WH + col) * sq(y1.x, y1.y) + __ldg(wt + ky2 * WH + col) * sq(y2.x, y2.y));
      } else if (j == 0) {
        s = __ldg(wt + ky1 * WH) * sq(y1.x, 0.f) + __ldg(wt + ky1 * WH + G::W / 2) * sq(y1.y, 0.f) +
            __ldg(wt + ky2 * WH) * sq(y2.x, 0.f) + __ldg(wt + ky2 * WH + G::W / 2) * sq(y2.y, 0.f);
      } else {
        const float2 y2c = cconj(y2);
        const float2 A = cscale(cadd(y1, y2c), 0.5f);
        const float2 B = cmul_mi(cscale(csub(y1, y2c), 0.5f));
        s = 2.0 * (__ldg(wt + ky1 * WH) * sq(A.x, A.y) + __ldg(wt + ky1 * WH + G::W / 2) * sq(B.x, B.y));
      }
      acc[t] += s;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ double block_sum_128(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  const double s = red[0] + red[1] + red[2] + red[3];
  __syncthreads();
  return s;
}

template <int N>
__global__ void __launch_bounds__(128, 3) k_global(GlobalArgs a) {
  using G = GGeo<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);
  __shared__ double red[4];
  const Scalars sc = *a.sc;
  if (sc.status != 0) {
    if (a.mode == 1 && blockIdx.x == 0 && threadIdx.x == 0) a.st->status = sc.status;
    return;
  }
  const unsigned int nb = gridDim.x;
  const int row_items = G::ROW_ITEMS * a.n_fields, col_items = G::COL_ITEMS * a.n_fields;

  auto rows = [&](int done, bool first, bool emit_only, float ltau) {
    for (int it = blockIdx.x; it < row_items; it += nb) {
      const int f = it / G::ROW_ITEMS;
      if (a.mode == 2 && f >= sc.n_levels) continue;  // level fields past the schedule
      row_item<N>(a, buf, f, (it % G::ROW_ITEMS) * G::RB, done, first, emit_only, ltau, sc);
    }
  };
  auto cols = [&](int done, float ltau, bool cmp, bool store) -> double {
    double acc = 0.0;
    for (int it = blockIdx.x; it < col_items; it += nb)
      acc += col_item<N>(a, buf, it / G::COL_ITEMS, (it % G::COL_ITEMS) * G::CB, done, ltau, cmp, store);
    return acc;
  };

  if (a.mode == 0) {
    rows(0, true, false, 0.f);
    for (int i = 0; i < a.n_sweeps; ++i) {
      if (!grid_barrier(a.bar, nb)) return;
      cols(i, 0.f, false, false);
      if (!grid_barrier(a.bar, nb)) return;
      rows(i + 1, false, i + 1 == a.n_sweeps, 0.f);
    }
    return;
  }
  if (a.mode == 3) {  // weighted power of given fields
    rows(0, true, false, 0.f);
    if (!grid_barrier(a.bar, nb)) return;
    for (int it = blockIdx.x; it < col_items; it += nb) {
      const int f = it / G::COL_ITEMS;
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      col_wpower<N>(a, buf, f, (it % G::COL_ITEMS) * G::CB, acc);
      for (int t = 0; t < a.nw; ++t) {
        const double s = block_sum_128(acc[t], red);
        if (threadIdx.x == 0) atomicAdd(a.wout + f * a.nw + t, s / double(G::H * G::W));
      }
    }
    return;
  }
  if (a.mode == 2) {  // level norms, fields = levels
    rows(0, true, false, 0.f);
    if (!grid_barrier(a.bar, nb)) return;
    for (int it = blockIdx.x; it < col_items; it += nb) {
      const int f = it / G::COL_ITEMS;
      if (f >= sc.n_levels) continue;
      const double s = block_sum_128(col_item<N>(a, buf, f, (it % G::COL_ITEMS) * G::CB, 0, 0.f, false, false), red);
      if (threadIdx.x == 0) atomicAdd(a.bnorm_out + f, s / double(G::H * G::W));
    }
    return;
  }
  // Wiener filter with lambda-cooling, one field; every CTA follows the same schedule
  const double tau = sc.tau;
  int lev = 0;
  double lam = sc.lam0;
  float ltau = float(lam * tau);
  const int last_level = sc.n_levels - 1;
  int it = 0, k = 0, status = 1, parity = 0;
  double rho = -1.0;
  rows(0, true, false, ltau);
  while (true) {
    ++k;
    ++it;
    const bool cmp = (k % a.check == 0) && k >= 2;
    const bool store = ((k + 1) % a.check == 0);
    if (!grid_barrier(a.bar, nb)) return;
    const double part = block_sum_128(cols(it, ltau, cmp, store), red);
    if (cmp && threadIdx.x == 0) atomicAdd(a.acc + parity, part);
    if (!grid_barrier(a.bar, nb)) return;
    if (cmp) {
      const double tot = __ldcg(a.acc + parity) * double(G::H * G::W);
      if (blockIdx.x == 0 && threadIdx.x == 0) a.acc[parity ^ 1] = 0.0;  // next check's accumulator
      parity ^= 1;
      const double bn = a.bnorm2[lev];
      const double r2 = bn > 0.0 ? tot / bn : tot;
      rho = sqrt(r2);
      if (!(r2 == r2) || r2 > 1e300) {
        status = 6;
      } else if (lev < last_level) {
        if (rho < a.level_tol || k >= a.level_max) {
          ++lev;
          lam = level_lambda(sc, lev, a.eta);
          ltau = float(lam * tau);
          k = 0;
        }
      } else if (rho < a.tol) {
        status = 0;
      }
    }
    if (status == 1 && it >= a.max_iter) status = 5;
    rows(it, false, status != 1, ltau);
    if (status != 1) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.st->status = status;
    a.st->iters = it;
    a.st->resid = rho;
  }
}

}  // namespace wf
