// Cluster-resident sampler for 256 x 256 and 512 x 512 images (Alg. 1 of the paper with A = I).
//
// A 256^2 field's packed half spectrum (256 KB) does not fit one SM, but it fits the distributed shared
// memory of a thread-block cluster. One field (one chain) is a cluster of P = N / 64 CTAs of N / 2 threads;
// CTA b keeps the global rows y = P a + b (a < 64), each row as N / 2 float2 slots, for all sweeps.
//
// Row transforms (length L = N / 2 complex, real-to-complex packing) stay inside a CTA: the R = L / 64
// threads of a row (neighbouring lanes of one warp) each run a 64-point register FFT over every R-th slot,
// then radix-R butterflies across them, with the real-transform pre/post pass of the mode pairs
// (K, L - K) fused into the butterflies. The half spectrum of a row is kept in digit-reversed slot
// order, X[K] at slot R (K mod 64) + K / 64, which the column pass simply follows.
//
// Column transforms (length N) are split over the cluster by decimation in time over the CTA rank:
// each CTA runs a 64-point register FFT down every column of its rows (twiddled by W_N^(b k')), then one
// radix-P stage combines the P partial transforms through distributed shared memory; the s-draw happens
// right there, on the complete column spectrum, followed by the inverse radix-P stage, the inverse twiddle
// and the local inverse FFTs. Two cluster barriers per sweep (hardware barriers, no spin waits).
// Draws follow the Philox counter layout of the on-chip sampler, so the chain is the same Markov chain
// draw for draw.
#pragma once

#include <cooperative_groups.h>

#include "wf_gbatch.cuh"

namespace wf {

template <int N_>
struct CGeo {
  static constexpr int N = N_, H = N_, W = N_;
  static constexpr int P = N / 64;   // CTAs per cluster
  static constexpr int A = 64;       // rows per CTA
  static constexpr int L = N / 2;    // complex length of a row transform = threads per CTA
  static constexpr int R = L / 64;   // threads per row in the row passes
  static constexpr int SP = L + R;   // float2 stride of a row: a half-warp's R-strided loads hit distinct banks
  static constexpr int ROWS_BYTES = A * SP * 8;
  static constexpr int SMEM = ROWS_BYTES + N * 8;  // rows, then the twiddles exp(-2 pi i j / N)
  static constexpr int WH = W / 2 + 1;
};

// ---------------------------------------------------------------------------------------------
// row passes (R threads per row, h = the thread's index within its row)
// ---------------------------------------------------------------------------------------------
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
template <int N>
__device__ __forceinline__ void crow_fwd(float2* row, int h, const float2* tw) {
  using G = CGeo<N>;
  constexpr int R = G::R;
  {
    float2 x[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) x[i] = row[R * i + h];
    fft<64, false>(x);
#pragma unroll
    for (int k = 0; k < 64; ++k) row[R * k + h] = k == 0 ? x[0] : cmul(x[k], tw[2 * h * k]);  // W_L^(h k)
  }
  __syncwarp();
  for (int u = h; u <= 32; u += R) {  // butterfly unit k' = u with its mirror v = 64 - u
    const int v = 64 - u;
    const bool two = u != 0 && u != 32;
    float2 p[R], q[R];
#pragma unroll
    for (int j = 0; j < R; ++j) p[j] = row[R * u + j];
    fft<R, false>(p);  // p[m] = C[u + 64 m]
    if (two) {
#pragma unroll
      for (int j = 0; j < R; ++j) q[j] = row[R * v + j];
      fft<R, false>(q);  // q[m] = C[v + 64 m]
    }
    if (u == 0) {
      p[0] = make_float2(p[0].x + p[0].y, p[0].x - p[0].y);  // (R[0], R[L])
#pragma unroll
      for (int m = 1; m < R; ++m) {
        if (2 * m == R) p[m] = cconj(p[m]);
        else if (m < R - m) c_r2c_pair(p[m], p[R - m], tw[64 * m]);
      }
    } else if (u == 32) {
#pragma unroll
      for (int m = 0; m < R / 2; ++m) c_r2c_pair(p[m], p[R - 1 - m], tw[32 + 64 * m]);
    } else {
#pragma unroll
      for (int m = 0; m < R; ++m) c_r2c_pair(p[m], q[R - 1 - m], tw[u + 64 * m]);
    }
#pragma unroll
    for (int m = 0; m < R; ++m) row[R * u + m] = p[m];
    if (two) {
#pragma unroll
      for (int m = 0; m < R; ++m) row[R * v + m] = q[m];
    }
  }
}

// inverse: packed half spectrum (digit-reversed slots) -> real row in natural slots (unnormalised)
template <int N>
__device__ __forceinline__ void crow_inv(float2* row, int h, const float2* tw) {
  using G = CGeo<N>;
  constexpr int R = G::R;
  for (int u = h; u <= 32; u += R) {
    const int v = 64 - u;
    const bool two = u != 0 && u != 32;
    float2 p[R], q[R];
#pragma unroll
    for (int m = 0; m < R; ++m) p[m] = row[R * u + m];
    if (two) {
#pragma unroll
      for (int m = 0; m < R; ++m) q[m] = row[R * v + m];
    }
    if (u == 0) {
      p[0] = make_float2(p[0].x + p[0].y, p[0].x - p[0].y);
#pragma unroll
      for (int m = 1; m < R; ++m) {
        if (2 * m == R) p[m] = cscale(cconj(p[m]), 2.0f);
        else if (m < R - m) c_c2r_pair(p[m], p[R - m], tw[64 * m]);
      }
    } else if (u == 32) {
#pragma unroll
      for (int m = 0; m < R / 2; ++m) c_c2r_pair(p[m], p[R - 1 - m], tw[32 + 64 * m]);
    } else {
#pragma unroll
      for (int m = 0; m < R; ++m) c_c2r_pair(p[m], q[R - 1 - m], tw[u + 64 * m]);
    }
    fft<R, true>(p);  // p[j] = sum_m exp(+2 pi i j m / R) C'[u + 64 m]
#pragma unroll
    for (int j = 0; j < R; ++j) row[R * u + j] = j == 0 ? p[0] : cmul(p[j], cconj(tw[2 * j * u]));
    if (two) {
      fft<R, true>(q);
#pragma unroll
      for (int j = 0; j < R; ++j) row[R * v + j] = j == 0 ? q[0] : cmul(q[j], cconj(tw[2 * j * v]));
    }
  }
  __syncwarp();
  float2 x[64];
#pragma unroll
  for (int k = 0; k < 64; ++k) x[k] = row[R * k + h];
  fft<64, true>(x);
#pragma unroll
  for (int i = 0; i < 64; ++i) row[R * i + h] = x[i];
}

// t-draw of global row y on its staged row: t = a + q (q s + sqrt(tau) xi), table aq[x*H + y] =
// ((1 - w) d, sqrt(w)); Philox stream 0, group y*W/4 + q feeds pixels 4q .. 4q+3 (q = h, h + R, ...)
template <int N>
__device__ __forceinline__ void ct_draw(float2* row, int y, int h, const float2* __restrict__ aq, float sqrt_tau,
                                        uint32_t step, uint32_t chain, uint32_t k0, uint32_t k1) {
  using G = CGeo<N>;
#pragma unroll 2
  for (int q = h; q < G::W / 4; q += G::R) {
    float z[4];
    normals4(uint32_t(y * (G::W / 4) + q), step, chain, 0u, k0, k1, z);
    float2 p0 = row[2 * q], p1 = row[2 * q + 1];
    const float2 c0 = WF_LDG(aq + (4 * q) * G::H + y), c1 = WF_LDG(aq + (4 * q + 1) * G::H + y);
    const float2 c2 = WF_LDG(aq + (4 * q + 2) * G::H + y), c3 = WF_LDG(aq + (4 * q + 3) * G::H + y);
    p0.x = fmaf(c0.y, fmaf(c0.y, p0.x, sqrt_tau * z[0]), c0.x);
    p0.y = fmaf(c1.y, fmaf(c1.y, p0.y, sqrt_tau * z[1]), c1.x);
    p1.x = fmaf(c2.y, fmaf(c2.y, p1.x, sqrt_tau * z[2]), c2.x);
    p1.y = fmaf(c3.y, fmaf(c3.y, p1.y, sqrt_tau * z[3]), c3.x);
    row[2 * q] = p0;
    row[2 * q + 1] = p1;
  }
}

// ---------------------------------------------------------------------------------------------
// column passes
// ---------------------------------------------------------------------------------------------
// local forward: 64-point FFT down slot t of this CTA's rows, output k' twiddled by W_N^(b k')
template <int N>
__device__ __forceinline__ void ccol_fwd(float2* rows, int t, int b, const float2* tw) {
  using G = CGeo<N>;
  float2 x[64];
#pragma unroll
  for (int a = 0; a < 64; ++a) x[a] = rows[a * G::SP + t];
  fft<64, false>(x);
#pragma unroll
  for (int k = 0; k < 64; ++k) rows[k * G::SP + t] = k == 0 ? x[0] : cmul(x[k], tw[b * k]);
}
// local inverse: untwiddle by W_N^(-b k'), inverse 64-point FFT back to the rows
template <int N>
__device__ __forceinline__ void ccol_inv(float2* rows, int t, int b, const float2* tw) {
  using G = CGeo<N>;
  float2 x[64];
#pragma unroll
  for (int k = 0; k < 64; ++k) {
    const float2 v = rows[k * G::SP + t];
    x[k] = k == 0 ? v : cmul(v, cconj(tw[b * k]));
  }
  fft<64, true>(x);
#pragma unroll
  for (int a = 0; a < 64; ++a) rows[a * G::SP + t] = x[a];
}

// One mode pair (ky1, ky2 = N - ky1, or N/2 when ky1 = 0) of packed column slot t (kx = K) with the
// s-draw s_hat = f t_hat + g zeta, table fg[ky*WH + kx] = (f / n, g / sqrt(2 n)). Interior columns: Philox
// stream 1 group K*H/2 + ky1, variates 0, 1 for ky1 and 2, 3 for ky2. Packed edge column (K = 0: kx = 0 as
// A and kx = W/2 as B in Y = A + i B): group ky1 draws (ky1, 0) from variates 0, 1 and (ky1, W/2) from
// 2, 3, the conjugates filling ky2; group 0 holds the four real modes (0,0), (H/2,0), (0,W/2), (H/2,W/2).
template <int N>
__device__ __forceinline__ void cdraw_pair(float2& y1, float2& y2, int K, int ky1, int ky2,
                                           const float2* __restrict__ fg, uint32_t step, uint32_t chain,
                                           uint32_t k0, uint32_t k1) {
  using G = CGeo<N>;
  float z[4];
  normals4(uint32_t(K * (G::H / 2) + ky1), step, chain, 1u, k0, k1, z);
  if (K != 0) {
    const float2 m1 = WF_LDG(fg + ky1 * G::WH + K), m2 = WF_LDG(fg + ky2 * G::WH + K);
    y1 = make_float2(fmaf(m1.x, y1.x, m1.y * z[0]), fmaf(m1.x, y1.y, m1.y * z[1]));
    y2 = make_float2(fmaf(m2.x, y2.x, m2.y * z[2]), fmaf(m2.x, y2.y, m2.y * z[3]));
    return;
  }
  const float2 a1 = WF_LDG(fg + ky1 * G::WH), b1 = WF_LDG(fg + ky1 * G::WH + G::W / 2);
  if (ky1 == 0) {
    const float2 a2 = WF_LDG(fg + ky2 * G::WH), b2 = WF_LDG(fg + ky2 * G::WH + G::W / 2);
    constexpr float R2 = 1.41421356237309505f;
    y1 = make_float2(fmaf(a1.x, y1.x, R2 * a1.y * z[0]), fmaf(b1.x, y1.y, R2 * b1.y * z[2]));
    y2 = make_float2(fmaf(a2.x, y2.x, R2 * a2.y * z[1]), fmaf(b2.x, y2.y, R2 * b2.y * z[3]));
  } else {
    const float2 y2c = cconj(y2);
    const float2 Am = cscale(cadd(y1, y2c), 0.5f);
    const float2 Bm = cmul_mi(cscale(csub(y1, y2c), 0.5f));
    const float2 Ap = make_float2(fmaf(a1.x, Am.x, a1.y * z[0]), fmaf(a1.x, Am.y, a1.y * z[1]));
    const float2 Bp = make_float2(fmaf(b1.x, Bm.x, b1.y * z[2]), fmaf(b1.x, Bm.y, b1.y * z[3]));
    y1 = cadd(Ap, cmul_i(Bp));
    y2 = cadd(cconj(Ap), cmul_i(cconj(Bp)));
  }
}

// cross-cluster radix-P stage with the s-draw. Work unit (slot t, k' = u with its mirror v = 64 - u):
// gathers Y_j[u] (and Y_j[v]) from every CTA j, forms the column spectrum t_hat[u + 64 m], draws, and
// scatters the inverse stage back. g = the thread's index in the cluster.
template <int N>
__device__ __forceinline__ void ccol_draw(cooperative_groups::cluster_group& cl, float2* rows, int g,
                                          const float2* __restrict__ fg, uint32_t step, uint32_t chain,
                                          uint32_t k0, uint32_t k1) {
  using G = CGeo<N>;
  constexpr int P = G::P, L = G::L, R = G::R;
  for (int w = g; w < L * 33; w += P * L) {
    const int t = w % L, u = w / L, v = 64 - u;
    const int K = (t % R) * 64 + t / R;  // kx held by slot t
    const bool two = u != 0 && u != 32;
    float2 p[P], q[P];
#pragma unroll
    for (int j = 0; j < P; ++j) p[j] = cl.map_shared_rank(rows, j)[u * G::SP + t];
    if (two) {
#pragma unroll
      for (int j = 0; j < P; ++j) q[j] = cl.map_shared_rank(rows, j)[v * G::SP + t];
    }
    fft<P, false>(p);  // p[m] = t_hat[u + 64 m]
    if (u == 0) {
      cdraw_pair<N>(p[0], p[P / 2], K, 0, N / 2, fg, step, chain, k0, k1);
#pragma unroll
      for (int m = 1; m < P / 2; ++m) cdraw_pair<N>(p[m], p[P - m], K, 64 * m, N - 64 * m, fg, step, chain, k0, k1);
    } else if (u == 32) {
#pragma unroll
      for (int m = 0; m < P / 2; ++m)
        cdraw_pair<N>(p[m], p[P - 1 - m], K, 32 + 64 * m, N - 32 - 64 * m, fg, step, chain, k0, k1);
    } else {
      fft<P, false>(q);  // q[m] = t_hat[v + 64 m]
#pragma unroll
      for (int m = 0; m < P / 2; ++m) {
        cdraw_pair<N>(p[m], q[P - 1 - m], K, u + 64 * m, N - u - 64 * m, fg, step, chain, k0, k1);
        cdraw_pair<N>(q[m], p[P - 1 - m], K, v + 64 * m, N - v - 64 * m, fg, step, chain, k0, k1);
      }
      fft<P, true>(q);
#pragma unroll
      for (int j = 0; j < P; ++j) cl.map_shared_rank(rows, j)[v * G::SP + t] = q[j];
    }
    fft<P, true>(p);
#pragma unroll
    for (int j = 0; j < P; ++j) cl.map_shared_rank(rows, j)[u * G::SP + t] = p[j];
  }
}

// ---------------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------------
template <int N>
constexpr int csample_min_ctas() { return N == 256 ? 3 : 1; }

// the sweeps of one chain by its cluster: s_0 from init (row-major [H][W], nullptr: zero), sample m (the
// state after sweep burn_in + (m + 1) thin) to out + m H W elements of type out_dtype
template <int N>
__device__ __forceinline__ void csample_chain(cooperative_groups::cluster_group& cl, unsigned char* smem_raw,
                                              const float2* __restrict__ aq, const float2* __restrict__ fg,
                                              float sqrt_tau, const float* init, void* out_v, int out_dtype,
                                              int n_sweeps, int burn_in, int thin, uint32_t step0, uint32_t chain,
                                              uint32_t k0, uint32_t k1) {
  using G = CGeo<N>;
  float2* rows = reinterpret_cast<float2*>(smem_raw);
  float2* tw = reinterpret_cast<float2*>(smem_raw + G::ROWS_BYTES);
  const int tid = threadIdx.x, b = int(cl.block_rank());
  for (int j = tid; j < N; j += G::L) {  // exp(-2 pi i j / N), FP64 then rounded once
    double sn, cs;
    sincospi(-2.0 * double(j) / double(N), &sn, &cs);
    tw[j] = make_float2(float(cs), float(sn));
  }
  for (int e = tid; e < G::A * G::L; e += G::L) {
    const int ar = e / G::L, i = e % G::L;
    float2 v = make_float2(0.f, 0.f);
    if (init != nullptr) v = WF_LDG(reinterpret_cast<const float2*>(init + (long long)(G::P * ar + b) * G::W) + i);
    rows[ar * G::SP + i] = v;
  }
  __syncthreads();
  const int ar = tid / G::R, h = tid % G::R, y = G::P * ar + b;
  float2* row = rows + ar * G::SP;
  const int eb = out_elem_bytes(out_dtype);
  char* out = reinterpret_cast<char*>(out_v);
  for (int done = 0;;) {
    const uint32_t step = step0 + uint32_t(done);
    ct_draw<N>(row, y, h, aq, sqrt_tau, step, chain, k0, k1);
    __syncwarp();
    crow_fwd<N>(row, h, tw);
    __syncthreads();
    ccol_fwd<N>(rows, tid, b, tw);
    cl.sync();  // every CTA's partial column transforms are in place
    ccol_draw<N>(cl, rows, b * G::L + tid, fg, step, chain, k0, k1);
    cl.sync();  // every unit's inverse stage has landed
    ccol_inv<N>(rows, tid, b, tw);
    __syncthreads();
    crow_inv<N>(row, h, tw);
    ++done;
    if (done > burn_in && (done - burn_in) % thin == 0) {
      const long long m = (done - burn_in) / thin - 1;
      __syncthreads();
      char* dst = out + m * (long long)(G::H * G::W) * eb;
      for (int e = tid; e < G::A * G::L; e += G::L) {
        const int r2 = e / G::L, i = e % G::L;
        store_pair(dst, (long long)(G::P * r2 + b) * G::L + i, rows[r2 * G::SP + i], out_dtype);
      }
      __syncthreads();
    }
    if (done == n_sweeps) break;
    __syncwarp();
  }
  cl.sync();  // no CTA leaves while another may still address its shared memory
}

// one problem, grid = n_chains clusters of P CTAs (chain = cluster index)
template <int N>
__global__ void __launch_bounds__(N / 2, csample_min_ctas<N>()) k_csample(SampleArgs a) {
  using G = CGeo<N>;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (a.sc->status != 0) return;  // uniform over the grid
  const long long ci = blockIdx.x / G::P;
  const int eb = out_elem_bytes(a.out_dtype);
  csample_chain<N>(cl, smem_raw, a.aq, a.fg, a.sc->sqrt_tau, a.init_s ? a.init_s + ci * a.init_stride : nullptr,
                   reinterpret_cast<char*>(a.out) + ci * a.n_samples * (long long)(G::H * G::W) * eb, a.out_dtype,
                   a.n_sweeps, a.burn_in, a.thin, a.step0, a.chain0 + uint32_t(ci), a.key0, a.key1);
}

// the sampling phase of a batch of large images (one cluster per image, after the Wiener solve): image f
// samples n_samples sweeps from its s_W (fields[f].out_wf) with step words 0, 1, ... and its own chain and
// key, into fields[f].out_samples; images whose set-up failed are skipped
struct CBArgs {
  const GBField* fields;
  const Scalars* sc;
  int F;
  int n_samples;
};
template <int N>
__global__ void __launch_bounds__(N / 2, csample_min_ctas<N>()) k_csample_batch(CBArgs a) {
  using G = CGeo<N>;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int f = blockIdx.x / G::P;
  const GBField fd = a.fields[f];
  const Scalars sc = a.sc[f];
  if (sc.status != 0 || fd.out_samples == nullptr || fd.out_wf == nullptr) return;  // uniform over the cluster
  csample_chain<N>(cl, smem_raw, fd.aq, fd.fg, sc.sqrt_tau, fd.out_wf, fd.out_samples, kOutF32, a.n_samples, 0, 1,
                   0u, fd.chain, fd.key0, fd.key1);
}

}  // namespace wf
