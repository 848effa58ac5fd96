// Batched persistent form: many independent images (one Wiener-filter solve to tol, then posterior
// samples from s_W, per image). Images up to 128 x 128 go through k_batch<N>: a persistent kernel whose
// CTAs (N threads, one field in shared memory) take images from an atomic work counter and run the whole
// pipeline for each on chip: input checks and tau, coefficient tables, per-level norms, the cooled
// G -> 0 iteration (§2.2) and the Alg. 1 sweeps.
#pragma once

#include "wf_gibbs.cuh"

namespace wf {

struct BatchItem {
  const float* d;
  const float* Ndiag;
  const uint8_t* mask;
  const float* Pk;
  float* out_wf;       // [H][W] or nullptr
  float* out_samples;  // [n_samples][H][W] or nullptr
  unsigned long long seed;
  unsigned int chain;
  int H;
};

struct BatchResult {
  double resid;
  int iters;
  int status;
};

struct BatchArgs {
  const BatchItem* items;
  const int* order;  // item indices of this size class
  int n;             // items in this class
  BatchResult* res;  // indexed by item
  int* queue;        // work counter, starts at 0
  char* scratch;     // per-CTA tables, slot_bytes each
  long long slot_bytes;
  double tau;        // <= 0: each image's minimum observed Ndiag
  double tol, eta, level_tol;
  int max_iter, level_max, check;
  int n_samples;
  int grid_pct;      // host side: percent of the occupancy-limited persistent grid (0 or >= 100: all)
};

template <int N>
constexpr long long batch_slot_bytes() {
  // aq, dn [N*N] + fg [N*(N/2+1)] + prev [N*N/2], float2 each, 256-byte aligned pieces
  return ((long long)N * N * 8 + 255) / 256 * 256 * 2 + ((long long)N * (N / 2 + 1) * 8 + 255) / 256 * 256 +
         ((long long)N * (N / 2) * 8 + 255) / 256 * 256;
}
template <int N>
constexpr int batch_smem_bytes() { return Geo<N>::FIELD_BYTES + (33 + kMaxLevels) * 8 + 8 * 4; }

template <int N>
__global__ void __launch_bounds__(N, N >= 128 ? 3 : 4) k_batch(BatchArgs b) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* S = reinterpret_cast<float2*>(smem_raw);
  double* red = reinterpret_cast<double*>(smem_raw + G::FIELD_BYTES);
  double* bn = red + 33;
  int* si = reinterpret_cast<int*>(bn + kMaxLevels);
  const int lt = threadIdx.x;
  constexpr int n = N * N, nm = N * (N / 2 + 1);
  char* slot = b.scratch + (long long)blockIdx.x * b.slot_bytes;
  float2* aq = reinterpret_cast<float2*>(slot);
  float2* dn = reinterpret_cast<float2*>(slot + ((long long)n * 8 + 255) / 256 * 256);
  float2* fg = reinterpret_cast<float2*>(slot + ((long long)n * 8 + 255) / 256 * 256 * 2);
  float2* prev = reinterpret_cast<float2*>(slot + ((long long)n * 8 + 255) / 256 * 256 * 2 +
                                           ((long long)nm * 8 + 255) / 256 * 256);
  while (true) {
    if (lt == 0) si[0] = atomicAdd(b.queue, 1);
    __syncthreads();
    const int q = si[0];
    __syncthreads();
    if (q >= b.n) break;
    const int idx = b.order[q];
    const BatchItem it = b.items[idx];

    // input checks, tau, max P (Alg. 1 definitions), as in the single-image set-up
    if (lt == 0) {
      si[1] = 0x7f800000;  // +inf bits: min over positive floats by integer order
      si[2] = 0;
      si[3] = 0;
      si[4] = 0;
      si[5] = 0;
    }
    __syncthreads();
    {
      float vmin = wf_inf(), vmax = 0.0f;
      int nobs = 0, bad = 0, neg = 0;
      for (int i = lt; i < n; i += N) {
        if (it.mask[i] == 0) {
          const float nv = it.Ndiag[i], dv = it.d[i];
          ++nobs;
          if (!isfinite(nv) || !isfinite(dv)) bad = 1;
          else if (!(nv > 0.0f)) neg = 1;
          else vmin = fminf(vmin, nv);
        }
      }
      for (int i = lt; i < nm; i += N) {
        const float pv = it.Pk[i];
        if (!isfinite(pv)) bad = 1;
        else if (pv < 0.0f) neg = 1;
        else vmax = fmaxf(vmax, pv);
      }
      atomicMin(si + 1, __float_as_int(vmin));
      atomicMax(si + 2, __float_as_int(vmax));
      atomicAdd(si + 3, nobs);
      atomicOr(si + 4, bad);
      atomicOr(si + 5, neg);
    }
    __syncthreads();
    const Scalars sc = make_scalars(__int_as_float(si[1]), si[3], __int_as_float(si[2]), si[4], si[5], b.tau, b.eta);
    __syncthreads();
    if (sc.status != 0) {
      if (lt == 0) b.res[idx] = BatchResult{-1.0, 0, sc.status};
      continue;
    }
    const double inv_n = 1.0 / double(n);
    for (int i = lt; i < n; i += N) {
      const int y = i / N, x = i % N;
      float2 a2, d2;
      table_pixel(it.d[i], it.Ndiag[i], it.mask[i] == 0, sc.tau, &a2, &d2);
      aq[x * N + y] = a2;
      dn[x * N + y] = d2;
    }
    for (int j = lt; j < nm; j += N) fg[j] = table_mode(it.Pk[j], sc.tau, inv_n);
    __syncthreads();
    for (int lev = 0; lev < sc.n_levels; ++lev) {
      const double v = level_norm<N>(S, red, lt, dn, it.Pk, float(level_lambda(sc, lev, b.eta) * sc.tau));
      if (lt == 0) bn[lev] = v;
      __syncthreads();
    }
    float2 c[G::LR];
#pragma unroll
    for (int m = 0; m < G::LR; ++m) c[m] = make_float2(0.f, 0.f);
    int iters = 0;
    double rho = -1.0;
    const int status = solve_sweeps<N>(S, red, lt, c, dn, it.Pk, sc, bn, prev, b.tol, b.eta, b.level_tol,
                                       b.max_iter, b.level_max, b.check, iters, rho);
    if (it.out_wf != nullptr) {
      float* stg = reinterpret_cast<float*>(S);
      stage_row<N>(stg, lt, c);
      __syncthreads();
      copy_out<N>(stg, lt, it.out_wf);
    }
    __syncthreads();
    if (b.n_samples > 0 && it.out_samples != nullptr)
      sample_sweeps<N>(S, lt, c, aq, TableCoef{fg, G::WH}, sc.sqrt_tau, 0u, it.chain, uint32_t(it.seed & 0xffffffffu),
                       uint32_t(it.seed >> 32), b.n_samples, 0, 1, it.out_samples, true);
    if (lt == 0) b.res[idx] = BatchResult{rho, iters, status};
    __syncthreads();
  }
}

}  // namespace wf
