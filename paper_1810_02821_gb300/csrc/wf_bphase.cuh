// Batched form for images up to 128 x 128, in phases: the images of a size class go through a few
// launches instead of one persistent kernel that runs the whole pipeline per image:
//   set-up    per-image tau, lambda_0 and checks, then every image's coefficient tables (wf_api.cu);
//   k_blevels a few CTAs per image: the level norms ||S N_lambda^-1 d||^2 of its cooling levels;
//   k_bsolve  one CTA per image, images with more cooling levels (longer solves) first, so that the
//             long solves do not start last: the lambda-cooled G -> 0 iteration (§2.2), s_W to the
//             image's output (or scratch), status / sweeps / residual to the batch results;
//   k_bsample fields of several images per CTA (as the single-image sampler): n_samples sweeps of
//             Alg. 1 from s_W, each image with its own tables, chain and key.
// Each kernel holds one stage's code only (the fused kernel's instruction footprint stalled its warps on
// instruction fetch), the block scheduler balances the unequal solves, and the sampler packs as many
// fields per SM as the single-image sampler does.
#pragma once

#include "wf_gbatch.cuh"

namespace wf {

struct BSolveArgs {
  const GBField* fields;  // [F]: dn, Pk, prev, out_wf (never null here), item
  const Scalars* sc;      // [F]
  BatchResult* res;       // indexed by GBField::item
  double* bnorm;          // [F][kMaxLevels] level norms (written by k_blevels, read by k_bsolve)
  const int* order;       // [F] image of each solve CTA, longest expected solves first (null: in order)
  int F;
  double tol, eta, level_tol;
  int max_iter, level_max, check;
};

struct BSampleArgs {
  const GBField* fields;  // [F]: aq, fg, out_wf (s_W, the chains' start), out_samples, chain, key0, key1
  const Scalars* sc;      // [F]
  int F;
  int n_samples;
};

template <int N>
constexpr int bsolve_min_ctas() { return N >= 128 ? 3 : (N == 64 ? 8 : 16); }
template <int N>
constexpr int bsolve_smem_bytes() { return Geo<N>::FIELD_BYTES + 33 * 8; }

// CTAs per image of k_blevels: CTA y of image x computes levels y, y + kLevelCtas, ... (most images have
// fewer levels than this, so few CTAs start only to exit)
constexpr int kLevelCtas = 16;

// ||S N_lambda^-1 d||^2 of every cooling level of image blockIdx.x, levels strided over blockIdx.y
template <int N>
__global__ void __launch_bounds__(N) k_blevels(BSolveArgs a) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* S = reinterpret_cast<float2*>(smem_raw);
  double* red = reinterpret_cast<double*>(smem_raw + G::FIELD_BYTES);
  const int f = blockIdx.x;
  const Scalars sc = a.sc[f];
  if (sc.status != 0) return;  // uniform over the CTA
  const GBField fd = a.fields[f];
  for (int lev = blockIdx.y; lev < sc.n_levels; lev += gridDim.y) {
    const double v = level_norm<N>(S, red, threadIdx.x, fd.dn, fd.Pk, float(level_lambda(sc, lev, a.eta) * sc.tau));
    if (threadIdx.x == 0) a.bnorm[f * kMaxLevels + lev] = v;
    __syncthreads();  // the field buffer is reused by the next level
  }
}

// one image per CTA: cooled solve from s = 0 with the level norms of k_blevels, s_W out
template <int N>
__global__ void __launch_bounds__(N, bsolve_min_ctas<N>()) k_bsolve(BSolveArgs a) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* S = reinterpret_cast<float2*>(smem_raw);
  double* red = reinterpret_cast<double*>(smem_raw + G::FIELD_BYTES);
  const int lt = threadIdx.x;
  const int f = a.order ? a.order[blockIdx.x] : int(blockIdx.x);
  const GBField fd = a.fields[f];
  const Scalars sc = a.sc[f];
  if (sc.status != 0) {  // uniform over the CTA
    if (lt == 0) a.res[fd.item] = BatchResult{-1.0, 0, sc.status};
    return;
  }
  float2 c[G::LR];
#pragma unroll
  for (int m = 0; m < G::LR; ++m) c[m] = make_float2(0.f, 0.f);
  int iters = 0;
  double rho = -1.0;
  const int status = solve_sweeps<N>(S, red, lt, c, fd.dn, fd.Pk, sc, a.bnorm + f * kMaxLevels, fd.prev,
                                     a.tol, a.eta, a.level_tol, a.max_iter, a.level_max, a.check, iters, rho);
  float* stg = reinterpret_cast<float*>(S);
  stage_row<N>(stg, lt, c);
  __syncthreads();
  copy_out<N>(stg, lt, fd.out_wf);
  if (lt == 0) a.res[fd.item] = BatchResult{rho, iters, status};
}

// FPC images per CTA (N threads each): every image's chain from its s_W. Images whose set-up failed (and
// the padding fields of the last CTA) run the same sweeps, so that the CTA's barriers line up, but write
// nothing.
template <int N, int FPC>
__global__ void __launch_bounds__(N * FPC, sample_min_ctas<N>()) k_bsample(BSampleArgs a) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int fld = threadIdx.x / N, lt = threadIdx.x % N;
  const int f0 = blockIdx.x * FPC + fld;
  const int f = f0 < a.F ? f0 : a.F - 1;
  const GBField fd = a.fields[f];
  const Scalars sc = a.sc[f];
  const bool active = f0 < a.F && sc.status == 0;
  float2* S = reinterpret_cast<float2*>(smem_raw + fld * G::FIELD_BYTES);
  float2 c[G::LR];
  const float2* src = reinterpret_cast<const float2*>(fd.out_wf + lt * G::W);
#pragma unroll
  for (int m = 0; m < G::LR; ++m) c[m] = active ? src[m] : make_float2(0.f, 0.f);
  sample_sweeps<N>(S, lt, c, fd.aq, TableCoef{fd.fg, G::WH}, sc.sqrt_tau, 0u, fd.chain, fd.key0, fd.key1,
                   a.n_samples, 0, 1, fd.out_samples, active);
}

}  // namespace wf
