// Size-specialised launchers of the fused kernels (one translation unit per image size).
#pragma once

#include <cuda_runtime.h>

#include "wf_gibbs.cuh"

namespace wf {

// optional CUDA-event bracket around the main kernel of a launch
struct LaunchTimer {
  virtual void start() = 0;
  virtual void stop() = 0;
};

// fields (chains) per CTA of the sampler: 128 threads per CTA for every size
template <int N>
constexpr int fields_per_cta() { return N >= 128 ? 1 : 128 / N; }

template <int N>
cudaError_t launch_sample(const SampleArgs& a, cudaStream_t st, LaunchTimer* t);

template <int N>
cudaError_t launch_solve(const SolveArgs& a, const BnormArgs& b, cudaStream_t st, LaunchTimer* t);

// definitions, included by the per-size translation units only
#if defined(WF_LAUNCH_DEFINE)
template <int N>
cudaError_t launch_sample(const SampleArgs& a, cudaStream_t st, LaunchTimer* t) {
  constexpr int FPC = fields_per_cta<N>();
  const int smem = FPC * Geo<N>::FIELD_BYTES;
  auto kern = k_sample<N, FPC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int blocks = (a.n_chains + FPC - 1) / FPC;
  if (t) t->start();
  kern<<<blocks, N * FPC, smem, st>>>(a);
  if (t) t->stop();
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_solve(const SolveArgs& a, const BnormArgs& b, cudaStream_t st, LaunchTimer* t) {
  const int smem = Geo<N>::FIELD_BYTES + 33 * 8;
  cudaError_t e = cudaFuncSetAttribute(k_bnorm<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_solve<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_bnorm<N><<<kMaxLevels, N, smem, st>>>(b);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (t) t->start();
  k_solve<N><<<1, N, smem, st>>>(a);
  if (t) t->stop();
  return cudaGetLastError();
}

#define WF_INSTANTIATE(N)                                                              \
  template cudaError_t launch_sample<N>(const SampleArgs&, cudaStream_t, LaunchTimer*); \
  template cudaError_t launch_solve<N>(const SolveArgs&, const BnormArgs&, cudaStream_t, LaunchTimer*);
#endif

}  // namespace wf
