// Size-specialised launchers of the fused kernels (one translation unit per image size).
#pragma once

#include <cuda_runtime.h>

#include "wf_gibbs.cuh"
#include "wf_global.cuh"
#include "wf_batch.cuh"
#include "wf_gbatch.cuh"
#include "wf_cluster.cuh"
#include "wf_cluster_ext.cuh"
#include "wf_bphase.cuh"

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
cudaError_t launch_sample_band(const SampleArgs& a, cudaStream_t st, LaunchTimer* t);

template <int N>
cudaError_t launch_sample_spin2(const Spin2Args& a, cudaStream_t st, LaunchTimer* t);

template <int N>
cudaError_t launch_solve(const SolveArgs& a, const BnormArgs& b, cudaStream_t st, LaunchTimer* t);

// batched persistent form for N <= 128: grid = min(items, resident CTAs), per-CTA scratch slots
template <int N>
cudaError_t launch_batch(const BatchArgs& b, int* grid_out, cudaStream_t st);

// batched form for N <= 128 in phases (after the per-image set-up kernels): a few CTAs per image for the
// level norms, one CTA per image for the cooled solves, then the samplers with fpc images per CTA
template <int N>
cudaError_t launch_bsolve(const BSolveArgs& a, cudaStream_t st);
template <int N>
cudaError_t launch_bsample(const BSampleArgs& a, int fpc, cudaStream_t st);

// weighted spectral power of real fields (N <= 128, one CTA per field)
template <int N>
cudaError_t launch_wpower(const WpowerArgs& p, cudaStream_t st);
template <int N>
cudaError_t batch_grid(int n_items, int grid_pct, int* grid_out);

// large images (N >= 256): one cooperative launch of k_global<N> (all CTAs co-resident)
template <int N>
cudaError_t launch_global(const GlobalArgs& a, cudaStream_t st, LaunchTimer* t);

// batched large images (N >= 256): one cooperative launch of k_gbatch<N> over all fields of a size class
template <int N>
cudaError_t launch_gbatch(const GBArgs& a, cudaStream_t st);

// cluster-resident sampler (N in {256, 512}): one cluster of N / MR CTAs of MR rows each per chain
// (MR = 64 at 256; 32 or 64 at 512). cudaErrorNotSupported when no cluster of that shape can be resident.
template <int N, int MR>
cudaError_t launch_csample(const SampleArgs& a, cudaStream_t st, LaunchTimer* t);
// clusters of k_csample<N, MR> that can be resident at once on the current device (0: none)
template <int N, int MR>
cudaError_t csample_clusters(int* clusters);
// whole pipeline (level norms, cooled solve, samples) of a batch of large images: one cluster per image
template <int N, int MR>
cudaError_t launch_cpipe(const CBArgs& a, cudaStream_t st, LaunchTimer* t);

// cluster-resident hierarchical sampler (a.band_clusters clusters of N / MR CTAs looping over the chains;
// a.fg and a.band_map in slot order) and
// spin-2 sampler (both components per cluster). cudaErrorNotSupported when no cluster of that shape
// can be resident.
template <int N, int MR>
cudaError_t launch_csample_band(const SampleArgs& a, cudaStream_t st, LaunchTimer* t);
// clusters of k_csample_band<N, MR> with n_bins bands that can be resident at once (0: none)
template <int N, int MR>
cudaError_t csample_band_clusters(int n_bins, int* clusters);
template <int N, int MR>
cudaError_t launch_csample_spin2(const Spin2Args& a, cudaStream_t st, LaunchTimer* t);

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
cudaError_t launch_sample_band(const SampleArgs& a, cudaStream_t st, LaunchTimer* t) {
  constexpr int FPC = fields_per_cta<N>();
  const int smem = FPC * (Geo<N>::FIELD_BYTES + band_bytes(a.n_bins));
  auto kern = k_sample_band<N, FPC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int blocks = (a.n_chains + FPC - 1) / FPC;
  if (t) t->start();
  kern<<<blocks, N * FPC, smem, st>>>(a);
  if (t) t->stop();
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_sample_spin2(const Spin2Args& a, cudaStream_t st, LaunchTimer* t) {
  constexpr int FPC = fields_per_cta<N>();  // images per CTA; two component fields each
  const int smem = 2 * FPC * Geo<N>::FIELD_BYTES;
  auto kern = k_sample_spin2<N, FPC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int blocks = (a.n_chains + FPC - 1) / FPC;
  if (t) t->start();
  kern<<<blocks, 2 * N * FPC, smem, st>>>(a);
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
  if (!a.rhs_mode) {  // rhs mode: the level norms are supplied
    k_bnorm<N><<<kMaxLevels, N, smem, st>>>(b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (t) t->start();
  k_solve<N><<<1, N, smem, st>>>(a);
  if (t) t->stop();
  return cudaGetLastError();
}


template <int N>
cudaError_t batch_grid(int n_items, int grid_pct, int* grid_out) {
  const int smem = batch_smem_bytes<N>();
  cudaError_t e = cudaFuncSetAttribute(k_batch<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<N>, N, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int full = per_sm * sms;
  if (grid_pct > 0 && grid_pct < 100) full = (full * grid_pct + 99) / 100;
  *grid_out = n_items < full ? n_items : full;
  return cudaSuccess;
}

template <int N>
cudaError_t launch_batch(const BatchArgs& b, int* grid_out, cudaStream_t st) {
  int grid = 0;
  cudaError_t e = batch_grid<N>(b.n, b.grid_pct, &grid);
  if (e != cudaSuccess) return e;
  if (grid_out) *grid_out = grid;
  if (grid > 0) k_batch<N><<<grid, N, batch_smem_bytes<N>(), st>>>(b);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_bsolve(const BSolveArgs& a, cudaStream_t st) {
  const int smem = bsolve_smem_bytes<N>();
  cudaError_t e = cudaFuncSetAttribute(k_blevels<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_bsolve<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (a.F > 0) {
    k_blevels<N><<<dim3(a.F, kLevelCtas), N, smem, st>>>(a);
    k_bsolve<N><<<a.F, N, smem, st>>>(a);
  }
  return cudaGetLastError();
}

template <int N, int FPC>
cudaError_t launch_bsample_fpc(const BSampleArgs& a, cudaStream_t st) {
  const int smem = FPC * Geo<N>::FIELD_BYTES;
  auto kern = k_bsample<N, FPC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (a.F > 0 && a.n_samples > 0) kern<<<(a.F + FPC - 1) / FPC, N * FPC, smem, st>>>(a);
  return cudaGetLastError();
}

// fields (images) per CTA fpc in 1 .. 128 / N (0: fields_per_cta<N>())
template <int N>
cudaError_t launch_bsample(const BSampleArgs& a, int fpc, cudaStream_t st) {
  if (fpc == 0) fpc = fields_per_cta<N>();
  if (fpc < 1 || fpc > fields_per_cta<N>()) return cudaErrorInvalidValue;
  switch (fpc) {
    case 1: return launch_bsample_fpc<N, 1>(a, st);
    case 2: if constexpr (fields_per_cta<N>() >= 2) return launch_bsample_fpc<N, 2>(a, st); break;
    case 4: if constexpr (fields_per_cta<N>() >= 4) return launch_bsample_fpc<N, 4>(a, st); break;
    case 8: if constexpr (fields_per_cta<N>() >= 8) return launch_bsample_fpc<N, 8>(a, st); break;
  }
  return cudaErrorInvalidValue;
}

template <int N>
cudaError_t launch_wpower(const WpowerArgs& p, cudaStream_t st) {
  const int smem = Geo<N>::FIELD_BYTES + 33 * 8;
  cudaError_t e = cudaFuncSetAttribute(k_wpower<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (p.n_fields > 0) k_wpower<N><<<p.n_fields, N, smem, st>>>(p);
  return cudaGetLastError();
}

#define WF_INSTANTIATE(N)                                                              \
  template cudaError_t launch_sample<N>(const SampleArgs&, cudaStream_t, LaunchTimer*); \
  template cudaError_t launch_sample_band<N>(const SampleArgs&, cudaStream_t, LaunchTimer*); \
  template cudaError_t launch_sample_spin2<N>(const Spin2Args&, cudaStream_t, LaunchTimer*); \
  template cudaError_t launch_solve<N>(const SolveArgs&, const BnormArgs&, cudaStream_t, LaunchTimer*); \
  template cudaError_t launch_batch<N>(const BatchArgs&, int*, cudaStream_t);                     \
  template cudaError_t batch_grid<N>(int, int, int*);                                                   \
  template cudaError_t launch_bsolve<N>(const BSolveArgs&, cudaStream_t);                                \
  template cudaError_t launch_bsample<N>(const BSampleArgs&, int, cudaStream_t);                         \
  template cudaError_t launch_wpower<N>(const WpowerArgs&, cudaStream_t);
#endif

#if defined(WF_LAUNCH_DEFINE_GLOBAL)
template <int N>
cudaError_t launch_global(const GlobalArgs& a, cudaStream_t st, LaunchTimer* t) {
  using G = GGeo<N>;
  cudaError_t e = cudaFuncSetAttribute(k_global<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_global<N>, 128, G::SMEM)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long items = (long long)(G::ROW_ITEMS > G::COL_ITEMS ? G::ROW_ITEMS : G::COL_ITEMS) * a.n_fields;
  long long full = (long long)per_sm * sms;
  if (a.grid_pct > 0 && a.grid_pct < 100) full = (full * a.grid_pct + 99) / 100;
  const int grid = int(items < full ? items : full);
  GlobalArgs arg = a;
  void* args[] = {&arg};
  if (t) t->start();
  e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_global<N>), dim3(grid), dim3(128), args, G::SMEM, st);
  if (t) t->stop();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
template <int N>
cudaError_t launch_gbatch(const GBArgs& a, cudaStream_t st) {
  using G = GGeo<N>;
  cudaError_t e = cudaFuncSetAttribute(k_gbatch<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gbatch<N>, 128, G::SMEM)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long items = (long long)(G::ROW_ITEMS > G::COL_ITEMS ? G::ROW_ITEMS : G::COL_ITEMS) * a.F;
  long long full = (long long)per_sm * sms;
  if (a.grid_pct > 0 && a.grid_pct < 100) full = (full * a.grid_pct + 99) / 100;
  const int grid = int(items < full ? items : full);
  GBArgs arg = a;
  void* args[] = {&arg};
  e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_gbatch<N>), dim3(grid), dim3(128), args, G::SMEM, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
#define WF_INSTANTIATE_GLOBAL(N)                                                               \
  template cudaError_t launch_global<N>(const GlobalArgs&, cudaStream_t, LaunchTimer*);         \
  template cudaError_t launch_gbatch<N>(const GBArgs&, cudaStream_t);
#endif

#if defined(WF_LAUNCH_DEFINE_CLUSTER)
template <int N, int MR>
cudaError_t csample_config(cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr, int n_chains, cudaStream_t st) {
  using G = CGeo<N, MR>;
  cudaError_t e = cudaFuncSetAttribute(k_csample<N, MR>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_cpipe<N, MR>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
  if (e != cudaSuccess) return e;
  if (G::P > 8) {  // clusters above the portable size of 8
    e = cudaFuncSetAttribute(k_csample<N, MR>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_cpipe<N, MR>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G::P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = dim3(unsigned(n_chains) * G::P, 1, 1);
  cfg->blockDim = dim3(G::L, 1, 1);
  cfg->dynamicSmemBytes = G::SMEM;
  cfg->stream = st;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
  return cudaSuccess;
}
template <int N, int MR>
cudaError_t csample_clusters(int* clusters) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cudaError_t e = csample_config<N, MR>(&cfg, attr, 1, nullptr);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveClusters(clusters, k_csample<N, MR>, &cfg);
}
template <int N, int MR>
cudaError_t launch_csample(const SampleArgs& a, cudaStream_t st, LaunchTimer* t) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cudaError_t e = csample_config<N, MR>(&cfg, attr, a.n_chains, st);
  if (e != cudaSuccess) return e;
  if (t) t->start();
  e = cudaLaunchKernelEx(&cfg, k_csample<N, MR>, a);
  if (t) t->stop();
  return e != cudaSuccess ? e : cudaGetLastError();
}
template <int N, int MR>
cudaError_t launch_cpipe(const CBArgs& a, cudaStream_t st, LaunchTimer* t) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cudaError_t e = csample_config<N, MR>(&cfg, attr, a.F, st);
  if (e != cudaSuccess) return e;
  if (t) t->start();
  e = cudaLaunchKernelEx(&cfg, k_cpipe<N, MR>, a);
  if (t) t->stop();
  return e != cudaSuccess ? e : cudaGetLastError();
}
#define WF_INSTANTIATE_CLUSTER(N, MR)                                                          \
  template cudaError_t launch_csample<N, MR>(const SampleArgs&, cudaStream_t, LaunchTimer*);   \
  template cudaError_t csample_clusters<N, MR>(int*);                                          \
  template cudaError_t launch_cpipe<N, MR>(const CBArgs&, cudaStream_t, LaunchTimer*);
#endif

#if defined(WF_LAUNCH_DEFINE_CLUSTER_EXT)
// launch configuration of `clusters` clusters of P CTAs of `threads` threads with `smem` dynamic shared
// bytes each; cudaErrorNotSupported when not one such cluster can be resident
template <class Kern>
cudaError_t cluster_launch_config(Kern kern, int P, int threads, int smem, int clusters, cudaStream_t st,
                                  cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (P > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = unsigned(P);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = dim3(unsigned(clusters) * unsigned(P), 1, 1);
  cfg->blockDim = dim3(unsigned(threads), 1, 1);
  cfg->dynamicSmemBytes = size_t(smem);
  cfg->stream = st;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
  int resident = 0;
  e = cudaOccupancyMaxActiveClusters(&resident, kern, cfg);
  if (e != cudaSuccess) return e;
  return resident > 0 ? cudaSuccess : cudaErrorNotSupported;
}
template <int N, int MR>
cudaError_t csample_band_clusters(int n_bins, int* clusters) {
  using G = CGeo<N, MR>;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  *clusters = 0;
  cudaError_t e = cluster_launch_config(k_csample_band<N, MR>, G::P, G::L, cband_smem<N, MR>(n_bins), 1, nullptr,
                                        &cfg, attr);
  if (e == cudaErrorNotSupported) return cudaSuccess;
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveClusters(clusters, k_csample_band<N, MR>, &cfg);
}
template <int N, int MR>
cudaError_t launch_csample_band(const SampleArgs& a, cudaStream_t st, LaunchTimer* t) {
  using G = CGeo<N, MR>;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cudaError_t e = cluster_launch_config(k_csample_band<N, MR>, G::P, G::L, cband_smem<N, MR>(a.n_bins),
                                        a.band_clusters, st, &cfg, attr);
  if (e != cudaSuccess) return e;
  if (t) t->start();
  e = cudaLaunchKernelEx(&cfg, k_csample_band<N, MR>, a);
  if (t) t->stop();
  return e != cudaSuccess ? e : cudaGetLastError();
}
template <int N, int MR>
cudaError_t launch_csample_spin2(const Spin2Args& a, cudaStream_t st, LaunchTimer* t) {
  using G = CGeo<N, MR>;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cudaError_t e =
      cluster_launch_config(k_csample_spin2<N, MR>, G::P, cspin2_threads<N, MR>(), cspin2_smem<N, MR>(), a.n_chains,
                            st, &cfg, attr);
  if (e != cudaSuccess) return e;
  if (t) t->start();
  e = cudaLaunchKernelEx(&cfg, k_csample_spin2<N, MR>, a);
  if (t) t->stop();
  return e != cudaSuccess ? e : cudaGetLastError();
}
#define WF_INSTANTIATE_CLUSTER_BAND(N, MR)                                                      \
  template cudaError_t launch_csample_band<N, MR>(const SampleArgs&, cudaStream_t, LaunchTimer*); \
  template cudaError_t csample_band_clusters<N, MR>(int, int*);
#define WF_INSTANTIATE_CLUSTER_SPIN2(N, MR) \
  template cudaError_t launch_csample_spin2<N, MR>(const Spin2Args&, cudaStream_t, LaunchTimer*);
#endif

}  // namespace wf
