// C ABI of the messenger-field Wiener filter / sampler: argument checks, device set-up kernels, scratch,
// launches of the fused kernels in wf_gibbs.cuh, and the status read-back.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/wf.h"
#include "wf_launch.h"
#include "wf_refine.h"

namespace {

thread_local int g_last_cuda_error = 0;
thread_local int g_timing = 0;
thread_local int g_large_sampler = 0;  // 0: automatic, 1: global-memory kernels, 2: clusters where they fit
thread_local double g_kernel_ms = -1.0;

// CUDA events around the main kernel of a call (only when timing is enabled on this thread)
struct KernelTimer : wf::LaunchTimer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t st;
  explicit KernelTimer(cudaStream_t s) : st(s) {
    g_kernel_ms = -1.0;
    if (!g_timing) return;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) e0 = e1 = nullptr;
  }
  void start() override { if (e0) cudaEventRecord(e0, st); }
  void stop() override { if (e1) cudaEventRecord(e1, st); }
  // after the stream has been synchronised
  void collect() {
    float ms = -1.0f;
    if (e0 && e1 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) g_kernel_ms = ms;
  }
  ~KernelTimer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

using wf::kMaxLevels;

wf_status cuda_fail(cudaError_t e) {
  g_last_cuda_error = int(e);
  return WF_ERR_CUDA;
}

#define WF_CUDA(call)                           \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

// ---------------------------------------------------------------------------------------------
// set-up kernels
// ---------------------------------------------------------------------------------------------
// One block: tau = min observed Ndiag (or the caller's), max_k P_k, input checks, lambda_0, levels.
__device__ void prep_block(const float* __restrict__ d, const float* __restrict__ Ndiag,
                           const uint8_t* __restrict__ mask, const float* __restrict__ Pk, int H, int W,
                           double tau_user, double eta, wf::Scalars* sc) {
  __shared__ float s_min[32], s_max[32];
  __shared__ int s_obs[32], s_bad[32], s_neg[32];
  float vmin = INFINITY, vmax = 0.0f;
  int nobs = 0, bad = 0, neg = 0;
  const int n = H * W, nm = H * (W / 2 + 1);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (mask[i] == 0) {
      const float nv = Ndiag[i], dv = d[i];
      ++nobs;
      if (!isfinite(nv) || !isfinite(dv)) bad = 1;
      else if (!(nv > 0.0f)) neg = 1;
      else vmin = fminf(vmin, nv);
    }
  }
  for (int i = threadIdx.x; i < nm; i += blockDim.x) {
    const float p = Pk[i];
    if (!isfinite(p)) bad = 1;
    else if (p < 0.0f) neg = 1;
    else vmax = fmaxf(vmax, p);
  }
  for (int o = 16; o > 0; o >>= 1) {
    vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
    vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    nobs += __shfl_xor_sync(0xffffffffu, nobs, o);
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    neg |= __shfl_xor_sync(0xffffffffu, neg, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = int(blockDim.x >> 5);
  if (l == 0) { s_min[w] = vmin; s_max[w] = vmax; s_obs[w] = nobs; s_bad[w] = bad; s_neg[w] = neg; }
  __syncthreads();
  if (threadIdx.x != 0) return;
  int total_obs = 0;
  for (int i = 0; i < nw; ++i) {
    vmin = fminf(vmin, s_min[i]);
    vmax = fmaxf(vmax, s_max[i]);
    total_obs += s_obs[i];
    bad |= s_bad[i];
    neg |= s_neg[i];
  }
  wf::Scalars r = wf::make_scalars(vmin, total_obs, vmax, bad, neg, tau_user, eta);
  *sc = r;
}

__global__ void k_prep(const float* __restrict__ d, const float* __restrict__ Ndiag, const uint8_t* __restrict__ mask,
                       const float* __restrict__ Pk, int H, int W, double tau_user, double eta, wf::Scalars* sc) {
  prep_block(d, Ndiag, mask, Pk, H, W, tau_user, eta, sc);
}

// Per-pixel tables ([W][H], x-major so that row threads read consecutive addresses) and the
// per-mode sample table (table_pixel, table_mode: within 2 ulp of the exact coefficients).
// Pixel tables are x-major, aq[x*H + ty] and dn[x*H + ty], with ty = y, or with perm = P > 0 (the
// cluster kernels, CTA b holding the rows y = P a + b) ty = (y mod P) H/P + y / P, so that the rows of one
// CTA are contiguous and its row threads read consecutive addresses.
__host__ __device__ inline int table_row(int y, int H, int perm) { return perm ? (y % perm) * (H / perm) + y / perm : y; }

// Position of half-spectrum entry j = ky (W/2 + 1) + kx in a mode table: natural (cm = 0), or the column slot
// order of the cluster kernels with cm rows per CTA (kx < W/2 at ky W/2 + t, t = (kx mod cm) R + kx / cm,
// R = (W/2) / cm, the slot holding kx; kx = W/2 at H W/2 + ky), so that a column unit's threads read
// consecutive addresses.
__host__ __device__ inline int mode_pos(int j, int H, int W, int cm) {
  if (!cm) return j;
  const int L = W / 2, ky = j / (L + 1), kx = j % (L + 1);
  return kx < L ? ky * L + (kx % cm) * (L / cm) + kx / cm : H * L + ky;
}

// pks (optional): P in the same order as the mode table (the cluster solve reads it there)
__global__ void k_tables(const float* __restrict__ d, const float* __restrict__ Ndiag, const uint8_t* __restrict__ mask,
                         const float* __restrict__ Pk, int H, int W, const wf::Scalars* __restrict__ sc,
                         float2* __restrict__ aq, float2* __restrict__ dn, float2* __restrict__ fg, int perm = 0,
                         int cm = 0, float* __restrict__ pks = nullptr) {
  if (sc->status != 0) return;
  const double tau = sc->tau;
  const int n = H * W, nm = H * (W / 2 + 1);
  const double inv_n = 1.0 / double(n);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + nm; i += gridDim.x * blockDim.x) {
    if (i < n) {
      const int y = i / W, x = i % W, ty = table_row(y, H, perm);
      float2 a2, d2;
      wf::table_pixel(d[i], Ndiag[i], mask[i] == 0, tau, &a2, &d2);
      if (aq) aq[x * H + ty] = a2;
      if (dn) dn[x * H + ty] = d2;
    } else {
      const int j = i - n, q = mode_pos(j, H, W, cm);
      if (fg) fg[q] = wf::table_mode(Pk[j], tau, inv_n);
      if (pks) pks[q] = Pk[j];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// launch helpers per size
// ---------------------------------------------------------------------------------------------
bool size_ok(int H, int W) {
  return H == W && (H == 16 || H == 32 || H == 64 || H == 128 || H == 256 || H == 512 || H == 1024);
}
bool size_on_chip(int H) { return H <= 128; }

bool cluster_fits(int H, int rows = 0);

// Path for `units` independent fields (chains or images) of H x H, H in {256, 512}: one thread-block
// cluster per field, or the global-memory kernels. Automatic choice (measured on GB300, 50 sweeps): the
// global-memory kernels (16-point sub-transforms, many CTAs per field) are faster for few fields, the
// clusters from about 32 fields at 256^2 (24 chains: 1.40 vs 1.84 ms; 32 chains: 2.46 vs 1.88 ms) and
// from about 8 at 512^2 (4 chains: 1.39 vs 1.58 ms; 8 chains: 2.88 vs 2.07 ms).
int cluster_min_units(int H) { return H == 256 ? 32 : 8; }

// rows per CTA of the cluster kernels: 64 at 256; at 512 the caller's choice of 32 or 64 (0: the default)
int cluster_rows_of(int H, int rows) { return H == 512 && (rows == 32 || rows == 64) ? rows : wf::cluster_rows(H); }

cudaError_t csample_clusters_any(int H, int rows, int* n) {
  if (H == 256) return wf::csample_clusters<256, 64>(n);
  return rows == 64 ? wf::csample_clusters<512, 64>(n) : wf::csample_clusters<512, 32>(n);
}
cudaError_t launch_csample_any(int H, int rows, const wf::SampleArgs& a, cudaStream_t st, wf::LaunchTimer* t) {
  if (H == 256) return wf::launch_csample<256, 64>(a, st, t);
  return rows == 64 ? wf::launch_csample<512, 64>(a, st, t) : wf::launch_csample<512, 32>(a, st, t);
}
cudaError_t launch_cpipe_any(int H, int rows, const wf::CBArgs& a, cudaStream_t st, wf::LaunchTimer* t) {
  if (H == 256) return wf::launch_cpipe<256, 64>(a, st, t);
  return rows == 64 ? wf::launch_cpipe<512, 64>(a, st, t) : wf::launch_cpipe<512, 32>(a, st, t);
}

bool use_cluster(int H, int units, int rows = 0) {
  if ((H != 256 && H != 512) || g_large_sampler == 1 || !cluster_fits(H, rows)) return false;
  return g_large_sampler == 2 || units >= cluster_min_units(H);
}

// whether at least one sampler cluster of that geometry fits on the current device (queried once per device)
bool cluster_fits(int H, int rows) {
  static std::mutex mu;
  static int known[3][64] = {};  // 0 unknown, 1 fits, 2 does not
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return false;
  }
  const int k = H == 256 ? 0 : (cluster_rows_of(H, rows) == 64 ? 2 : 1);
  std::lock_guard<std::mutex> lock(mu);
  if (known[k][dev] == 0) {
    int clusters = 0;
    const cudaError_t e = csample_clusters_any(H, cluster_rows_of(H, rows), &clusters);
    if (e != cudaSuccess) cudaGetLastError();
    known[k][dev] = (e == cudaSuccess && clusters > 0) ? 1 : 2;
  }
  return known[k][dev] == 1;
}

// An output the kernels may store to: device or managed memory, or page-locked host memory that is
// mapped into the device address space at the same address (cudaHostAlloc, or cudaHostRegister with
// mapping, under unified addressing). Page-locked memory without that mapping cannot be written by a
// kernel and is refused here instead of faulting in the kernel.
bool out_ptr_ok(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;  // not known to the runtime: left to the caller
  }
  if (at.type == cudaMemoryTypeHost) return at.devicePointer == p;
  if (at.type == cudaMemoryTypeUnregistered) {  // pageable host memory: only where the GPU can reach it
    int dev = 0, pageable = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return pageable != 0;
  }
  return true;
}

// Twiddle tables of the large-image path, in FP64 then rounded once:
// tw_row[j] = exp(-2 pi i j / (W/2)), tw_col[j] = exp(-2 pi i j / H), tw_real[k] = exp(-2 pi i k / W).
__global__ void k_twiddles(int H, int W, float2* tw_row, float2* tw_col, float2* tw_real) {
  const int LR = W / 2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < LR + H + LR; i += gridDim.x * blockDim.x) {
    double sn, cs;
    if (i < LR) {
      sincospi(-2.0 * double(i) / double(LR), &sn, &cs);
      tw_row[i] = make_float2(float(cs), float(sn));
    } else if (i < LR + H) {
      const int j = i - LR;
      sincospi(-2.0 * double(j) / double(H), &sn, &cs);
      tw_col[j] = make_float2(float(cs), float(sn));
    } else {
      const int k = i - LR - H;
      sincospi(-2.0 * double(k) / double(W), &sn, &cs);
      tw_real[k] = make_float2(float(cs), float(sn));
    }
  }
}

cudaError_t launch_global_any(int H, const wf::GlobalArgs& a, cudaStream_t st, wf::LaunchTimer* t) {
  switch (H) {
    case 256: return wf::launch_global<256>(a, st, t);
    case 512: return wf::launch_global<512>(a, st, t);
    case 1024: return wf::launch_global<1024>(a, st, t);
  }
  return cudaErrorInvalidValue;
}

// scratch carved from one stream-ordered allocation
struct Scratch {
  void* base = nullptr;
  cudaStream_t st = nullptr;
  ~Scratch() {
    if (base) cudaFreeAsync(base, st);
  }
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// bump allocator over one cudaMallocAsync block
struct Carve {
  size_t off = 0;
  template <class T>
  size_t take(size_t count) {
    const size_t o = off;
    off += align256(count * sizeof(T));
    return o;
  }
};

// Diagonal pixel response A of d = A s + n (Alg. 1 definitions with A_i^2 > 0): the t-update with A equals
// the A = I update for data d / A and noise N / A^2, and A_i = 0 leaves pixel i without data. Values are
// formed in FP64 and rounded once.
__global__ void k_response(int n, const float* __restrict__ d, const float* __restrict__ Nd,
                           const uint8_t* __restrict__ mask, const float* __restrict__ A, float* d2, float* N2,
                           uint8_t* m2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double a = A[i];
    if (mask[i] != 0 || a == 0.0) {
      d2[i] = 0.0f;
      N2[i] = 1.0f;
      m2[i] = 1;
    } else {
      d2[i] = float(double(d[i]) / a);
      N2[i] = float(double(Nd[i]) / (a * a));
      m2[i] = 0;
    }
  }
}

// transformed inputs of a call with a response (scratch freed with the object, stream-ordered)
struct Response {
  Scratch scr;
  const float* d = nullptr;
  const float* Nd = nullptr;
  const uint8_t* mask = nullptr;
};

cudaError_t apply_response(const float* d, const float* Nd, const uint8_t* mask, const float* A, size_t n,
                           cudaStream_t st, Response* r) {
  Carve cv;
  const size_t o_d = cv.take<float>(n), o_n = cv.take<float>(n), o_m = cv.take<uint8_t>(n);
  r->scr.st = st;
  cudaError_t e = cudaMallocAsync(&r->scr.base, cv.off, st);
  if (e != cudaSuccess) return e;
  char* b = static_cast<char*>(r->scr.base);
  float* d2 = reinterpret_cast<float*>(b + o_d);
  float* n2 = reinterpret_cast<float*>(b + o_n);
  uint8_t* m2 = reinterpret_cast<uint8_t*>(b + o_m);
  const long long blocks = (long long)(n + 255) / 256;
  k_response<<<int(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(int(n), d, Nd, mask, A, d2, n2, m2);
  r->d = d2;
  r->Nd = n2;
  r->mask = m2;
  return cudaGetLastError();
}

// Sampler for H >= 256: fields = chains, state in global memory, one cooperative launch.
wf_status sample_global(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, int H, int W,
                        uint64_t seed, const wf_sample_opts& o, long long sweeps, float* out, cudaStream_t st,
                        wf::LaunchTimer* timer) {
  const size_t n = size_t(H) * W, nm = size_t(H) * (W / 2 + 1), nz = size_t(H) * (W / 2);
  Carve cv;
  const size_t o_sc = cv.take<wf::Scalars>(1), o_bar = cv.take<wf::GridBar>(1), o_aq = cv.take<float2>(n),
               o_fg = cv.take<float2>(nm), o_tr = cv.take<float2>(W / 2), o_tc = cv.take<float2>(H),
               o_tw = cv.take<float2>(W / 2), o_z = cv.take<float2>(nz * size_t(o.n_chains));
  Scratch scr;
  scr.st = st;
  WF_CUDA(cudaMallocAsync(&scr.base, cv.off, st));
  char* b = static_cast<char*>(scr.base);
  auto* sc = reinterpret_cast<wf::Scalars*>(b + o_sc);
  auto* bar = reinterpret_cast<wf::GridBar*>(b + o_bar);
  WF_CUDA(cudaMemsetAsync(bar, 0, sizeof(wf::GridBar), st));
  k_prep<<<1, 1024, 0, st>>>(d, Ndiag, mask, Pk, H, W, o.tau, 0.5, sc);
  WF_CUDA(cudaGetLastError());
  k_tables<<<int((n + nm + 255) / 256), 256, 0, st>>>(d, Ndiag, mask, Pk, H, W, sc,
                                                       reinterpret_cast<float2*>(b + o_aq), nullptr,
                                                       reinterpret_cast<float2*>(b + o_fg));
  WF_CUDA(cudaGetLastError());
  k_twiddles<<<8, 256, 0, st>>>(H, W, reinterpret_cast<float2*>(b + o_tr), reinterpret_cast<float2*>(b + o_tc),
                                reinterpret_cast<float2*>(b + o_tw));
  WF_CUDA(cudaGetLastError());
  wf::GlobalArgs a{};
  a.Z = reinterpret_cast<float2*>(b + o_z);
  a.tw_row = reinterpret_cast<float2*>(b + o_tr);
  a.tw_col = reinterpret_cast<float2*>(b + o_tc);
  a.tw_real = reinterpret_cast<float2*>(b + o_tw);
  a.aq = reinterpret_cast<float2*>(b + o_aq);
  a.fg = reinterpret_cast<float2*>(b + o_fg);
  a.Pk = Pk;
  a.sc = sc;
  a.bar = bar;
  a.init_s = o.init_s;
  a.init_stride = (o.init_s && o.init_per_chain) ? (long long)n : 0;
  a.out = out;
  a.n_samples = o.n_samples;
  a.n_fields = o.n_chains;
  a.n_sweeps = int(sweeps);
  a.burn_in = o.burn_in;
  a.thin = o.thin;
  a.chain0 = o.chain_offset;
  a.step0 = o.start_step;
  a.key0 = uint32_t(seed & 0xffffffffu);
  a.key1 = uint32_t(seed >> 32);
  a.out_dtype = o.out_dtype;
  a.mode = 0;
  cudaError_t e = launch_global_any(H, a, st, timer);
  if (e != cudaSuccess) return cuda_fail(e);
  wf::Scalars hsc;
  wf::GridBar hb;
  WF_CUDA(cudaMemcpyAsync(&hsc, sc, sizeof(hsc), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaMemcpyAsync(&hb, bar, sizeof(hb), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  if (hsc.status != WF_OK) return wf_status(hsc.status);
  return hb.err ? wf_status(hb.err) : WF_OK;
}

// Wiener filter for H >= 256: level norms (fields = levels), then the cooled iteration, field in
// global memory.
wf_status solve_global(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, int H, int W,
                       const wf_solve_opts& o, float* out_s, int32_t* iters_out, double* resid_out, cudaStream_t st,
                       wf::LaunchTimer* timer, const float2* rhs_tab = nullptr, const double* rhs_norms = nullptr) {
  const size_t n = size_t(H) * W, nz = size_t(H) * (W / 2);
  // scalars first: the number of cooling levels sizes the level-norm pass
  Scratch s1;
  s1.st = st;
  WF_CUDA(cudaMallocAsync(&s1.base, sizeof(wf::Scalars), st));
  auto* sc1 = static_cast<wf::Scalars*>(s1.base);
  k_prep<<<1, 1024, 0, st>>>(d, Ndiag, mask, Pk, H, W, o.tau, o.eta, sc1);
  WF_CUDA(cudaGetLastError());
  wf::Scalars hsc;
  WF_CUDA(cudaMemcpyAsync(&hsc, sc1, sizeof(hsc), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  if (hsc.status != WF_OK) return wf_status(hsc.status);
  const int levels = hsc.n_levels;
  Carve cv;
  const size_t o_sc = cv.take<wf::Scalars>(1), o_bar = cv.take<wf::GridBar>(2), o_dn = cv.take<float2>(n),
               o_tr = cv.take<float2>(W / 2), o_tc = cv.take<float2>(H), o_tw = cv.take<float2>(W / 2),
               o_bn = cv.take<double>(wf::kMaxLevels), o_acc = cv.take<double>(2), o_st = cv.take<wf::SolveStatus>(1),
               o_prev = cv.take<float2>(nz),
               o_z = cv.take<float2>(nz * size_t(levels > 1 && !rhs_tab ? levels : 1));
  Scratch scr;
  scr.st = st;
  WF_CUDA(cudaMallocAsync(&scr.base, cv.off, st));
  char* b = static_cast<char*>(scr.base);
  auto* sc = reinterpret_cast<wf::Scalars*>(b + o_sc);
  auto* bar = reinterpret_cast<wf::GridBar*>(b + o_bar);
  WF_CUDA(cudaMemcpyAsync(sc, &hsc, sizeof(hsc), cudaMemcpyHostToDevice, st));
  WF_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(wf::GridBar), st));
  WF_CUDA(cudaMemsetAsync(b + o_bn, 0, wf::kMaxLevels * sizeof(double), st));
  WF_CUDA(cudaMemsetAsync(b + o_acc, 0, 2 * sizeof(double), st));
  WF_CUDA(cudaMemsetAsync(b + o_st, 0, sizeof(wf::SolveStatus), st));
  if (!rhs_tab) {
    k_tables<<<int((n + 255) / 256), 256, 0, st>>>(d, Ndiag, mask, Pk, H, W, sc, nullptr,
                                                   reinterpret_cast<float2*>(b + o_dn), nullptr);
    WF_CUDA(cudaGetLastError());
  }
  k_twiddles<<<8, 256, 0, st>>>(H, W, reinterpret_cast<float2*>(b + o_tr), reinterpret_cast<float2*>(b + o_tc),
                                reinterpret_cast<float2*>(b + o_tw));
  WF_CUDA(cudaGetLastError());
  wf::GlobalArgs a{};
  a.Z = reinterpret_cast<float2*>(b + o_z);
  a.tw_row = reinterpret_cast<float2*>(b + o_tr);
  a.tw_col = reinterpret_cast<float2*>(b + o_tc);
  a.tw_real = reinterpret_cast<float2*>(b + o_tw);
  a.dn = rhs_tab ? rhs_tab : reinterpret_cast<float2*>(b + o_dn);
  a.Pk = Pk;
  a.sc = sc;
  a.bar = bar;
  a.eta = o.eta;
  cudaError_t e = cudaSuccess;
  if (!rhs_tab) {  // level norms (rhs mode: supplied)
    a.mode = 2;
    a.n_fields = levels;
    a.bnorm_out = reinterpret_cast<double*>(b + o_bn);
    e = launch_global_any(H, a, st, nullptr);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  a.mode = 1;
  a.rhs_mode = rhs_tab ? 1 : 0;
  a.n_fields = 1;
  a.bar = bar + 1;
  a.bnorm2 = rhs_tab ? rhs_norms : reinterpret_cast<double*>(b + o_bn);
  a.acc = reinterpret_cast<double*>(b + o_acc);
  a.prev = reinterpret_cast<float2*>(b + o_prev);
  a.st = reinterpret_cast<wf::SolveStatus*>(b + o_st);
  a.out = out_s;
  a.tol = o.tol;
  a.level_tol = o.level_tol;
  a.max_iter = o.max_iter;
  a.level_max = o.level_max;
  a.check = o.check;
  e = launch_global_any(H, a, st, timer);
  if (e != cudaSuccess) return cuda_fail(e);
  wf::SolveStatus hst;
  wf::GridBar hb[2];
  WF_CUDA(cudaMemcpyAsync(&hst, a.st, sizeof(hst), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaMemcpyAsync(hb, bar, sizeof(hb), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  if (hb[0].err || hb[1].err) return wf_status(hb[0].err ? hb[0].err : hb[1].err);
  if (iters_out) *iters_out = hst.iters;
  if (resid_out) *resid_out = hst.resid;
  return wf_status(hst.status);
}

}  // namespace

extern "C" {

void wf_solve_opts_default(wf_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tau = 0.0;
  o->tol = 1e-6;
  o->eta = 0.5;
  o->level_tol = 1e-2;
  o->level_max = 64;
  o->check = 4;
  o->max_iter = 20000;
  o->refine = 3;  // the returned residual is the FP64 residual of the returned map
  o->init_s = nullptr;
  o->refine_tol = 1e-3;
}

void wf_sample_opts_default(wf_sample_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tau = 0.0;
  o->n_samples = 0;
  o->n_chains = 1;
  o->chain_offset = 0;
  o->start_step = 0;
  o->burn_in = 0;
  o->thin = 1;
  o->init_per_chain = 0;
  o->init_s = nullptr;
}

int32_t wf_supported_size(int32_t H, int32_t W) { return size_ok(H, W) ? 1 : 0; }

int32_t wf_abi_version(void) { return (1 << 16) | 0; }

int32_t wf_last_cuda_error(void) { return g_last_cuda_error; }

void wf_set_kernel_timing(int32_t enable) { g_timing = enable ? 1 : 0; }

int32_t wf_set_large_image_sampler(int32_t mode) {
  const int prev = g_large_sampler;
  g_large_sampler = (mode == 1 || mode == 2) ? mode : 0;
  return prev;
}

double wf_last_kernel_ms(void) { return g_kernel_ms; }

const char* wf_status_string(wf_status s) {
  switch (s) {
    case WF_OK: return "ok";
    case WF_ERR_ARG: return "invalid argument";
    case WF_ERR_TAU: return "tau exceeds the minimum observed noise variance";
    case WF_ERR_SHAPE: return "unsupported image shape";
    case WF_ERR_CUDA: return "CUDA runtime error";
    case WF_ERR_NOT_CONVERGED: return "not converged within max_iter";
    case WF_ERR_NONFINITE: return "non-finite input or residual";
    case WF_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

}  // extern "C"

namespace {

// Wiener filter for 256 and 512 on one thread-block cluster (k_cpipe with one image and no samples): level
// norms, then the cooled iteration from zero, the field in distributed shared memory.
wf_status solve_cluster(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, int H, int W,
                        const wf_solve_opts& o, float* out_s, int32_t* iters_out, double* resid_out, cudaStream_t st,
                        wf::LaunchTimer* timer) {
  const size_t n = size_t(H) * W, nz = size_t(H) * (W / 2);
  Carve cv;
  const size_t nm = size_t(H) * (W / 2 + 1);
  const size_t o_sc = cv.take<wf::Scalars>(1), o_res = cv.take<wf::BatchResult>(1), o_f = cv.take<wf::GBField>(1),
               o_dn = cv.take<float2>(n), o_prev = cv.take<float2>(nz), o_pk = cv.take<float>(nm);
  Scratch scr;
  scr.st = st;
  WF_CUDA(cudaMallocAsync(&scr.base, cv.off, st));
  char* b = static_cast<char*>(scr.base);
  auto* sc = reinterpret_cast<wf::Scalars*>(b + o_sc);
  auto* res = reinterpret_cast<wf::BatchResult*>(b + o_res);
  k_prep<<<1, 1024, 0, st>>>(d, Ndiag, mask, Pk, H, W, o.tau, o.eta, sc);
  WF_CUDA(cudaGetLastError());
  const int rows = cluster_rows_of(H, 0);
  k_tables<<<int((n + nm + 255) / 256), 256, 0, st>>>(d, Ndiag, mask, Pk, H, W, sc, nullptr,
                                                      reinterpret_cast<float2*>(b + o_dn), nullptr, H / rows, rows,
                                                      reinterpret_cast<float*>(b + o_pk));
  WF_CUDA(cudaGetLastError());
  wf::GBField fd{};
  fd.dn = reinterpret_cast<const float2*>(b + o_dn);
  fd.Pk = reinterpret_cast<const float*>(b + o_pk);  // slot order of the cluster kernels
  fd.prev = reinterpret_cast<float2*>(b + o_prev);
  fd.out_wf = out_s;
  fd.item = 0;
  WF_CUDA(cudaMemcpyAsync(b + o_f, &fd, sizeof(fd), cudaMemcpyHostToDevice, st));
  wf::CBArgs cb{};
  cb.fields = reinterpret_cast<const wf::GBField*>(b + o_f);
  cb.sc = sc;
  cb.res = res;
  cb.F = 1;
  cb.tol = o.tol;
  cb.eta = o.eta;
  cb.level_tol = o.level_tol;
  cb.max_iter = o.max_iter;
  cb.level_max = o.level_max;
  cb.check = o.check;
  cb.n_samples = 0;
  const cudaError_t e = launch_cpipe_any(H, cluster_rows_of(H, 0), cb, st, timer);
  if (e != cudaSuccess) return cuda_fail(e);
  wf::BatchResult hr;
  WF_CUDA(cudaMemcpyAsync(&hr, res, sizeof(hr), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  if (iters_out) *iters_out = hr.iters;
  if (resid_out) *resid_out = hr.resid;
  return wf_status(hr.status);
}

// One cooled messenger solve (data mode, or rhs mode when rhs_tab is given: solves (S^-1 + N^-1) s = r
// with the table's r and the supplied per-level norms).
wf_status solve_pass(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, int32_t H, int32_t W,
                     const wf_solve_opts& o, float* out_s, int32_t* iters_out, double* resid_out, cudaStream_t st,
                     wf::LaunchTimer* timer, const float2* rhs_tab = nullptr, const double* rhs_norms = nullptr) {
  if (!size_on_chip(H)) {
    if (o.init_s) return WF_ERR_ARG;  // the large-image solve starts from zero
    if (!rhs_tab && use_cluster(H, 1))
      return solve_cluster(d, Ndiag, mask, Pk, H, W, o, out_s, iters_out, resid_out, st, timer);
    return solve_global(d, Ndiag, mask, Pk, H, W, o, out_s, iters_out, resid_out, st, timer, rhs_tab, rhs_norms);
  }
  const size_t n = size_t(H) * W, nm = size_t(H) * (W / 2 + 1);
  Carve cv;
  const size_t off_sc = cv.take<wf::Scalars>(1), off_st = cv.take<wf::SolveStatus>(1),
               off_bn = cv.take<double>(kMaxLevels), off_dn = cv.take<float2>(n),
               off_prev = cv.take<float2>(size_t(H) * (W / 2));
  Scratch scr;
  scr.st = st;
  WF_CUDA(cudaMallocAsync(&scr.base, cv.off, st));
  char* b = static_cast<char*>(scr.base);
  auto* sc = reinterpret_cast<wf::Scalars*>(b + off_sc);
  auto* sst = reinterpret_cast<wf::SolveStatus*>(b + off_st);
  auto* bn = reinterpret_cast<double*>(b + off_bn);
  auto* dn = reinterpret_cast<float2*>(b + off_dn);
  auto* prev = reinterpret_cast<float2*>(b + off_prev);
  WF_CUDA(cudaMemsetAsync(sst, 0, sizeof(wf::SolveStatus), st));
  k_prep<<<1, 1024, 0, st>>>(d, Ndiag, mask, Pk, H, W, o.tau, o.eta, sc);
  WF_CUDA(cudaGetLastError());
  if (!rhs_tab) {
    k_tables<<<int((n + nm + 255) / 256), 256, 0, st>>>(d, Ndiag, mask, Pk, H, W, sc, nullptr, dn, nullptr);
    WF_CUDA(cudaGetLastError());
  }
  wf::SolveArgs a{};
  a.dn = rhs_tab ? rhs_tab : dn;
  a.Pk = Pk;
  a.sc = sc;
  a.bnorm2 = rhs_tab ? rhs_norms : bn;
  a.init_s = o.init_s;
  a.prev = prev;
  a.out = out_s;
  a.st = sst;
  a.tol = o.tol;
  a.eta = o.eta;
  a.level_tol = o.level_tol;
  a.max_iter = o.max_iter;
  a.level_max = o.level_max;
  a.check = o.check;
  a.rhs_mode = rhs_tab ? 1 : 0;
  wf::BnormArgs bb{dn, Pk, sc, bn, o.eta};
  cudaError_t e = cudaSuccess;
  switch (H) {
    case 16: e = wf::launch_solve<16>(a, bb, st, timer); break;
    case 32: e = wf::launch_solve<32>(a, bb, st, timer); break;
    case 64: e = wf::launch_solve<64>(a, bb, st, timer); break;
    case 128: e = wf::launch_solve<128>(a, bb, st, timer); break;
  }
  if (e != cudaSuccess) return cuda_fail(e);
  wf::Scalars hsc;
  wf::SolveStatus hst;
  WF_CUDA(cudaMemcpyAsync(&hsc, sc, sizeof(hsc), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaMemcpyAsync(&hst, sst, sizeof(hst), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  if (hsc.status != WF_OK) return wf_status(hsc.status);
  if (iters_out) *iters_out = hst.iters;
  if (resid_out) *resid_out = hst.resid;
  return wf_status(hst.status);
}

// Mixed-precision iterative refinement: FP32 messenger solves, FP64 residuals (wf_refine.cu).
// The FP32 solves use (d, Ndiag, mask); the FP64 residual uses the caller's inputs (d0, N0, m0) and
// response A0 (null: the same inputs, A = I).
wf_status solve_refined(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, int32_t H, int32_t W,
                        const wf_solve_opts& o, float* out_s, int32_t* iters_out, double* resid_out, cudaStream_t st,
                        wf::LaunchTimer* timer, const float* d0, const float* N0, const uint8_t* m0,
                        const float* A0) {
  wf_solve_opts first = o;
  first.tol = o.tol > 1e-5 ? o.tol : 1e-5;  // the FP32 iteration alone stops above its floor
  int32_t it = 0, total = 0;
  double rs = 0.0;
  wf_status r = solve_pass(d, Ndiag, mask, Pk, H, W, first, out_s, &it, &rs, st, timer);
  total += it;
  if (r != WF_OK && r != WF_ERR_NOT_CONVERGED) return r;
  const size_t n = size_t(H) * W, nm = size_t(H) * (W / 2 + 1);
  Carve cv;
  const size_t o_sc = cv.take<wf::Scalars>(1), o_dn = cv.take<float2>(n), o_rt = cv.take<float2>(n),
               o_e = cv.take<float>(n), o_nr = cv.take<double>(4), o_ln = cv.take<double>(kMaxLevels),
               o_fft = cv.take<char>(wf::refine_scratch_bytes(H, W));
  Scratch scr;
  scr.st = st;
  WF_CUDA(cudaMallocAsync(&scr.base, cv.off, st));
  char* b = static_cast<char*>(scr.base);
  auto* sc = reinterpret_cast<wf::Scalars*>(b + o_sc);
  k_prep<<<1, 1024, 0, st>>>(d, Ndiag, mask, Pk, H, W, o.tau, o.eta, sc);
  WF_CUDA(cudaGetLastError());
  k_tables<<<int((n + nm + 255) / 256), 256, 0, st>>>(d, Ndiag, mask, Pk, H, W, sc, nullptr,
                                                       reinterpret_cast<float2*>(b + o_dn), nullptr);
  WF_CUDA(cudaGetLastError());
  double* norms = reinterpret_cast<double*>(b + o_nr);
  wf::RefineArgs ra{};
  ra.H = H;
  ra.W = W;
  ra.d = d0;
  ra.Nd = N0;
  ra.mask = m0;
  ra.A = A0;
  ra.Pk = Pk;
  ra.s = out_s;
  ra.dn = reinterpret_cast<float2*>(b + o_dn);
  ra.rtab = reinterpret_cast<float2*>(b + o_rt);
  ra.rnorm = norms;
  ra.bnorm = norms + 1;
  ra.level_norms = reinterpret_cast<double*>(b + o_ln);
  ra.n_levels = kMaxLevels;
  ra.scratch = b + o_fft;
  cudaError_t e = wf::refine_bnorm(ra, st);
  if (e != cudaSuccess) return cuda_fail(e);
  wf_solve_opts corr = o;
  corr.tol = o.refine_tol;
  corr.init_s = nullptr;
  float* ev = reinterpret_cast<float*>(b + o_e);
  double rho = -1.0;
  wf_status status = WF_ERR_NOT_CONVERGED;
  for (int k = 0; k <= o.refine; ++k) {
    if ((e = wf::refine_residual(ra, st)) != cudaSuccess) return cuda_fail(e);
    double h[2];
    WF_CUDA(cudaMemcpyAsync(h, norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    WF_CUDA(cudaStreamSynchronize(st));
    rho = h[1] > 0.0 ? sqrt(h[0] / h[1]) : sqrt(h[0]);
    if (!(rho == rho)) { status = WF_ERR_NONFINITE; break; }
    if (rho < o.tol) { status = WF_OK; break; }
    if (k == o.refine) break;
    r = solve_pass(d, Ndiag, mask, Pk, H, W, corr, ev, &it, &rs, st, nullptr, ra.rtab, ra.level_norms);
    total += it;
    if (r != WF_OK && r != WF_ERR_NOT_CONVERGED) return r;
    if ((e = wf::refine_update(int(n), out_s, ev, st)) != cudaSuccess) return cuda_fail(e);
  }
  WF_CUDA(cudaStreamSynchronize(st));
  if (iters_out) *iters_out = total;
  if (resid_out) *resid_out = rho;
  return status;
}

}  // namespace

extern "C" {

wf_status wf_solve_ex(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, int32_t H, int32_t W,
                      const wf_solve_opts* opts, float* out_s, int32_t* iters_out, double* resid_out,
                      wf_stream_t stream) {
  wf_solve_opts o;
  wf_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!d || !Ndiag || !mask || !Pk || !out_s) return WF_ERR_ARG;
  if (!size_ok(H, W)) return WF_ERR_SHAPE;
  if (!(o.tol >= 0.0) || !(o.eta > 0.0 && o.eta < 1.0) || !(o.level_tol >= 0.0) || o.level_max < 1 || o.check < 1 ||
      o.max_iter < 1 || o.refine < 0 || (o.refine > 0 && !(o.refine_tol > 0.0)))
    return WF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const float* d0 = d;
  const float* N0 = Ndiag;
  const uint8_t* m0 = mask;
  Response resp;
  if (o.A) {
    WF_CUDA(apply_response(d, Ndiag, mask, o.A, size_t(H) * W, st, &resp));
    d = resp.d;
    Ndiag = resp.Nd;
    mask = resp.mask;
  }
  KernelTimer timer(st);
  const wf_status r = o.refine > 0 ? solve_refined(d, Ndiag, mask, Pk, H, W, o, out_s, iters_out, resid_out, st, &timer,
                                                   d0, N0, m0, o.A)
                                   : solve_pass(d, Ndiag, mask, Pk, H, W, o, out_s, iters_out, resid_out, st, &timer);
  timer.collect();
  return r;
}

wf_status wf_solve(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, int32_t H, int32_t W,
                   double tau, double tol, float* out_s, int32_t* iters_out, double* resid_out, wf_stream_t stream) {
  wf_solve_opts o;
  wf_solve_opts_default(&o);
  o.tau = tau;
  o.tol = tol;
  return wf_solve_ex(d, Ndiag, mask, Pk, H, W, &o, out_s, iters_out, resid_out, stream);
}

wf_status wf_sample_ex(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, int32_t H, int32_t W,
                       uint64_t seed, const wf_sample_opts* opts, float* out, wf_stream_t stream) {
  if (!opts) return WF_ERR_ARG;
  const wf_sample_opts o = *opts;
  if (!d || !Ndiag || !mask || !Pk) return WF_ERR_ARG;
  if (!size_ok(H, W)) return WF_ERR_SHAPE;
  if (o.n_samples < 0 || o.n_chains < 1 || o.burn_in < 0 || o.thin < 1) return WF_ERR_ARG;
  if (o.out_dtype < WF_OUT_F32 || o.out_dtype > WF_OUT_F16) return WF_ERR_ARG;
  if (o.n_samples == 0) return WF_OK;
  if (!out || !out_ptr_ok(out)) return WF_ERR_ARG;
  const long long sweeps = (long long)o.burn_in + o.n_samples * (long long)o.thin;
  if (sweeps > 0x7fffffffLL || o.n_samples > 0x7fffffffLL) return WF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Response resp;
  if (o.A) {
    WF_CUDA(apply_response(d, Ndiag, mask, o.A, size_t(H) * W, st, &resp));
    d = resp.d;
    Ndiag = resp.Nd;
    mask = resp.mask;
  }
  // 256 and 512: one cluster per chain when the device can host the cluster, else the field in global memory
  const bool cluster = use_cluster(H, o.n_chains);
  if (!size_on_chip(H) && !cluster) {
    KernelTimer gt(st);
    const wf_status r = sample_global(d, Ndiag, mask, Pk, H, W, seed, o, sweeps, out, st, &gt);
    gt.collect();
    return r;
  }
  const size_t n = size_t(H) * W, nm = size_t(H) * (W / 2 + 1);
  const size_t off_sc = 0, off_aq = align256(sizeof(wf::Scalars)), off_fg = off_aq + align256(n * sizeof(float2)),
               total = off_fg + align256(nm * sizeof(float2));
  Scratch scr;
  scr.st = st;
  WF_CUDA(cudaMallocAsync(&scr.base, total, st));
  char* b = static_cast<char*>(scr.base);
  auto* sc = reinterpret_cast<wf::Scalars*>(b + off_sc);
  auto* aq = reinterpret_cast<float2*>(b + off_aq);
  auto* fg = reinterpret_cast<float2*>(b + off_fg);
  k_prep<<<1, 1024, 0, st>>>(d, Ndiag, mask, Pk, H, W, o.tau, 0.5, sc);
  WF_CUDA(cudaGetLastError());
  k_tables<<<int((n + nm + 255) / 256), 256, 0, st>>>(d, Ndiag, mask, Pk, H, W, sc, aq, nullptr, fg,
                                                       cluster ? H / cluster_rows_of(H, 0) : 0,
                                                       cluster ? cluster_rows_of(H, 0) : 0);
  WF_CUDA(cudaGetLastError());
  wf::SampleArgs a{};
  a.aq = aq; a.fg = fg; a.sc = sc; a.init_s = o.init_s;
  a.init_stride = (o.init_s && o.init_per_chain) ? (long long)n : 0;
  a.out = out; a.n_samples = o.n_samples; a.n_chains = o.n_chains; a.n_sweeps = int(sweeps);
  a.burn_in = o.burn_in; a.thin = o.thin; a.chain0 = o.chain_offset; a.step0 = o.start_step;
  a.key0 = uint32_t(seed & 0xffffffffu); a.key1 = uint32_t(seed >> 32);
  a.out_dtype = o.out_dtype;
  KernelTimer timer(st);
  cudaError_t e = cudaSuccess;
  switch (H) {
    case 16: e = wf::launch_sample<16>(a, st, &timer); break;
    case 32: e = wf::launch_sample<32>(a, st, &timer); break;
    case 64: e = wf::launch_sample<64>(a, st, &timer); break;
    case 128: e = wf::launch_sample<128>(a, st, &timer); break;
    case 256:
    case 512: e = launch_csample_any(H, cluster_rows_of(H, 0), a, st, &timer); break;
  }
  if (e != cudaSuccess) return cuda_fail(e);
  wf::Scalars hsc;
  WF_CUDA(cudaMemcpyAsync(&hsc, sc, sizeof(hsc), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  timer.collect();
  return wf_status(hsc.status);
}

}  // extern "C"

namespace {
// bins in [-1, n_bins) and band powers finite and >= 0, else WF_ERR_ARG in sc->status
__global__ void k_check_band(const int32_t* __restrict__ bins, int nm, int n_bins, const float* __restrict__ P0,
                             wf::Scalars* sc) {
  bool bad = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nm + n_bins; i += gridDim.x * blockDim.x) {
    if (i < nm) {
      bad |= bins[i] < -1 || bins[i] >= n_bins;
    } else {
      const float p = P0[i - nm];
      bad |= !(p >= 0.0f) || !isfinite(p);
    }
  }
  if (bad && sc->status == 0) sc->status = WF_ERR_ARG;
}

// Plan of the hierarchical sampler's band sums. bmap, in the order of the mode tables (natural for cm = 0,
// else the column slot order of the cluster kernels with cm rows per CTA, mode_pos) = (bin, position):
// the modes the s-draw visits as themselves (every interior mode, and on the columns kx = 0 and W/2 the
// rows ky <= H/2, whose conjugates count through their mirror weight) with a bin get consecutive
// positions per bin, bins in order and modes in table order within a bin (so the sums run in the same
// order every call); the others get position -2. off[b] = first position of bin b; lo[j] = first bin
// summed by CTA j of a cluster of P (contiguous ranges of about equal mode counts).
__global__ void k_band_map(const int32_t* __restrict__ bins, int H, int W, int cm, int n_bins, int2* __restrict__ bmap,
                           int* __restrict__ cnt) {
  const int WH = W / 2 + 1, nm = H * WH;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nm; j += gridDim.x * blockDim.x) {
    const int ky = j / WH, kx = j % WH, b = bins[j];
    const bool counted = b >= 0 && b < n_bins && ((kx != 0 && kx != W / 2) || ky <= H / 2);
    bmap[mode_pos(j, H, W, cm)] = make_int2(b, counted ? -1 : -2);
    if (counted) atomicAdd(cnt + b, 1);
  }
}
__global__ void k_band_offsets(const int* __restrict__ cnt, int n_bins, int P, int* __restrict__ off,
                               int* __restrict__ lo) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int acc = 0;
  for (int b = 0; b < n_bins; ++b) {
    off[b] = acc;
    acc += cnt[b];
  }
  off[n_bins] = acc;
  int b = 0;
  for (int j = 0; j < P; ++j) {  // CTA j starts at the first bin whose modes begin at or after j/P of all
    const long long target = (long long)acc * j / P;
    while (b < n_bins && off[b] < target) ++b;
    lo[j] = b;
  }
  lo[P] = n_bins;
}
// one block per bin: the bin's counted modes in table order get positions off[b], off[b] + 1, ...
__global__ void k_band_positions(int nm, const int* __restrict__ off, int2* __restrict__ bmap) {
  __shared__ int wsum[8];
  const int b = blockIdx.x;
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  int base = off[b];
  for (int c = 0; c < nm; c += 256) {
    const int i = c + int(threadIdx.x);
    bool f = false;
    if (i < nm) {
      const int2 e = bmap[i];
      f = e.x == b && e.y == -1;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (l == 0) wsum[w] = __popc(bal);
    __syncthreads();
    int pre = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      pre += k < w ? wsum[k] : 0;
      tot += wsum[k];
    }
    if (f) bmap[i].y = base + pre + __popc(bal & ((1u << l) - 1u));
    base += tot;
    __syncthreads();  // wsum is rewritten in the next chunk
  }
}

// clusters of the hierarchical sampler at size H that can be resident at once
cudaError_t band_clusters_any(int H, int n_bins, int* n) {
  return H == 256 ? wf::csample_band_clusters<256, 64>(n_bins, n) : wf::csample_band_clusters<512, 32>(n_bins, n);
}

// largest number of bins of the hierarchical sampler at size H
int band_max_bins(int H) { return H <= 256 ? 256 : 512; }
}  // namespace

extern "C" {

wf_status wf_sample_band(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, const int32_t* bins,
                         int32_t n_bins, const float* P0, int32_t H, int32_t W, uint64_t seed,
                         const wf_sample_opts* opts, float* out, float* out_P, wf_stream_t stream) {
  if (!opts) return WF_ERR_ARG;
  const wf_sample_opts o = *opts;
  if (!d || !Ndiag || !mask || !Pk || !bins || (n_bins > 0 && !P0)) return WF_ERR_ARG;
  if (!size_ok(H, W) || H > 512) return WF_ERR_SHAPE;
  if (n_bins < 0 || n_bins > band_max_bins(H)) return WF_ERR_ARG;
  if (o.n_samples < 0 || o.n_chains < 1 || o.burn_in < 0 || o.thin < 1) return WF_ERR_ARG;
  if (o.out_dtype < WF_OUT_F32 || o.out_dtype > WF_OUT_F16) return WF_ERR_ARG;
  if (o.n_samples == 0) return WF_OK;
  if (!out || !out_ptr_ok(out) || (out_P && !out_ptr_ok(out_P))) return WF_ERR_ARG;
  const long long sweeps = (long long)o.burn_in + o.n_samples * (long long)o.thin;
  if (sweeps > 0x7fffffffLL || o.n_samples > 0x7fffffffLL) return WF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Response resp;  // a pixel response A: data d / A and noise N / A^2, A = 0 as missing (as wf_sample_ex)
  if (o.A) {
    WF_CUDA(apply_response(d, Ndiag, mask, o.A, size_t(H) * W, st, &resp));
    d = resp.d;
    Ndiag = resp.Nd;
    mask = resp.mask;
  }
  const size_t n = size_t(H) * W, nm = size_t(H) * (W / 2 + 1);
  // the band-sum plan, and one statistics buffer per field of the grid (up to 128^2) or per cluster (256
  // and 512: thread-block clusters, as many as can be resident, each looping over chains, with tables in
  // the cluster kernels' orders)
  const bool cluster = !size_on_chip(H);
  const int cm = cluster ? wf::cluster_rows(H) : 0, perm = cluster ? H / cm : 1;
  long long n_buf = 0;
  int n_cl = 0;
  if (cluster) {
    WF_CUDA(band_clusters_any(H, n_bins, &n_cl));
    if (n_cl < 1) return cuda_fail(cudaErrorNotSupported);
    if (n_cl > o.n_chains) n_cl = o.n_chains;
    n_buf = n_cl;
  } else {
    const int fpc = H >= 128 ? 1 : 128 / H;  // fields per CTA of k_sample_band
    n_buf = (o.n_chains + fpc - 1) / fpc * (long long)fpc;
  }
  Carve cv;
  const size_t off_sc = cv.take<wf::Scalars>(1), off_aq = cv.take<float2>(n), off_fg = cv.take<float2>(nm),
               off_map = cv.take<int2>(nm), off_cnt = cv.take<int>(n_bins + 1), off_off = cv.take<int>(n_bins + 1),
               off_lo = cv.take<int>(perm + 1), off_buf = cv.take<float2>(size_t(n_buf) * nm);
  Scratch scr;
  scr.st = st;
  WF_CUDA(cudaMallocAsync(&scr.base, cv.off, st));
  char* b = static_cast<char*>(scr.base);
  auto* sc = reinterpret_cast<wf::Scalars*>(b + off_sc);
  auto* aq = reinterpret_cast<float2*>(b + off_aq);
  auto* fg = reinterpret_cast<float2*>(b + off_fg);
  k_prep<<<1, 1024, 0, st>>>(d, Ndiag, mask, Pk, H, W, o.tau, 0.5, sc);
  WF_CUDA(cudaGetLastError());
  k_check_band<<<int((nm + n_bins + 255) / 256), 256, 0, st>>>(bins, int(nm), n_bins, P0, sc);
  WF_CUDA(cudaGetLastError());
  k_tables<<<int((n + nm + 255) / 256), 256, 0, st>>>(d, Ndiag, mask, Pk, H, W, sc, aq, nullptr, fg, perm, cm);
  WF_CUDA(cudaGetLastError());
  // the plan (built before k_check_band's status is read: invalid bins are never counted, and the
  // sampler does not run when that status is set)
  int2* bmap = reinterpret_cast<int2*>(b + off_map);
  int* band_off = reinterpret_cast<int*>(b + off_off);
  int* band_lo = reinterpret_cast<int*>(b + off_lo);
  int* cnt = reinterpret_cast<int*>(b + off_cnt);
  WF_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (n_bins + 1), st));
  k_band_map<<<int((nm + 255) / 256), 256, 0, st>>>(bins, H, W, cm, n_bins, bmap, cnt);
  k_band_offsets<<<1, 32, 0, st>>>(cnt, n_bins, perm, band_off, band_lo);
  if (n_bins > 0) k_band_positions<<<n_bins, 256, 0, st>>>(int(nm), band_off, bmap);
  WF_CUDA(cudaGetLastError());
  wf::SampleArgs a{};
  a.aq = aq; a.fg = fg; a.sc = sc; a.init_s = o.init_s;
  a.init_stride = (o.init_s && o.init_per_chain) ? (long long)n : 0;
  a.out = out; a.n_samples = o.n_samples; a.n_chains = o.n_chains; a.n_sweeps = int(sweeps);
  a.burn_in = o.burn_in; a.thin = o.thin; a.chain0 = o.chain_offset; a.step0 = o.start_step;
  a.key0 = uint32_t(seed & 0xffffffffu); a.key1 = uint32_t(seed >> 32);
  a.out_dtype = o.out_dtype;
  a.n_bins = n_bins; a.P0 = P0; a.out_P = out_P;
  a.band_map = bmap; a.band_off = band_off; a.band_lo = band_lo;
  a.band_buf = reinterpret_cast<float2*>(b + off_buf); a.band_clusters = n_cl;
  KernelTimer timer(st);
  cudaError_t e = cudaSuccess;
  switch (H) {
    case 16: e = wf::launch_sample_band<16>(a, st, &timer); break;
    case 32: e = wf::launch_sample_band<32>(a, st, &timer); break;
    case 64: e = wf::launch_sample_band<64>(a, st, &timer); break;
    case 128: e = wf::launch_sample_band<128>(a, st, &timer); break;
    case 256: e = wf::launch_csample_band<256, 64>(a, st, &timer); break;
    case 512: e = wf::launch_csample_band<512, 32>(a, st, &timer); break;
  }
  if (e != cudaSuccess) return cuda_fail(e);
  wf::Scalars hsc;
  WF_CUDA(cudaMemcpyAsync(&hsc, sc, sizeof(hsc), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  timer.collect();
  return wf_status(hsc.status);
}

}  // extern "C"

namespace {
// the spin-2 messenger variance: the smaller of the two components' minima (statuses combined)
__global__ void k_min_tau(wf::Scalars* a, const wf::Scalars* b, double tau_user) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (a->status == 0 && b->status != 0) a->status = b->status;
  if (a->status != 0) return;
  const double t = tau_user > 0.0 ? tau_user : fmin(a->tau, b->tau);
  a->tau = t;
  a->sqrt_tau = float(sqrt(t));
}
}  // namespace

extern "C" {

wf_status wf_sample_spin2(const float* d1, const float* d2, const float* N1, const float* N2, const uint8_t* mask,
                          const float* PE, const float* PB, int32_t H, int32_t W, uint64_t seed,
                          const wf_sample_opts* opts, float* out, wf_stream_t stream) {
  if (!opts) return WF_ERR_ARG;
  const wf_sample_opts o = *opts;
  if (!d1 || !d2 || !N1 || !N2 || !mask || !PE || !PB) return WF_ERR_ARG;
  if (!size_ok(H, W) || H > 512) return WF_ERR_SHAPE;
  if (o.n_samples < 0 || o.n_chains < 1 || o.burn_in < 0 || o.thin < 1) return WF_ERR_ARG;
  if (o.out_dtype < WF_OUT_F32 || o.out_dtype > WF_OUT_F16) return WF_ERR_ARG;
  if (o.n_samples == 0) return WF_OK;
  if (!out || !out_ptr_ok(out)) return WF_ERR_ARG;
  const long long sweeps = (long long)o.burn_in + o.n_samples * (long long)o.thin;
  if (sweeps > 0x7fffffffLL || o.n_samples > 0x7fffffffLL) return WF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Response r1, r2;  // one pixel response A for both components (the same mask results for both)
  if (o.A) {
    WF_CUDA(apply_response(d1, N1, mask, o.A, size_t(H) * W, st, &r1));
    WF_CUDA(apply_response(d2, N2, mask, o.A, size_t(H) * W, st, &r2));
    d1 = r1.d;
    N1 = r1.Nd;
    d2 = r2.d;
    N2 = r2.Nd;
    mask = r1.mask;
  }
  const size_t n = size_t(H) * W, nm = size_t(H) * (W / 2 + 1);
  Carve cv;
  const size_t o_sc = cv.take<wf::Scalars>(2), o_aq = cv.take<float2>(2 * n), o_fe = cv.take<float2>(nm),
               o_fb = cv.take<float2>(nm);
  Scratch scr;
  scr.st = st;
  WF_CUDA(cudaMallocAsync(&scr.base, cv.off, st));
  char* b = static_cast<char*>(scr.base);
  auto* sc = reinterpret_cast<wf::Scalars*>(b + o_sc);
  auto* aq = reinterpret_cast<float2*>(b + o_aq);
  auto* fgE = reinterpret_cast<float2*>(b + o_fe);
  auto* fgB = reinterpret_cast<float2*>(b + o_fb);
  // each component's set-up checks the caller's tau against its own noise (or finds its own minimum);
  // the pair then uses the caller's tau or the smaller minimum
  k_prep<<<1, 1024, 0, st>>>(d1, N1, mask, PE, H, W, o.tau, 0.5, sc);
  k_prep<<<1, 1024, 0, st>>>(d2, N2, mask, PB, H, W, o.tau, 0.5, sc + 1);
  k_min_tau<<<1, 32, 0, st>>>(sc, sc + 1, o.tau);
  WF_CUDA(cudaGetLastError());
  // 256 and 512: both components of a chain in one thread-block cluster of 32-row CTAs, tables in the
  // cluster kernels' orders
  const int cm = size_on_chip(H) ? 0 : 32, perm = cm ? H / cm : 0;
  k_tables<<<int((n + nm + 255) / 256), 256, 0, st>>>(d1, N1, mask, PE, H, W, sc, aq, nullptr, fgE, perm, cm);
  k_tables<<<int((n + nm + 255) / 256), 256, 0, st>>>(d2, N2, mask, PB, H, W, sc, aq + n, nullptr, fgB, perm, cm);
  WF_CUDA(cudaGetLastError());
  wf::Spin2Args a{};
  a.aq2 = aq; a.fgE = fgE; a.fgB = fgB; a.sc = sc; a.init_s = o.init_s;
  a.init_stride = (o.init_s && o.init_per_chain) ? 2 * (long long)n : 0;
  a.out = out; a.n_samples = o.n_samples; a.n_chains = o.n_chains; a.n_sweeps = int(sweeps);
  a.burn_in = o.burn_in; a.thin = o.thin; a.chain0 = o.chain_offset; a.step0 = o.start_step;
  a.key0 = uint32_t(seed & 0xffffffffu); a.key1 = uint32_t(seed >> 32);
  a.out_dtype = o.out_dtype;
  KernelTimer timer(st);
  cudaError_t e = cudaSuccess;
  switch (H) {
    case 16: e = wf::launch_sample_spin2<16>(a, st, &timer); break;
    case 32: e = wf::launch_sample_spin2<32>(a, st, &timer); break;
    case 64: e = wf::launch_sample_spin2<64>(a, st, &timer); break;
    case 128: e = wf::launch_sample_spin2<128>(a, st, &timer); break;
    case 256: e = wf::launch_csample_spin2<256, 32>(a, st, &timer); break;
    case 512: e = wf::launch_csample_spin2<512, 32>(a, st, &timer); break;
  }
  if (e != cudaSuccess) return cuda_fail(e);
  wf::Scalars hsc;
  WF_CUDA(cudaMemcpyAsync(&hsc, sc, sizeof(hsc), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  timer.collect();
  return wf_status(hsc.status);
}

}  // extern "C"

namespace {
// Wiener-filter tables of one shear component at level lambda for the spin-2 sweep: aq = ((1 - w) d, sqrt w)
// with w = N_bar / (N_bar + lambda tau), N_bar = N - tau (missing pixels: w = 1); fg = (f / n, 0) with
// f = P / (P + lambda tau) (no draws). perm, cm: the cluster kernels' table orders (k_tables), 0: natural.
__global__ void k_s2_level_tables(const float* __restrict__ d, const float* __restrict__ Nd,
                                  const uint8_t* __restrict__ mask, const float* __restrict__ Pk, int H, int W,
                                  const wf::Scalars* __restrict__ sc, double lam, float2* aq, float2* fg, int perm,
                                  int cm) {
  const int n = H * W, nm = H * (W / 2 + 1);
  const double tau = sc->tau, lt = lam * tau;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + nm; i += gridDim.x * blockDim.x) {
    if (i < n) {
      const int y = i / W, x = i % W;
      double a = 0.0, w = 1.0;
      if (mask[i] == 0) {
        const double nb = double(Nd[i]) - tau;
        w = nb / (nb + lt);
        a = (1.0 - w) * double(d[i]);
      }
      aq[x * H + table_row(y, H, perm)] = make_float2(float(a), float(sqrt(w)));
    } else {
      const int j = i - n;
      const double P = double(Pk[j]);
      fg[mode_pos(j, H, W, cm)] = make_float2(P > 0.0 ? float(P / (P + lt) / double(n)) : 0.0f, 0.0f);
    }
  }
}
__global__ void k_s2_quiet(const wf::Scalars* a, wf::Scalars* b) {  // the draws' scale set to zero
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *b = *a;
    b->sqrt_tau = 0.0f;
  }
}
}  // namespace

extern "C" {

wf_status wf_solve_spin2(const float* d1, const float* d2, const float* N1, const float* N2, const uint8_t* mask,
                         const float* PE, const float* PB, int32_t H, int32_t W, const wf_solve_opts* opts, float* out,
                         int32_t* iters_out, double* resid_out, wf_stream_t stream) {
  wf_solve_opts o;
  wf_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!d1 || !d2 || !N1 || !N2 || !mask || !PE || !PB || !out) return WF_ERR_ARG;
  if (!size_ok(H, W) || H > 512) return WF_ERR_SHAPE;
  if (!(o.tol > 0.0) || !(o.eta > 0.0 && o.eta < 1.0) || o.level_max < 1 || o.check < 1 || o.max_iter < 1)
    return WF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // a pixel response A (one for both components): the Wiener filter of (d / A, N / A^2, A = 0 as missing)
  // is that of the response problem, and so is its relative residual (both are A-weighted forms of the
  // same system), so the solve and its FP64 residual run on the transformed data
  Response r1, r2;
  if (o.A) {
    WF_CUDA(apply_response(d1, N1, mask, o.A, size_t(H) * W, st, &r1));
    WF_CUDA(apply_response(d2, N2, mask, o.A, size_t(H) * W, st, &r2));
    d1 = r1.d;
    N1 = r1.Nd;
    d2 = r2.d;
    N2 = r2.Nd;
    mask = r1.mask;
  }
  const size_t n = size_t(H) * W, nm = size_t(H) * (W / 2 + 1);
  Carve cv;
  const size_t o_sc = cv.take<wf::Scalars>(3), o_aq = cv.take<float2>(2 * n), o_fe = cv.take<float2>(nm),
               o_fb = cv.take<float2>(nm), o_r = cv.take<double>(2), o_x = cv.take<double2>(8 * n);
  Scratch scr;
  scr.st = st;
  WF_CUDA(cudaMallocAsync(&scr.base, cv.off, st));
  char* b = static_cast<char*>(scr.base);
  auto* sc = reinterpret_cast<wf::Scalars*>(b + o_sc);
  auto* aq = reinterpret_cast<float2*>(b + o_aq);
  auto* fgE = reinterpret_cast<float2*>(b + o_fe);
  auto* fgB = reinterpret_cast<float2*>(b + o_fb);
  auto* rn = reinterpret_cast<double*>(b + o_r);
  k_prep<<<1, 1024, 0, st>>>(d1, N1, mask, PE, H, W, o.tau, o.eta, sc);
  k_prep<<<1, 1024, 0, st>>>(d2, N2, mask, PB, H, W, o.tau, o.eta, sc + 1);
  k_min_tau<<<1, 32, 0, st>>>(sc, sc + 1, o.tau);
  k_s2_quiet<<<1, 32, 0, st>>>(sc, sc + 2);
  WF_CUDA(cudaGetLastError());
  wf::Scalars hs[2];
  WF_CUDA(cudaMemcpyAsync(hs, sc, 2 * sizeof(wf::Scalars), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaMemsetAsync(out, 0, 2 * n * sizeof(float), st));
  WF_CUDA(cudaMemsetAsync(rn, 0, 2 * sizeof(double), st));
  WF_CUDA(cudaStreamSynchronize(st));
  if (hs[0].status != WF_OK) return wf_status(hs[0].status);
  const double tau = hs[0].tau, pmax = hs[0].pmax > hs[1].pmax ? hs[0].pmax : hs[1].pmax;
  const double lam0 = pmax / tau > 1.0 ? pmax / tau : 1.0;
  cudaError_t e = wf::spin2_residual_f64(out, d1, d2, N1, N2, mask, PE, PB, H, W, true, rn, b + o_x, st);
  if (e != cudaSuccess) return cuda_fail(e);
  double hb[2];
  WF_CUDA(cudaMemcpyAsync(hb, rn, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  const double bnorm = hb[1];
  wf::Spin2Args a{};
  a.aq2 = aq; a.fgE = fgE; a.fgB = fgB; a.sc = sc + 2; a.init_s = out; a.init_stride = 0;
  a.out = out; a.n_samples = 1; a.n_chains = 1; a.burn_in = 0; a.thin = 1; a.out_dtype = 0;
  const int cm = size_on_chip(H) ? 0 : 32, perm = cm ? H / cm : 0;  // 256, 512: the cluster sampler's orders
  auto run = [&](double lam, int sweeps) -> wf_status {
    k_s2_level_tables<<<int((n + nm + 255) / 256), 256, 0, st>>>(d1, N1, mask, PE, H, W, sc, lam, aq, fgE, perm, cm);
    k_s2_level_tables<<<int((n + nm + 255) / 256), 256, 0, st>>>(d2, N2, mask, PB, H, W, sc, lam, aq + n, fgB, perm,
                                                                 cm);
    WF_CUDA(cudaGetLastError());
    a.n_sweeps = sweeps;
    a.thin = sweeps;  // the state after the last sweep is the only sample
    cudaError_t e2 = cudaSuccess;
    switch (H) {
      case 16: e2 = wf::launch_sample_spin2<16>(a, st, nullptr); break;
      case 32: e2 = wf::launch_sample_spin2<32>(a, st, nullptr); break;
      case 64: e2 = wf::launch_sample_spin2<64>(a, st, nullptr); break;
      case 128: e2 = wf::launch_sample_spin2<128>(a, st, nullptr); break;
      case 256: e2 = wf::launch_csample_spin2<256, 32>(a, st, nullptr); break;
      case 512: e2 = wf::launch_csample_spin2<512, 32>(a, st, nullptr); break;
    }
    if (e2 != cudaSuccess) return cuda_fail(e2);
    return WF_OK;
  };
  int iters = 0;
  wf_status r = WF_OK;
  for (int lev = 0; lev < wf::kMaxLevels; ++lev) {  // cooling levels above lambda = 1
    double lam = lam0;
    for (int j = 0; j < lev; ++j) lam = lam * o.eta > 1.0 ? lam * o.eta : 1.0;
    if (lam <= 1.0) break;
    if ((r = run(lam, o.level_max)) != WF_OK) return r;
    iters += o.level_max;
  }
  double rho = -1.0;
  wf_status status = WF_ERR_NOT_CONVERGED;
  while (iters < o.max_iter) {
    const int k = o.check < o.max_iter - iters ? o.check : o.max_iter - iters;
    if ((r = run(1.0, k)) != WF_OK) return r;
    iters += k;
    WF_CUDA(cudaMemsetAsync(rn, 0, sizeof(double), st));
    e = wf::spin2_residual_f64(out, d1, d2, N1, N2, mask, PE, PB, H, W, false, rn, b + o_x, st);
    if (e != cudaSuccess) return cuda_fail(e);
    double h;
    WF_CUDA(cudaMemcpyAsync(&h, rn, sizeof(double), cudaMemcpyDeviceToHost, st));
    WF_CUDA(cudaStreamSynchronize(st));
    rho = bnorm > 0.0 ? sqrt(h / bnorm) : sqrt(h);
    if (!(rho == rho)) { status = WF_ERR_NONFINITE; break; }
    if (rho < o.tol) { status = WF_OK; break; }
  }
  if (iters_out) *iters_out = iters;
  if (resid_out) *resid_out = rho;
  return status;
}

wf_status wf_shear_to_convergence(const float* gamma, int64_t n_fields, int32_t H, int32_t W, float* kappa,
                                  wf_stream_t stream) {
  if (!gamma || !kappa || n_fields < 0) return WF_ERR_ARG;
  if (!size_ok(H, W)) return WF_ERR_SHAPE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t n = size_t(H) * W;
  Scratch scr;
  scr.st = st;
  WF_CUDA(cudaMallocAsync(&scr.base, 4 * n * sizeof(double2), st));
  for (int64_t i = 0; i < n_fields; ++i) {
    const float* g = gamma + i * 2 * n;
    float* k = kappa + i * 2 * n;
    cudaError_t e = wf::shear_to_convergence_f64(g, g + n, H, W, k, k + n, scr.base, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  WF_CUDA(cudaStreamSynchronize(st));
  return WF_OK;
}

}  // extern "C"

namespace {
// a grid barrier that expects one arrival more than the grid: every CTA's wait runs out
__global__ void k_wait_timeout(wf::GridBar* bar) {
  wf::grid_barrier(bar, gridDim.x + 1);
}
}  // namespace

extern "C" {

wf_status wf_selftest_wait_timeout(int32_t n_blocks, double* elapsed_ms) {
  if (n_blocks < 1 || n_blocks > 1024) return WF_ERR_ARG;
  int dev = 0, sms = 0, per_sm = 0;
  WF_CUDA(cudaGetDevice(&dev));
  WF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  WF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wait_timeout, 32, 0));
  if ((long long)per_sm * sms < n_blocks) return WF_ERR_ARG;  // the grid must be co-resident
  cudaStream_t st;
  WF_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  wf::GridBar* bar = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  wf::GridBar hb{};
  float ms = 0.f;
  cudaError_t e = cudaMallocAsync(&bar, sizeof(wf::GridBar), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, sizeof(wf::GridBar), st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    void* args[] = {&bar};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_wait_timeout), dim3(n_blocks), dim3(32), args, 0, st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, bar, sizeof(hb), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (bar) cudaFreeAsync(bar, st);
  cudaStreamSynchronize(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (e != cudaSuccess) return cuda_fail(e);
  if (elapsed_ms) *elapsed_ms = ms;
  return hb.err ? wf_status(hb.err) : WF_OK;
}

wf_status wf_sample(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, int32_t H, int32_t W,
                    int64_t n_samples, uint64_t seed, float* out, wf_stream_t stream) {
  wf_sample_opts o;
  wf_sample_opts_default(&o);
  o.n_samples = n_samples;
  return wf_sample_ex(d, Ndiag, mask, Pk, H, W, seed, &o, out, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// batched form
// ---------------------------------------------------------------------------------------------
namespace {

cudaError_t launch_batch_any(int H, const wf::BatchArgs& b, cudaStream_t st) {
  switch (H) {
    case 16: return wf::launch_batch<16>(b, nullptr, st);
    case 32: return wf::launch_batch<32>(b, nullptr, st);
    case 64: return wf::launch_batch<64>(b, nullptr, st);
    case 128: return wf::launch_batch<128>(b, nullptr, st);
  }
  return cudaErrorInvalidValue;
}
cudaError_t batch_grid_any(int H, int n, int pct, int* g) {
  switch (H) {
    case 16: return wf::batch_grid<16>(n, pct, g);
    case 32: return wf::batch_grid<32>(n, pct, g);
    case 64: return wf::batch_grid<64>(n, pct, g);
    case 128: return wf::batch_grid<128>(n, pct, g);
  }
  return cudaErrorInvalidValue;
}
long long batch_slot_any(int H) {
  switch (H) {
    case 16: return wf::batch_slot_bytes<16>();
    case 32: return wf::batch_slot_bytes<32>();
    case 64: return wf::batch_slot_bytes<64>();
    case 128: return wf::batch_slot_bytes<128>();
  }
  return 0;
}

// Large images (H >= 256) of a batch: the images of a size class are split into chunks, and every chunk
// is one cooperative launch of k_gbatch with one field per image (see wf_gbatch.cuh). Per-field buffers:
// pixel tables aq, dn [n], mode table fg [nm], state Z and previous Wiener iterate [H][W/2].
// With `cluster` (256 and 512 where a cluster fits the device) the chunk is one k_cpipe launch instead:
// one thread-block cluster per image runs its level norms, cooled solve and samples with the field in
// distributed shared memory (Z unused).
struct GBChunk {
  int H = 0, stream = 0;
  bool cluster = false;
  int rows = 0;  // rows per CTA of the cluster kernels
  std::vector<int> items;  // batch item indices
  size_t o_fields = 0, o_idx = 0, o_sc = 0, o_state = 0, o_acc = 0, o_bn = 0, o_active = 0, o_bar = 0, o_tr = 0,
         o_tc = 0, o_tw = 0, o_data = 0, per_field = 0;
  size_t f_aq = 0, f_dn = 0, f_fg = 0, f_z = 0, f_prev = 0, f_pk = 0;
};

void layout_chunk(GBChunk& c, Carve& cv) {
  const int H = c.H, F = int(c.items.size());
  const size_t n = size_t(H) * H, nm = size_t(H) * (H / 2 + 1), nz = size_t(H) * (H / 2);
  c.o_fields = cv.take<wf::GBField>(F);
  c.o_idx = cv.take<int>(F);
  c.o_sc = cv.take<wf::Scalars>(F);
  c.o_state = cv.take<wf::GBState>(2 * size_t(F));
  c.o_acc = cv.take<double>(2 * size_t(F));
  c.o_bn = cv.take<double>(size_t(F) * wf::kMaxLevels);
  c.o_active = cv.take<int>(1);
  c.o_bar = cv.take<wf::GridBar>(1);
  c.o_tr = cv.take<float2>(H / 2);
  c.o_tc = cv.take<float2>(H);
  c.o_tw = cv.take<float2>(H / 2);
  Carve f;
  c.f_aq = f.take<float2>(n);
  c.f_dn = f.take<float2>(n);
  c.f_fg = f.take<float2>(nm);
  if (!c.cluster) c.f_z = f.take<float2>(nz);
  if (c.cluster) c.f_pk = f.take<float>(nm);  // P in the clusters' slot order
  c.f_prev = f.take<float2>(nz);
  c.per_field = f.off;
  c.o_data = cv.take<char>(c.per_field * size_t(F));
}

// device descriptors of a chunk's fields (host side, from the scratch base address)
std::vector<wf::GBField> chunk_fields(const GBChunk& c, const std::vector<wf::BatchItem>& items, char* b) {
  std::vector<wf::GBField> v(c.items.size());
  for (size_t f = 0; f < c.items.size(); ++f) {
    const wf::BatchItem& it = items[c.items[f]];
    char* base = b + c.o_data + f * c.per_field;
    wf::GBField& g = v[f];
    g.aq = reinterpret_cast<const float2*>(base + c.f_aq);
    g.dn = reinterpret_cast<const float2*>(base + c.f_dn);
    g.fg = reinterpret_cast<const float2*>(base + c.f_fg);
    g.Pk = c.cluster ? reinterpret_cast<const float*>(base + c.f_pk) : it.Pk;
    g.Z = c.cluster ? nullptr : reinterpret_cast<float2*>(base + c.f_z);
    g.prev = reinterpret_cast<float2*>(base + c.f_prev);
    g.out_wf = it.out_wf;
    g.out_samples = it.out_samples;
    g.chain = it.chain;
    g.key0 = uint32_t(it.seed & 0xffffffffu);
    g.key1 = uint32_t(it.seed >> 32);
    g.item = c.items[f];
  }
  return v;
}

// A size class up to 128 x 128 in the phased form (small_path 0): per-image set-up, tables, then one
// k_bsolve launch and one k_bsample launch over all its images. Per-image buffers: pixel tables aq, dn [n],
// mode table fg [nm], previous Wiener iterate [H][W/2], and s_W [n] for images without an out_wf.
struct SmallClass {
  int H = 0;
  std::vector<int> items;
  size_t o_fields = 0, o_idx = 0, o_sc = 0, o_bn = 0, o_order = 0, o_data = 0, per_field = 0;
  size_t f_aq = 0, f_dn = 0, f_fg = 0, f_prev = 0, f_sw = 0;
};

void layout_small(SmallClass& c, Carve& cv) {
  const int H = c.H, F = int(c.items.size());
  const size_t n = size_t(H) * H, nm = size_t(H) * (H / 2 + 1), nz = size_t(H) * (H / 2);
  c.o_fields = cv.take<wf::GBField>(F);
  c.o_idx = cv.take<int>(F);
  c.o_sc = cv.take<wf::Scalars>(F);
  c.o_bn = cv.take<double>(size_t(F) * wf::kMaxLevels);
  c.o_order = cv.take<int>(F);
  Carve f;
  c.f_aq = f.take<float2>(n);
  c.f_dn = f.take<float2>(n);
  c.f_fg = f.take<float2>(nm);
  c.f_prev = f.take<float2>(nz);
  c.f_sw = f.take<float>(n);
  c.per_field = f.off;
  c.o_data = cv.take<char>(c.per_field * size_t(F));
}

std::vector<wf::GBField> small_fields(const SmallClass& c, const std::vector<wf::BatchItem>& items, char* b) {
  std::vector<wf::GBField> v(c.items.size());
  for (size_t f = 0; f < c.items.size(); ++f) {
    const wf::BatchItem& it = items[c.items[f]];
    char* base = b + c.o_data + f * c.per_field;
    wf::GBField& g = v[f];
    g.aq = reinterpret_cast<const float2*>(base + c.f_aq);
    g.dn = reinterpret_cast<const float2*>(base + c.f_dn);
    g.fg = reinterpret_cast<const float2*>(base + c.f_fg);
    g.Pk = it.Pk;
    g.Z = nullptr;
    g.prev = reinterpret_cast<float2*>(base + c.f_prev);
    g.out_wf = it.out_wf ? it.out_wf : reinterpret_cast<float*>(base + c.f_sw);  // s_W always kept
    g.out_samples = it.out_samples;
    g.chain = it.chain;
    g.key0 = uint32_t(it.seed & 0xffffffffu);
    g.key1 = uint32_t(it.seed >> 32);
    g.item = c.items[f];
  }
  return v;
}

// per-field set-up: one block per field (as k_prep)
__global__ void k_prep_fields(const wf::BatchItem* __restrict__ items, const int* __restrict__ idx, int H,
                              double tau_user, double eta, wf::Scalars* sc) {
  const wf::BatchItem it = items[idx[blockIdx.x]];
  prep_block(it.d, it.Ndiag, it.mask, it.Pk, H, H, tau_user, eta, sc + blockIdx.x);
}

// per-field tables (as k_tables), grid-stride over fields x (n + nm)
// cm > 0 (cluster chunks, cm rows per CTA): the mode table in the clusters' slot order, and a copy of P in
// that order at the field's Pk (chunk scratch)
__global__ void k_tables_fields(const wf::BatchItem* __restrict__ items, const int* __restrict__ idx,
                                const wf::GBField* __restrict__ fields, const wf::Scalars* __restrict__ sc, int F,
                                int H, int perm, int cm = 0) {
  const long long n = (long long)H * H, nm = (long long)H * (H / 2 + 1), per = n + nm;
  const double inv_n = 1.0 / double(n);
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < per * F;
       g += (long long)gridDim.x * blockDim.x) {
    const int f = int(g / per);
    const long long i = g % per;
    const wf::Scalars s = sc[f];
    if (s.status != 0) continue;
    const wf::BatchItem it = items[idx[f]];
    const wf::GBField fd = fields[f];
    if (i < n) {
      const int y = int(i / H), x = int(i % H), ty = table_row(y, H, perm);
      float2 a2, d2;
      wf::table_pixel(it.d[i], it.Ndiag[i], it.mask[i] == 0, s.tau, &a2, &d2);
      const_cast<float2*>(fd.aq)[x * H + ty] = a2;
      const_cast<float2*>(fd.dn)[x * H + ty] = d2;
    } else {
      const int j = int(i - n), q = mode_pos(j, H, H, cm);
      const_cast<float2*>(fd.fg)[q] = wf::table_mode(it.Pk[j], s.tau, inv_n);
      if (cm) const_cast<float*>(fd.Pk)[q] = it.Pk[j];
    }
  }
}

// zero the schedule state, residual sums and level norms; active = F
__global__ void k_gb_init(wf::GBState* state, double* acc, double* bnorm, int* active, wf::GridBar* bar, int F) {
  const long long words = 2LL * F * (sizeof(wf::GBState) / 4);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < words; i += (long long)gridDim.x * blockDim.x)
    reinterpret_cast<int*>(state)[i] = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 2LL * F; i += (long long)gridDim.x * blockDim.x)
    acc[i] = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)F * wf::kMaxLevels;
       i += (long long)gridDim.x * blockDim.x)
    bnorm[i] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *active = F;
    bar->count = 0;
    bar->gen = 0;
    bar->err = 0;
    bar->pad = 0;
  }
}

cudaError_t launch_gbatch_any(int H, const wf::GBArgs& a, cudaStream_t st) {
  switch (H) {
    case 256: return wf::launch_gbatch<256>(a, st);
    case 512: return wf::launch_gbatch<512>(a, st);
    case 1024: return wf::launch_gbatch<1024>(a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_bsolve_any(int H, const wf::BSolveArgs& a, cudaStream_t st) {
  switch (H) {
    case 16: return wf::launch_bsolve<16>(a, st);
    case 32: return wf::launch_bsolve<32>(a, st);
    case 64: return wf::launch_bsolve<64>(a, st);
    case 128: return wf::launch_bsolve<128>(a, st);
  }
  return cudaErrorInvalidValue;
}
// fpc: images per sampler CTA, clamped to 1 .. 128 / H (0: 128 / H)
cudaError_t launch_bsample_any(int H, const wf::BSampleArgs& a, int fpc, cudaStream_t st) {
  if (fpc > 128 / H) fpc = 128 / H;
  switch (H) {
    case 16: return wf::launch_bsample<16>(a, fpc, st);
    case 32: return wf::launch_bsample<32>(a, fpc, st);
    case 64: return wf::launch_bsample<64>(a, fpc, st);
    case 128: return wf::launch_bsample<128>(a, fpc, st);
  }
  return cudaErrorInvalidValue;
}

// Solve order of a small size class: images by decreasing number of cooling levels (a cheap predictor
// of the solve's length), failed set-ups last. One CTA: counting sort over the level counts; the order
// within a count is arbitrary (every image's result is independent of it).
__global__ void k_order_by_levels(const wf::Scalars* __restrict__ sc, int F, int* order) {
  __shared__ int start[wf::kMaxLevels + 1];
  for (int b = threadIdx.x; b <= wf::kMaxLevels; b += blockDim.x) start[b] = 0;
  __syncthreads();
  auto bin = [&](int f) {
    const wf::Scalars s = sc[f];
    return s.status == 0 ? wf::kMaxLevels - s.n_levels : wf::kMaxLevels;  // more levels -> smaller bin
  };
  for (int f = threadIdx.x; f < F; f += blockDim.x) atomicAdd(&start[bin(f)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int b = 0; b <= wf::kMaxLevels; ++b) {
      const int c = start[b];
      start[b] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int f = threadIdx.x; f < F; f += blockDim.x) order[atomicAdd(&start[bin(f)], 1)] = f;
}

// the phased pipeline of one small size class on stream st (item table uploaded, descriptors in place)
wf_status run_small(const SmallClass& c, const wf::BatchItem* d_items, wf::BatchResult* d_res,
                    const wf_batch_opts& o, char* b, cudaStream_t st) {
  const int F = int(c.items.size()), H = c.H;
  auto* fields = reinterpret_cast<wf::GBField*>(b + c.o_fields);
  auto* idx = reinterpret_cast<int*>(b + c.o_idx);
  auto* sc = reinterpret_cast<wf::Scalars*>(b + c.o_sc);
  k_prep_fields<<<F, 1024, 0, st>>>(d_items, idx, H, o.tau, o.eta, sc);
  WF_CUDA(cudaGetLastError());
  const long long tab = (long long)F * (size_t(H) * H + size_t(H) * (H / 2 + 1));
  k_tables_fields<<<int((tab + 255) / 256 < 4096 ? (tab + 255) / 256 : 4096), 256, 0, st>>>(d_items, idx, fields,
                                                                                           sc, F, H, 0);
  WF_CUDA(cudaGetLastError());
  wf::BSolveArgs sa{};
  sa.fields = fields;
  sa.sc = sc;
  sa.res = d_res;
  sa.bnorm = reinterpret_cast<double*>(b + c.o_bn);
  sa.order = reinterpret_cast<const int*>(b + c.o_order);
  sa.F = F;
  k_order_by_levels<<<1, 1024, 0, st>>>(sc, F, reinterpret_cast<int*>(b + c.o_order));
  WF_CUDA(cudaGetLastError());
  sa.tol = o.tol;
  sa.eta = o.eta;
  sa.level_tol = o.level_tol;
  sa.max_iter = o.max_iter;
  sa.level_max = o.level_max;
  sa.check = o.check;
  cudaError_t e = launch_bsolve_any(H, sa, st);
  if (e != cudaSuccess) return cuda_fail(e);
  wf::BSampleArgs pa{};
  pa.fields = fields;
  pa.sc = sc;
  pa.F = F;
  pa.n_samples = o.n_samples;
  if ((e = launch_bsample_any(H, pa, o.small_fields_per_cta, st)) != cudaSuccess) return cuda_fail(e);
  return WF_OK;
}

// set-up and launch of one chunk on stream st (item table uploaded, descriptors in place)
wf_status run_chunk(const GBChunk& c, const wf::BatchItem* d_items, wf::BatchResult* d_res, const wf_batch_opts& o,
                    char* b, cudaStream_t st) {
  const int F = int(c.items.size()), H = c.H;
  auto* fields = reinterpret_cast<wf::GBField*>(b + c.o_fields);
  auto* idx = reinterpret_cast<int*>(b + c.o_idx);
  auto* sc = reinterpret_cast<wf::Scalars*>(b + c.o_sc);
  auto* state = reinterpret_cast<wf::GBState*>(b + c.o_state);
  auto* acc = reinterpret_cast<double*>(b + c.o_acc);
  auto* bn = reinterpret_cast<double*>(b + c.o_bn);
  auto* active = reinterpret_cast<int*>(b + c.o_active);
  auto* bar = reinterpret_cast<wf::GridBar*>(b + c.o_bar);
  k_prep_fields<<<F, 1024, 0, st>>>(d_items, idx, H, o.tau, o.eta, sc);
  WF_CUDA(cudaGetLastError());
  const long long tab = (long long)F * (size_t(H) * H + size_t(H) * (H / 2 + 1));
  k_tables_fields<<<int((tab + 255) / 256 < 4096 ? (tab + 255) / 256 : 4096), 256, 0, st>>>(
      d_items, idx, fields, sc, F, H, c.cluster ? H / c.rows : 0, c.cluster ? c.rows : 0);
  WF_CUDA(cudaGetLastError());
  if (c.cluster) {
    wf::CBArgs cb{};
    cb.fields = fields;
    cb.sc = sc;
    cb.res = d_res;
    cb.F = F;
    cb.tol = o.tol;
    cb.eta = o.eta;
    cb.level_tol = o.level_tol;
    cb.max_iter = o.max_iter;
    cb.level_max = o.level_max;
    cb.check = o.check;
    cb.n_samples = o.n_samples;
    const cudaError_t e = launch_cpipe_any(H, c.rows, cb, st, nullptr);
    if (e != cudaSuccess) return cuda_fail(e);
    return WF_OK;
  }
  const long long init_words = 2LL * F * 16;
  k_gb_init<<<int((init_words + 255) / 256 < 1024 ? (init_words + 255) / 256 : 1024), 256, 0, st>>>(state, acc, bn,
                                                                                                   active, bar, F);
  WF_CUDA(cudaGetLastError());
  k_twiddles<<<8, 256, 0, st>>>(H, H, reinterpret_cast<float2*>(b + c.o_tr), reinterpret_cast<float2*>(b + c.o_tc),
                                reinterpret_cast<float2*>(b + c.o_tw));
  WF_CUDA(cudaGetLastError());
  wf::GBArgs a{};
  a.fields = fields;
  a.sc = sc;
  a.state = state;
  a.acc = acc;
  a.bnorm = bn;
  a.res = d_res;
  a.active = active;
  a.bar = bar;
  a.tw_row = reinterpret_cast<float2*>(b + c.o_tr);
  a.tw_col = reinterpret_cast<float2*>(b + c.o_tc);
  a.tw_real = reinterpret_cast<float2*>(b + c.o_tw);
  a.F = F;
  a.tol = o.tol;
  a.eta = o.eta;
  a.level_tol = o.level_tol;
  a.max_iter = o.max_iter;
  a.level_max = o.level_max;
  a.check = o.check;
  a.n_samples = o.n_samples;
  a.grid_pct = o.large_grid_pct;
  const cudaError_t e = launch_gbatch_any(H, a, st);
  if (e != cudaSuccess) return cuda_fail(e);
  return WF_OK;
}

}  // namespace

extern "C" {

void wf_batch_opts_default(wf_batch_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tau = 0.0;
  o->tol = 1e-5;
  o->eta = 0.5;
  o->level_tol = 1e-2;
  o->level_max = 64;
  o->check = 4;
  o->max_iter = 20000;
  o->n_samples = 0;
  o->large_streams = 8;
}

}  // extern "C"

namespace {

const int kBatchSizes[7] = {16, 32, 64, 128, 256, 512, 1024};

// Host-side plan of a batch: validated items grouped by size class and the layout of its one scratch block.
struct BatchPlan {
  int n_items = 0;
  wf_batch_opts o{};
  std::vector<std::vector<int>> cls;
  std::vector<wf::BatchItem> dev_items;
  std::vector<int> order;
  size_t o_items = 0, o_order = 0, o_res = 0, o_q = 0, o_slot[4] = {0, 0, 0, 0}, bytes = 0;
  int nls = 0;                  // streams of the large-image chunks
  std::vector<GBChunk> chunks;  // large images: one cooperative launch each
  std::vector<SmallClass> small;  // phased small classes (small_path 0)
};

bool batch_opts_ok(const wf_batch_opts& o) {
  return o.tol >= 0.0 && o.eta > 0.0 && o.eta < 1.0 && o.level_max >= 1 && o.check >= 1 && o.max_iter >= 1 &&
         o.n_samples >= 0 && o.large_streams >= 1 && o.small_grid_pct >= 0 && o.small_grid_pct <= 100 &&
         o.large_grid_pct >= 0 && o.large_grid_pct <= 100 && (o.small_path == 0 || o.small_path == 1) &&
         (o.large_cluster_rows == 0 || o.large_cluster_rows == 32 || o.large_cluster_rows == 64) &&
         (o.small_fields_per_cta == 0 || o.small_fields_per_cta == 1 || o.small_fields_per_cta == 2 ||
          o.small_fields_per_cta == 4 || o.small_fields_per_cta == 8);
}

wf_status plan_batch(const wf_batch_item* items, int n_items, const wf_batch_opts& o, BatchPlan* p) {
  p->n_items = n_items;
  p->o = o;
  p->cls.assign(7, {});
  p->dev_items.resize(n_items);
  for (int i = 0; i < n_items; ++i) {
    const wf_batch_item& it = items[i];
    if (!it.d || !it.Ndiag || !it.mask || !it.Pk) return WF_ERR_ARG;
    if (!size_ok(it.H, it.W)) return WF_ERR_SHAPE;
    if (o.n_samples > 0 && !it.out_samples) return WF_ERR_ARG;
    int c = 0;
    while (kBatchSizes[c] != it.H) ++c;
    p->cls[c].push_back(i);
    p->dev_items[i] = wf::BatchItem{it.d, it.Ndiag, it.mask, it.Pk, it.out_wf, it.out_samples, it.seed, it.chain, it.H};
  }
  // one block: items, order, results, queues, per-class CTA slots, per-stream large scratch
  Carve cv;
  p->o_items = cv.take<wf::BatchItem>(n_items);
  p->o_order = cv.take<int>(n_items);
  p->o_res = cv.take<wf::BatchResult>(n_items);
  p->o_q = cv.take<int>(8);
  p->small.clear();
  for (int c = 0; c < 4; ++c) {
    if (p->cls[c].empty()) continue;
    if (o.small_path == 0) {
      SmallClass sc;
      sc.H = kBatchSizes[c];
      sc.items = p->cls[c];
      layout_small(sc, cv);
      p->small.push_back(std::move(sc));
      continue;
    }
    int grid = 0;
    cudaError_t e = batch_grid_any(kBatchSizes[c], int(p->cls[c].size()), o.small_grid_pct, &grid);
    if (e != cudaSuccess) return cuda_fail(e);
    p->o_slot[c] = cv.take<char>(size_t(grid) * size_t(batch_slot_any(kBatchSizes[c])));
  }
  // large images: each size class split into up to large_streams chunks, chunk k on stream k
  p->chunks.clear();
  p->nls = 0;
  for (int c = 4; c < 7; ++c) {
    const int nc = int(p->cls[c].size());
    if (!nc) continue;
    const int parts = o.large_streams < nc ? o.large_streams : nc;
    for (int k = 0; k < parts; ++k) {
      GBChunk ch;
      ch.H = kBatchSizes[c];
      ch.stream = k;
      for (int i = k * nc / parts; i < (k + 1) * nc / parts; ++i) ch.items.push_back(p->cls[c][i]);
      ch.cluster = use_cluster(ch.H, int(ch.items.size()), o.large_cluster_rows);
      ch.rows = cluster_rows_of(ch.H, o.large_cluster_rows);
      layout_chunk(ch, cv);
      p->chunks.push_back(std::move(ch));
    }
    if (parts > p->nls) p->nls = parts;
  }
  p->order.clear();
  for (int c = 0; c < 7; ++c) p->order.insert(p->order.end(), p->cls[c].begin(), p->cls[c].end());
  p->bytes = cv.off;
  return WF_OK;
}

// Streams and events of one recorded batch (destroyed after the work, or after the capture, has ended).
struct ForkJoin {
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> evs;
  ~ForkJoin() {
    for (auto e : evs) cudaEventDestroy(e);
    for (auto s2 : side) cudaStreamDestroy(s2);
  }
};

// Enqueue the whole batch on `st` (work counters and statuses reset, per-class persistent launches and
// the large-image pipelines forked over side streams, joined back into `st`). The item table and order
// must already be in the scratch block `b`.
wf_status record_batch(const BatchPlan& p, char* b, cudaStream_t st, ForkJoin& fj) {
  const wf_batch_opts& o = p.o;
  auto* d_items = reinterpret_cast<wf::BatchItem*>(b + p.o_items);
  auto* d_order = reinterpret_cast<int*>(b + p.o_order);
  auto* d_res = reinterpret_cast<wf::BatchResult*>(b + p.o_res);
  auto* d_q = reinterpret_cast<int*>(b + p.o_q);
  WF_CUDA(cudaMemsetAsync(d_q, 0, 8 * sizeof(int), st));
  WF_CUDA(cudaMemsetAsync(d_res, 0, p.n_items * sizeof(wf::BatchResult), st));
  cudaEvent_t ready;
  WF_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  fj.evs.push_back(ready);
  WF_CUDA(cudaEventRecord(ready, st));
  auto new_stream = [&](cudaStream_t* out) -> cudaError_t {
    cudaError_t e = cudaStreamCreateWithFlags(out, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    fj.side.push_back(*out);
    return cudaStreamWaitEvent(*out, ready, 0);
  };
  wf_status fail = WF_OK;
  for (size_t k = 0; k < p.small.size() && fail == WF_OK; ++k) {
    cudaStream_t s2;
    cudaError_t e = new_stream(&s2);
    if (e != cudaSuccess) { fail = cuda_fail(e); break; }
    fail = run_small(p.small[k], d_items, d_res, o, b, s2);
  }
  int offset = 0;
  for (int c = 0; c < 4 && fail == WF_OK && o.small_path == 1; ++c) {
    if (p.cls[c].empty()) continue;
    cudaStream_t s2;
    cudaError_t e = new_stream(&s2);
    if (e != cudaSuccess) { fail = cuda_fail(e); break; }
    wf::BatchArgs ba{};
    ba.items = d_items;
    ba.order = d_order + offset;
    ba.n = int(p.cls[c].size());
    ba.res = d_res;
    ba.queue = d_q + c;
    ba.scratch = b + p.o_slot[c];
    ba.slot_bytes = batch_slot_any(kBatchSizes[c]);
    ba.tau = o.tau;
    ba.tol = o.tol;
    ba.eta = o.eta;
    ba.level_tol = o.level_tol;
    ba.max_iter = o.max_iter;
    ba.level_max = o.level_max;
    ba.check = o.check;
    ba.n_samples = o.n_samples;
    ba.grid_pct = o.small_grid_pct;
    if ((e = launch_batch_any(kBatchSizes[c], ba, s2)) != cudaSuccess) fail = cuda_fail(e);
    offset += int(p.cls[c].size());
  }
  if (fail == WF_OK && p.nls) {
    std::vector<cudaStream_t> pool(p.nls);
    for (int k = 0; k < p.nls && fail == WF_OK; ++k) {
      cudaError_t e = new_stream(&pool[k]);
      if (e != cudaSuccess) fail = cuda_fail(e);
    }
    for (size_t k = 0; k < p.chunks.size() && fail == WF_OK; ++k) {
      const GBChunk& c = p.chunks[k];
      fail = run_chunk(c, d_items, d_res, o, b, pool[c.stream]);
    }
  }
  // join (also after a failure, so that a capture can end)
  for (auto s2 : fj.side) {
    cudaEvent_t done;
    if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) continue;
    fj.evs.push_back(done);
    cudaEventRecord(done, s2);
    cudaStreamWaitEvent(st, done, 0);
  }
  return fail;
}

// Item table, order and the large-image field descriptors into the scratch block. The host copies stay
// alive in `keep` until the stream has passed them.
wf_status upload_batch(const BatchPlan& p, char* b, cudaStream_t st, std::vector<std::vector<char>>& keep) {
  WF_CUDA(cudaMemcpyAsync(b + p.o_items, p.dev_items.data(), p.n_items * sizeof(wf::BatchItem), cudaMemcpyHostToDevice,
                          st));
  WF_CUDA(cudaMemcpyAsync(b + p.o_order, p.order.data(), p.n_items * sizeof(int), cudaMemcpyHostToDevice, st));
  for (const SmallClass& c : p.small) {
    const std::vector<wf::GBField> fv = small_fields(c, p.dev_items, b);
    keep.emplace_back(reinterpret_cast<const char*>(fv.data()),
                      reinterpret_cast<const char*>(fv.data()) + fv.size() * sizeof(wf::GBField));
    WF_CUDA(cudaMemcpyAsync(b + c.o_fields, keep.back().data(), keep.back().size(), cudaMemcpyHostToDevice, st));
    keep.emplace_back(reinterpret_cast<const char*>(c.items.data()),
                      reinterpret_cast<const char*>(c.items.data()) + c.items.size() * sizeof(int));
    WF_CUDA(cudaMemcpyAsync(b + c.o_idx, keep.back().data(), keep.back().size(), cudaMemcpyHostToDevice, st));
  }
  for (const GBChunk& c : p.chunks) {
    const std::vector<wf::GBField> fv = chunk_fields(c, p.dev_items, b);
    keep.emplace_back(reinterpret_cast<const char*>(fv.data()),
                      reinterpret_cast<const char*>(fv.data()) + fv.size() * sizeof(wf::GBField));
    WF_CUDA(cudaMemcpyAsync(b + c.o_fields, keep.back().data(), keep.back().size(), cudaMemcpyHostToDevice, st));
    keep.emplace_back(reinterpret_cast<const char*>(c.items.data()),
                      reinterpret_cast<const char*>(c.items.data()) + c.items.size() * sizeof(int));
    WF_CUDA(cudaMemcpyAsync(b + c.o_idx, keep.back().data(), keep.back().size(), cudaMemcpyHostToDevice, st));
  }
  return WF_OK;
}

// device results -> items[].status/iters/resid (after the stream has been synchronised)
wf_status batch_results(const std::vector<wf::BatchResult>& hres, wf_batch_item* items, int n_items) {
  wf_status first = WF_OK;
  for (int i = 0; i < n_items; ++i) {
    items[i].status = hres[i].status;
    items[i].iters = hres[i].iters;
    items[i].resid = hres[i].resid;
    if (first == WF_OK && hres[i].status != WF_OK) first = wf_status(hres[i].status);
  }
  return first;
}

}  // namespace

struct wf_batch_graph_s {
  BatchPlan plan;
  void* base = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~wf_batch_graph_s() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (base) cudaFree(base);
  }
};

extern "C" {

wf_status wf_batch_run(wf_batch_item* items, int32_t n_items, const wf_batch_opts* opts, wf_stream_t stream) {
  wf_batch_opts o;
  wf_batch_opts_default(&o);
  if (opts) o = *opts;
  if (n_items < 0 || (n_items > 0 && !items)) return WF_ERR_ARG;
  if (!batch_opts_ok(o)) return WF_ERR_ARG;
  if (n_items == 0) return WF_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  BatchPlan p;
  wf_status r = plan_batch(items, n_items, o, &p);
  if (r != WF_OK) return r;
  Scratch scr;
  scr.st = st;
  WF_CUDA(cudaMallocAsync(&scr.base, p.bytes, st));
  char* b = static_cast<char*>(scr.base);
  std::vector<std::vector<char>> keep;
  if ((r = upload_batch(p, b, st, keep)) != WF_OK) return r;
  wf_status fail;
  {
    ForkJoin fj;
    fail = record_batch(p, b, st, fj);
    std::vector<wf::BatchResult> hres(n_items);
    cudaError_t e = cudaMemcpyAsync(hres.data(), b + p.o_res, n_items * sizeof(wf::BatchResult),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (fail != WF_OK) return fail;
    if (e != cudaSuccess) return cuda_fail(e);
    return batch_results(hres, items, n_items);
  }
}

wf_status wf_batch_graph_create(const wf_batch_item* items, int32_t n_items, const wf_batch_opts* opts,
                                wf_batch_graph* out) {
  if (!out) return WF_ERR_ARG;
  *out = nullptr;
  wf_batch_opts o;
  wf_batch_opts_default(&o);
  if (opts) o = *opts;
  if (n_items < 1 || !items || !batch_opts_ok(o)) return WF_ERR_ARG;
  auto* g = new wf_batch_graph_s();
  wf_status r = plan_batch(items, n_items, o, &g->plan);
  cudaStream_t cs = nullptr;
  auto fail = [&](wf_status s) {
    if (cs) cudaStreamDestroy(cs);
    delete g;
    return s;
  };
  if (r != WF_OK) return fail(r);
  cudaError_t e = cudaMalloc(&g->base, g->plan.bytes);
  if (e != cudaSuccess) return fail(cuda_fail(e));
  if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return fail(cuda_fail(e));
  char* b = static_cast<char*>(g->base);
  std::vector<std::vector<char>> keep;
  if ((r = upload_batch(g->plan, b, cs, keep)) != WF_OK) return fail(r);
  if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return fail(cuda_fail(e));
  if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed)) != cudaSuccess) return fail(cuda_fail(e));
  {
    ForkJoin fj;
    r = record_batch(g->plan, b, cs, fj);
    e = cudaStreamEndCapture(cs, &g->graph);
  }
  if (r != WF_OK) return fail(r);
  if (e != cudaSuccess) return fail(cuda_fail(e));
  if ((e = cudaGraphInstantiate(&g->exec, g->graph, 0)) != cudaSuccess) return fail(cuda_fail(e));
  cudaStreamDestroy(cs);
  *out = g;
  return WF_OK;
}

wf_status wf_batch_graph_launch(wf_batch_graph g, wf_stream_t stream) {
  if (!g || !g->exec) return WF_ERR_ARG;
  WF_CUDA(cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)));
  return WF_OK;
}

wf_status wf_batch_graph_results(wf_batch_graph g, wf_batch_item* items, int32_t n_items, wf_stream_t stream) {
  if (!g || !items || n_items != g->plan.n_items) return WF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::vector<wf::BatchResult> hres(n_items);
  WF_CUDA(cudaMemcpyAsync(hres.data(), static_cast<char*>(g->base) + g->plan.o_res,
                          n_items * sizeof(wf::BatchResult), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  return batch_results(hres, items, n_items);
}

void wf_batch_graph_destroy(wf_batch_graph g) { delete g; }

wf_status wf_batch_autotune(const wf_batch_item* items, int32_t n_items, wf_batch_opts* opts, int32_t reps,
                            double* best_ms, wf_stream_t stream) {
  if (!opts || !items || n_items < 1 || reps < 1) return WF_ERR_ARG;
  if (!batch_opts_ok(*opts)) return WF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  bool has_large = false;
  for (int i = 0; i < n_items; ++i) has_large |= items[i].H > 128;
  cudaEvent_t e0, e1;
  WF_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError());
  }
  // time one candidate: capture, one warm-up replay, `reps` timed replays
  auto time_opts = [&](const wf_batch_opts& c, double* ms) -> wf_status {
    wf_batch_graph g = nullptr;
    wf_status r = wf_batch_graph_create(items, n_items, &c, &g);
    if (r != WF_OK) return r;
    cudaError_t e = cudaGraphLaunch(g->exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int k = 0; k < reps && e == cudaSuccess; ++k) e = cudaGraphLaunch(g->exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    wf_batch_graph_destroy(g);
    if (e != cudaSuccess) return cuda_fail(e);
    *ms = double(t) / reps;
    return WF_OK;
  };
  wf_batch_opts best = *opts;
  double best_t = 0.0;
  wf_status r = time_opts(best, &best_t);
  auto try_knob = [&](int32_t wf_batch_opts::*knob, std::initializer_list<int> vals) {
    for (int v : vals) {
      if (r != WF_OK) return;
      if (best.*knob == v) continue;
      wf_batch_opts c = best;
      c.*knob = v;
      double t = 0.0;
      r = time_opts(c, &t);
      if (r == WF_OK && t < best_t) {
        best_t = t;
        best = c;
      }
    }
  };
  bool has_512 = false;
  for (int i = 0; i < n_items; ++i) has_512 |= items[i].H == 512;
  if (has_large) {
    try_knob(&wf_batch_opts::large_grid_pct, {100, 50, 25, 12});
    try_knob(&wf_batch_opts::large_streams, {1, 2, 4, 8, 16});
  }
  if (has_512) try_knob(&wf_batch_opts::large_cluster_rows, {32, 64});
  bool has_small = false;
  for (int i = 0; i < n_items; ++i) has_small |= items[i].H <= 128;
  int min_small = 1024;
  for (int i = 0; i < n_items; ++i)
    if (items[i].H < min_small) min_small = items[i].H;
  if (has_small) {
    try_knob(&wf_batch_opts::small_path, {0, 1});
    if (best.small_path == 1) try_knob(&wf_batch_opts::small_grid_pct, {100, 50, 25});
    if (best.small_path == 0 && min_small < 128) try_knob(&wf_batch_opts::small_fields_per_cta, {1, 2, 4, 8});
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (r != WF_OK) return r;
  *opts = best;
  if (best_ms) *best_ms = best_t;
  return WF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// differentiation form: spectral powers and the log-likelihood gradient
// ---------------------------------------------------------------------------------------------
namespace {

// P = amp (k/k0)^slope, dP/damp = P/amp, dP/dslope = P ln(k/k0) on the half spectrum (FP64, rounded once),
// k = sqrt((ky/H)^2 + (kx/W)^2) with ky folded to [-1/2, 1/2); and N = alpha * sigma2 per pixel.
__global__ void k_psd(int H, int W, double amp, double slope, double k0, double alpha, const float* __restrict__ sigma2,
                      float* P, float* dPa, float* dPn, float* Nd) {
  const int WH = W / 2 + 1, nm = H * WH, n = H * W;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nm + n; i += gridDim.x * blockDim.x) {
    if (i < nm) {
      const int ky = i / WH, kx = i % WH;
      const double fy = double(ky < H / 2 ? ky : ky - H) / H, fx = double(kx) / W;
      const double k = sqrt(fy * fy + fx * fx);
      double p = 0.0, dn = 0.0;
      if (k > 0.0) {
        p = amp * pow(k / k0, slope);
        dn = p * log(k / k0);
      }
      P[i] = float(p);
      dPa[i] = float(p / amp);
      dPn[i] = float(dn);
    } else {
      const int j = i - nm;
      Nd[j] = float(alpha * double(sigma2[j]));
    }
  }
}

// x = (v - s) / N on observed pixels (0 on missing) and the FP64 sums
//   sums[0] += v x,  sums[1] += sigma2 x v,  sums[2] += sigma2 x^2   (observed pixels)
__global__ void k_xres(int n, const float* __restrict__ v, const float* __restrict__ s, const float* __restrict__ Nd,
                       const float* __restrict__ sigma2, const uint8_t* __restrict__ mask, float* x, double* sums) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float xi = 0.0f;
    if (mask[i] == 0) {
      xi = (v[i] - s[i]) / Nd[i];
      const double xd = xi, vd = v[i], s2 = sigma2[i];
      a0 += vd * xd;
      a1 += s2 * xd * vd;
      a2 += s2 * xd * xd;
    }
    x[i] = xi;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(sums + 0, a0);
    atomicAdd(sums + 1, a1);
    atomicAdd(sums + 2, a2);
  }
}

// Rademacher probe z (+-1 on observed pixels, 0 on missing): Philox stream 5, counter (i/4, probe, 0, 5),
// word i mod 4, sign from its top bit.
__global__ void k_rademacher(int n, uint32_t probe, uint32_t k0, uint32_t k1, const uint8_t* __restrict__ mask,
                             float* z) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n / 4; g += gridDim.x * blockDim.x) {
    const wf::u4 r = wf::philox4x32_10(wf::u4{uint32_t(g), probe, 0u, 5u}, k0, k1);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int i = 4 * g + e;
      z[i] = mask[i] ? 0.0f : ((w[e] >> 31) ? -1.0f : 1.0f);
    }
  }
}

// v = g - y (all pixels; y is 0 on missing ones) and sum[0] += sum_o sigma2 y x
__global__ void k_vjp_mix(int n, const float* __restrict__ g, const float* __restrict__ y, const float* __restrict__ x,
                          const float* __restrict__ sigma2, const uint8_t* __restrict__ mask, float* v, double* sum) {
  double a = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    v[i] = g[i] - y[i];
    if (mask[i] == 0) a += double(sigma2[i]) * double(y[i]) * double(x[i]);
  }
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(sum, a);
}

// weighted spectral power into device memory dout[n_fields * nw]
cudaError_t spectral_power_dev(const float* a, const float* b, float sgn, int n_fields, const float* w, int nw, int H,
                               int W, double* dout, cudaStream_t st) {
  if (size_on_chip(H)) {
    wf::WpowerArgs p{a, b, sgn, n_fields, w, nw, dout};
    switch (H) {
      case 16: return wf::launch_wpower<16>(p, st);
      case 32: return wf::launch_wpower<32>(p, st);
      case 64: return wf::launch_wpower<64>(p, st);
      case 128: return wf::launch_wpower<128>(p, st);
    }
    return cudaErrorInvalidValue;
  }
  // large images: mode 3 of the cooperative kernel (tables and twiddles in a scratch block)
  const size_t nz = size_t(H) * (W / 2);
  Carve cv;
  const size_t o_sc = cv.take<wf::Scalars>(1), o_bar = cv.take<wf::GridBar>(1), o_tr = cv.take<float2>(W / 2),
               o_tc = cv.take<float2>(H), o_tw = cv.take<float2>(W / 2), o_z = cv.take<float2>(nz * size_t(n_fields));
  void* base = nullptr;
  cudaError_t e = cudaMallocAsync(&base, cv.off, st);
  if (e != cudaSuccess) return e;
  char* bb = static_cast<char*>(base);
  wf::Scalars sc{};
  sc.status = 0;
  sc.n_levels = 1;
  sc.tau = 1.0;
  e = cudaMemcpyAsync(bb + o_sc, &sc, sizeof(sc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bb + o_bar, 0, sizeof(wf::GridBar), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dout, 0, sizeof(double) * size_t(n_fields) * nw, st);
  if (e == cudaSuccess) {
    k_twiddles<<<8, 256, 0, st>>>(H, W, reinterpret_cast<float2*>(bb + o_tr), reinterpret_cast<float2*>(bb + o_tc),
                                  reinterpret_cast<float2*>(bb + o_tw));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    wf::GlobalArgs g{};
    g.Z = reinterpret_cast<float2*>(bb + o_z);
    g.tw_row = reinterpret_cast<float2*>(bb + o_tr);
    g.tw_col = reinterpret_cast<float2*>(bb + o_tc);
    g.tw_real = reinterpret_cast<float2*>(bb + o_tw);
    g.sc = reinterpret_cast<wf::Scalars*>(bb + o_sc);
    g.bar = reinterpret_cast<wf::GridBar*>(bb + o_bar);
    g.mode = 3;
    g.n_fields = n_fields;
    g.va = a;
    g.vb = b;
    g.vsign = sgn;
    g.wts = w;
    g.nw = nw;
    g.wout = dout;
    e = launch_global_any(H, g, st, nullptr);
  }
  const cudaError_t e2 = cudaFreeAsync(base, st);
  return e != cudaSuccess ? e : e2;
}

}  // namespace

extern "C" {

wf_status wf_spectral_power(const float* a, const float* b, float sgn, int32_t n_fields, const float* w, int32_t nw,
                            int32_t H, int32_t W, double* out, wf_stream_t stream) {
  if (!a || !w || !out || n_fields < 0 || nw < 1 || nw > 4) return WF_ERR_ARG;
  if (!size_ok(H, W)) return WF_ERR_SHAPE;
  if (n_fields == 0) return WF_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Scratch scr;
  scr.st = st;
  WF_CUDA(cudaMallocAsync(&scr.base, sizeof(double) * size_t(n_fields) * nw, st));
  auto* dout = static_cast<double*>(scr.base);
  cudaError_t e = spectral_power_dev(a, b, sgn, n_fields, w, nw, H, W, dout, st);
  if (e != cudaSuccess) return cuda_fail(e);
  WF_CUDA(cudaMemcpyAsync(out, dout, sizeof(double) * size_t(n_fields) * nw, cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  return WF_OK;
}

wf_status wf_loglike_grad(const float* d, const float* sigma2, const uint8_t* mask, int32_t H, int32_t W,
                          const double* params, int32_t n_probes, uint64_t seed, double tol, double* out_quad,
                          double* out_grad_quad, double* out_grad, double* out_grad_var, float* out_wf,
                          wf_stream_t stream) {
  if (!d || !sigma2 || !mask || !params) return WF_ERR_ARG;
  if (!size_ok(H, W)) return WF_ERR_SHAPE;
  const double amp = params[0], slope = params[1], k0 = params[2], alpha = params[3];
  if (!(amp > 0.0) || !(k0 > 0.0) || !(alpha > 0.0) || !std::isfinite(slope) || n_probes < 0 || !(tol > 0.0))
    return WF_ERR_ARG;
  if (out_grad && n_probes < 1) return WF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t n = size_t(H) * W, nm = size_t(H) * (W / 2 + 1);
  Carve cv;
  const size_t o_P = cv.take<float>(3 * nm), o_N = cv.take<float>(n), o_s = cv.take<float>(n), o_x = cv.take<float>(n),
               o_z = cv.take<float>(n), o_w = cv.take<float>(n), o_sum = cv.take<double>(4),
               o_pow = cv.take<double>(8);
  Scratch scr;
  scr.st = st;
  WF_CUDA(cudaMallocAsync(&scr.base, cv.off, st));
  char* b = static_cast<char*>(scr.base);
  float* P = reinterpret_cast<float*>(b + o_P);
  float* dPa = P + nm;
  float* dPn = P + 2 * nm;
  float* Nd = reinterpret_cast<float*>(b + o_N);
  float* sW = out_wf ? out_wf : reinterpret_cast<float*>(b + o_s);
  float* x = reinterpret_cast<float*>(b + o_x);
  float* z = reinterpret_cast<float*>(b + o_z);
  float* wv = reinterpret_cast<float*>(b + o_w);
  double* sums = reinterpret_cast<double*>(b + o_sum);
  double* pw = reinterpret_cast<double*>(b + o_pow);
  const int nblk = int((nm + n + 255) / 256);
  k_psd<<<nblk < 1024 ? nblk : 1024, 256, 0, st>>>(H, W, amp, slope, k0, alpha, sigma2, P, dPa, dPn, Nd);
  WF_CUDA(cudaGetLastError());
  wf_solve_opts so;
  wf_solve_opts_default(&so);
  so.tol = tol;
  int32_t it = 0;
  double rs = 0.0;
  wf_status r = wf_solve_ex(d, Nd, mask, P, H, W, &so, sW, &it, &rs, stream);
  if (r != WF_OK) return r;
  // x = C^-1 d on observed pixels; Q = -1/2 d.x, dQ/dalpha = 1/2 sigma2 x.x
  WF_CUDA(cudaMemsetAsync(sums, 0, 4 * sizeof(double), st));
  const int xb = int((n + 255) / 256) < 1024 ? int((n + 255) / 256) : 1024;
  k_xres<<<xb, 256, 0, st>>>(int(n), d, sW, Nd, sigma2, mask, x, sums);
  WF_CUDA(cudaGetLastError());
  // dQ/d(amp, slope) = 1/2 sum_k dP |U x|^2
  cudaError_t e = spectral_power_dev(x, nullptr, 0.f, 1, dPa, 2, H, W, pw, st);
  if (e != cudaSuccess) return cuda_fail(e);
  double hs[4], hp[2];
  WF_CUDA(cudaMemcpyAsync(hs, sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaMemcpyAsync(hp, pw, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  const double gq[3] = {0.5 * hp[0], 0.5 * hp[1], 0.5 * hs[2]};
  if (out_quad) *out_quad = -0.5 * hs[0];
  if (out_grad_quad)
    for (int i = 0; i < 3; ++i) out_grad_quad[i] = gq[i];
  if (!out_grad && !out_grad_var) return WF_OK;
  // trace terms: t = z^T C^-1 dC z per probe, C^-1 z = N^-1 (z - s_W(z))
  // the probe solves only need an error far below the Monte-Carlo error of the trace estimate
  wf_solve_opts sp = so;
  sp.tol = tol > 1e-5 ? tol : 1e-5;
  sp.refine = 0;  // plain FP32 iteration: its error is far below the trace estimate's
  double tsum[3] = {0, 0, 0}, tsq[3] = {0, 0, 0};
  for (int j = 0; j < n_probes; ++j) {
    k_rademacher<<<int((n / 4 + 255) / 256), 256, 0, st>>>(int(n), uint32_t(j), uint32_t(seed & 0xffffffffu),
                                                          uint32_t(seed >> 32), mask, z);
    WF_CUDA(cudaGetLastError());
    r = wf_solve_ex(z, Nd, mask, P, H, W, &sp, wv, &it, &rs, stream);  // wv = s_W(z)
    if (r != WF_OK) return r;
    WF_CUDA(cudaMemsetAsync(sums, 0, 4 * sizeof(double), st));
    k_xres<<<xb, 256, 0, st>>>(int(n), z, wv, Nd, sigma2, mask, x, sums);  // x = C^-1 z
    WF_CUDA(cudaGetLastError());
    // w^T dS z = (|U(w+z)|^2_dP - |U(w-z)|^2_dP) / 4
    if ((e = spectral_power_dev(x, z, 1.f, 1, dPa, 2, H, W, pw, st)) != cudaSuccess) return cuda_fail(e);
    if ((e = spectral_power_dev(x, z, -1.f, 1, dPa, 2, H, W, pw + 2, st)) != cudaSuccess) return cuda_fail(e);
    double hq[4];
    WF_CUDA(cudaMemcpyAsync(hs, sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    WF_CUDA(cudaMemcpyAsync(hq, pw, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    WF_CUDA(cudaStreamSynchronize(st));
    const double t[3] = {0.25 * (hq[0] - hq[2]), 0.25 * (hq[1] - hq[3]), hs[1]};
    for (int i = 0; i < 3; ++i) {
      tsum[i] += t[i];
      tsq[i] += t[i] * t[i];
    }
  }
  for (int i = 0; i < 3; ++i) {
    const double mean = tsum[i] / n_probes;
    const double var = n_probes > 1 ? (tsq[i] - n_probes * mean * mean) / (n_probes - 1) : 0.0;
    if (out_grad) out_grad[i] = gq[i] - 0.5 * mean;
    if (out_grad_var) out_grad_var[i] = 0.25 * var / n_probes;
  }
  return WF_OK;
}

wf_status wf_loglike_grad_batch(wf_lik_item* items, int32_t n_items, int32_t n_probes, double tol,
                                wf_stream_t stream) {
  if (n_items < 0 || (n_items > 0 && !items) || n_probes < 0 || !(tol > 0.0)) return WF_ERR_ARG;
  for (int i = 0; i < n_items; ++i) {
    const wf_lik_item& it = items[i];
    if (!it.d || !it.sigma2 || !it.mask) return WF_ERR_ARG;
    if (!size_ok(it.H, it.W)) return WF_ERR_SHAPE;
    if (!(it.params[0] > 0.0) || !(it.params[2] > 0.0) || !(it.params[3] > 0.0) || !std::isfinite(it.params[1]))
      return WF_ERR_ARG;
  }
  if (n_items == 0) return WF_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // per item: P, dP/damp, dP/dslope [3 nm], N [n], s_W [n], x [n], sums [4], powers [2];
  // per item and probe: z [n], s_W(z) [n], sums [4], powers [4]
  Carve cv;
  std::vector<size_t> o_P(n_items), o_N(n_items), o_s(n_items), o_x(n_items), o_z(n_items), o_w(n_items);
  for (int i = 0; i < n_items; ++i) {
    const size_t n = size_t(items[i].H) * items[i].W, nm = size_t(items[i].H) * (items[i].W / 2 + 1);
    o_P[i] = cv.take<float>(3 * nm);
    o_N[i] = cv.take<float>(n);
    o_s[i] = cv.take<float>(n);
    o_x[i] = cv.take<float>(n);
    o_z[i] = cv.take<float>(n * size_t(n_probes));
    o_w[i] = cv.take<float>(n * size_t(n_probes));
  }
  const size_t o_sum = cv.take<double>(4 * size_t(n_items) * (1 + n_probes)),
               o_pow = cv.take<double>(4 * size_t(n_items) * (1 + n_probes));
  Scratch scr;
  scr.st = st;
  WF_CUDA(cudaMallocAsync(&scr.base, cv.off, st));
  char* b = static_cast<char*>(scr.base);
  double* sums = reinterpret_cast<double*>(b + o_sum);
  double* pws = reinterpret_cast<double*>(b + o_pow);
  WF_CUDA(cudaMemsetAsync(sums, 0, 4 * sizeof(double) * size_t(n_items) * (1 + n_probes), st));
  auto F = [&](size_t off) { return reinterpret_cast<float*>(b + off); };
  std::vector<wf_batch_item> fwd(n_items);
  for (int i = 0; i < n_items; ++i) {
    const wf_lik_item& it = items[i];
    const size_t n = size_t(it.H) * it.W, nm = size_t(it.H) * (it.W / 2 + 1);
    float* P = F(o_P[i]);
    const int nblk = int((nm + n + 255) / 256);
    k_psd<<<nblk < 1024 ? nblk : 1024, 256, 0, st>>>(it.H, it.W, it.params[0], it.params[1], it.params[2],
                                                     it.params[3], it.sigma2, P, P + nm, P + 2 * nm, F(o_N[i]));
    WF_CUDA(cudaGetLastError());
    wf_batch_item& bi = fwd[i];
    std::memset(&bi, 0, sizeof(bi));
    bi.d = it.d; bi.Ndiag = F(o_N[i]); bi.mask = it.mask; bi.Pk = P; bi.H = it.H; bi.W = it.W;
    bi.out_wf = F(o_s[i]);
  }
  wf_batch_opts bo;
  wf_batch_opts_default(&bo);
  bo.tol = tol;
  bo.n_samples = 0;
  wf_status r = wf_batch_run(fwd.data(), n_items, &bo, stream);
  if (r != WF_OK && r != WF_ERR_NOT_CONVERGED) {
    for (int i = 0; i < n_items; ++i) items[i].status = fwd[i].status;
    return r;
  }
  // x = C^-1 d; Q and dQ/dalpha from the sums, dQ/d(amp, slope) from weighted powers of x
  for (int i = 0; i < n_items; ++i) {
    const wf_lik_item& it = items[i];
    const size_t n = size_t(it.H) * it.W, nm = size_t(it.H) * (it.W / 2 + 1);
    const int xb = int((n + 255) / 256) < 1024 ? int((n + 255) / 256) : 1024;
    k_xres<<<xb, 256, 0, st>>>(int(n), it.d, F(o_s[i]), F(o_N[i]), it.sigma2, it.mask, F(o_x[i]), sums + 4 * i);
    WF_CUDA(cudaGetLastError());
    cudaError_t e = spectral_power_dev(F(o_x[i]), nullptr, 0.f, 1, F(o_P[i]) + nm, 2, it.H, it.W, pws + 4 * i, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  // probes: all images x probes as one batch of solves, C^-1 z = N^-1 (z - s_W(z))
  if (n_probes > 0) {
    std::vector<wf_batch_item> pr(size_t(n_items) * n_probes);
    for (int i = 0; i < n_items; ++i) {
      const wf_lik_item& it = items[i];
      const size_t n = size_t(it.H) * it.W;
      for (int j = 0; j < n_probes; ++j) {
        float* z = F(o_z[i]) + size_t(j) * n;
        k_rademacher<<<int((n / 4 + 255) / 256), 256, 0, st>>>(int(n), uint32_t(j), uint32_t(it.seed & 0xffffffffu),
                                                              uint32_t(it.seed >> 32), it.mask, z);
        WF_CUDA(cudaGetLastError());
        wf_batch_item& bi = pr[size_t(i) * n_probes + j];
        std::memset(&bi, 0, sizeof(bi));
        bi.d = z; bi.Ndiag = F(o_N[i]); bi.mask = it.mask; bi.Pk = F(o_P[i]); bi.H = it.H; bi.W = it.W;
        bi.out_wf = F(o_w[i]) + size_t(j) * n;
      }
    }
    wf_batch_opts bp = bo;
    bp.tol = tol > 1e-5 ? tol : 1e-5;
    r = wf_batch_run(pr.data(), int32_t(pr.size()), &bp, stream);
    if (r != WF_OK && r != WF_ERR_NOT_CONVERGED) return r;
    for (int i = 0; i < n_items; ++i) {
      const wf_lik_item& it = items[i];
      const size_t n = size_t(it.H) * it.W, nm = size_t(it.H) * (it.W / 2 + 1);
      const int xb = int((n + 255) / 256) < 1024 ? int((n + 255) / 256) : 1024;
      for (int j = 0; j < n_probes; ++j) {
        const size_t q = size_t(n_items) + size_t(i) * n_probes + j;
        float* z = F(o_z[i]) + size_t(j) * n;
        float* wv = F(o_w[i]) + size_t(j) * n;
        k_xres<<<xb, 256, 0, st>>>(int(n), z, wv, F(o_N[i]), it.sigma2, it.mask, F(o_x[i]), sums + 4 * q);
        WF_CUDA(cudaGetLastError());
        cudaError_t e = spectral_power_dev(F(o_x[i]), z, 1.f, 1, F(o_P[i]) + nm, 2, it.H, it.W, pws + 4 * q, st);
        if (e == cudaSuccess)
          e = spectral_power_dev(F(o_x[i]), z, -1.f, 1, F(o_P[i]) + nm, 2, it.H, it.W, pws + 4 * q + 2, st);
        if (e != cudaSuccess) return cuda_fail(e);
      }
    }
  }
  const size_t nq = size_t(n_items) * (1 + n_probes);
  std::vector<double> hs(4 * nq), hp(4 * nq);
  WF_CUDA(cudaMemcpyAsync(hs.data(), sums, 4 * nq * sizeof(double), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaMemcpyAsync(hp.data(), pws, 4 * nq * sizeof(double), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  wf_status first = WF_OK;
  for (int i = 0; i < n_items; ++i) {
    wf_lik_item& it = items[i];
    it.status = fwd[i].status;
    const double gq[3] = {0.5 * hp[4 * i], 0.5 * hp[4 * i + 1], 0.5 * hs[4 * i + 2]};
    it.quad = -0.5 * hs[4 * i];
    for (int k = 0; k < 3; ++k) it.grad_quad[k] = gq[k];
    if (n_probes > 0) {
      double tsum[3] = {0, 0, 0}, tsq[3] = {0, 0, 0};
      for (int j = 0; j < n_probes; ++j) {
        const size_t q = size_t(n_items) + size_t(i) * n_probes + j;
        const double t[3] = {0.25 * (hp[4 * q] - hp[4 * q + 2]), 0.25 * (hp[4 * q + 1] - hp[4 * q + 3]), hs[4 * q + 1]};
        for (int k = 0; k < 3; ++k) {
          tsum[k] += t[k];
          tsq[k] += t[k] * t[k];
        }
      }
      for (int k = 0; k < 3; ++k) {
        const double mean = tsum[k] / n_probes;
        const double var = n_probes > 1 ? (tsq[k] - n_probes * mean * mean) / (n_probes - 1) : 0.0;
        it.grad[k] = gq[k] - 0.5 * mean;
        it.grad_var[k] = 0.25 * var / n_probes;
      }
    }
    if (first == WF_OK && it.status != WF_OK) first = wf_status(it.status);
  }
  return first;
}

wf_status wf_wiener_vjp(const float* d, const float* sigma2, const uint8_t* mask, int32_t H, int32_t W,
                        const double* params, const float* g, const float* s_w_in, double tol, double* out_vjp,
                        float* out_wf, wf_stream_t stream) {
  if (!d || !sigma2 || !mask || !params || (g && !out_vjp)) return WF_ERR_ARG;
  if (!size_ok(H, W)) return WF_ERR_SHAPE;
  const double amp = params[0], slope = params[1], k0 = params[2], alpha = params[3];
  if (!(amp > 0.0) || !(k0 > 0.0) || !(alpha > 0.0) || !std::isfinite(slope) || !(tol > 0.0)) return WF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t n = size_t(H) * W, nm = size_t(H) * (W / 2 + 1);
  Carve cv;
  const size_t o_P = cv.take<float>(3 * nm), o_N = cv.take<float>(n), o_s = cv.take<float>(n), o_x = cv.take<float>(n),
               o_b = cv.take<float>(n), o_y = cv.take<float>(n), o_w = cv.take<float>(n), o_sum = cv.take<double>(4),
               o_pow = cv.take<double>(8), o_f64 = cv.take<double2>(2 * n);
  Scratch scr;
  scr.st = st;
  WF_CUDA(cudaMallocAsync(&scr.base, cv.off, st));
  char* b = static_cast<char*>(scr.base);
  float* P = reinterpret_cast<float*>(b + o_P);
  float* dPa = P + nm;
  float* dPn = P + 2 * nm;
  float* Nd = reinterpret_cast<float*>(b + o_N);
  float* sW = out_wf ? out_wf : reinterpret_cast<float*>(b + o_s);
  float* x = reinterpret_cast<float*>(b + o_x);
  float* bv = reinterpret_cast<float*>(b + o_b);
  float* y = reinterpret_cast<float*>(b + o_y);
  float* wv = reinterpret_cast<float*>(b + o_w);
  double* sums = reinterpret_cast<double*>(b + o_sum);
  double* pw = reinterpret_cast<double*>(b + o_pow);
  const int nblk = int((nm + n + 255) / 256);
  k_psd<<<nblk < 1024 ? nblk : 1024, 256, 0, st>>>(H, W, amp, slope, k0, alpha, sigma2, P, dPa, dPn, Nd);
  WF_CUDA(cudaGetLastError());
  wf_solve_opts so;
  wf_solve_opts_default(&so);
  so.tol = tol;
  if (tol < 1e-6) so.refine = 8;  // below the FP32 iteration's floor
  int32_t it = 0;
  double rs = 0.0;
  wf_status r = WF_OK;
  if (s_w_in) {
    if (s_w_in != sW) WF_CUDA(cudaMemcpyAsync(sW, s_w_in, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
  } else if ((r = wf_solve_ex(d, Nd, mask, P, H, W, &so, sW, &it, &rs, stream)) != WF_OK) {
    return r;
  }
  if (!g) {
    WF_CUDA(cudaStreamSynchronize(st));
    return WF_OK;
  }
  const int xb = int((n + 255) / 256) < 1024 ? int((n + 255) / 256) : 1024;
  WF_CUDA(cudaMemsetAsync(sums, 0, 4 * sizeof(double), st));
  k_xres<<<xb, 256, 0, st>>>(int(n), d, sW, Nd, sigma2, mask, x, sums);  // x = C^-1 d (0 on missing)
  WF_CUDA(cudaGetLastError());
  cudaError_t e = wf::apply_S_f64(g, P, H, W, bv, b + o_f64, st);    // b = S g
  if (e != cudaSuccess) return cuda_fail(e);
  if ((r = wf_solve_ex(bv, Nd, mask, P, H, W, &so, wv, &it, &rs, stream)) != WF_OK) return r;  // s_W(S g)
  k_xres<<<xb, 256, 0, st>>>(int(n), bv, wv, Nd, sigma2, mask, y, sums);  // y = C^-1 (S g)_o
  WF_CUDA(cudaGetLastError());
  WF_CUDA(cudaMemsetAsync(sums, 0, sizeof(double), st));
  k_vjp_mix<<<xb, 256, 0, st>>>(int(n), g, y, x, sigma2, mask, bv, sums);  // bv = g - y
  WF_CUDA(cudaGetLastError());
  // (g - y)^T dS x = (|U(x + v)|^2_dP - |U(x - v)|^2_dP) / 4
  if ((e = spectral_power_dev(x, bv, 1.f, 1, dPa, 2, H, W, pw, st)) != cudaSuccess) return cuda_fail(e);
  if ((e = spectral_power_dev(x, bv, -1.f, 1, dPa, 2, H, W, pw + 2, st)) != cudaSuccess) return cuda_fail(e);
  double hs, hq[4];
  WF_CUDA(cudaMemcpyAsync(&hs, sums, sizeof(double), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaMemcpyAsync(hq, pw, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  out_vjp[0] = 0.25 * (hq[0] - hq[2]);
  out_vjp[1] = 0.25 * (hq[1] - hq[3]);
  out_vjp[2] = -hs;
  return WF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// wf_sample_noalloc: the sampler with its scratch in a static device array instead of cudaMallocAsync,
// for callers that cannot allocate device memory when they call (real-time loops that cannot wait on the
// allocator, hosts whose device memory is all owned by their own pool or fixed in advance).
// ---------------------------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocBytes = 262144;  // tables of a 128 x 128 image: 256 + 131072 + 66560 bytes
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once per device. In host code
// the array's name is only a host-side stand-in, so the kernels must be given this address. The cached
// address belongs to the device's primary context: it does not survive cudaDeviceReset, after which the
// module is loaded again and the array may move (a process that resets a device must not call this
// entry point on it afterwards).
cudaError_t noalloc_scratch(void** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *ptr = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" {

wf_status wf_sample_noalloc(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, int32_t H,
                            int32_t W, uint64_t seed, const wf_sample_opts* opts, float* out, wf_stream_t stream) {
  if (!opts) return WF_ERR_ARG;
  const wf_sample_opts o = *opts;
  if (!d || !Ndiag || !mask || !Pk) return WF_ERR_ARG;
  if (!size_ok(H, W)) return WF_ERR_SHAPE;
  const size_t n = size_t(H) * W, nm = size_t(H) * (W / 2 + 1);
  const size_t off_aq = align256(sizeof(wf::Scalars)), off_fg = off_aq + align256(n * sizeof(float2)),
               total = off_fg + align256(nm * sizeof(float2));
  if (total > kNoAllocBytes) return WF_ERR_SHAPE;  // image too large for the static scratch array
  if (o.n_samples < 0 || o.n_chains < 1 || o.burn_in < 0 || o.thin < 1) return WF_ERR_ARG;
  if (o.A) return WF_ERR_ARG;  // the response needs transformed copies of the inputs (device memory)
  if (o.out_dtype < WF_OUT_F32 || o.out_dtype > WF_OUT_F16) return WF_ERR_ARG;
  if (o.n_samples == 0) return WF_OK;
  if (!out || !out_ptr_ok(out)) return WF_ERR_ARG;
  const long long sweeps = (long long)o.burn_in + o.n_samples * (long long)o.thin;
  if (sweeps > 0x7fffffffLL || o.n_samples > 0x7fffffffLL) return WF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  void* base = nullptr;
  WF_CUDA(noalloc_scratch(&base));
  char* b = static_cast<char*>(base);
  auto* sc = reinterpret_cast<wf::Scalars*>(b);
  auto* aq = reinterpret_cast<float2*>(b + off_aq);
  auto* fg = reinterpret_cast<float2*>(b + off_fg);
  // k_prep rewrites every field of sc and k_tables every table entry before the sampler reads them
  k_prep<<<1, 1024, 0, st>>>(d, Ndiag, mask, Pk, H, W, o.tau, 0.5, sc);
  WF_CUDA(cudaGetLastError());
  k_tables<<<int((n + nm + 255) / 256), 256, 0, st>>>(d, Ndiag, mask, Pk, H, W, sc, aq, nullptr, fg);
  WF_CUDA(cudaGetLastError());
  wf::SampleArgs a{};
  a.aq = aq; a.fg = fg; a.sc = sc; a.init_s = o.init_s;
  a.init_stride = (o.init_s && o.init_per_chain) ? (long long)n : 0;
  a.out = out; a.n_samples = o.n_samples; a.n_chains = o.n_chains; a.n_sweeps = int(sweeps);
  a.burn_in = o.burn_in; a.thin = o.thin; a.chain0 = o.chain_offset; a.step0 = o.start_step;
  a.key0 = uint32_t(seed & 0xffffffffu); a.key1 = uint32_t(seed >> 32);
  a.out_dtype = o.out_dtype;
  cudaError_t e = cudaSuccess;
  switch (H) {
    case 16: e = wf::launch_sample<16>(a, st, nullptr); break;
    case 32: e = wf::launch_sample<32>(a, st, nullptr); break;
    case 64: e = wf::launch_sample<64>(a, st, nullptr); break;
    case 128: e = wf::launch_sample<128>(a, st, nullptr); break;
  }
  if (e != cudaSuccess) return cuda_fail(e);
  wf::Scalars hsc;
  WF_CUDA(cudaMemcpyAsync(&hsc, sc, sizeof(hsc), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  return wf_status(hsc.status);
}

}  // extern "C"
