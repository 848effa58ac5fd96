// FP32 fused multiply-add throughput of the device, measured: the denominator of the FP32 roofline that
// the messenger-field transforms (5 n log2 n flops per sweep) are reported against. Every SM is filled
// with independent FMA chains (16 per thread, 2048 threads per SM), scalar FFMA or the paired FFMA2
// form, and the launch is timed with CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include "../../include/wf.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

__device__ float g_fma_sink;

// Each thread runs kChains independent recurrences x <- x a + b (float rounding makes every step
// necessary, so nothing can be folded); the sums are stored only under a condition the data never meet,
// which keeps the work live without a store per thread.
__global__ void __launch_bounds__(kThreads) k_fma_rate(long long iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = float(threadIdx.x) * 1e-3f + float(j);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == -1.0f) g_fma_sink = s;
}

// The same with the paired form: one FFMA2 instruction is two FP32 FMAs (per-lane rounding as fmaf).
__global__ void __launch_bounds__(kThreads) k_fma2_rate(long long iters, float a, float b) {
  float2 x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = make_float2(float(threadIdx.x) * 1e-3f + float(j), float(j) - 0.5f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = __ffma2_rn(x[j], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j].x + x[j].y;
  if (s == -1.0f) g_fma_sink = s;
}

}  // namespace

extern "C" {

wf_status wf_measure_fp32_peak(int32_t paired, int64_t iters, double* tflops_out, double* ms_out,
                               wf_stream_t stream) {
  if (iters < 1 || iters > (int64_t(1) << 40) || (paired != 0 && paired != 1)) return WF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    return WF_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, paired ? k_fma2_rate : k_fma_rate, kThreads, 0) !=
          cudaSuccess ||
      per_sm < 1)
    return WF_ERR_CUDA;
  const int blocks = sms * per_sm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return WF_ERR_CUDA;
  }
  cudaEventRecord(e0, st);
  // a = 1 - 2^-12 and b = 2^-4: every chain contracts towards b / (1 - a) = 256 and stays finite
  if (paired)
    k_fma2_rate<<<blocks, kThreads, 0, st>>>(iters, 0.999755859375f, 0.0625f);
  else
    k_fma_rate<<<blocks, kThreads, 0, st>>>(iters, 0.999755859375f, 0.0625f);
  cudaError_t e = cudaGetLastError();
  cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || !(ms > 0.f)) return WF_ERR_CUDA;
  const double fmas = double(blocks) * kThreads * double(iters) * kChains * (paired ? 2.0 : 1.0);
  if (tflops_out) *tflops_out = 2.0 * fmas / (double(ms) * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return WF_OK;
}

}  // extern "C"
