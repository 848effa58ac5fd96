// FP64 iterative-refinement helpers of the Wiener filter (see wf_refine.cu).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace wf {

struct RefineArgs {
  int H, W;
  const float* d;
  const float* Nd;       // noise variance (observed pixels)
  const uint8_t* mask;
  const float* A;        // diagonal pixel response of d = A s + n, or null for A = I
  const float* Pk;       // [H][W/2+1]
  const float* s;        // current FP32 iterate [H][W]
  const float2* dn;      // Wiener-filter pixel table [W][H] (d, 1/N_bar)
  float2* rtab;          // out: correction right-hand-side table [W][H] (r, 1/N_bar)
  double* rnorm;         // out: ||S r||^2
  double* bnorm;         // out (refine_bnorm): ||S N^-1 d||^2
  double* level_norms;   // out: rnorm copied into n_levels entries
  int n_levels;
  void* scratch;         // refine_scratch_bytes(H, W)
};

// forward (sign = -1) or inverse (+1) unnormalised 2D FFT of a [H][W] complex FP64 array; a and b are
// ping-pong buffers, *result points to the one holding the transform
cudaError_t fft2_f64(double2* a, double2* b, int H, int W, int sign, cudaStream_t st, double2** result);

size_t refine_scratch_bytes(int H, int W);
cudaError_t refine_bnorm(const RefineArgs& a, cudaStream_t st);
cudaError_t refine_residual(const RefineArgs& a, cudaStream_t st);
cudaError_t refine_update(int n, float* s, const float* e, cudaStream_t st);
// (kappa_E, kappa_B) of a shear pair by the inverse Kaiser-Squires rotation; scratch: 4 H W double2
cudaError_t shear_to_convergence_f64(const float* g1, const float* g2, int H, int W, float* kE, float* kB, void* scratch,
                                     cudaStream_t st);
// spin-2 Wiener-filter residual in FP64: out[0] += ||g + S N^-1 (g - d)||^2 (g = (g1, g2), the shear
// covariance S of the E/B spectra), out[1] += ||S N^-1 d||^2 (when with_b); scratch: 8 H W double2
cudaError_t spin2_residual_f64(const float* g, const float* d1, const float* d2, const float* N1, const float* N2,
                               const uint8_t* mask, const float* PE, const float* PB, int H, int W, bool with_b,
                               double* out, void* scratch, cudaStream_t st);
// out = S v = U^dagger diag(P) U v in FP64 (rounded once to float); scratch: 2 H W double2
cudaError_t apply_S_f64(const float* v, const float* Pk, int H, int W, float* out, void* scratch, cudaStream_t st);

}  // namespace wf
