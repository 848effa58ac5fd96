// FP64 pieces of the mixed-precision iterative refinement of the Wiener filter:
//   * a batched radix-2 Stockham FFT in FP64 over rows or columns of a [H][W] complex array in global
//     memory (self-sorting, one kernel per stage; Govindaraju et al., "High performance discrete Fourier
//     transforms on graphics processors", SC'08);
//   * the refinement residual r = A N^-1 (d - A s) - S^-1 s of an FP32 iterate s and its norm ||S r||,
//     with S = U^dagger diag(P) U applied through the FP64 transforms (S^-1 only on modes with P > 0) and
//     A the diagonal pixel response (A = I unless given).
// The Wiener-filter equation (S^-1 + A N^-1 A) s = A N^-1 d (Eq. 2-3 with a diagonal response, N^-1 = 0
// on missing pixels) gives (I + S A N^-1 A) s - S A N^-1 d = -S r, so ||S r|| / ||S A N^-1 d|| is the
// relative residual used everywhere else in the library, here evaluated in FP64.
#include <cuda_runtime.h>

#include "wf_refine.h"

namespace wf {

namespace {

__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 dsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 dmul(double2 a, double2 w) {
  return make_double2(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}

// One radix-2 Stockham stage (sub-transform size Ns -> 2 Ns) of `batch` sequences of length n; element i
// of sequence b at [b * bstride + i * estride]. sign = -1 forward, +1 inverse (unnormalised).
__global__ void k_stockham2(const double2* __restrict__ in, double2* __restrict__ out, int n, int Ns, int batch,
                            long long bstride, long long estride, double sign) {
  const long long half = n / 2;
  const long long total = half * batch;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long b, j;
    if (estride == 1) {  // rows: consecutive threads walk along a sequence
      b = t / half;
      j = t % half;
    } else {  // columns: consecutive threads walk across sequences (coalesced)
      j = t / batch;
      b = t % batch;
    }
    const double2* x = in + b * bstride;
    double2* y = out + b * bstride;
    const double2 v0 = x[j * estride];
    double2 v1 = x[(j + half) * estride];
    const long long k = j % Ns;
    double sn, cs;
    sincospi(sign * double(k) / double(Ns), &sn, &cs);  // exp(sign * i pi k / Ns)
    v1 = dmul(v1, make_double2(cs, sn));
    const long long d = (j / Ns) * Ns * 2 + k;
    y[d * estride] = dadd(v0, v1);
    y[(d + Ns) * estride] = dsub(v0, v1);
  }
}

int ilog2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// s -> (s, 0) complex; rpix = A N^-1 (d - A s) on observed pixels with A != 0 (A = 1 when null), else 0
__global__ void k_ir_start(int n, const float* __restrict__ d, const float* __restrict__ Nd,
                           const uint8_t* __restrict__ mask, const float* __restrict__ A, const float* __restrict__ s,
                           double2* xs, double* rpix) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    xs[i] = make_double2(double(s[i]), 0.0);
    const double a = A ? double(A[i]) : 1.0;
    rpix[i] = (mask[i] || a == 0.0) ? 0.0 : a * (double(d[i]) - a * double(s[i])) / double(Nd[i]);
  }
}

// P on the full spectrum from the half table (P depends on |k|: (ky, kx) for kx > W/2 is (-ky, W - kx))
__device__ __forceinline__ double p_full(const float* __restrict__ Pk, int H, int W, int ky, int kx) {
  const int WH = W / 2 + 1;
  return kx <= W / 2 ? double(Pk[ky * WH + kx]) : double(Pk[((H - ky) % H) * WH + (W - kx)]);
}

// X <- X / (n P) on modes with P > 0, 0 elsewhere (forward then inverse unnormalised transforms give n).
// On the modes with P = 0 the residual s + S A N^-1 (A s - d) is s itself: out += sum |X|^2 / n there.
__global__ void k_ir_divp(int H, int W, const float* __restrict__ Pk, double2* X, double* out) {
  const int n = H * W;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double p = p_full(Pk, H, W, i / W, i % W);
    if (p > 0.0) {
      X[i] = make_double2(X[i].x / (double(n) * p), X[i].y / (double(n) * p));
    } else {
      acc += (X[i].x * X[i].x + X[i].y * X[i].y) / double(n);
      X[i] = make_double2(0.0, 0.0);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(out, acc);
}

// r = rpix - Re(q); xr = (r, 0); rtab[x*H + y] = (float(r), 1/N_bar) for the correction solve
__global__ void k_ir_finish(int H, int W, const double* __restrict__ rpix, const double2* __restrict__ q,
                            const float2* __restrict__ dn, double2* xr, float2* rtab) {
  const int n = H * W;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double r = rpix[i] - q[i].x;
    xr[i] = make_double2(r, 0.0);
    const int y = i / W, x = i % W;
    rtab[x * H + y] = make_float2(float(r), dn[x * H + y].y);
  }
}

// v -> (v, 0) with v = A N^-1 d on observed pixels with A != 0
__global__ void k_ir_rhs(int n, const float* __restrict__ d, const float* __restrict__ Nd,
                         const uint8_t* __restrict__ mask, const float* __restrict__ A, double2* x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double a = A ? double(A[i]) : 1.0;
    x[i] = make_double2((mask[i] || a == 0.0) ? 0.0 : a * double(d[i]) / double(Nd[i]), 0.0);
  }
}

// out += sum_k P_k^2 |X_k|^2 / n (full spectrum, unnormalised X)
__global__ void k_ir_pnorm(int H, int W, const float* __restrict__ Pk, const double2* __restrict__ X, double* out) {
  const int n = H * W;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double p = p_full(Pk, H, W, i / W, i % W);
    acc += p * p * (X[i].x * X[i].x + X[i].y * X[i].y);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc / double(n));
}

__global__ void k_fill(double* a, int n, const double* v) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = *v;
}

__global__ void k_add_f32(int n, float* s, const float* __restrict__ e) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s[i] += e[i];
}

int grid_for(long long n) {
  const long long g = (n + 255) / 256;
  return int(g < 2048 ? (g < 1 ? 1 : g) : 2048);
}

}  // namespace

cudaError_t fft2_f64(double2* a, double2* b, int H, int W, int sign, cudaStream_t st, double2** result) {
  double2* in = a;
  double2* out = b;
  const double sg = sign < 0 ? -1.0 : 1.0;
  for (int s = 0; s < ilog2i(W); ++s) {  // rows
    k_stockham2<<<grid_for((long long)H * W / 2), 256, 0, st>>>(in, out, W, 1 << s, H, W, 1, sg);
    double2* t = in;
    in = out;
    out = t;
  }
  for (int s = 0; s < ilog2i(H); ++s) {  // columns
    k_stockham2<<<grid_for((long long)H * W / 2), 256, 0, st>>>(in, out, H, 1 << s, W, 1, W, sg);
    double2* t = in;
    in = out;
    out = t;
  }
  *result = in;
  return cudaGetLastError();
}

size_t refine_scratch_bytes(int H, int W) {
  const size_t n = size_t(H) * W;
  return 2 * n * sizeof(double2) + n * sizeof(double) + 4 * sizeof(double) + 64;
}

cudaError_t refine_bnorm(const RefineArgs& a, cudaStream_t st) {
  const int n = a.H * a.W;
  double2* xa = reinterpret_cast<double2*>(a.scratch);
  double2* xb = xa + n;
  cudaError_t e = cudaMemsetAsync(a.bnorm, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  k_ir_rhs<<<grid_for(n), 256, 0, st>>>(n, a.d, a.Nd, a.mask, a.A, xa);
  double2* X = nullptr;
  if ((e = fft2_f64(xa, xb, a.H, a.W, -1, st, &X)) != cudaSuccess) return e;
  k_ir_pnorm<<<grid_for(n), 256, 0, st>>>(a.H, a.W, a.Pk, X, a.bnorm);
  return cudaGetLastError();
}

cudaError_t refine_residual(const RefineArgs& a, cudaStream_t st) {
  const int n = a.H * a.W;
  double2* xa = reinterpret_cast<double2*>(a.scratch);
  double2* xb = xa + n;
  double* rpix = reinterpret_cast<double*>(xb + n);
  cudaError_t e = cudaMemsetAsync(a.rnorm, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  k_ir_start<<<grid_for(n), 256, 0, st>>>(n, a.d, a.Nd, a.mask, a.A, a.s, xa, rpix);
  double2* X = nullptr;
  if ((e = fft2_f64(xa, xb, a.H, a.W, -1, st, &X)) != cudaSuccess) return e;
  k_ir_divp<<<grid_for(n), 256, 0, st>>>(a.H, a.W, a.Pk, X, a.rnorm);
  double2* other = X == xa ? xb : xa;
  double2* q = nullptr;
  if ((e = fft2_f64(X, other, a.H, a.W, +1, st, &q)) != cudaSuccess) return e;  // q = S^-1 s
  double2* xr = q == xa ? xb : xa;
  k_ir_finish<<<grid_for(n), 256, 0, st>>>(a.H, a.W, rpix, q, a.dn, xr, a.rtab);
  double2* other2 = xr == xa ? xb : xa;
  double2* R = nullptr;
  if ((e = fft2_f64(xr, other2, a.H, a.W, -1, st, &R)) != cudaSuccess) return e;
  k_ir_pnorm<<<grid_for(n), 256, 0, st>>>(a.H, a.W, a.Pk, R, a.rnorm);
  // every cooling level of the correction solve measures its residual against ||S r||
  k_fill<<<1, 64, 0, st>>>(a.level_norms, a.n_levels, a.rnorm);
  return cudaGetLastError();
}

namespace {

// X <- X P / n on the full spectrum (forward then inverse unnormalised transforms give n)
__global__ void k_ir_mulp(int H, int W, const float* __restrict__ Pk, double2* X) {
  const int n = H * W;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double p = p_full(Pk, H, W, i / W, i % W) / double(n);
    X[i] = make_double2(X[i].x * p, X[i].y * p);
  }
}

__global__ void k_ir_load(int n, const float* __restrict__ v, double2* x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x[i] = make_double2(double(v[i]), 0.0);
}

__global__ void k_ir_store(int n, const double2* __restrict__ x, float* v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = float(x[i].x);
}

}  // namespace

cudaError_t apply_S_f64(const float* v, const float* Pk, int H, int W, float* out, void* scratch, cudaStream_t st) {
  const int n = H * W;
  double2* xa = reinterpret_cast<double2*>(scratch);
  double2* xb = xa + n;
  k_ir_load<<<grid_for(n), 256, 0, st>>>(n, v, xa);
  double2* X = nullptr;
  cudaError_t e = fft2_f64(xa, xb, H, W, -1, st, &X);
  if (e != cudaSuccess) return e;
  k_ir_mulp<<<grid_for(n), 256, 0, st>>>(H, W, Pk, X);
  double2* q = nullptr;
  if ((e = fft2_f64(X, X == xa ? xb : xa, H, W, +1, st, &q)) != cudaSuccess) return e;
  k_ir_store<<<grid_for(n), 256, 0, st>>>(n, q, out);
  return cudaGetLastError();
}

namespace {

// rotation (c, s) of the Kaiser-Squires operator at full-spectrum mode (ky, kx), as in the samplers
__device__ __forceinline__ void ks_rot_d(int H, int W, int ky, int kx, double& c, double& s) {
  const int y = ky < H / 2 ? ky : ky - H, x = kx < W / 2 ? kx : kx - W;
  if ((x == 0 && y == 0) || ky == H / 2 || kx == W / 2) {
    c = 1.0;
    s = 0.0;
    return;
  }
  const double k1 = x, k2 = y, r = 1.0 / (k1 * k1 + k2 * k2);
  c = (k1 * k1 - k2 * k2) * r;
  s = 2.0 * k1 * k2 * r;
}

// (A, B) <- (c A + s B, -s A + c B) / n on the full spectra
__global__ void k_ks_inverse(int H, int W, double2* A, double2* B) {
  const int n = H * W;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double c, s;
    ks_rot_d(H, W, i / W, i % W, c, s);
    const double2 a = A[i], b = B[i];
    A[i] = make_double2((c * a.x + s * b.x) / n, (c * a.y + s * b.y) / n);
    B[i] = make_double2((-s * a.x + c * b.x) / n, (-s * a.y + c * b.y) / n);
  }
}

}  // namespace

cudaError_t shear_to_convergence_f64(const float* g1, const float* g2, int H, int W, float* kE, float* kB, void* scratch,
                                     cudaStream_t st) {
  const int n = H * W;
  double2* a0 = reinterpret_cast<double2*>(scratch);
  double2* a1 = a0 + n;
  double2* b0 = a1 + n;
  double2* b1 = b0 + n;
  k_ir_load<<<grid_for(n), 256, 0, st>>>(n, g1, a0);
  k_ir_load<<<grid_for(n), 256, 0, st>>>(n, g2, b0);
  double2 *A = nullptr, *B = nullptr;
  cudaError_t e = fft2_f64(a0, a1, H, W, -1, st, &A);
  if (e == cudaSuccess) e = fft2_f64(b0, b1, H, W, -1, st, &B);
  if (e != cudaSuccess) return e;
  k_ks_inverse<<<grid_for(n), 256, 0, st>>>(H, W, A, B);
  double2 *ka = nullptr, *kb = nullptr;
  if ((e = fft2_f64(A, A == a0 ? a1 : a0, H, W, +1, st, &ka)) != cudaSuccess) return e;
  if ((e = fft2_f64(B, B == b0 ? b1 : b0, H, W, +1, st, &kb)) != cudaSuccess) return e;
  k_ir_store<<<grid_for(n), 256, 0, st>>>(n, ka, kE);
  k_ir_store<<<grid_for(n), 256, 0, st>>>(n, kb, kB);
  return cudaGetLastError();
}

namespace {

// G_c = (g_c, 0); V_c = (g_c - d_c) / N_c on observed pixels (b: V_c = d_c / N_c, G = 0)
__global__ void k_s2_load(int n, const float* __restrict__ g, const float* __restrict__ d1,
                          const float* __restrict__ d2, const float* __restrict__ N1, const float* __restrict__ N2,
                          const uint8_t* __restrict__ mask, int rhs, double2* G1, double2* G2, double2* V1,
                          double2* V2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double a = rhs ? 0.0 : double(g[i]), b = rhs ? 0.0 : double(g[n + i]);
    G1[i] = make_double2(a, 0.0);
    G2[i] = make_double2(b, 0.0);
    const bool obs = mask[i] == 0;
    V1[i] = make_double2(obs ? (rhs ? double(d1[i]) : a - double(d1[i])) / double(N1[i]) : 0.0, 0.0);
    V2[i] = make_double2(obs ? (rhs ? double(d2[i]) : b - double(d2[i])) / double(N2[i]) : 0.0, 0.0);
  }
}

// out += sum_k |G_k + S V_k|^2 / n with S V = rotate(P_E e, P_B b), (e, b) = rotate^T V
__global__ void k_s2_norm(int H, int W, const float* __restrict__ PE, const float* __restrict__ PB,
                          const double2* __restrict__ G1, const double2* __restrict__ G2,
                          const double2* __restrict__ V1, const double2* __restrict__ V2, double* out) {
  const int n = H * W;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int ky = i / W, kx = i % W;
    double c, s;
    ks_rot_d(H, W, ky, kx, c, s);
    const double pe = p_full(PE, H, W, ky, kx), pb = p_full(PB, H, W, ky, kx);
    const double2 v1 = V1[i], v2 = V2[i];
    const double2 e = make_double2(pe * (c * v1.x + s * v2.x), pe * (c * v1.y + s * v2.y));
    const double2 b = make_double2(pb * (-s * v1.x + c * v2.x), pb * (-s * v1.y + c * v2.y));
    const double2 r1 = make_double2(G1[i].x + c * e.x - s * b.x, G1[i].y + c * e.y - s * b.y);
    const double2 r2 = make_double2(G2[i].x + s * e.x + c * b.x, G2[i].y + s * e.y + c * b.y);
    acc += (r1.x * r1.x + r1.y * r1.y + r2.x * r2.x + r2.y * r2.y) / double(n);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

}  // namespace

cudaError_t spin2_residual_f64(const float* g, const float* d1, const float* d2, const float* N1, const float* N2,
                               const uint8_t* mask, const float* PE, const float* PB, int H, int W, bool with_b,
                               double* out, void* scratch, cudaStream_t st) {
  const int n = H * W;
  double2* x = reinterpret_cast<double2*>(scratch);  // 4 arrays and their ping-pong partners
  cudaError_t e = cudaSuccess;
  for (int pass = 0; pass < (with_b ? 2 : 1) && e == cudaSuccess; ++pass) {
    const int rhs = pass;  // pass 0: the residual of g; pass 1: the right-hand side S N^-1 d
    k_s2_load<<<grid_for(n), 256, 0, st>>>(n, g, d1, d2, N1, N2, mask, rhs, x, x + 2 * n, x + 4 * n, x + 6 * n);
    double2* F[4];
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = fft2_f64(x + 2 * k * n, x + (2 * k + 1) * n, H, W, -1, st, &F[k]);
    if (e != cudaSuccess) break;
    k_s2_norm<<<grid_for(n), 256, 0, st>>>(H, W, PE, PB, F[0], F[1], F[2], F[3], out + pass);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t refine_update(int n, float* s, const float* e, cudaStream_t st) {
  k_add_f32<<<grid_for(n), 256, 0, st>>>(n, s, e);
  return cudaGetLastError();
}

}  // namespace wf
