// Fused messenger-field Gibbs step (Alg. 1 of the paper, A = I) with the field resident in shared memory.
//
// One field (one chain of one image, N x N pixels, N in {16, 32, 64, 128}) is owned by N threads and
// one shared-memory buffer holding the packed half-spectrum [H][W/2] (float2, row stride W/2 + 1):
//   element (y, 0) packs the real kx = 0 and kx = W/2 values as (re, im); (y, kx) is kx otherwise.
//
// A sweep is two passes, each ending in a CTA barrier:
//   column pass (thread = column c, role r = parity of ky):
//       radix-2 split on load -> in-register FFT of length H/2 -> Fourier-space draw
//       s_hat = f t_hat + g zeta for every mode it holds (Alg. 1 s-update, Philox stream 1)
//       -> inverse FFT -> radix-2 twiddle -> store
//   row pass (thread = row y):
//       radix-2 combine on load -> C2R row transform -> s (real row in registers) -> [write sample]
//       -> pixel draw t = w s + (1 - w) d + sqrt(tau w) xi (Alg. 1 t-update, Philox stream 0)
//       -> R2C row transform -> store
// Scale factors of the unnormalised transforms are folded into the Fourier-space coefficients:
// f' = f / n and g' = g / sqrt(2 n) (per real component of an interior mode).
#pragma once

#include <cmath>
#include <cstdint>
#include <limits>
#include <type_traits>

#include "wf_math.cuh"

namespace wf {

template <int I>
using ic = std::integral_constant<int, I>;
template <class F, int... I>
WF_HD void sfor_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(ic<I>{}), ...);
}
// compile-time loop: f(ic<0>), ..., f(ic<N-1>)
template <int N, class F>
WF_HD void sfor(F&& f) {
  sfor_impl(f, std::make_integer_sequence<int, N>{});
}

#if defined(__CUDA_ARCH__)
#define WF_LDG(p) __ldg(p)
#else
#define WF_LDG(p) (*(p))
#endif

WF_HD float wf_rcp(float x) {
#if defined(__CUDA_ARCH__)
  return __frcp_rn(x);
#else
  return 1.0f / x;
#endif
}
// a / b with the fast device division (about 2 ulp); used where a few ulp do not matter
WF_HD float wf_fdiv(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fdividef(a, b);
#else
  return a / b;
#endif
}
// 1 / sqrt(x) for x > 0 (hardware approximation on the device)
WF_HD float wf_rsqrt(float x) {
#if defined(__CUDA_ARCH__)
  return rsqrtf(x);
#else
  return 1.0f / std::sqrt(x);
#endif
}
WF_HD float wf_inf() {
#if defined(__CUDA_ARCH__)
  return __int_as_float(0x7f800000);
#else
  return std::numeric_limits<float>::infinity();
#endif
}

template <int N_>
struct Geo {
  static constexpr int N = N_, H = N_, W = N_;
  static constexpr int LR = N / 2;  // complex length of a row transform
  static constexpr int LC = N / 2;  // half length of a column (radix-2 split)
  static constexpr int SP = LR + 1;  // float2 stride of a spectrum row in shared memory
  static constexpr int STG = W + 2;  // float stride of a staged real row (= the spectrum row's span)
  static constexpr int SPEC_BYTES = H * SP * 8;
  static constexpr int STG_BYTES = H * STG * 4;
  static constexpr int FIELD_BYTES = ((SPEC_BYTES > STG_BYTES ? SPEC_BYTES : STG_BYTES) + 15) / 16 * 16;
  static constexpr int WH = W / 2 + 1;  // columns of the [H][W/2+1] mode tables
};

// Per-call scalars computed on the device by the set-up kernel.
struct Scalars {
  double tau;      // messenger variance T = tau I (Alg. 1: min observed noise variance)
  double lam0;     // first lambda-cooling level
  double pmax;     // max_k P_k
  float sqrt_tau;
  int n_levels;    // number of cooling levels including lambda = 1
  int status;      // wf_status of the set-up; kernels do nothing unless 0
  int pad;
};

// Result of one Wiener-filter solve.
struct SolveStatus {
  double resid;
  int iters;
  int status;
};

// ---------------------------------------------------------------------------------------------
// set-up arithmetic (FP64, once per call)
// ---------------------------------------------------------------------------------------------
constexpr int kMaxLevels = 64;

// tau, lambda_0 and the number of cooling levels from the reductions over the inputs.
// lambda_j = max(1, lambda_0 eta^j); the last level (index n_levels - 1) is lambda = 1.
WF_HD Scalars make_scalars(float min_obs, int n_obs, float pmax, int bad, int neg, double tau_user, double eta) {
  Scalars r{};
  r.status = 0;
  if (bad) r.status = 6;       // WF_ERR_NONFINITE
  else if (neg) r.status = 1;  // WF_ERR_ARG
  double tau;
  if (tau_user > 0.0) {
    tau = tau_user;
    if (n_obs > 0 && tau_user > double(min_obs) && r.status == 0) r.status = 2;  // WF_ERR_TAU
  } else {
    tau = n_obs > 0 ? double(min_obs) : (pmax > 0.0f ? double(pmax) : 1.0);
  }
  r.tau = tau;
  r.sqrt_tau = float(sqrt(tau));
  r.pmax = double(pmax);
  r.lam0 = fmax(1.0, double(pmax) / tau);
  int levels = 1;
  double lam = r.lam0;
  while (lam > 1.0 && levels < kMaxLevels) {
    lam = fmax(1.0, lam * eta);
    ++levels;
  }
  r.n_levels = levels;
  return r;
}

// lambda of cooling level lev. eta^lev by binary powers (at most a dozen FP64 products): every thread of a
// CTA evaluates this at each level change, and the library pow() is a long FP64 instruction sequence on a
// GPU whose FP64 rate is a small fraction of its FP32 rate.
WF_HD double level_lambda(const Scalars& sc, int lev, double eta) {
  if (lev >= sc.n_levels - 1) return 1.0;
  double p = 1.0, b = eta;
  for (int e = lev; e > 0; e >>= 1) {
    if (e & 1) p *= b;
    b *= b;
  }
  return fmax(1.0, sc.lam0 * p);
}

// correctly rounded FP32 division, reciprocal and square root (IEEE round to nearest even)
WF_HD float fdiv_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fdiv_rn(a, b);
#else
  return a / b;
#endif
}
WF_HD float fsqrt_rn(float a) {
#if defined(__CUDA_ARCH__)
  return __fsqrt_rn(a);
#else
  return std::sqrt(a);
#endif
}

// per-pixel tables of pixel i = y*W + x, stored at x*H + y:
//   aq = ((1 - w) d, sqrt(w)) with w = N_bar/(tau + N_bar)  (sampler, lambda = 1; w = 1, a = 0 if missing)
//   dn = (d, 1/N_bar)                                        (Wiener filter; (0, 0) if missing)
// N_bar = N - tau is formed by one FP64 subtraction (exact for a tau taken from the data) and rounded once;
// since tau + N_bar = N, w = N_bar / N and 1 - w = tau / N, each from one correctly rounded FP32 division,
// so every entry is within 2 ulp of its exact value (FP64 division and square root, run per pixel, would
// cost tens of FP64 instructions each on a GPU whose FP64 rate is a small fraction of its FP32 rate).
WF_HD void table_pixel(float dv_in, float nv, bool obs, double tau, float2* aq, float2* dn) {
  float a = 0.0f, wgt = 1.0f, dv = 0.0f, inb = 0.0f;
  if (obs) {
    dv = dv_in;
    const float nbar = float(double(nv) - tau);  // >= 0 since tau <= min observed Ndiag
    wgt = fdiv_rn(nbar, nv);
    a = fdiv_rn(float(tau), nv) * dv;
    inb = nbar > 0.0f ? fdiv_rn(1.0f, nbar) : wf_inf();
  }
  *aq = make_float2(a, fsqrt_rn(wgt));
  *dn = make_float2(dv, inb);
}

// per-mode sampler table: (f / n, g / sqrt(2 n)), f = P/(P + tau), g^2 = P tau/(P + tau) = f tau (Alg. 1);
// correctly rounded FP32 operations (1/n and 1/(2n) are powers of two), within 2 ulp of the exact values
WF_HD float2 table_mode(float Pv, double tau, double inv_n) {
  if (!(Pv > 0.0f)) return make_float2(0.0f, 0.0f);
  const float t = float(tau), in = float(inv_n);
  const float f = fdiv_rn(Pv, Pv + t);
  return make_float2(f * in, fsqrt_rn(f * t * (0.5f * in)));
}

// ---------------------------------------------------------------------------------------------
// shared-memory passes (lt = thread index within the field, in [0, N))
// ---------------------------------------------------------------------------------------------
template <int N>
WF_HD void row_load_spec(const float2* S, int lt, float2 (&c)[N / 2]) {
  using G = Geo<N>;
  const int col = lt % G::LC, r = lt / G::LC;
  const float2* e = S + col * G::SP;
  const float2* o = S + (col + G::LC) * G::SP;
  if (r == 0) {
#pragma unroll
    for (int k = 0; k < G::LR; ++k) c[k] = cadd(e[k], o[k]);
  } else {
#pragma unroll
    for (int k = 0; k < G::LR; ++k) c[k] = csub(e[k], o[k]);
  }
}

template <int N>
WF_HD void row_store_spec(float2* S, int y, const float2 (&c)[N / 2]) {
  using G = Geo<N>;
#pragma unroll
  for (int k = 0; k < G::LR; ++k) S[y * G::SP + k] = c[k];
}

// c[m] = (t[2m], t[2m+1]) -> packed half-spectrum row
template <int N>
WF_HD void row_forward(float2 (&c)[N / 2]) {
  fft<N / 2, false>(c);
  r2c_post_all<N / 2>(c, std::make_integer_sequence<int, N / 2>{});
}

// column load with the radix-2 decimation-in-frequency split; x[k'] -> Y[2k' + r] after fft
template <int N>
WF_HD void col_load(const float2* S, int lt, float2 (&x)[N / 2]) {
  using G = Geo<N>;
  const int col = lt % G::LC, r = lt / G::LC;
  if (r == 0) {
#pragma unroll
    for (int n = 0; n < G::LC; ++n) x[n] = cadd(S[n * G::SP + col], S[(n + G::LC) * G::SP + col]);
  } else {
    sfor<G::LC>([&](auto I) {
      constexpr int n = decltype(I)::value;
      x[n] = twiddle<n, G::H, false>(csub(S[n * G::SP + col], S[(n + G::LC) * G::SP + col]));
    });
  }
}

// after the inverse column transform: store e[n] (r = 0, rows [0, LC)) or exp(+2 pi i n / H) * o[n]
// (r = 1, rows [LC, H)); x holds the transform already.
template <int N>
WF_HD void col_store_inv(float2* S, int lt, const float2 (&x)[N / 2]) {
  using G = Geo<N>;
  const int col = lt % G::LC, r = lt / G::LC;
  if (r == 0) {
#pragma unroll
    for (int n = 0; n < G::LC; ++n) S[n * G::SP + col] = x[n];
  } else {
    sfor<G::LC>([&](auto I) {
      constexpr int n = decltype(I)::value;
      S[(n + G::LC) * G::SP + col] = twiddle<n, G::H, true>(x[n]);
    });
  }
}

// order shared-memory accesses between the edge thread and its helpers (threads of columns 0 .. LC/2-1
// of the same role): they always share a warp
template <int N>
WF_HD void sync_field() {
#if defined(__CUDA_ARCH__)
  __syncwarp();
#endif
}

template <int L>
WF_HD void conj_all(float2 (&x)[L]) {
#pragma unroll
  for (int k = 0; k < L; ++k) x[k].y = -x[k].y;
}

// mode pairs held by a column thread: register kp and its mirror register, with their ky values.
// role 0 holds even ky: (kp, LC/2) for kp = 0 (ky 0 and H/2), (kp, LC - kp) otherwise (ky, H - ky).
// role 1 holds odd ky: (kp, LC - 1 - kp) (ky = 2kp + 1 and H - ky).
// f(kp, kq, ky1, ky2, ic<IS_ZERO_GROUP>) is called with compile-time register indices.
template <int N, class F>
WF_HD void for_mode_pairs(int r, F&& f) {
  using G = Geo<N>;
  if (r == 0) {
    sfor<G::LC / 2>([&](auto I) {
      constexpr int kp = decltype(I)::value;
      constexpr int kq = kp == 0 ? G::LC / 2 : G::LC - kp;
      f(ic<kp>{}, ic<kq>{}, 2 * kp, kp == 0 ? G::H / 2 : G::H - 2 * kp, ic<kp == 0>{});
    });
  } else {
    sfor<G::LC / 2>([&](auto I) {
      constexpr int kp = decltype(I)::value;
      constexpr int kq = G::LC - 1 - kp;
      f(ic<kp>{}, ic<kq>{}, 2 * kp + 1, G::H - 2 * kp - 1, ic<0>{});
    });
  }
}

// Staging of one real field (row y held as c[m] = (s[2m], s[2m+1])) and a coalesced copy to global.
// A staged row occupies exactly the floats of spectrum row y, so a thread's staged row and its
// spectrum row are the same memory.
template <int N>
WF_HD void stage_row(float* stg, int y, const float2 (&c)[N / 2]) {
  using G = Geo<N>;
  float2* r = reinterpret_cast<float2*>(stg) + y * G::SP;
#pragma unroll
  for (int m = 0; m < G::LR; ++m) r[m] = c[m];
}
template <int N>
WF_HD void copy_out(const float* stg, int lt, float* __restrict__ out) {
  using G = Geo<N>;
  const float2* s2 = reinterpret_cast<const float2*>(stg);
  float2* o2 = reinterpret_cast<float2*>(out);
#pragma unroll 4
  for (int e = lt; e < G::H * G::LR; e += N) {
    const int y = e / G::LR, m = e % G::LR;
    o2[e] = s2[y * G::SP + m];
  }
}
// the staged field to an output image of element type t (OutType)
#if defined(__CUDACC__)
template <int N>
__device__ __forceinline__ void copy_out_t(const float* stg, int lt, void* __restrict__ out, int t) {
  using G = Geo<N>;
  if (t == kOutF32) {
    copy_out<N>(stg, lt, static_cast<float*>(out));
    return;
  }
  const float2* s2 = reinterpret_cast<const float2*>(stg);
#pragma unroll 4
  for (int e = lt; e < G::H * G::LR; e += N) {
    const int y = e / G::LR, m = e % G::LR;
    store_pair(out, e, s2[y * G::SP + m], t);
  }
}
#endif

// ---------------------------------------------------------------------------------------------
// pixel-space updates (Alg. 1 t-update), row y, c[m] = (s[2m], s[2m+1]) -> (t[2m], t[2m+1])
// ---------------------------------------------------------------------------------------------
// right-hand side of the level-lambda Wiener equation, N_lambda^-1 d = d / (N_bar + lambda tau)
template <int N>
WF_HD void rhs_row(float2 (&c)[N / 2], int y, const float2* __restrict__ dn, float lt_) {
  using G = Geo<N>;
#pragma unroll
  for (int x = 0; x < G::W; ++x) {
    const float2 co = WF_LDG(dn + x * G::H + y);
    const float nbar = co.y > 0.0f ? wf_rcp(co.y) : wf_inf();
    const float v = co.x / (nbar + lt_);
    if (x & 1) c[x / 2].y = v; else c[x / 2].x = v;
  }
}

// ---------------------------------------------------------------------------------------------
// Fourier-space updates (Alg. 1 s-update) on the modes held by a column thread
// ---------------------------------------------------------------------------------------------
// sum over the full spectrum of P^2 |V|^2 for the forward transform V held by this thread
// (edge columns separated into kx = 0 and kx = W/2)
template <int N>
WF_HD double p2_power(const float2 (&x)[N / 2], int lt, const float* __restrict__ Pk) {
  using G = Geo<N>;
  constexpr int WH = G::WH;
  const int col = lt % G::LC, r = lt / G::LC;
  float acc = 0.0f;  // the thread's LC modes in FP32; the caller sums the threads in FP64
  auto p2 = [](float P, float re, float im) -> float { return P * P * fmaf(re, re, im * im); };
  for_mode_pairs<N>(r, [&](auto KP, auto KQ, int ky1, int ky2, auto ZG) {
    constexpr int kp = decltype(KP)::value, kq = decltype(KQ)::value;
    constexpr bool zero_group = decltype(ZG)::value != 0;
    if (col != 0) {
      acc += 2.0f * (p2(WF_LDG(Pk + ky1 * WH + col), x[kp].x, x[kp].y) + p2(WF_LDG(Pk + ky2 * WH + col), x[kq].x, x[kq].y));
    } else if constexpr (zero_group) {
      acc += p2(WF_LDG(Pk + ky1 * WH), x[kp].x, 0.f) + p2(WF_LDG(Pk + ky1 * WH + G::W / 2), x[kp].y, 0.f) +
             p2(WF_LDG(Pk + ky2 * WH), x[kq].x, 0.f) + p2(WF_LDG(Pk + ky2 * WH + G::W / 2), x[kq].y, 0.f);
    } else {
      const float2 y1 = x[kp], y2c = cconj(x[kq]);
      const float2 A = cscale(cadd(y1, y2c), 0.5f);
      const float2 B = cmul_mi(cscale(csub(y1, y2c), 0.5f));
      acc += 2.0f * (p2(WF_LDG(Pk + ky1 * WH), A.x, A.y) + p2(WF_LDG(Pk + ky1 * WH + G::W / 2), B.x, B.y));
    }
  });
  return double(acc);
}

// sum over the full spectrum of w_j(k) |V_k|^2, j < nw <= 4, for the forward transform V held by this
// thread; tables w_j = w + j*H*(W/2+1) on the half spectrum; edge columns separated into kx = 0 and W/2
template <int N>
WF_HD void wpower_acc(const float2 (&x)[N / 2], int lt, const float* __restrict__ w, int nw, double (&acc)[4]) {
  using G = Geo<N>;
  constexpr int WH = G::WH, TS = G::H * G::WH;
  const int col = lt % G::LC, r = lt / G::LC;
  auto sq = [](float a, float b) -> double { return double(a) * a + double(b) * b; };
  for_mode_pairs<N>(r, [&](auto KP, auto KQ, int ky1, int ky2, auto ZG) {
    constexpr int kp = decltype(KP)::value, kq = decltype(KQ)::value;
    constexpr bool zero_group = decltype(ZG)::value != 0;
    for (int j = 0; j < nw; ++j) {
      const float* wt = w + j * TS;
      double v;
      if (col != 0) {
        v = 2.0 * (WF_LDG(wt + ky1 * WH + col) * sq(x[kp].x, x[kp].y) +
                   WF_LDG(wt + ky2 * WH + col) * sq(x[kq].x, x[kq].y));
      } else if (zero_group) {
        v = WF_LDG(wt + ky1 * WH) * sq(x[kp].x, 0.f) + WF_LDG(wt + ky1 * WH + G::W / 2) * sq(x[kp].y, 0.f) +
            WF_LDG(wt + ky2 * WH) * sq(x[kq].x, 0.f) + WF_LDG(wt + ky2 * WH + G::W / 2) * sq(x[kq].y, 0.f);
      } else {
        const float2 y1 = x[kp], y2c = cconj(x[kq]);
        const float2 A = cscale(cadd(y1, y2c), 0.5f);
        const float2 B = cmul_mi(cscale(csub(y1, y2c), 0.5f));
        v = 2.0 * (WF_LDG(wt + ky1 * WH) * sq(A.x, A.y) + WF_LDG(wt + ky1 * WH + G::W / 2) * sq(B.x, B.y));
      }
      acc[j] += v;
    }
  });
}

// block-wide double sum; every thread gets the result. red must hold >= 33 doubles. Blocks of fewer than
// 32 threads (power of two) reduce within their partial warp only.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int nt = blockDim.x;
  if (nt < 32) {
    const unsigned int mask = (1u << nt) - 1u;
    for (int o = nt / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    __syncthreads();
    return v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (nt + 31) >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += red[i];
    red[32] = s;
  }
  __syncthreads();
  const double s = red[32];
  __syncthreads();
  return s;
}

// ---------------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------------
struct SampleArgs {
  const float2* aq;      // [W][H] pixel table (a, q)
  const float2* fg;      // [H][W/2+1] mode table (f/n, g/sqrt(2n))
  const Scalars* sc;
  const float* init_s;   // nullptr -> zeros; else [n_chains or 1][H][W]
  long long init_stride; // elements between chains' initial states (0: shared)
  float* out;            // [n_chains][n_samples][H][W]
  long long n_samples;
  int n_chains;
  int n_sweeps;
  int burn_in;
  int thin;
  uint32_t chain0;
  uint32_t step0;
  uint32_t key0, key1;
  int out_dtype;         // OutType of out
  // hierarchical samplers (k_sample_band, k_csample_band) only
  int n_bins;
  const float* P0;       // [n_bins] initial band powers
  float* out_P;          // [n_chains][n_samples][n_bins] or nullptr
  const int2* band_map;  // mode table order: (bin or -1, position in the bin-ordered statistics buffer or < 0)
  const int* band_off;   // [n_bins + 1] start of each bin in the statistics buffer
  float2* band_buf;      // statistics buffers: one per chain (on-chip form), one per cluster (k_csample_band)
  // cluster form of the hierarchical sampler (k_csample_band) only
  const int* band_lo;    // [CTAs per cluster + 1] bins summed by each CTA of a cluster
  int band_clusters;     // clusters launched; each runs chains c, c + band_clusters, ...
};

// shared bytes per field of the hierarchical sampler: the per-band s-draw coefficients (float2) and the
// band powers (floats)
WF_HD int band_bytes(int n_bins) { return ((n_bins * 12 + 15) / 16) * 16; }

// CTAs per SM the sample kernel is compiled for (register budget 65536 / (threads * CTAs)):
// 128^2 fields are limited to three per SM by shared memory (66.5 KB each).
// Philox calls in flight in the rolled pointwise-draw loops (the field registers are dead there)
#ifndef WF_RNG_UNROLL
#define WF_RNG_UNROLL 4
#endif
constexpr int kRngUnroll = WF_RNG_UNROLL;
#ifndef WF_SAMPLE_MIN_CTAS_128
#define WF_SAMPLE_MIN_CTAS_128 3
#endif
template <int N>
constexpr int sample_min_ctas() { return N >= 128 ? WF_SAMPLE_MIN_CTAS_128 : (N == 64 ? 4 : 8); }

// ---------------------------------------------------------------------------------------------
// pointwise draws as rolled loops over shared memory: the thread parks the data it holds in its own
// slots of the (dead) field buffer, updates it in place with the Philox draws generated inline, and
// reloads it. The field registers are dead meanwhile, which keeps register pressure off these loops.
// ---------------------------------------------------------------------------------------------
// t-draw of row y, staged as stg[y*STG + x] (the same layout as stage_row):
// t = a + q (q s + sqrt(tau) xi), table aq[x*H + y] = ((1 - w) d, sqrt(w)); Philox stream 0,
// group y*W/4 + q feeds pixels 4q .. 4q+3.
template <int N>
WF_HD void t_draw_staged(float* stg, int y, const float2* __restrict__ aq, float sqrt_tau, uint32_t step,
                         uint32_t chain, uint32_t k0, uint32_t k1, uint32_t stream = 0u) {
  using G = Geo<N>;
  float2* row = reinterpret_cast<float2*>(stg) + y * G::SP;  // (s[2m], s[2m+1]) pairs
#pragma unroll (kRngUnroll)
  for (int q = 0; q < G::W / 4; ++q) {
    float z[4];
    normals4(uint32_t(y * (G::W / 4) + q), step, chain, stream, k0, k1, z);
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

// Wiener-filter t-update at level lambda of the staged row y: table dn[x*H + y] = (d, 1/N_bar) ((0, 0) on
// missing pixels), w = N_bar / (lambda tau + N_bar) = 1 / (1 + lambda tau / N_bar), t = d + w (s - d).
// rhs mode (refinement corrections): dn holds (r, 1/N_bar) and t = lambda tau r + w s, whose fixed point
// solves (S^-1 + N_lambda^-1) s = r for any pixel-space r (r need not vanish on missing pixels).
// Rolled over groups of four pixels: the row's registers are dead meanwhile, so more table loads are in
// flight.
template <int N>
WF_HD void t_update_wf_staged(float* stg, int y, const float2* __restrict__ dn, float lt_, bool rhs) {
  using G = Geo<N>;
  float2* row = reinterpret_cast<float2*>(stg) + y * G::SP;
  const float g = rhs ? 0.0f : 1.0f, h = rhs ? lt_ : 1.0f;
#pragma unroll (kRngUnroll)
  for (int q = 0; q < G::W / 4; ++q) {
    float2 p0 = row[2 * q], p1 = row[2 * q + 1];
    const float2 c0 = WF_LDG(dn + (4 * q) * G::H + y), c1 = WF_LDG(dn + (4 * q + 1) * G::H + y);
    const float2 c2 = WF_LDG(dn + (4 * q + 2) * G::H + y), c3 = WF_LDG(dn + (4 * q + 3) * G::H + y);
    const float w0 = wf_rcp(fmaf(lt_, c0.y, 1.0f)), w1 = wf_rcp(fmaf(lt_, c1.y, 1.0f));
    const float w2 = wf_rcp(fmaf(lt_, c2.y, 1.0f)), w3 = wf_rcp(fmaf(lt_, c3.y, 1.0f));
    p0.x = fmaf(w0, fmaf(-g, c0.x, p0.x), h * c0.x);
    p0.y = fmaf(w1, fmaf(-g, c1.x, p0.y), h * c1.x);
    p1.x = fmaf(w2, fmaf(-g, c2.x, p1.x), h * c2.x);
    p1.y = fmaf(w3, fmaf(-g, c3.x, p1.y), h * c3.x);
    row[2 * q] = p0;
    row[2 * q + 1] = p1;
  }
}

template <int N>
WF_HD void load_staged_row(const float* stg, int y, float2 (&c)[N / 2]) {
  using G = Geo<N>;
  const float2* r = reinterpret_cast<const float2*>(stg) + y * G::SP;
#pragma unroll
  for (int m = 0; m < G::LR; ++m) c[m] = r[m];
}

// The modes of column thread (col, r) are parked in the slots it stores to after the inverse column
// transform: register k at cs[(k + r*LC) * SP + col] (rows r*LC .. r*LC+LC-1 of its column).
template <int N>
WF_HD int park_index(int lt, int k) {
  using G = Geo<N>;
  return (k + (lt / G::LC) * G::LC) * G::SP + lt % G::LC;
}
template <int N>
WF_HD void park_modes(float2* cs, int lt, const float2 (&x)[N / 2]) {
#pragma unroll
  for (int k = 0; k < N / 2; ++k) cs[park_index<N>(lt, k)] = x[k];
}
template <int N>
WF_HD void unpark_modes(const float2* cs, int lt, float2 (&x)[N / 2]) {
#pragma unroll
  for (int k = 0; k < N / 2; ++k) x[k] = cs[park_index<N>(lt, k)];
}

// s-draw on parked modes: s_hat = f t_hat + g zeta, table fg[ky*WH + kx] = (f / n, g / sqrt(2 n)).
// Mode pair kp of role r: registers kp and kq with ky1 = 2kp + r and its mirror ky2 (for_mode_pairs);
// Philox stream 1, group col*H/2 + ky1.
template <int N>
WF_HD void mode_pair(int r, int kp, int& kq, int& ky1, int& ky2) {
  using G = Geo<N>;
  kq = r == 0 ? (kp == 0 ? G::LC / 2 : G::LC - kp) : G::LC - 1 - kp;
  ky1 = 2 * kp + r;
  ky2 = r == 0 ? (kp == 0 ? G::H / 2 : G::H - 2 * kp) : G::H - 2 * kp - 1;
}

// Wiener-filter s-update at level lambda on the thread's parked modes (park_modes): s_hat = f t_hat with
// f = P/(P + lambda tau) (scaled by 1/n), rolled over the thread's mode pairs (the column registers are dead
// meanwhile, so more Pk / prev loads are in flight; each thread touches only its own parked slots, the
// packed edge column included). With CMP the residual of the previous iterate, |r_k| = |s_hat_new -
// s_hat_old| / (1 - f), is accumulated over the full spectrum (returned, scaled 1/n): per-mode terms and
// the thread's partial sum (its 2 x LC/2 modes) in FP32 (a residual estimate needs a few digits, and FP64
// arithmetic runs at a small fraction of the FP32 rate), the threads' partial sums in FP64 by the caller.
// With STORE the new modes go to prev[ky*LR + col].
template <int N>
WF_HD double s_update_wf_parked(float2* cs, int lt, const float* __restrict__ Pk, float lt_,
                                float2* __restrict__ prev, bool CMP, bool STORE) {
  using G = Geo<N>;
  constexpr int WH = G::WH, LC = G::LC;
  constexpr float INV_N = 1.0f / float(G::H * G::W);
  const int col = lt % LC, r = lt / LC;
  float acc = 0.0f;
  const float inv_lt = 1.0f / lt_;
  auto wres = [&](float P, float dre, float dim) -> float {
    const float g = fmaf(P, inv_lt, 1.0f);
    return fmaf(dre, dre, dim * dim) * (g * g);
  };
  auto fcoef = [&](float P) { return wf_fdiv(P, P + lt_) * INV_N; };
#pragma unroll 4
  for (int kp = 0; kp < LC / 2; ++kp) {
    int kq, ky1, ky2;
    mode_pair<N>(r, kp, kq, ky1, ky2);
    const int i1 = park_index<N>(lt, kp), i2 = park_index<N>(lt, kq);
    const float2 x1 = cs[i1], x2 = cs[i2];
    float2 n1, n2;
    if (col != 0) {
      const float P1 = WF_LDG(Pk + ky1 * WH + col), P2 = WF_LDG(Pk + ky2 * WH + col);
      n1 = cscale(x1, fcoef(P1));
      n2 = cscale(x2, fcoef(P2));
      if (CMP) {
        const float2 o1 = prev[ky1 * G::LR + col], o2 = prev[ky2 * G::LR + col];
        acc += 2.0f * (wres(P1, n1.x - o1.x, n1.y - o1.y) + wres(P2, n2.x - o2.x, n2.y - o2.y));
      }
    } else {
      const float Pa1 = WF_LDG(Pk + ky1 * WH), Pb1 = WF_LDG(Pk + ky1 * WH + G::W / 2);
      const float fa1 = fcoef(Pa1), fb1 = fcoef(Pb1);
      if (r == 0 && kp == 0) {  // the four self-conjugate modes
        const float Pa2 = WF_LDG(Pk + ky2 * WH), Pb2 = WF_LDG(Pk + ky2 * WH + G::W / 2);
        n1 = make_float2(fa1 * x1.x, fb1 * x1.y);
        n2 = make_float2(fcoef(Pa2) * x2.x, fcoef(Pb2) * x2.y);
        if (CMP) {
          const float2 o1 = prev[ky1 * G::LR], o2 = prev[ky2 * G::LR];
          acc += wres(Pa1, n1.x - o1.x, 0.f) + wres(Pb1, n1.y - o1.y, 0.f) + wres(Pa2, n2.x - o2.x, 0.f) +
                 wres(Pb2, n2.y - o2.y, 0.f);
        }
      } else {
        const float2 y2c = cconj(x2);
        const float2 A = cscale(cscale(cadd(x1, y2c), 0.5f), fa1);
        const float2 B = cscale(cmul_mi(cscale(csub(x1, y2c), 0.5f)), fb1);
        n1 = cadd(A, cmul_i(B));
        n2 = cadd(cconj(A), cmul_i(cconj(B)));
        if (CMP) {
          const float2 o1 = prev[ky1 * G::LR], o2c = cconj(prev[ky2 * G::LR]);
          const float2 oA = cscale(cadd(o1, o2c), 0.5f);
          const float2 oB = cmul_mi(cscale(csub(o1, o2c), 0.5f));
          // modes ky1 and H - ky1 of each edge column have equal magnitude: weight 2
          acc += 2.0f * (wres(Pa1, A.x - oA.x, A.y - oA.y) + wres(Pb1, B.x - oB.x, B.y - oB.y));
        }
      }
    }
    cs[i1] = n1;
    cs[i2] = n2;
    if (STORE) {
      prev[ky1 * G::LR + col] = n1;
      prev[ky2 * G::LR + col] = n2;
    }
  }
  return double(acc);
}

// Mode coefficients (f/n, g/sqrt(2n)) of the s-draw. TableCoef reads the per-call table; BandCoef (the
// hierarchical sampler) takes them from the per-band table cb = band_coef(P_b) in shared memory for modes
// with a bin (bmap[j].x >= 0, j = ky (W/2+1) + kx; -1: the table's coefficients) and stores the band
// statistics of each new mode, (n |s_hat|^2 with its mirror weight, the squares of its stream-6 normals),
// to its own position bmap[j].y of the chain's bin-ordered buffer in global memory (< 0: not summed), so
// that the band sums need no atomics and run in a fixed order.
// s-draw coefficients (f/n, g/sqrt(2n)) of band power P (table_mode's formulas in FP32; (0, 0) for P <= 0)
WF_HD float2 band_coef(float P, float tau, float inv_n) {
  if (!(P > 0.0f)) return make_float2(0.0f, 0.0f);
  const float q = P * wf_rcp(P + tau);
  const float g2 = q * tau * 0.5f * inv_n;
  return make_float2(q * inv_n, g2 * wf_rsqrt(g2));
}

struct TableCoef {
  static constexpr bool kBand = false;
  const float2* __restrict__ fg;
  int wh;
  WF_HD float2 coef(int ky, int kx) const { return WF_LDG(fg + ky * wh + kx); }
  WF_HD void add(int, int, float, float) const {}
};
struct BandCoef {
  static constexpr bool kBand = true;
  const float2* __restrict__ fg;
  int wh;
  const int2* __restrict__ bmap;  // [H][W/2+1]: (bin, position in the statistics buffer)
  float2* cb;                     // shared [n_bins]: band_coef of each band power
  float* Pb;                      // shared [n_bins]
  float2* buf;                    // this chain's statistics, bin-ordered (global, L2)
  const int* off;                 // [n_bins + 1] start of each bin in buf
  int n_bins;
  float tau, inv_n, n;
  WF_HD float2 coef(int ky, int kx) const {
    const int b = WF_LDG(bmap + ky * wh + kx).x;
    return b < 0 ? WF_LDG(fg + ky * wh + kx) : cb[b];
  }
  WF_HD void add(int ky, int kx, float s2, float x2) const {
#if defined(__CUDA_ARCH__)
    const int pos = WF_LDG(bmap + ky * wh + kx).y;
    if (pos >= 0) __stcg(buf + pos, make_float2(s2 * n, x2));
#endif
  }
};

// interior columns (col > 0): every thread but the edge thread updates its own parked modes
template <int N, class Coef>
WF_HD void s_draw_interior(float2* cs, int lt, const Coef& cf, uint32_t step, uint32_t chain, uint32_t k0,
                           uint32_t k1) {
  using G = Geo<N>;
  constexpr int LC = G::LC, H = G::H;
  const int col = lt % LC, r = lt / LC;
  if (col == 0) return;
#pragma unroll (kRngUnroll)
  for (int kp = 0; kp < LC / 2; ++kp) {
    int kq, ky1, ky2;
    mode_pair<N>(r, kp, kq, ky1, ky2);
    float z[4];
    normals4(uint32_t(col * (H / 2) + ky1), step, chain, 1u, k0, k1, z);
    const int i1 = park_index<N>(lt, kp), i2 = park_index<N>(lt, kq);
    float2 y1 = cs[i1], y2 = cs[i2];
    const float2 m1 = cf.coef(ky1, col), m2 = cf.coef(ky2, col);
    y1 = make_float2(fmaf(m1.x, y1.x, m1.y * z[0]), fmaf(m1.x, y1.y, m1.y * z[1]));
    y2 = make_float2(fmaf(m2.x, y2.x, m2.y * z[2]), fmaf(m2.x, y2.y, m2.y * z[3]));
    cs[i1] = y1;
    cs[i2] = y2;
    if constexpr (Coef::kBand) {  // both modes have their mirror in the other half plane: weight 2
      float zb[4];
      normals4(uint32_t(col * (H / 2) + ky1), step, chain, 6u, k0, k1, zb);
      cf.add(ky1, col, 2.0f * (y1.x * y1.x + y1.y * y1.y), zb[0] * zb[0] + zb[1] * zb[1]);
      cf.add(ky2, col, 2.0f * (y2.x * y2.x + y2.y * y2.y), zb[2] * zb[2] + zb[3] * zb[3]);
    }
  }
}

// the packed edge column (col 0: kx = 0 as A and kx = W/2 as B in Y = A + i B, both Hermitian in ky):
// its LC/2 mode pairs of role r are shared out to the threads of columns 0 .. LC/2-1 of that role
// (one pair each), which read and write the edge thread's parked slots. Group ky1 (col 0) feeds the pair.
template <int N, class Coef>
WF_HD void s_draw_edge(float2* cs, int lt, const Coef& cf, uint32_t step, uint32_t chain, uint32_t k0,
                       uint32_t k1) {
  using G = Geo<N>;
  constexpr int LC = G::LC;
  const int kp = lt % LC, r = lt / LC;
  if (kp >= LC / 2) return;
  const int edge = r * LC;  // thread index of the edge thread of this role
  int kq, ky1, ky2;
  mode_pair<N>(r, kp, kq, ky1, ky2);
  float z[4];
  normals4(uint32_t(ky1), step, chain, 1u, k0, k1, z);
  const int i1 = park_index<N>(edge, kp), i2 = park_index<N>(edge, kq);
  float2 y1 = cs[i1], y2 = cs[i2];
  const float2 a1 = cf.coef(ky1, 0), b1 = cf.coef(ky1, G::W / 2);
  float zb[4] = {0.f, 0.f, 0.f, 0.f};
  if constexpr (Coef::kBand) normals4(uint32_t(ky1), step, chain, 6u, k0, k1, zb);
  if (ky1 == 0) {
    // group 0: the four self-conjugate modes, real with variance g^2
    const float2 a2 = cf.coef(ky2, 0), b2 = cf.coef(ky2, G::W / 2);
    constexpr float R2 = 1.41421356237309505f;
    y1 = make_float2(fmaf(a1.x, y1.x, R2 * a1.y * z[0]), fmaf(b1.x, y1.y, R2 * b1.y * z[2]));
    y2 = make_float2(fmaf(a2.x, y2.x, R2 * a2.y * z[1]), fmaf(b2.x, y2.y, R2 * b2.y * z[3]));
    if constexpr (Coef::kBand) {  // one real degree of freedom each
      cf.add(ky1, 0, y1.x * y1.x, zb[0] * zb[0]);
      cf.add(ky1, G::W / 2, y1.y * y1.y, zb[2] * zb[2]);
      cf.add(ky2, 0, y2.x * y2.x, zb[1] * zb[1]);
      cf.add(ky2, G::W / 2, y2.y * y2.y, zb[3] * zb[3]);
    }
  } else {
    const float2 y2c = cconj(y2);
    const float2 A = cscale(cadd(y1, y2c), 0.5f);
    const float2 B = cmul_mi(cscale(csub(y1, y2c), 0.5f));
    const float2 Ap = make_float2(fmaf(a1.x, A.x, a1.y * z[0]), fmaf(a1.x, A.y, a1.y * z[1]));
    const float2 Bp = make_float2(fmaf(b1.x, B.x, b1.y * z[2]), fmaf(b1.x, B.y, b1.y * z[3]));
    y1 = cadd(Ap, cmul_i(Bp));
    y2 = cadd(cconj(Ap), cmul_i(cconj(Bp)));
    if constexpr (Coef::kBand) {  // (ky1, 0) and (ky1, W/2) with their mirrors at H - ky1: weight 2
      cf.add(ky1, 0, 2.0f * (Ap.x * Ap.x + Ap.y * Ap.y), zb[0] * zb[0] + zb[1] * zb[1]);
      cf.add(ky1, G::W / 2, 2.0f * (Bp.x * Bp.x + Bp.y * Bp.y), zb[2] * zb[2] + zb[3] * zb[3]);
    }
  }
  cs[i1] = y1;
  cs[i2] = y2;
}

// Spin-2 (shear) sampler: the two shear components are two fields of one CTA (component = field index
// mod 2) and the s-draw couples them per mode: rotate (t1_hat, t2_hat) by the Kaiser-Squires angle into
// E and B, draw each with its own spectrum (tables fgE, fgB; E draws from stream 1, B from stream 9 in the
// counter layout of the scalar s-draw), rotate back. (c, s) = (cos 2 phi, sin 2 phi) of k = (kx, ky), with
// (1, 0) at k = 0 and on the Nyquist row and column.
struct Spin2Coef {
  static constexpr bool kBand = false;
  const float2* __restrict__ fgE;
  const float2* __restrict__ fgB;
  int wh;
  float2* cs0;  // parked modes of component 1 and 2 (shared)
  float2* cs1;
  int comp;
  WF_HD float2 coef(int, int) const { return make_float2(0.f, 0.f); }
  WF_HD void add(int, int, float, float) const {}
};

template <int N>
WF_HD void ks_rot(int ky, int kx, float& c, float& s) {
  using G = Geo<N>;
  const int y = ky < G::H / 2 ? ky : ky - G::H;  // folded row frequency
  if ((kx == 0 && y == 0) || ky == G::H / 2 || kx == G::W / 2) {
    c = 1.0f;
    s = 0.0f;
    return;
  }
  const float k1 = float(kx), k2 = float(y), r = 1.0f / (k1 * k1 + k2 * k2);
  c = (k1 * k1 - k2 * k2) * r;
  s = 2.0f * k1 * k2 * r;
}

// one complex mode: (a, b) = (t1_hat, t2_hat) -> new (gamma1_hat, gamma2_hat); mE, mB = (f/n, g/sqrt(2n))
WF_HD void spin2_mode(float2& a, float2& b, float c, float s, float2 mE, float2 mB, float zE0, float zE1, float zB0,
                      float zB1) {
  const float2 e = make_float2(fmaf(c, a.x, s * b.x), fmaf(c, a.y, s * b.y));
  const float2 q = make_float2(fmaf(c, b.x, -s * a.x), fmaf(c, b.y, -s * a.y));
  const float2 e2 = make_float2(fmaf(mE.x, e.x, mE.y * zE0), fmaf(mE.x, e.y, mE.y * zE1));
  const float2 q2 = make_float2(fmaf(mB.x, q.x, mB.y * zB0), fmaf(mB.x, q.y, mB.y * zB1));
  a = make_float2(fmaf(c, e2.x, -s * q2.x), fmaf(c, e2.y, -s * q2.y));
  b = make_float2(fmaf(s, e2.x, c * q2.x), fmaf(s, e2.y, c * q2.y));
}

// interior columns: the pairs of column thread (col, r) are shared out to the two components' threads
template <int N>
WF_HD void spin2_interior(const Spin2Coef& cf, int lt, uint32_t step, uint32_t chain, uint32_t k0, uint32_t k1) {
  using G = Geo<N>;
  constexpr int LC = G::LC, H = G::H;
  const int col = lt % LC, r = lt / LC;
  if (col == 0) return;
  const int kp0 = cf.comp == 0 ? 0 : LC / 4, kp1 = cf.comp == 0 ? LC / 4 : LC / 2;
#pragma unroll 2
  for (int kp = kp0; kp < kp1; ++kp) {
    int kq, ky1, ky2;
    mode_pair<N>(r, kp, kq, ky1, ky2);
    float zE[4], zB[4];
    normals4(uint32_t(col * (H / 2) + ky1), step, chain, 1u, k0, k1, zE);
    normals4(uint32_t(col * (H / 2) + ky1), step, chain, 9u, k0, k1, zB);
    const int i1 = park_index<N>(lt, kp), i2 = park_index<N>(lt, kq);
    float2 a1 = cf.cs0[i1], b1 = cf.cs1[i1], a2 = cf.cs0[i2], b2 = cf.cs1[i2];
    float c, s;
    ks_rot<N>(ky1, col, c, s);
    spin2_mode(a1, b1, c, s, WF_LDG(cf.fgE + ky1 * cf.wh + col), WF_LDG(cf.fgB + ky1 * cf.wh + col), zE[0], zE[1],
               zB[0], zB[1]);
    ks_rot<N>(ky2, col, c, s);
    spin2_mode(a2, b2, c, s, WF_LDG(cf.fgE + ky2 * cf.wh + col), WF_LDG(cf.fgB + ky2 * cf.wh + col), zE[2], zE[3],
               zB[2], zB[3]);
    cf.cs0[i1] = a1;
    cf.cs1[i1] = b1;
    cf.cs0[i2] = a2;
    cf.cs1[i2] = b2;
  }
}

// the packed edge column (kx = 0 as A and kx = W/2 as B in Y = A + i B) of both components, by the first
// component's threads of columns 0 .. LC/2-1 (one mode pair each)
template <int N>
WF_HD void spin2_edge(const Spin2Coef& cf, int lt, uint32_t step, uint32_t chain, uint32_t k0, uint32_t k1) {
  using G = Geo<N>;
  constexpr int LC = G::LC, WH2 = G::W / 2;
  const int kp = lt % LC, r = lt / LC;
  if (cf.comp != 0 || kp >= LC / 2) return;
  const int edge = r * LC;
  int kq, ky1, ky2;
  mode_pair<N>(r, kp, kq, ky1, ky2);
  float zE[4], zB[4];
  normals4(uint32_t(ky1), step, chain, 1u, k0, k1, zE);
  normals4(uint32_t(ky1), step, chain, 9u, k0, k1, zB);
  const int i1 = park_index<N>(edge, kp), i2 = park_index<N>(edge, kq);
  float2 y1a = cf.cs0[i1], y2a = cf.cs0[i2], y1b = cf.cs1[i1], y2b = cf.cs1[i2];
  const int wh = cf.wh;
  if (ky1 == 0) {
    // four real modes, each on k = 0 or a Nyquist line: no rotation, real draws with variance g^2
    constexpr float R2 = 1.41421356237309505f;
    auto upd = [&](float& a, float& b, int ky, int kx, float ze, float zb) {
      const float2 mE = WF_LDG(cf.fgE + ky * wh + kx), mB = WF_LDG(cf.fgB + ky * wh + kx);
      a = fmaf(mE.x, a, R2 * mE.y * ze);
      b = fmaf(mB.x, b, R2 * mB.y * zb);
    };
    upd(y1a.x, y1b.x, ky1, 0, zE[0], zB[0]);
    upd(y1a.y, y1b.y, ky1, WH2, zE[2], zB[2]);
    upd(y2a.x, y2b.x, ky2, 0, zE[1], zB[1]);
    upd(y2a.y, y2b.y, ky2, WH2, zE[3], zB[3]);
  } else {
    // unpack both components: A = value at (ky1, 0), B = value at (ky1, W/2)
    const float2 Aa = cscale(cadd(y1a, cconj(y2a)), 0.5f), Ba = cmul_mi(cscale(csub(y1a, cconj(y2a)), 0.5f));
    const float2 Ab = cscale(cadd(y1b, cconj(y2b)), 0.5f), Bb = cmul_mi(cscale(csub(y1b, cconj(y2b)), 0.5f));
    float2 A1 = Aa, A2 = Ab, B1 = Ba, B2 = Bb;
    float c, s;
    ks_rot<N>(ky1, 0, c, s);
    spin2_mode(A1, A2, c, s, WF_LDG(cf.fgE + ky1 * wh), WF_LDG(cf.fgB + ky1 * wh), zE[0], zE[1], zB[0], zB[1]);
    ks_rot<N>(ky1, WH2, c, s);
    spin2_mode(B1, B2, c, s, WF_LDG(cf.fgE + ky1 * wh + WH2), WF_LDG(cf.fgB + ky1 * wh + WH2), zE[2], zE[3], zB[2],
               zB[3]);
    y1a = cadd(A1, cmul_i(B1));
    y2a = cadd(cconj(A1), cmul_i(cconj(B1)));
    y1b = cadd(A2, cmul_i(B2));
    y2b = cadd(cconj(A2), cmul_i(cconj(B2)));
  }
  cf.cs0[i1] = y1a;
  cf.cs0[i2] = y2a;
  cf.cs1[i1] = y1b;
  cf.cs1[i2] = y2b;
}

// band-power draw after the s-draw (every mode's statistics stored and visible to the field's threads):
// the field's threads in groups of G = min(N, 32) lanes take four bins at a time, each lane summing its
// lane-strided entries of the four bins (16 loads in flight), then a fixed shuffle tree per bin: the same
// order every run; P_b = S_b / X_b and band_coef(P_b) to shared memory. Called by all lanes of every
// warp (the loop bounds are the same for every field of a warp).
template <int N>
__device__ __forceinline__ void band_update(const BandCoef& bc, int lt) {
  constexpr int G = N < 32 ? N : 32, NG = N / G, KB = 4, U = 4;
  const int gl = lt % G;
  for (int b0 = lt / G; b0 < bc.n_bins; b0 += NG * KB) {
    int o0[KB], len[KB], most = 0;
    float S[KB], X[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      const int b = b0 + k * NG;
      o0[k] = b < bc.n_bins ? bc.off[b] : 0;
      len[k] = b < bc.n_bins ? bc.off[b + 1] - o0[k] : 0;
      most = len[k] > most ? len[k] : most;
      S[k] = X[k] = 0.0f;
    }
    for (int j = gl; j < most; j += U * G) {
      float2 v[KB][U];
#pragma unroll
      for (int k = 0; k < KB; ++k)
#pragma unroll
        for (int u = 0; u < U; ++u)
          v[k][u] = j + G * u < len[k] ? __ldcg(bc.buf + o0[k] + j + G * u) : make_float2(0.0f, 0.0f);
#pragma unroll
      for (int k = 0; k < KB; ++k)
#pragma unroll
        for (int u = 0; u < U; ++u) {
          S[k] += v[k][u].x;
          X[k] += v[k][u].y;
        }
    }
#pragma unroll
    for (int k = 0; k < KB; ++k) {
#pragma unroll
      for (int d = G / 2; d > 0; d >>= 1) {
        S[k] += __shfl_xor_sync(0xffffffffu, S[k], d);
        X[k] += __shfl_xor_sync(0xffffffffu, X[k], d);
      }
      const int b = b0 + k * NG;
      if (gl == 0 && b < bc.n_bins) {
        const float P = X[k] > 0.0f ? S[k] / X[k] : 0.0f;
        bc.Pb[b] = P;
        bc.cb[b] = band_coef(P, bc.tau, bc.inv_n);
      }
    }
  }
}

// One sweep = four transforms, all run by the single forward-FFT block at the top of the loop (an
// inverse transform is conj(FFT(conj(x)))), so the kernel holds one copy of the transform code:
//   ROW_FWD: t (pixel space, after the t-draw) -> R2C rows -> store; load columns
//   COL_FWD: column FFT -> s-draw on the parked modes -> conj
//   COL_INV: conj -> store; load rows -> C2R pre-pass -> conj
//   ROW_INV: conj -> s (pixel space) -> [write sample] -> t-draw on the staged row for the next sweep
template <int N, class Coef>
__device__ __forceinline__ void sample_sweeps(float2* S, int lt, float2 (&c)[N / 2], const float2* __restrict__ aq,
                                              const Coef& cf, float sqrt_tau, uint32_t step0,
                                              uint32_t chain, uint32_t k0, uint32_t k1, int n_sweeps, int burn_in,
                                              int thin, void* out, bool active, int out_dtype = kOutF32,
                                              float* out_P = nullptr, uint32_t t_stream = 0u,
                                              long long out_stride = (long long)N * N) {
  using G = Geo<N>;
  float* stg = reinterpret_cast<float*>(S);  // staged rows (between the row load and the next store)
  float2* cs = S;                            // parked column modes (between the column load and store)
  stage_row<N>(stg, lt, c);
  t_draw_staged<N>(stg, lt, aq, sqrt_tau, step0, chain, k0, k1, t_stream);
  load_staged_row<N>(stg, lt, c);

  enum { ROW_FWD, COL_FWD, COL_INV, ROW_INV };
  int phase = ROW_FWD;
  int done = 0;  // sweeps completed
  while (true) {
    fft<G::LR, false>(c);
    if (phase == ROW_FWD) {
      r2c_post_all<G::LR>(c, std::make_integer_sequence<int, G::LR>{});
      row_store_spec<N>(S, lt, c);  // over this thread's own staged row
      __syncthreads();
      col_load<N>(S, lt, c);
      __syncthreads();  // buffer free for the parked modes
      phase = COL_FWD;
    } else if (phase == COL_FWD) {
      park_modes<N>(cs, lt, c);
      if constexpr (std::is_same<Coef, Spin2Coef>::value) {  // both components parked, then coupled
        __syncthreads();
        spin2_interior<N>(cf, lt, step0 + uint32_t(done), chain, k0, k1);
        spin2_edge<N>(cf, lt, step0 + uint32_t(done), chain, k0, k1);
        __syncthreads();
      } else {
        s_draw_interior<N>(cs, lt, cf, step0 + uint32_t(done), chain, k0, k1);
        sync_field<N>();  // the edge thread's parked modes are visible to its helpers
        s_draw_edge<N>(cs, lt, cf, step0 + uint32_t(done), chain, k0, k1);
        sync_field<N>();
      }
      if constexpr (Coef::kBand) {  // P | s: every mode's statistics are in before the band draw
        __syncthreads();
        band_update<N>(cf, lt);
      }
      unpark_modes<N>(cs, lt, c);
      conj_all<G::LC>(c);
      phase = COL_INV;
    } else if (phase == COL_INV) {
      conj_all<G::LC>(c);
      col_store_inv<N>(S, lt, c);  // over this thread's own parked slots
      __syncthreads();
      row_load_spec<N>(S, lt, c);
      __syncthreads();
      c2r_pre_all<G::LR>(c, std::make_integer_sequence<int, G::LR>{});
      conj_all<G::LR>(c);
      phase = ROW_INV;
    } else {
      conj_all<G::LR>(c);  // c[m] = (s[2m], s[2m+1]) after sweep done + 1
      ++done;
      stage_row<N>(stg, lt, c);
      if (done > burn_in && (done - burn_in) % thin == 0) {
        const long long m = (done - burn_in) / thin - 1;
        __syncthreads();
        if (active)
          copy_out_t<N>(stg, lt, static_cast<char*>(out) + m * out_stride * out_elem_bytes(out_dtype), out_dtype);
        if constexpr (Coef::kBand) {
          if (active && out_P)
            for (int b = lt; b < cf.n_bins; b += N) out_P[m * cf.n_bins + b] = cf.Pb[b];
        }
        __syncthreads();
      }
      if (done == n_sweeps) break;
      t_draw_staged<N>(stg, lt, aq, sqrt_tau, step0 + uint32_t(done), chain, k0, k1, t_stream);
      load_staged_row<N>(stg, lt, c);
      phase = ROW_FWD;
    }
  }
  __syncthreads();  // the buffer is reused by the caller
}

template <int N, int FPC>
__global__ void __launch_bounds__(N * FPC, sample_min_ctas<N>()) k_sample(SampleArgs a) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int fld = threadIdx.x / N, lt = threadIdx.x % N;
  const int ci = blockIdx.x * FPC + fld;
  const bool active = ci < a.n_chains;
  float2* S = reinterpret_cast<float2*>(smem_raw + fld * G::FIELD_BYTES);
  if (a.sc->status != 0) return;  // uniform over the grid
  float2 c[G::LR];
  if (a.init_s != nullptr && active) {
    const float2* src = reinterpret_cast<const float2*>(a.init_s + ci * a.init_stride + lt * G::W);
#pragma unroll
    for (int m = 0; m < G::LR; ++m) c[m] = WF_LDG(src + m);
  } else {
#pragma unroll
    for (int m = 0; m < G::LR; ++m) c[m] = make_float2(0.f, 0.f);
  }
  sample_sweeps<N>(S, lt, c, a.aq, TableCoef{a.fg, G::WH}, a.sc->sqrt_tau, a.step0, a.chain0 + uint32_t(ci),
                   a.key0, a.key1,
                   a.n_sweeps, a.burn_in, a.thin,
                   reinterpret_cast<char*>(a.out) +
                       ci * a.n_samples * (long long)(G::H * G::W) * out_elem_bytes(a.out_dtype),
                   active, a.out_dtype);
}

// The hierarchical sampler: k_sample's sweeps with the s-draw coefficients taken from band powers held in
// shared memory and a band-power draw (P | s) after every s-draw. Field fld's band region follows the FPC
// field buffers: the per-band draw coefficients [n_bins] float2, then the band powers [n_bins] floats; its
// mode statistics go to its own bin-ordered buffer in global memory (a.band_buf, a.band_off[n_bins]
// entries per field of the grid).
template <int N, int FPC>
__global__ void __launch_bounds__(N * FPC, sample_min_ctas<N>()) k_sample_band(SampleArgs a) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int fld = threadIdx.x / N, lt = threadIdx.x % N;
  const int ci = blockIdx.x * FPC + fld;
  const bool active = ci < a.n_chains;
  float2* S = reinterpret_cast<float2*>(smem_raw + fld * G::FIELD_BYTES);
  unsigned char* band = smem_raw + FPC * G::FIELD_BYTES + fld * band_bytes(a.n_bins);
  float2* cb = reinterpret_cast<float2*>(band);
  float* Pb = reinterpret_cast<float*>(cb + a.n_bins);
  if (a.sc->status != 0) return;  // uniform over the grid
  const float tau = float(a.sc->tau);
  constexpr float NPIX = float(G::H * G::W);
  for (int b = lt; b < a.n_bins; b += N) {
    Pb[b] = a.P0[b];
    cb[b] = band_coef(a.P0[b], tau, 1.0f / NPIX);
  }
  // one statistics buffer per field of the grid (inactive fields past the last chain run the sweeps with
  // the CTA, its barriers and warp shuffles, into their own buffer, and write no output)
  float2* buf = a.band_buf + (long long)ci * (a.n_bins > 0 ? a.band_off[a.n_bins] : 0);
  __syncthreads();
  float2 c[G::LR];
  if (a.init_s != nullptr && active) {
    const float2* src = reinterpret_cast<const float2*>(a.init_s + ci * a.init_stride + lt * G::W);
#pragma unroll
    for (int m = 0; m < G::LR; ++m) c[m] = WF_LDG(src + m);
  } else {
#pragma unroll
    for (int m = 0; m < G::LR; ++m) c[m] = make_float2(0.f, 0.f);
  }
  const BandCoef cf{a.fg, G::WH, a.band_map, cb, Pb, buf, a.band_off, a.n_bins, tau, 1.0f / NPIX, NPIX};
  sample_sweeps<N>(S, lt, c, a.aq, cf, a.sc->sqrt_tau, a.step0, a.chain0 + uint32_t(ci), a.key0, a.key1,
                   a.n_sweeps, a.burn_in, a.thin,
                   reinterpret_cast<char*>(a.out) +
                       ci * a.n_samples * (long long)(G::H * G::W) * out_elem_bytes(a.out_dtype),
                   active, a.out_dtype, a.out_P ? a.out_P + ci * a.n_samples * (long long)a.n_bins : nullptr);
}

// Spin-2 sampler: CTA = FPC images x 2 shear components, component fields interleaved (field 2 i + comp);
// tables aq2 [2][W][H] (per component), fgE and fgB [H][W/2+1]; out [n_chains][n_samples][2][H][W];
// init_s [2][H][W] per image when given (init_stride elements between chains).
struct Spin2Args {
  const float2* aq2;
  const float2* fgE;
  const float2* fgB;
  const Scalars* sc;
  const float* init_s;
  long long init_stride;
  float* out;
  long long n_samples;
  int n_chains;
  int n_sweeps;
  int burn_in;
  int thin;
  uint32_t chain0;
  uint32_t step0;
  uint32_t key0, key1;
  int out_dtype;
};

template <int N, int FPC>
__global__ void __launch_bounds__(2 * N * FPC, 1) k_sample_spin2(Spin2Args a) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int fld = threadIdx.x / N, lt = threadIdx.x % N;
  const int img = fld / 2, comp = fld % 2;
  const int ci = blockIdx.x * FPC + img;
  const bool active = ci < a.n_chains;
  float2* S = reinterpret_cast<float2*>(smem_raw + fld * G::FIELD_BYTES);
  float2* S0 = reinterpret_cast<float2*>(smem_raw + (2 * img) * G::FIELD_BYTES);
  float2* S1 = reinterpret_cast<float2*>(smem_raw + (2 * img + 1) * G::FIELD_BYTES);
  if (a.sc->status != 0) return;  // uniform over the grid
  float2 c[G::LR];
  if (a.init_s != nullptr && active) {
    const float2* src =
        reinterpret_cast<const float2*>(a.init_s + ci * a.init_stride + comp * (long long)(G::H * G::W) + lt * G::W);
#pragma unroll
    for (int m = 0; m < G::LR; ++m) c[m] = WF_LDG(src + m);
  } else {
#pragma unroll
    for (int m = 0; m < G::LR; ++m) c[m] = make_float2(0.f, 0.f);
  }
  const Spin2Coef cf{a.fgE, a.fgB, G::WH, S0, S1, comp};
  const long long n = (long long)(G::H * G::W);
  sample_sweeps<N>(S, lt, c, a.aq2 + comp * n, cf, a.sc->sqrt_tau, a.step0, a.chain0 + uint32_t(ci), a.key0, a.key1,
                   a.n_sweeps, a.burn_in, a.thin,
                   reinterpret_cast<char*>(a.out) + (ci * a.n_samples * 2 + comp) * n * out_elem_bytes(a.out_dtype),
                   active, a.out_dtype, nullptr, comp == 0 ? 0u : 8u, 2 * n);
}

struct SolveArgs {
  const float2* dn;      // [W][H] pixel table (d, 1/N_bar), or (r, 1/N_bar) in rhs mode
  const float* Pk;       // [H][W/2+1]
  const Scalars* sc;
  const double* bnorm2;  // [n_levels] ||S N_lambda^-1 d||^2 per level (rhs mode: ||S r||^2)
  const float* init_s;   // nullptr -> zeros
  float2* prev;          // [H][W/2] scratch: previous s_hat at check sweeps
  float* out;            // [H][W]
  SolveStatus* st;
  double tol;
  double eta;
  double level_tol;
  int max_iter;
  int level_max;
  int check;
  int rhs_mode;          // 1: solve (S^-1 + N^-1) s = r with the table's r (refinement correction)
};

// The G -> 0 iteration with lambda-cooling for one field (one CTA of N threads). On entry c holds the
// starting iterate as pixel rows; on exit the last iterate. Returns the wf_status (0 converged,
// 5 not converged, 6 non-finite); it and rho receive the sweeps done and the last measured residual.
template <int N>
__device__ __forceinline__ int solve_sweeps(float2* S, double* red, int lt, float2 (&c)[N / 2],
                                            const float2* __restrict__ dn, const float* __restrict__ Pk,
                                            const Scalars& sc, const double* bnorm2, float2* prev, double tol,
                                            double eta, double level_tol, int max_iter, int level_max, int check,
                                            int& it, double& rho, bool rhs = false) {
  using G = Geo<N>;
  const double tau = sc.tau;
  int lev = 0;
  double lam = sc.lam0;
  float ltau = float(lam * tau);
  const int last_level = sc.n_levels - 1;
  // t-update on the thread's own staged row (the spectrum row it stores to next)
  float* stg = reinterpret_cast<float*>(S);
  auto t_update = [&](float lt_) {
    stage_row<N>(stg, lt, c);
    t_update_wf_staged<N>(stg, lt, dn, lt_, rhs);
    load_staged_row<N>(stg, lt, c);
  };
  t_update(ltau);
  // One sweep = four transforms, all run by the single forward FFT at the top of the loop (an inverse
  // transform is conj(FFT(conj(x)))), as in the sampler: one copy of the transform code.
  enum { ROW_FWD, COL_FWD, COL_INV, ROW_INV };
  int phase = ROW_FWD;
  it = 0;
  int k = 0;       // sweeps at the current level
  int status = 1;  // 1 = running
  rho = -1.0;
  while (true) {
    fft<G::LR, false>(c);
    if (phase == ROW_FWD) {
      r2c_post_all<G::LR>(c, std::make_integer_sequence<int, G::LR>{});
      row_store_spec<N>(S, lt, c);
      __syncthreads();
      col_load<N>(S, lt, c);
      __syncthreads();
      phase = COL_FWD;
    } else if (phase == COL_FWD) {
      ++k;
      ++it;
      const bool cmp = (k % check == 0) && k >= 2;
      const bool store = ((k + 1) % check == 0);
      // s-update on the parked modes (the slots this thread stores to after the inverse transform)
      park_modes<N>(S, lt, c);
      const double acc = s_update_wf_parked<N>(S, lt, Pk, ltau, prev, cmp, store);
      unpark_modes<N>(S, lt, c);
      if (cmp) {
        const double tot = block_sum(acc, red) * double(G::H * G::W);
        const double bn = bnorm2[lev];
        const double r2 = bn > 0.0 ? tot / bn : tot;
        rho = sqrt(r2);
        if (!(r2 == r2) || r2 > 1e300) {
          status = 6;  // non-finite residual
        } else if (lev < last_level) {
          if (rho < level_tol || k >= level_max) {
            ++lev;
            lam = level_lambda(sc, lev, eta);
            ltau = float(lam * tau);
            k = 0;
          }
        } else if (rho < tol) {
          status = 0;
        }
      }
      if (status == 1 && it >= max_iter) status = 5;  // not converged
      conj_all<G::LC>(c);
      phase = COL_INV;
    } else if (phase == COL_INV) {
      conj_all<G::LC>(c);
      col_store_inv<N>(S, lt, c);
      __syncthreads();
      row_load_spec<N>(S, lt, c);
      __syncthreads();
      c2r_pre_all<G::LR>(c, std::make_integer_sequence<int, G::LR>{});
      conj_all<G::LR>(c);
      phase = ROW_INV;
    } else {
      conj_all<G::LR>(c);  // c[m] = (s[2m], s[2m+1])
      if (status != 1) break;
      t_update(ltau);
      phase = ROW_FWD;
    }
  }
  return status;
}

template <int N>
__global__ void __launch_bounds__(N) k_solve(SolveArgs a) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* S = reinterpret_cast<float2*>(smem_raw);
  float* stg = reinterpret_cast<float*>(S);
  double* red = reinterpret_cast<double*>(smem_raw + G::FIELD_BYTES);
  const int lt = threadIdx.x;
  const Scalars sc = *a.sc;
  if (sc.status != 0) return;
  float2 c[G::LR];
  if (a.init_s != nullptr) {
    const float2* src = reinterpret_cast<const float2*>(a.init_s + lt * G::W);
#pragma unroll
    for (int m = 0; m < G::LR; ++m) c[m] = WF_LDG(src + m);
  } else {
#pragma unroll
    for (int m = 0; m < G::LR; ++m) c[m] = make_float2(0.f, 0.f);
  }
  int it = 0;
  double rho = -1.0;
  const int status = solve_sweeps<N>(S, red, lt, c, a.dn, a.Pk, sc, a.bnorm2, a.prev, a.tol, a.eta, a.level_tol,
                                     a.max_iter, a.level_max, a.check, it, rho, a.rhs_mode != 0);
  stage_row<N>(stg, lt, c);
  __syncthreads();
  copy_out<N>(stg, lt, a.out);
  if (lt == 0) {
    a.st->status = status;
    a.st->iters = it;
    a.st->resid = rho;
  }
}

// ||S N_lambda^-1 d||^2 of one cooling level (all N threads of the CTA; every thread gets the sum)
template <int N>
__device__ __forceinline__ double level_norm(float2* S, double* red, int lt, const float2* __restrict__ dn,
                                             const float* __restrict__ Pk, float ltau) {
  using G = Geo<N>;
  float2 c[G::LR];
  rhs_row<N>(c, lt, dn, ltau);
  row_forward<N>(c);
  row_store_spec<N>(S, lt, c);
  __syncthreads();
  col_load<N>(S, lt, c);
  fft<G::LC, false>(c);
  const double tot = block_sum(p2_power<N>(c, lt, Pk), red);
  return tot / double(G::H * G::W);
}

// ||S N_lambda^-1 d||^2 for every cooling level (one CTA per level)
struct BnormArgs {
  const float2* dn;
  const float* Pk;
  const Scalars* sc;
  double* bnorm2;
  double eta;
};

template <int N>
__global__ void __launch_bounds__(N) k_bnorm(BnormArgs a) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* S = reinterpret_cast<float2*>(smem_raw);
  double* red = reinterpret_cast<double*>(smem_raw + G::FIELD_BYTES);
  const int lev = blockIdx.x, lt = threadIdx.x;
  const Scalars sc = *a.sc;
  if (sc.status != 0 || lev >= sc.n_levels) return;
  const double v = level_norm<N>(S, red, lt, a.dn, a.Pk, float(level_lambda(sc, lev, a.eta) * sc.tau));
  if (lt == 0) a.bnorm2[lev] = v;
}

// Weighted spectral power of real fields v_f = a_f + sgn * b_f (b may be null): out[f*nw + j] =
// sum_k w_j(k) |(U v_f)_k|^2 with U the unitary 2D DFT (one CTA per field).
struct WpowerArgs {
  const float* a;
  const float* b;
  float sgn;
  int n_fields;
  const float* w;
  int nw;
  double* out;
};

template <int N>
__global__ void __launch_bounds__(N) k_wpower(WpowerArgs p) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* S = reinterpret_cast<float2*>(smem_raw);
  double* red = reinterpret_cast<double*>(smem_raw + G::FIELD_BYTES);
  const int f = blockIdx.x, lt = threadIdx.x;
  const long long base = (long long)f * G::H * G::W + (long long)lt * G::W;
  float2 c[G::LR];
#pragma unroll
  for (int m = 0; m < G::LR; ++m) {
    float2 v = reinterpret_cast<const float2*>(p.a + base)[m];
    if (p.b) {
      const float2 u = reinterpret_cast<const float2*>(p.b + base)[m];
      v = make_float2(fmaf(p.sgn, u.x, v.x), fmaf(p.sgn, u.y, v.y));
    }
    c[m] = v;
  }
  row_forward<N>(c);
  row_store_spec<N>(S, lt, c);
  __syncthreads();
  col_load<N>(S, lt, c);
  fft<G::LC, false>(c);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  wpower_acc<N>(c, lt, p.w, p.nw, acc);
  for (int j = 0; j < p.nw; ++j) {
    const double tot = block_sum(acc[j], red);
    if (lt == 0) p.out[f * p.nw + j] = tot / double(G::H * G::W);
  }
}

}  // namespace wf
