// Register-resident building blocks of the messenger-field Gibbs step (Alg. 1 of the paper):
//   * compile-time twiddle factors,
//   * an in-register radix-2 complex FFT of length L (natural order in and out),
//   * the real <-> half-length-complex packing used for the row transforms,
//   * Philox4x32-10 and the Box-Muller transform for the G(0,1) draws.
// Everything here is __host__ __device__ so the same arithmetic can be exercised on the host.
#pragma once

#include <cstdint>
#include <utility>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#if defined(__CUDA_ARCH__)
#define WF_HD __host__ __device__ __forceinline__
#else
#define WF_HD inline
#endif

namespace wf {

// ---------------------------------------------------------------------------------------------
// complex helpers (float2 = re, im)
// ---------------------------------------------------------------------------------------------
// On sm_100 and later the component-wise operations use the paired FP32 instructions (two lanes of a
// float2 per instruction, each rounded as the scalar operation): one issue slot instead of two. The
// results are bit-identical to the scalar forms (measured: same samples, 14-17% faster Gibbs sweeps).
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000) && !defined(WF_NO_F32X2)
#define WF_F32X2 1
#endif
WF_HD float2 cadd(float2 a, float2 b) {
#if defined(WF_F32X2)
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
WF_HD float2 csub(float2 a, float2 b) {
#if defined(WF_F32X2)
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);  // a - b, exact product then one rounding
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}
WF_HD float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
WF_HD float2 cscale(float2 a, float s) {
#if defined(WF_F32X2)
  return __fmul2_rn(a, make_float2(s, s));
#else
  return make_float2(a.x * s, a.y * s);
#endif
}
// a + conj(b) and a - conj(b)
WF_HD float2 cadd_conj(float2 a, float2 b) {
#if defined(WF_F32X2)
  return __ffma2_rn(b, make_float2(1.0f, -1.0f), a);
#else
  return make_float2(a.x + b.x, a.y - b.y);
#endif
}
WF_HD float2 csub_conj(float2 a, float2 b) {
#if defined(WF_F32X2)
  return __ffma2_rn(b, make_float2(-1.0f, 1.0f), a);
#else
  return make_float2(a.x - b.x, a.y + b.y);
#endif
}
// (measured on GB300: a paired form of this product needs broadcast operands and raises register
// pressure enough to spill, so it stays scalar)
WF_HD float2 cmul(float2 a, float2 w) {
  return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
// multiply by i and by -i
WF_HD float2 cmul_i(float2 a) { return make_float2(-a.y, a.x); }
WF_HD float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }

// ---------------------------------------------------------------------------------------------
// compile-time twiddles: cos/sin(2 pi k / n) in double, from the Taylor series after folding the
// angle into [0, pi/4] with the octant symmetries of the circle. Only evaluated in constant
// expressions (template arguments), never at run time.
// ---------------------------------------------------------------------------------------------
constexpr double kPi = 3.14159265358979323846264338327950288;

__host__ __device__ constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int i = 1; i < 14; ++i) {
    term *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int i = 1; i < 14; ++i) {
    term *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
    sum += term;
  }
  return sum;
}
// cos(2 pi k / n) for integer k, n > 0
__host__ __device__ constexpr double cos2pi(long k, long n) {
  k %= n;
  if (k < 0) k += n;
  // reduce with exact integer arithmetic on the numerator 8k over denominator 8n (octants)
  long m = 8 * k;             // angle = 2 pi m / (8 n)
  long N8 = 8 * n;
  // quadrant handling: cos(2pi - a) = cos a
  if (m > N8 / 2) m = N8 - m;                      // now angle in [0, pi]
  bool neg = false;
  if (m > N8 / 4) { m = N8 / 2 - m; neg = true; }  // cos(pi - a) = -cos a, angle in [0, pi/2]
  double r = 0.0;
  if (m > N8 / 8) r = taylor_sin(2.0 * kPi * double(N8 / 4 - m) / double(N8));   // cos a = sin(pi/2 - a)
  else r = taylor_cos(2.0 * kPi * double(m) / double(N8));
  return neg ? -r : r;
}
// sin(2 pi k / n) = cos(2 pi (k - n/4) / n) computed exactly via  sin a = cos(a - pi/2) with 4n denominators
__host__ __device__ constexpr double sin2pi(long k, long n) { return cos2pi(4 * k - n, 4 * n); }

// exp(-2 pi i k / n) (forward) or exp(+2 pi i k / n) (inverse), rounded once to float
template <long K, long N, bool INV>
struct Tw {
  static constexpr float re = float(cos2pi(K, N));
  static constexpr float im = INV ? float(sin2pi(K, N)) : float(-sin2pi(K, N));
};

// multiply a by the twiddle exp(-+2 pi i K / N), skipping the trivial cases
template <long K, long N, bool INV>
WF_HD float2 twiddle(float2 a) {
  constexpr long k = ((K % N) + N) % N;
  if constexpr (k == 0) {
    return a;
  } else if constexpr (4 * k == N) {
    return INV ? cmul_i(a) : cmul_mi(a);
  } else if constexpr (2 * k == N) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (4 * k == 3 * N) {
    return INV ? cmul_mi(a) : cmul_i(a);
  } else {
    return cmul(a, make_float2(Tw<k, N, INV>::re, Tw<k, N, INV>::im));
  }
}

// ---------------------------------------------------------------------------------------------
// in-register radix-2 FFT, length L (power of two), unnormalised, natural order in and out.
// Decimation in time: bit-reverse the register order (free after unrolling), then log2(L) stages.
// ---------------------------------------------------------------------------------------------
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
__host__ __device__ constexpr int bitrev(int v, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((v >> i) & 1) << (bits - 1 - i);
  return r;
}

template <int L, int I>
WF_HD void bitrev_swap(float2 (&x)[L]) {
  constexpr int J = bitrev(I, ilog2(L));
  if constexpr (I < J) {
    float2 t = x[I];
    x[I] = x[J];
    x[J] = t;
  }
}
template <int L, int... I>
WF_HD void bitrev_all(float2 (&x)[L], std::integer_sequence<int, I...>) {
  (bitrev_swap<L, I>(x), ...);
}

template <int L, int HALF, bool INV, int B>
WF_HD void butterfly(float2 (&x)[L]) {
  constexpr int j = B % HALF;
  constexpr int i0 = (B / HALF) * 2 * HALF + j;
  constexpr int i1 = i0 + HALF;
  float2 b = twiddle<j, 2 * HALF, INV>(x[i1]);
  float2 a = x[i0];
  x[i0] = cadd(a, b);
  x[i1] = csub(a, b);
}
template <int L, int HALF, bool INV, int... B>
WF_HD void stage(float2 (&x)[L], std::integer_sequence<int, B...>) {
  (butterfly<L, HALF, INV, B>(x), ...);
}
template <int L, int HALF, bool INV>
WF_HD void stages(float2 (&x)[L]) {
  if constexpr (HALF < L) {
    stage<L, HALF, INV>(x, std::make_integer_sequence<int, L / 2>{});
    stages<L, 2 * HALF, INV>(x);
  }
}

// X[k] = sum_m x[m] exp(-+2 pi i m k / L)
template <int L, bool INV>
WF_HD void fft_radix2(float2 (&x)[L]) {
  static_assert((L & (L - 1)) == 0 && L >= 2, "power-of-two length");
  bitrev_all<L>(x, std::make_integer_sequence<int, L>{});
  stages<L, 1, INV>(x);
}

// Two consecutive radix-2 decimation-in-time stages (halves HALF and 2*HALF) fused into one radix-4
// butterfly on x[b+j], x[b+j+H], x[b+j+2H], x[b+j+3H] with w = exp(-+2 pi i j / 4H):
//   y0 = (a0 + w^2 a1) + (w a2 + w^3 a3)     y2 = (a0 + w^2 a1) - (w a2 + w^3 a3)
//   y1 = (a0 - w^2 a1) -+ i (w a2 - w^3 a3)  y3 = (a0 - w^2 a1) +- i (w a2 - w^3 a3)
// (three twiddle products instead of four).
// s = a + w x and d = a - w x for the compile-time twiddle w = exp(-+2 pi i K / N). For a general w the
// product is fused into s (four FMAs) and d = 2a - s (two FMAs) instead of a product and two sums.
template <long K, long N, bool INV>
WF_HD void tw_addsub(float2 a, float2 x, float2& s, float2& d) {
  constexpr long k = ((K % N) + N) % N;
  if constexpr (k == 0 || 4 * k == N || 2 * k == N || 4 * k == 3 * N) {
    const float2 t = twiddle<K, N, INV>(x);  // 1, -+i, -1, +-i: no multiplications
    s = cadd(a, t);
    d = csub(a, t);
  } else {
    constexpr float wr = Tw<k, N, INV>::re, wi = Tw<k, N, INV>::im;
#if defined(WF_F32X2)
    // the same two roundings per component as the scalar form, as two paired FMAs
    s = __ffma2_rn(x, make_float2(wr, wr), __ffma2_rn(make_float2(x.y, x.x), make_float2(-wi, wi), a));
#else
    s = make_float2(fmaf(wr, x.x, fmaf(-wi, x.y, a.x)), fmaf(wr, x.y, fmaf(wi, x.x, a.y)));
#endif
    d = make_float2(fmaf(2.0f, a.x, -s.x), fmaf(2.0f, a.y, -s.y));  // scalar: measured faster here
  }
}

// Two consecutive radix-2 decimation-in-time stages (halves HALF and 2*HALF) fused into one radix-4
// butterfly on x[b+j], x[b+j+H], x[b+j+2H], x[b+j+3H] with w = exp(-+2 pi i j / 4H):
//   y0 = (a0 + w^2 a1) + (w a2 + w^3 a3)     y2 = (a0 + w^2 a1) - (w a2 + w^3 a3)
//   y1 = (a0 - w^2 a1) -+ i (w a2 - w^3 a3)  y3 = (a0 - w^2 a1) +- i (w a2 - w^3 a3)
// (three twiddle products instead of four, two of them fused into the sums).
template <int L, int HALF, bool INV, int B>
WF_HD void butterfly4(float2 (&x)[L]) {
  constexpr int j = B % HALF;
  constexpr int i0 = (B / HALF) * 4 * HALF + j;
  float2 s01, d01, s23, d23;
  tw_addsub<2 * j, 4 * HALF, INV>(x[i0], x[i0 + HALF], s01, d01);
  tw_addsub<3 * j, 4 * HALF, INV>(twiddle<j, 4 * HALF, INV>(x[i0 + 2 * HALF]), x[i0 + 3 * HALF], s23, d23);
  x[i0] = cadd(s01, s23);
  x[i0 + 2 * HALF] = csub(s01, s23);
  // d01 -+ i d23 (forward: -i d23 = (d23.y, -d23.x)), component by component
  if (INV) {
    x[i0 + HALF] = make_float2(d01.x - d23.y, d01.y + d23.x);
    x[i0 + 3 * HALF] = make_float2(d01.x + d23.y, d01.y - d23.x);
  } else {
    x[i0 + HALF] = make_float2(d01.x + d23.y, d01.y - d23.x);
    x[i0 + 3 * HALF] = make_float2(d01.x - d23.y, d01.y + d23.x);
  }
}
template <int L, int HALF, bool INV, int... B>
WF_HD void stage4(float2 (&x)[L], std::integer_sequence<int, B...>) {
  (butterfly4<L, HALF, INV, B>(x), ...);
}
template <int L, int HALF, bool INV>
WF_HD void stages4(float2 (&x)[L]) {
  if constexpr (4 * HALF <= L) {
    stage4<L, HALF, INV>(x, std::make_integer_sequence<int, L / 4>{});
    stages4<L, 4 * HALF, INV>(x);
  }
}

// X[k] = sum_m x[m] exp(-+2 pi i m k / L): bit reversal, one radix-2 stage if log2 L is odd, then
// radix-4 stages.
template <int L, bool INV>
WF_HD void fft(float2 (&x)[L]) {
  static_assert((L & (L - 1)) == 0 && L >= 2, "power-of-two length");
  bitrev_all<L>(x, std::make_integer_sequence<int, L>{});
  if constexpr (ilog2(L) % 2 == 1) {
    stage<L, 1, INV>(x, std::make_integer_sequence<int, L / 2>{});
    stages4<L, 2, INV>(x);
  } else {
    stages4<L, 1, INV>(x);
  }
}

// ---------------------------------------------------------------------------------------------
// real transforms of length 2L through one complex transform of length L.
// Packed half-spectrum: X[0] = (R[0], R[L]) (both real), X[k] = R[k] for 0 < k < L,
// where R[k] = sum_x r[x] exp(-2 pi i k x / (2L)).
// ---------------------------------------------------------------------------------------------
template <int L, int K>
WF_HD void r2c_post_pair(float2 (&c)[L]) {
  // c holds C = FFT_L(r[2m] + i r[2m+1]); produce R[K] and R[L-K]
  if constexpr (K == 0) {
    float2 c0 = c[0];
    c[0] = make_float2(c0.x + c0.y, c0.x - c0.y);
  } else if constexpr (2 * K == L) {
    c[K] = cconj(c[K]);
  } else if constexpr (K < L - K) {
    const float2 a = c[K], bc = c[L - K];            // b = conj(bc)
    float2 E = cscale(cadd_conj(a, bc), 0.5f);       // transform of the even samples
    float2 O = cmul_mi(cscale(csub_conj(a, bc), 0.5f));  // transform of the odd samples
    float2 WO = twiddle<K, 2 * L, false>(O);
    c[K] = cadd(E, WO);
    c[L - K] = cconj(csub(E, WO));
  }
}
template <int L, int... K>
WF_HD void r2c_post_all(float2 (&c)[L], std::integer_sequence<int, K...>) {
  (r2c_post_pair<L, K>(c), ...);
}

// inverse: packed half-spectrum R -> C' so that IFFT_L(C')[m] = r[2m] + i r[2m+1] with
// r[x] = sum_k R[k] exp(+2 pi i k x / (2L)) over the full (Hermitian) spectrum (unnormalised).
template <int L, int K>
WF_HD void c2r_pre_pair(float2 (&c)[L]) {
  if constexpr (K == 0) {
    float2 r = c[0];  // (R0, RL)
    c[0] = make_float2(r.x + r.y, r.x - r.y);
  } else if constexpr (2 * K == L) {
    c[K] = cscale(cconj(c[K]), 2.0f);
  } else if constexpr (K < L - K) {
    // E'[K] = R[K] + conj R[L-K] (even samples), O'[K] = (R[K] - conj R[L-K]) exp(+2 pi i K / 2L)
    // (odd samples); both are Hermitian in K <-> L-K, so C'[L-K] = conj E' + i conj O'.
    const float2 a = c[K], bc = c[L - K];  // b = conj(bc)
    float2 E = cadd_conj(a, bc);
    float2 O = twiddle<K, 2 * L, true>(csub_conj(a, bc));
    c[K] = cadd(E, cmul_i(O));
    c[L - K] = cadd(cconj(E), cmul_i(cconj(O)));
  }
}
template <int L, int... K>
WF_HD void c2r_pre_all(float2 (&c)[L], std::integer_sequence<int, K...>) {
  (c2r_pre_pair<L, K>(c), ...);
}

// ---------------------------------------------------------------------------------------------
// sample output element types: FP32, or the state rounded once (to nearest even) to BF16 or FP16
// ---------------------------------------------------------------------------------------------
enum OutType { kOutF32 = 0, kOutBF16 = 1, kOutF16 = 2 };
WF_HD int out_elem_bytes(int t) { return t == kOutF32 ? 4 : 2; }
// pair e = (value 2e, value 2e+1) of an output array of type t
#if defined(__CUDACC__)
__device__ __forceinline__ void store_pair(void* out, long long e, float2 v, int t) {
  if (t == kOutBF16)
    reinterpret_cast<__nv_bfloat162*>(out)[e] = __floats2bfloat162_rn(v.x, v.y);
  else if (t == kOutF16)
    reinterpret_cast<__half2*>(out)[e] = __floats2half2_rn(v.x, v.y);
  else
    reinterpret_cast<float2*>(out)[e] = v;
}
#endif

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) and Box-Muller
// ---------------------------------------------------------------------------------------------
struct u4 { uint32_t x, y, z, w; };

WF_HD void mulhilo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
#if defined(__CUDA_ARCH__)
  hi = __umulhi(a, b);
  lo = a * b;
#else
  uint64_t p = uint64_t(a) * uint64_t(b);
  hi = uint32_t(p >> 32);
  lo = uint32_t(p);
#endif
}

WF_HD u4 philox4x32_10(u4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo(0xD2511F53u, c.x, hi0, lo0);
    mulhilo(0xCD9E8D57u, c.z, hi1, lo1);
    c = u4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// 32-bit word -> odd multiple of 2^-24 in (0, 1), exact in float
WF_HD float to_uniform(uint32_t x) { return float(2u * (x >> 9) + 1u) * 5.9604644775390625e-08f; }

// (z0, z1) = sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1), u = (2 floor(x / 2^9) + 1) 2^-24.
// Device: the 23 bits k = floor(x / 2^9) become v = 1 + k 2^-23 by placing them under the exponent of 1
// (exact, no integer-to-float conversion), and u = v - (1 - 2^-24) = (2k + 1) 2^-24 exactly (the operands
// are within a factor of two, so the difference is exact); -2 ln u0 = -2 ln(2) log2(u0) from the hardware
// log2, clamped at the smallest normal float (log2 of the largest u, 1 - 2^-24, may round to zero), its
// square root as x * rsqrt(x); the angle 2 pi (u1 - 1/2) = 2 pi v1 - 2 pi (3/2 - 2^-24) in (-pi, pi) as one
// FMA (absolute error below 3.5e-7), for which cos(2 pi u) = -cos(2 pi (u - 1/2)) and likewise for sin.
WF_HD void box_muller(uint32_t a, uint32_t b, float& z0, float& z1) {
#if defined(__CUDA_ARCH__)
  const float u0 = __int_as_float(0x3f800000u | (a >> 9)) - 0.999999940395355224609375f;   // (2k + 1) 2^-24
  const float ang = fmaf(__int_as_float(0x3f800000u | (b >> 9)), 6.2831854820251465f,
                         -9.424777848530681f);                                              // 2 pi (u1 - 1/2)
  const float e = fmaxf(-1.3862943611198906f * __log2f(u0), 1.17549435e-38f);          // -2 ln u0
  const float r = e * rsqrtf(e);
  float sn, cs;
  __sincosf(ang, &sn, &cs);
  z0 = -r * cs;
  z1 = -r * sn;
#else
  const float u0 = to_uniform(a), u1 = to_uniform(b);
  const float r = sqrtf(-2.0f * logf(u0));
  const float a2 = 6.28318530717958647692f * (u1 - 0.5f);
  z0 = -r * cosf(a2);
  z1 = -r * sinf(a2);
#endif
}

WF_HD void normals4(uint32_t group, uint32_t step, uint32_t chain, uint32_t stream, uint32_t k0, uint32_t k1,
                    float (&z)[4]) {
  u4 r = philox4x32_10(u4{group, step, chain, stream}, k0, k1);
  box_muller(r.x, r.y, z[0], z[1]);
  box_muller(r.z, r.w, z[2], z[3]);
}

}  // namespace wf
