// Host-side driver around curand's own Philox4x32-10 (curand_philox4x32_x.h), used only by the CPU
// tests to pin the oracle's Philox implementation against an independent one. The header's functions
// are device-only by default; defining QUALIFIERS first makes them callable from host code, where the
// header already provides a host branch for the 32x32->64-bit multiply.
// Reads lines "c0 c1 c2 c3 k0 k1" (decimal uint32) from stdin, prints "r0 r1 r2 r3".
#include <cstdio>
#include <cuda_runtime.h>
#define QUALIFIERS static inline __host__ __device__
#include <curand_philox4x32_x.h>

int main() {
  unsigned c0, c1, c2, c3, k0, k1;
  while (std::scanf("%u %u %u %u %u %u", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
    uint4 c = make_uint4(c0, c1, c2, c3);
    uint2 k = make_uint2(k0, k1);
    uint4 r = curand_Philox4x32_10(c, k);
    std::printf("%u %u %u %u\n", r.x, r.y, r.z, r.w);
  }
  return 0;
}
