// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC 2011) and the
// exact conversions the sampler uses. The same counters give the same words on the host
// side, so every random draw of a sweep is reproducible and independent of scheduling.
#pragma once

#include <stdint.h>

namespace gbk {

struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  U4 r;
  r.x = c0; r.y = c1; r.z = c2; r.w = c3;
  return r;
}

// u53(a, b) = ((a >> 5) 2^26 + (b >> 6)) 2^-53 in [0, 1), exact.
__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}
// u32(a) = (a + 1/2) 2^-32 in (0, 1), exact.
__device__ __forceinline__ double u32(uint32_t a) { return ((double)a + 0.5) * (1.0 / 4294967296.0); }
// u24(a) = (a >> 8) 2^-24 in [0, 1), exact.
__device__ __forceinline__ double u24(uint32_t a) { return (double)(a >> 8) * (1.0 / 16777216.0); }
// (a * n) >> 32 in [0, n).
__device__ __forceinline__ uint32_t ranged(uint32_t a, uint32_t n) {
  return (uint32_t)(((uint64_t)a * (uint64_t)n) >> 32);
}

}  // namespace gbk
