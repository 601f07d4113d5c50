// Accumulators for per-bin sums: compensated float32 (mixed) and plain float64.
#pragma once

#include <cuda_runtime.h>

namespace gbk {

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest, no contraction).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// Compensated float32 sum (running sum plus accumulated rounding errors); the warp
// total combines lanes pairwise with TwoSum and returns hi + lo in float64.
struct CompF {
  float s, c;
  __device__ __forceinline__ void init() { s = 0.f; c = 0.f; }
  __device__ __forceinline__ void add(float x) {
    float t, e;
    two_sum(s, x, t, e);
    s = t;
    c = __fadd_rn(c, e);
  }
  // the warp's total as a float pair (hi, lo), hi + lo the compensated sum
  __device__ __forceinline__ float2 warp_pair() const {
    float hi = s, lo = c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
      const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
      float t, e;
      two_sum(hi, ohi, t, e);
      hi = t;
      lo = __fadd_rn(__fadd_rn(lo, olo), e);
    }
    return make_float2(hi, lo);
  }
  __device__ __forceinline__ double warp_total() const {
    float hi = s, lo = c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
      const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
      float t, e;
      two_sum(hi, ohi, t, e);
      hi = t;
      lo = __fadd_rn(__fadd_rn(lo, olo), e);
    }
    return (double)hi + (double)lo;
  }
};

// u = 1 + a rho for a PSD ratio a = S_acc / S_oms held as a float pair ah + al: the small term
// al rho enters before the product a rho is rounded, so the float rounding of a (the same in
// every bin of a walker) leaves no error common to all bins; what remains is random per bin.
__device__ __forceinline__ float one_plus(float ah, float al, float rho) { return 1.0f + fmaf(ah, rho, al * rho); }

// ln u for u >= 1, split as e ln 2 + ln m with m in [1, 2): returns ln m and adds the integer e
// to `e`. ln m < 0.7 keeps the float rounding of the returned part below 6e-8, where ln u itself
// (up to ~8 at low frequencies) would carry up to 5e-7 per bin, enough to add up to ~1e-2 over
// 2^20 bins; the caller multiplies the integer sum of e by ln 2 in float64.
__device__ __forceinline__ float log_split(float u, int& e) {
  const int bits = __float_as_int(u);
  e += (bits >> 23) - 127;
  return logf(__int_as_float((bits & 0x007fffff) | 0x3f800000));
}
constexpr double kLn2 = 0.6931471805599453094;

struct PlainD {
  double s;
  __device__ __forceinline__ void init() { s = 0.0; }
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double warp_total() const {
    double v = s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  }
};

}  // namespace gbk
