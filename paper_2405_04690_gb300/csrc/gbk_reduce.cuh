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
