// Truncated diagonal Gaussian mixture on the unit box: the learned birth / in-model
// proposal of the sampler (Eq. rj-acceptance needs its density exactly).
//
// A source of band b is mapped to u in [0, 1]^8 where the band's prior is uniform:
//   u0 = (ln A - ln A_min) / (ln A_max - ln A_min)   u1 = (f0 - lo_b) / (hi_b - lo_b)
//   u2 = (Mc - Mc_min) / (Mc_max - Mc_min)            u3 = phi0 / 2 pi    u4 = psi / pi
//   u5 = (cos i + 1) / 2    u6 = (sin beta + 1) / 2    u7 = lambda / 2 pi
// ([lo_b, hi_b) the band's f0 allowance, Mc the chirp mass of (f0, fdot)). The network
// gives 16 x (1 weight logit, 8 mean logits, 8 width logits): pi = softmax,
// mu = sigmoid, ln s = S_MIN + (S_MAX - S_MIN) sigmoid. Each component is a product of
// normals truncated to [0, 1] and renormalised by Z = Phi((1 - mu)/s) - Phi(-mu/s), so
// q integrates to 1 on the box. The sampler uses q_eps = eps + (1 - eps) q (a fraction
// eps of the draws from the prior, density 1).
#pragma once

#include <math.h>
#include <stdint.h>

namespace gbk {

constexpr int kMixComp = 16;
constexpr int kMixDim = 8;
constexpr int kMixOut = kMixComp * (1 + 2 * kMixDim);   // 272
constexpr double kMixSMin = -10.0, kMixSMax = 0.0;
constexpr double kLogSqrt2Pi = 0.91893853320467274178;

template <typename T>
struct __align__(16) MixRow {   // 16-byte aligned: rows are read with vector loads
  T lw[kMixComp];              // ln pi_k - sum_d (ln s_kd + ln Z_kd) - 8 ln sqrt(2 pi)
  T cw[kMixComp];              // cumulative weights pi_0 + ... + pi_k
  T mu[kMixComp][kMixDim];
  T is[kMixComp][kMixDim];     // 1 / s
  T s[kMixComp][kMixDim];
  T plo[kMixComp][kMixDim];    // Phi(-mu / s)
  T pw[kMixComp][kMixDim];     // Z
};

__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double m_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float m_cdf(float x) { return normcdff(x); }
__device__ __forceinline__ double m_cdf(double x) { return normcdf(x); }
__device__ __forceinline__ float m_icdf(float x) { return normcdfinvf(x); }
__device__ __forceinline__ double m_icdf(double x) { return normcdfinv(x); }

// Build one row from the network's raw outputs (one thread).
template <typename T>
__device__ void mix_build(const float* __restrict__ raw, MixRow<T>& m) {
  T mx = (T)raw[0];
  for (int k = 1; k < kMixComp; ++k) mx = fmax(mx, (T)raw[k * 17]);
  T se = 0;
  for (int k = 0; k < kMixComp; ++k) se += m_exp((T)raw[k * 17] - mx);
  const T lse = mx + m_log(se);
  T cum = 0;
  for (int k = 0; k < kMixComp; ++k) {
    const T lpi = (T)raw[k * 17] - lse;
    cum += m_exp(lpi);
    m.cw[k] = cum;
    T acc = lpi - (T)(kMixDim * kLogSqrt2Pi);
    for (int d = 0; d < kMixDim; ++d) {
      const T mu = (T)1 / ((T)1 + m_exp(-(T)raw[k * 17 + 1 + d]));
      const T sg = (T)1 / ((T)1 + m_exp(-(T)raw[k * 17 + 9 + d]));
      const T ls = (T)kMixSMin + (T)(kMixSMax - kMixSMin) * sg;
      const T s = m_exp(ls);
      const T lo = m_cdf(-mu / s);
      const T z = m_cdf(((T)1 - mu) / s) - lo;
      m.mu[k][d] = mu;
      m.s[k][d] = s;
      m.is[k][d] = (T)1 / s;
      m.plo[k][d] = lo;
      m.pw[k][d] = z;
      acc -= ls + m_log(z);
    }
    m.lw[k] = acc;
  }
}

// 8 (16) contiguous values of a row in vector loads (rows are 16-byte aligned), so that the
// loads of a component are in flight together.
__device__ __forceinline__ void ld8(const float* p, float* o) {
  const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
__device__ __forceinline__ void ld8(const double* p, double* o) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double2 a = *reinterpret_cast<const double2*>(p + 2 * i);
    o[2 * i] = a.x;
    o[2 * i + 1] = a.y;
  }
}

// ln q_eps(u): log-sum-exp over the components in one pass (running maximum).
template <typename T>
__device__ T mix_logq(const MixRow<T>& m, const T* u, T eps) {
  if (eps >= (T)1) return (T)0;
  T uu[kMixDim];
#pragma unroll
  for (int d = 0; d < kMixDim; ++d) uu[d] = u[d];
  T mx = -(T)INFINITY, se = (T)0;
#pragma unroll 4
  for (int k = 0; k < kMixComp; ++k) {
    T mu[kMixDim], is[kMixDim];
    ld8(m.mu[k], mu);
    ld8(m.is[k], is);
    T acc = m.lw[k];
#pragma unroll
    for (int d = 0; d < kMixDim; ++d) {
      const T z = (uu[d] - mu[d]) * is[d];
      acc -= (T)0.5 * z * z;
    }
    if (acc > mx) {
      se = se * m_exp(mx - acc) + (T)1;
      mx = acc;
    } else {
      se += m_exp(acc - mx);
    }
  }
  const T lq = mx + m_log(se);
  if (eps <= (T)0) return lq;
  // ln[eps + (1 - eps) e^lq] = logaddexp(ln eps, ln(1 - eps) + lq)
  const T a = m_log(eps), b = m_log1p(-eps) + lq;
  const T hi = fmax(a, b), lo = fmin(a, b);
  return hi + m_log1p(m_exp(lo - hi));
}

// (w + 1/2) 2^-32: a uniform in (0, 1) from one 32-bit word (exact in float64).
__device__ __forceinline__ double mix_u32(uint32_t w) { return ((double)w + 0.5) * 2.3283064365386963e-10; }

// Draw u from the mixture: component = first k with cw_k > u32(w_comp) (the last one if
// rounding leaves none); per dimension u_d = mu + s Phi^-1(plo + Z u32(w_d)), clamped.
template <typename T>
__device__ void mix_draw(const MixRow<T>& m, uint32_t w_comp, const uint32_t* w_dims, T* u) {
  const T v = (T)mix_u32(w_comp);
  T cw[kMixComp];
  ld8(m.cw, cw);
  ld8(m.cw + 8, cw + 8);
  int k = kMixComp - 1;
#pragma unroll
  for (int j = kMixComp - 1; j >= 0; --j)
    if (v < cw[j]) k = j;
  T pl[kMixDim], pw[kMixDim], mu[kMixDim], sg[kMixDim];
  ld8(m.plo[k], pl);
  ld8(m.pw[k], pw);
  ld8(m.mu[k], mu);
  ld8(m.s[k], sg);
#pragma unroll
  for (int d = 0; d < kMixDim; ++d) {
    const T p = pl[d] + pw[d] * (T)mix_u32(w_dims[d]);
    T x = mu[d] + sg[d] * m_icdf(p);
    x = x < (T)0 ? (T)0 : x;        // also maps a NaN-free -inf to 0
    x = x > (T)1 ? (T)1 : x;
    u[d] = x;
  }
}

}  // namespace gbk
