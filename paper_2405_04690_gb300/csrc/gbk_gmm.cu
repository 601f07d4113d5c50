// Batched Gaussian-mixture refit of the reversible-jump proposal (Sec. V.E, App. G): one CTA
// per group (band) fits a diagonal-covariance mixture to the group's points by EM (Dempster,
// Laird & Rubin 1977) and writes it as the mixture outputs the sampler reads.
#include <float.h>
#include <math.h>

#include "gbk_internal.cuh"
#include "gbk_mix.cuh"

namespace gbk {
namespace {

constexpr int kGmmCap = 2048;       // present points used per group (the first kGmmCap)
constexpr int kGmmThreads = 256;
constexpr int kGmmWarps = kGmmThreads / 32;
constexpr int kAcc = 1 + 2 * kMixDim;   // S0, S1[8], S2[8]
constexpr double kLog2Pi = 1.8378770664093454836;
constexpr double kWOff = -30.0;     // weight logit of a component left out of the proposal
constexpr double kClamp = 1e-9;

template <typename T>
struct GmmSmem {
  float pts[kGmmCap][kMixDim];
  T em[kMixComp][kMixDim], eiv[kMixComp][kMixDim], ec[kMixComp];   // E-step constants
  unsigned long long keys[kGmmCap];
  double acc[kGmmWarps][kMixComp][kAcc];
  double llw[kGmmWarps];
  double w[kMixComp], mu[kMixComp][kMixDim], var[kMixComp][kMixDim], nk[kMixComp];
  double red[kGmmWarps][kMixDim], mean[kMixDim];
  int cnt[kGmmThreads];
  int used[kMixComp];
  int n;
};

// float -> uint32 whose unsigned order is the float order
__device__ __forceinline__ uint32_t fkey(float v) {
  const uint32_t b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float g_exp(float x) { return expf(x); }
__device__ __forceinline__ double g_exp(double x) { return exp(x); }
__device__ __forceinline__ float g_log(float x) { return logf(x); }
__device__ __forceinline__ double g_log(double x) { return log(x); }

__device__ __forceinline__ double logit_c(double p) {
  p = fmin(fmax(p, kClamp), 1.0 - kClamp);
  return log(p / (1.0 - p));
}

// Per-dimension sum over the n points of f(x_d) (double, fixed order: thread-strided, then
// a shuffle tree per warp, then the warps in order); result in S.mean.
template <typename T, typename F>
__device__ void dim_sums(GmmSmem<T>& S, int n, F f) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double s[kMixDim];
#pragma unroll
  for (int d = 0; d < kMixDim; ++d) s[d] = 0.0;
  for (int i = tid; i < n; i += kGmmThreads)
#pragma unroll
    for (int d = 0; d < kMixDim; ++d) s[d] += f((double)S.pts[i][d], d);
#pragma unroll
  for (int d = 0; d < kMixDim; ++d) {
    for (int o = 16; o; o >>= 1) s[d] += __shfl_xor_sync(0xffffffffu, s[d], o);
    if (lane == 0) S.red[wid][d] = s[d];
  }
  __syncthreads();
  if (tid < kMixDim) {
    double t = 0.0;
    for (int w = 0; w < kGmmWarps; ++w) t += S.red[w][tid];
    S.mean[tid] = t;
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kGmmThreads) k_gmm_fit(const float* __restrict__ x, int n_points, int n_comp,
                                                         int n_iter, double reg, double min_weight, int n_groups,
                                                         int n_copies, float* __restrict__ raw_out,
                                                         double* __restrict__ fit_out, double* __restrict__ loglike) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GmmSmem<T>& S = *reinterpret_cast<GmmSmem<T>*>(smem_raw);
  const int g = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const float* xg = x + (int64_t)g * n_points * kMixDim;

  // ---- present rows (no NaN), compacted in order: per-thread chunk counts, scan, copy
  const int chunk = (n_points + kGmmThreads - 1) / kGmmThreads;
  const int r0 = min(n_points, tid * chunk), r1 = min(n_points, r0 + chunk);
  auto present = [&](int r) {
    bool ok = true;
#pragma unroll
    for (int d = 0; d < kMixDim; ++d) ok = ok && !isnan(xg[(int64_t)r * kMixDim + d]);
    return ok;
  };
  int c = 0;
  for (int r = r0; r < r1; ++r) c += present(r) ? 1 : 0;
  S.cnt[tid] = c;
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int i = 0; i < kGmmThreads; ++i) {
      const int v = S.cnt[i];
      S.cnt[i] = run;
      run += v;
    }
    S.n = min(run, kGmmCap);
  }
  __syncthreads();
  int o = S.cnt[tid];
  for (int r = r0; r < r1 && o < kGmmCap; ++r)
    if (present(r)) {
#pragma unroll
      for (int d = 0; d < kMixDim; ++d) S.pts[o][d] = xg[(int64_t)r * kMixDim + d];
      ++o;
    }
  __syncthreads();
  const int n = S.n;
  const int K = min(n_comp, n);

  // ---- start: points sorted by u1 (ties by position), means at ranks floor((k + 1/2) n / K)
  if (n > 0) {
    int p2 = 1;
    while (p2 < n) p2 <<= 1;
    for (int i = tid; i < p2; i += kGmmThreads)
      S.keys[i] = i < n ? ((unsigned long long)fkey(S.pts[i][1]) << 32) | (unsigned)i : ~0ull;
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < p2; i += kGmmThreads) {
          const int l = i ^ j;
          if (l > i) {
            const unsigned long long a = S.keys[i], b = S.keys[l];
            const bool up = (i & k) == 0;
            if ((a > b) == up) {
              S.keys[i] = b;
              S.keys[l] = a;
            }
          }
        }
        __syncthreads();
      }
    if (tid < K * kMixDim) {
      const int k = tid / kMixDim, d = tid % kMixDim;
      const int r = (int)floor(((double)k + 0.5) * (double)n / (double)K);
      S.mu[k][d] = (double)S.pts[(int)(S.keys[r] & 0xffffffffu)][d];
    }
    dim_sums(S, n, [](double v, int) { return v; });
    double mloc[kMixDim];   // per-dimension means (read before the next dim_sums overwrites them)
#pragma unroll
    for (int d = 0; d < kMixDim; ++d) mloc[d] = S.mean[d] / n;
    dim_sums(S, n, [&](double v, int d) { return (v - mloc[d]) * (v - mloc[d]); });
    if (tid < K * kMixDim) S.var[tid / kMixDim][tid % kMixDim] = S.mean[tid % kMixDim] / n + reg;
    if (tid < K) S.w[tid] = 1.0 / K;
    __syncthreads();
  }

  // ---- EM: n_iter (E, M) passes, then one E pass for the log-likelihood of the result
  const int h = lane >> 4, k = lane & 15;
  for (int it = 0; it <= n_iter && n > 0; ++it) {
    // E-step constants, once per CTA, one thread per (component, dimension) in warps 0-3:
    // (T) mu, (T) 1/var and ln w - 1/2 sum_d (ln var + ln 2 pi) (sum over the 8 lanes of k)
    if (tid < kMixComp * kMixDim) {
      const int kk = tid / kMixDim, d = tid % kMixDim;
      double lv = 0.0;
      if (kk < K) {
        S.em[kk][d] = (T)S.mu[kk][d];
        S.eiv[kk][d] = (T)(1.0 / S.var[kk][d]);
        lv = log(S.var[kk][d]) + kLog2Pi;
      }
      for (int o = 4; o; o >>= 1) lv += __shfl_xor_sync(0xffffffffu, lv, o, kMixDim);
      if (kk < K && d == 0) S.ec[kk] = (T)(log(S.w[kk]) - 0.5 * lv);
    }
    __syncthreads();
    T m_k[kMixDim], iv_k[kMixDim], c_k = (T)0;
    if (k < K) {
#pragma unroll
      for (int d = 0; d < kMixDim; ++d) {
        m_k[d] = S.em[k][d];
        iv_k[d] = S.eiv[k][d];
      }
      c_k = S.ec[k];
    } else {
#pragma unroll
      for (int d = 0; d < kMixDim; ++d) m_k[d] = iv_k[d] = (T)0;
    }
    T a[kAcc];
#pragma unroll
    for (int f = 0; f < kAcc; ++f) a[f] = (T)0;
    T ll = (T)0;   // per-point log-likelihoods (lanes 0 and 16); float64 only across lanes and warps
    for (int base = 2 * wid; base < n; base += 2 * kGmmWarps) {
      const int p = base + h;
      const bool pv = p < n;
      T xd[kMixDim];
#pragma unroll
      for (int d = 0; d < kMixDim; ++d) xd[d] = pv ? (T)S.pts[p][d] : (T)0;
      T q = (T)0;
#pragma unroll
      for (int d = 0; d < kMixDim; ++d) {
        const T z = xd[d] - m_k[d];
        q += z * z * iv_k[d];
      }
      const bool kv = k < K;
      const T lp = kv ? c_k - (T)0.5 * q : -(T)INFINITY;
      T mx = lp;
      for (int s = 8; s; s >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, s));
      const T e = kv ? g_exp(lp - mx) : (T)0;
      T sum = e;
      for (int s = 8; s; s >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, s);
      if (pv) {
        if (kv) {
          const T r = e / sum;
          a[0] += r;
#pragma unroll
          for (int d = 0; d < kMixDim; ++d) {
            const T z = xd[d] - m_k[d];
            a[1 + d] += r * z;
            a[1 + kMixDim + d] += r * z * z;
          }
        }
        if (k == 0) ll += mx + g_log(sum);
      }
    }
    // halves -> lanes 0..15 (double), warps -> shared memory
#pragma unroll
    for (int f = 0; f < kAcc; ++f) {
      const double v = (double)a[f];
      const double u = __shfl_down_sync(0xffffffffu, v, 16);
      if (lane < 16 && k < K) S.acc[wid][k][f] = v + u;
    }
    const double lld = (double)ll + (double)__shfl_down_sync(0xffffffffu, ll, 16);
    if (lane == 0) S.llw[wid] = lld;
    __syncthreads();
    if (it == n_iter) break;
    // M-step (fixed warp order): N_k = S0 + 10 eps, mu += S1 / N, var = S2 / N - (S1 / N)^2 + reg
    if (tid < K * kMixDim) {
      const int kk = tid / kMixDim, d = tid % kMixDim;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      for (int w = 0; w < kGmmWarps; ++w) {
        s0 += S.acc[w][kk][0];
        s1 += S.acc[w][kk][1 + d];
        s2 += S.acc[w][kk][1 + kMixDim + d];
      }
      const double nk = s0 + 10.0 * DBL_EPSILON;
      const double m1 = s1 / nk;
      S.mu[kk][d] = (double)(T)S.mu[kk][d] + m1;   // the sums are centred on the mean as the E pass used it
      S.var[kk][d] = s2 / nk - m1 * m1 + reg;
      if (d == 0) S.nk[kk] = nk;
    }
    __syncthreads();
    if (tid < K) {
      double tot = 0.0;
      for (int j = 0; j < K; ++j) tot += S.nk[j];
      S.w[tid] = S.nk[tid] / tot;
    }
    __syncthreads();
  }

  // ---- outputs
  if (tid == 0) {
    int any = 0, best = 0;
    for (int j = 0; j < K; ++j) {
      S.used[j] = S.w[j] >= min_weight ? 1 : 0;
      any |= S.used[j];
      if (S.w[j] > S.w[best]) best = j;
    }
    if (K > 0 && !any) S.used[best] = 1;
    if (loglike) {
      double t = 0.0;
      for (int w = 0; w < kGmmWarps; ++w) t += S.llw[w];
      loglike[g] = n > 0 ? t : 0.0;
    }
  }
  __syncthreads();
  for (int i = tid; i < kMixComp * kAcc; i += kGmmThreads) {
    const int kk = i / kAcc, f = i % kAcc;
    double v;
    if (kk < K) {
      if (f == 0) v = S.used[kk] ? 0.0 : kWOff;
      else if (f <= kMixDim) v = logit_c(S.mu[kk][f - 1]);
      else v = logit_c((0.5 * log(S.var[kk][f - 1 - kMixDim]) - kMixSMin) / (kMixSMax - kMixSMin));
    } else {
      v = f == 0 ? (K == 0 ? 0.0 : kWOff) : f <= kMixDim ? 0.0 : logit_c(1.0);
    }
    for (int c2 = 0; c2 < n_copies; ++c2) raw_out[((int64_t)c2 * n_groups + g) * kMixOut + i] = (float)v;
    if (fit_out) {
      double fv = 0.0;
      if (kk < K) fv = f == 0 ? S.w[kk] : f <= kMixDim ? S.mu[kk][f - 1] : S.var[kk][f - 1 - kMixDim];
      fit_out[((int64_t)g * kMixComp + kk) * kAcc + f] = fv;
    }
  }
}

}  // namespace
}  // namespace gbk

using namespace gbk;

extern "C" int32_t gmm_max_points(void) { return kGmmCap; }

extern "C" gbk_status gmm_fit(const float* x, int32_t n_groups, int32_t n_points, int32_t n_comp, int32_t n_iter,
                              double reg, double min_weight, int32_t precision, int32_t n_copies, float* raw_out,
                              double* fit_out, double* loglike, void* stream) {
  if (!x || !raw_out) return set_error(GBK_EINVAL, "gmm_fit: null device pointer");
  if (n_groups < 1 || n_points < 0 || n_comp < 1 || n_comp > kMixComp || n_iter < 0 || n_copies < 1)
    return set_error(GBK_EINVAL, "gmm_fit: bad sizes (groups %d, points %d, components %d, iterations %d)", n_groups,
                     n_points, n_comp, n_iter);
  if (!(reg > 0.0) || !(min_weight >= 0.0 && min_weight <= 1.0))
    return set_error(GBK_EINVAL, "gmm_fit: reg must be > 0 and min_weight in [0, 1]");
  if (precision != GBK_MIXED && precision != GBK_FP64) return set_error(GBK_EINVAL, "gmm_fit: bad precision");
  const size_t smem = precision == GBK_MIXED ? sizeof(GmmSmem<float>) : sizeof(GmmSmem<double>);
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == GBK_MIXED) {
    if (cudaFuncSetAttribute(k_gmm_fit<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return set_error(GBK_ECUDA, "gmm_fit: cannot set shared memory size");
    }
    k_gmm_fit<float><<<n_groups, kGmmThreads, smem, st>>>(x, n_points, n_comp, n_iter, reg, min_weight, n_groups,
                                                          n_copies, raw_out, fit_out, loglike);
  } else {
    if (cudaFuncSetAttribute(k_gmm_fit<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return set_error(GBK_ECUDA, "gmm_fit: cannot set shared memory size");
    }
    k_gmm_fit<double><<<n_groups, kGmmThreads, smem, st>>>(x, n_points, n_comp, n_iter, reg, min_weight, n_groups,
                                                           n_copies, raw_out, fit_out, loglike);
  }
  return check_launch("gmm_fit");
}
