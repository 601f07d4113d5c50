// total_loglike without any allocation: for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or anything that allocates): code running inside
// another framework's memory budget or allocator, a process whose allocations must all
// happen before a latency-critical phase, or a plug-in that is handed device buffers and
// may not grow the device footprint. They cannot create a gbk_ctx either (gbk_create
// allocates its tables). This entry point needs neither: the PSD shape is computed in
// a kernel, and its scratch (the shape tables and the cross-block partial sums) lives in a
// fixed file-scope __device__ array that the module holds for as long as the library is
// loaded on a device. The PSD shape is evaluated in float64 once per call into that array
// (float32 tables, like the context's), and the sum of ln Q is kept in float64.
#include <math.h>
#include <mutex>

#include "gbk_internal.cuh"
#include "gbk_reduce.cuh"

namespace gbk {

constexpr int kStChunk = kTlChunk;               // bins per block of the likelihood pass (total_loglike_parts)
constexpr int kStWalkers = 4;                    // walkers per block of that pass
constexpr int kStShapeThreads = 256;             // bins per block of the shape pass
constexpr int64_t kStScratchDoubles = 1 << 21;   // 16 MiB

// Scratch layout, in doubles: the float32 shape tables iq [n_bins] and rho [n_bins] (n_bins
// doubles together), then the likelihood pass's partial sums [chunk][walker][2], then the
// shape pass's sums of ln Q [shape block]. Every call writes all of the entries it later
// reads, so nothing needs clearing between calls.
static __device__ __align__(256) double g_static_scratch[kStScratchDoubles];

// Eq. psd split by noise power, S_n = S_oms Q(f) + S_acc P(f), in float64 with float64
// constants (as the context's tables are built): per bin iq = 2^-128 / Q and rho = P / Q
// rounded once to float32, and the float64 sum of ln Q over the block's bins. Float64 runs at
// a small fraction of the float32 rate here, so each thread takes kStRun consecutive bins and
// spends few float64 operations per bin: (sin x, cos x) advance by a rotation through the bin
// spacing of x, 1 / f and 1 / Q come from a float32 reciprocal refined by two Newton steps,
// and ln Q is summed as the log of a product of mantissas plus the sum of binary exponents.
constexpr int kStRun = 16;
__device__ __forceinline__ double recip_nr(double v) {
  double y = (double)__frcp_rn((float)v);
  y = y * (2.0 - v * y);
  return y * (2.0 - v * y);
}

__global__ void __launch_bounds__(kStShapeThreads)
k_static_shape(double tobs, int64_t k0, int64_t nb, double ck, double sk, float* __restrict__ iq,
               float* __restrict__ rho, double* __restrict__ lnq_part) {
  const int64_t kfirst = ((int64_t)blockIdx.x * kStShapeThreads + threadIdx.x) * kStRun;
  double lq = 0.0;
  if (kfirst < nb) {
    const double two_pi = 6.283185307179586;
    double sx, cx;
    sincos(two_pi * ((double)(k0 + kfirst) / tobs) * kLc, &sx, &cx);
    double prod = 1.0;
    int esum = 0;
    const int64_t kend = min(kfirst + (int64_t)kStRun, nb);
    for (int64_t k = kfirst; k < kend; ++k) {
      const double kk = (double)(k0 + k);
      const double f = kk / tobs;
      const double inv_f = tobs * recip_nr(kk);
      const double c2x = 2.0 * cx * cx - 1.0;
      const double tpcf = two_pi * kC * f;
      const double a = 0.4e-3 * inv_f, bq = f * (1.0 / 8e-3), o = 2e-3 * inv_f, tpfc = two_pi * f / kC;
      const double a2 = a * a, bq2 = bq * bq, o2 = o * o;
      const double inv_tpcf = recip_nr(tpcf);
      const double pm_unit = (1.0 + a2) * (1.0 + bq2 * bq2) * (inv_tpcf * inv_tpcf);
      const double op_unit = tpfc * tpfc * (1.0 + o2 * o2);
      const double s2 = 8.0 * sx * sx;
      const double p = s2 * 2.0 * pm_unit * (3.0 + 2.0 * cx + c2x);
      const double q = s2 * op_unit * (2.0 + cx);
      const double iqd = recip_nr(q);
      iq[k] = (float)(2.9387358770557188e-39 * iqd);   // 2^-128 / Q
      rho[k] = (float)(p * iqd);
      int e;
      prod *= frexp(q, &e);
      esum += e;
      const double sn = sx * ck + cx * sk;             // x advances by one bin
      cx = cx * ck - sx * sk;
      sx = sn;
    }
    lq = log(prod) + 0.6931471805599453094 * (double)esum;
  }
  for (int o = 16; o > 0; o >>= 1) lq += __shfl_xor_sync(0xffffffffu, lq, o);
  __shared__ double red[kStShapeThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kStShapeThreads / 32; ++w) t += red[w];
    lnq_part[blockIdx.x] = t;
  }
}

__global__ void k_static_final(const double* __restrict__ part, int nchunks, const double* __restrict__ lnq_part,
                               int nshape, const double* __restrict__ pp, int32_t nwl, int64_t nb, double df,
                               double* __restrict__ logl) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwl) return;
  double q = 0.0, l = 0.0, lq = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    q += part[((int64_t)c * nwl + w) * 2];
    l += part[((int64_t)c * nwl + w) * 2 + 1];
  }
  for (int c = 0; c < nshape; ++c) lq += lnq_part[c];
  const double so = pp[2 * w] * pp[2 * w];
  logl[w] = -0.5 * (4.0 * df / so) * q - 2.0 * ((double)nb * log(so) + lq + l);
}

// Device address of the scratch array, looked up once per device with that device
// current (in host code the array's name is only a host-side stand-in).
static std::mutex g_static_mutex;
static double* g_static_ptr[64];

static gbk_status static_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return set_error(GBK_ECUDA, "total_loglike_noalloc: no current CUDA device");
  }
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return set_error(GBK_ECUDA, "total_loglike_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    }
    g_static_ptr[dev] = (double*)p;
  }
  *out = g_static_ptr[dev];
  return GBK_OK;
}

}  // namespace gbk

using namespace gbk;

extern "C" int64_t total_loglike_noalloc_capacity(void) { return kStScratchDoubles; }

extern "C" gbk_status total_loglike_noalloc(double tobs, int64_t k0, int64_t n_bins, const float* residual,
                                            const double* psd_params, int32_t n_walkers, double* logl, void* stream) {
  if (!(tobs > 0) || k0 < 1 || n_bins < 1) return set_error(GBK_EINVAL, "total_loglike_noalloc: bad grid");
  if ((double)(k0 + n_bins) / tobs >= 0.5 / kLc)   // Eq. psd vanishes at f = c / (2L)
    return set_error(GBK_EINVAL, "total_loglike_noalloc: window reaches f = c/(2L)");
  if (n_walkers < 0) return set_error(GBK_EINVAL, "total_loglike_noalloc: n_walkers < 0");
  if (n_walkers == 0) return GBK_OK;
  if (!residual || !psd_params || !logl) return set_error(GBK_EINVAL, "total_loglike_noalloc: null device pointer");
  if (((uintptr_t)residual & 7) != 0) return set_error(GBK_EINVAL, "total_loglike_noalloc: residual must be 8-byte aligned");
  const int64_t nchunks = (n_bins + kStChunk - 1) / kStChunk;
  const int64_t nshape = (n_bins + kStShapeThreads * kStRun - 1) / (kStShapeThreads * kStRun);
  const int64_t ngroups = ((int64_t)n_walkers + kStWalkers - 1) / kStWalkers;
  if (ngroups > 65535)
    return set_error(GBK_ERANGE, "total_loglike_noalloc: %lld walkers exceed the %d the launch grid takes",
                     (long long)n_walkers, 65535 * kStWalkers);
  const int64_t need = n_bins + nchunks * (int64_t)n_walkers * 2 + nshape;
  if (need > kStScratchDoubles)
    return set_error(GBK_ERANGE,
                     "total_loglike_noalloc: %lld walkers x %lld bins need %lld scratch doubles, the fixed array holds %lld",
                     (long long)n_walkers, (long long)n_bins, (long long)need, (long long)kStScratchDoubles);
  double* scratch = nullptr;
  gbk_status s = static_scratch(&scratch);
  if (s) return s;
  float* iq = reinterpret_cast<float*>(scratch);
  float* rho = iq + n_bins;
  double* part = scratch + n_bins;
  double* lnq_part = part + nchunks * (int64_t)n_walkers * 2;
  cudaStream_t st = (cudaStream_t)stream;
  const double dx = 6.283185307179586 * kLc / tobs;   // x = 2 pi f L / c advances by dx per bin
  k_static_shape<<<(unsigned)nshape, kStShapeThreads, 0, st>>>(tobs, k0, n_bins, cos(dx), sin(dx), iq, rho, lnq_part);
  s = total_loglike_parts(residual, iq, rho, psd_params, 0, n_walkers, n_bins, part, st);
  if (s) return s;
  k_static_final<<<(n_walkers + 127) / 128, 128, 0, st>>>(part, (int)nchunks, lnq_part, (int)nshape, psd_params,
                                                          n_walkers, n_bins, 1.0 / tobs, logl);
  return check_launch("total_loglike_noalloc");
}
