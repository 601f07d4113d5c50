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

constexpr int kStThreads = 256;
constexpr int kStChunk = 4096;                   // bins per block of the likelihood pass
constexpr int kStWalkers = 8;                    // walkers per block
constexpr int kStShapeThreads = 256;             // bins per block of the shape pass
constexpr int64_t kStScratchDoubles = 1 << 21;   // 16 MiB

// Scratch layout, in doubles: the float32 shape tables iq [n_bins] and rho [n_bins] (n_bins
// doubles together), then the likelihood pass's partial sums [chunk][walker][2], then the
// shape pass's sums of ln Q [shape block]. Every call writes all of the entries it later
// reads, so nothing needs clearing between calls.
static __device__ __align__(256) double g_static_scratch[kStScratchDoubles];

// Eq. psd split by noise power, S_n = S_oms Q(f) + S_acc P(f), in float64 with float64
// constants (as the context's tables are built): per bin iq = 2^-128 / Q and rho = P / Q
// rounded once to float32, and the float64 sum of ln Q over the block's bins.
__global__ void __launch_bounds__(kStShapeThreads)
k_static_shape(double tobs, int64_t k0, int64_t nb, float* __restrict__ iq, float* __restrict__ rho,
               double* __restrict__ lnq_part) {
  const int64_t k = (int64_t)blockIdx.x * kStShapeThreads + threadIdx.x;
  double lq = 0.0;
  if (k < nb) {
    const double f = (double)(k0 + k) / tobs;
    const double x = 2.0 * 3.141592653589793 * f * kLc;
    double sx, cx;
    sincos(x, &sx, &cx);
    const double c2x = 2.0 * cx * cx - 1.0;
    const double tpcf = 2.0 * 3.141592653589793 * kC * f;
    const double a = 0.4e-3 / f, bq = f / 8e-3, o = 2e-3 / f, tpfc = 2.0 * 3.141592653589793 * f / kC;
    const double pm_unit = (1.0 + a * a) * (1.0 + bq * bq * bq * bq) / (tpcf * tpcf);
    const double op_unit = tpfc * tpfc * (1.0 + o * o * o * o);
    const double s2 = 8.0 * sx * sx;
    const double p = s2 * 2.0 * pm_unit * (3.0 + 2.0 * cx + c2x);
    const double q = s2 * op_unit * (2.0 + cx);
    iq[k] = (float)(2.9387358770557188e-39 / q);   // 2^-128 / Q
    rho[k] = (float)(p / q);
    lq = log(q);
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

__global__ void __launch_bounds__(kStThreads)
k_static_part(int64_t nb, const float* __restrict__ R, const double* __restrict__ pp, int32_t nwl,
              const float* __restrict__ iqt, const float* __restrict__ rhot, double* __restrict__ part) {
  const int chunk = blockIdx.x;
  const int wg = blockIdx.y * kStWalkers;
  const int64_t kbeg = (int64_t)chunk * kStChunk;
  const int64_t kend = min(kbeg + (int64_t)kStChunk, nb);
  // a = S_acc / S_oms as a float pair hi + lo (u = (1 + hi rho) + lo rho): the rounding of
  // a, the same in every bin of a walker, would otherwise bias the sum of ln u
  float aw[kStWalkers], awl[kStWalkers];
  const float* rw[kStWalkers];
  bool act[kStWalkers];
#pragma unroll
  for (int j = 0; j < kStWalkers; ++j) {
    const int w = wg + j;
    act[j] = w < nwl;
    const int ww = act[j] ? w : 0;
    const double so = pp[2 * ww] * pp[2 * ww], sa = pp[2 * ww + 1] * pp[2 * ww + 1];
    const double a = sa / so;
    aw[j] = (float)a;
    awl[j] = (float)(a - (double)aw[j]);
    rw[j] = R + (int64_t)ww * 2 * nb * 2;
  }
  CompF sq[kStWalkers], sl[kStWalkers];
#pragma unroll
  for (int j = 0; j < kStWalkers; ++j) { sq[j].init(); sl[j].init(); }
  const float up = 18446744073709551616.0f;  // 2^64
  for (int64_t k = kbeg + threadIdx.x; k < kend; k += kStThreads) {
    const float iq = __ldg(iqt + k), rh = __ldg(rhot + k);
#pragma unroll
    for (int j = 0; j < kStWalkers; ++j) {
      if (!act[j]) continue;
      const float2 a = *reinterpret_cast<const float2*>(rw[j] + 2 * k);
      const float2 e = *reinterpret_cast<const float2*>(rw[j] + 2 * (nb + k));
      const float u = fmaf(awl[j], rh, fmaf(aw[j], rh, 1.0f));
      const float ax = a.x * up, ay = a.y * up, ex = e.x * up, ey = e.y * up;
      sq[j].add((ax * ax + ay * ay + ex * ex + ey * ey) * iq * __frcp_rn(u));
      sl[j].add(logf(u));
    }
  }
  __shared__ double red[kStThreads / 32][kStWalkers][2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kStWalkers; ++j) {
    const double tq = sq[j].warp_total();
    const double tl = sl[j].warp_total();
    if (lane == 0) { red[wid][j][0] = tq; red[wid][j][1] = tl; }
  }
  __syncthreads();
  if (threadIdx.x < kStWalkers * 2) {
    const int j = threadIdx.x >> 1, which = threadIdx.x & 1;
    if (wg + j < nwl) {
      double s = 0.0;
      for (int w = 0; w < kStThreads / 32; ++w) s += red[w][j][which];
      part[((int64_t)chunk * nwl + wg + j) * 2 + which] = s;
    }
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
  const int64_t nshape = (n_bins + kStShapeThreads - 1) / kStShapeThreads;
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
  k_static_shape<<<(unsigned)nshape, kStShapeThreads, 0, st>>>(tobs, k0, n_bins, iq, rho, lnq_part);
  dim3 grid((unsigned)nchunks, (unsigned)ngroups);
  k_static_part<<<grid, kStThreads, 0, st>>>(n_bins, residual, psd_params, n_walkers, iq, rho, part);
  k_static_final<<<(n_walkers + 127) / 128, 128, 0, st>>>(part, (int)nchunks, lnq_part, (int)nshape, psd_params,
                                                          n_walkers, n_bins, 1.0 / tobs, logl);
  return check_launch("total_loglike_noalloc");
}
