// total_loglike without any allocation: for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or anything that allocates): code running inside
// another framework's memory budget or allocator, a process whose allocations must all
// happen before a latency-critical phase, or a plug-in that is handed device buffers and
// may not grow the device footprint. They cannot create a gbk_ctx either (gbk_create
// allocates its tables). This entry point needs neither: the PSD shape is computed in
// the kernel, and its one piece of scratch, the cross-block partial sums, lives in a
// fixed file-scope __device__ array that the module holds for as long as the library is
// loaded on a device.
#include <math.h>
#include <mutex>

#include "gbk_internal.cuh"
#include "gbk_reduce.cuh"

namespace gbk {

constexpr int kStThreads = 256;
constexpr int kStChunk = 4096;                   // bins per block
constexpr int kStWalkers = 8;                    // walkers per block
constexpr int64_t kStScratchDoubles = 1 << 20;   // 8 MiB of partial sums

// Partial sums [chunk][walker][2] followed by [chunk] sums of ln Q; every call writes all
// of the entries it later reads, so nothing needs clearing between calls.
static __device__ __align__(256) double g_static_scratch[kStScratchDoubles];

// Per-bin PSD shape in float32 (S = S_oms Q (1 + (S_acc/S_oms) rho), Eq. psd):
// returns iq = 2^-128 / Q and rho = P / Q for frequency f.
__device__ __forceinline__ void psd_shape_f(double f, float& iq, float& rho, double& q64) {
  const double x = 2.0 * 3.141592653589793 * f * kLc;
  const float xf = (float)x, ff = (float)f;
  float sx, cx;
  sincosf(xf, &sx, &cx);
  const float c2x = 2.0f * cx * cx - 1.0f;
  const float a = 0.4e-3f / ff, bq = ff / 8e-3f, o = 2e-3f / ff;
  const float tpcf = 6.283185307179586f * 299792458.0f * ff;
  const float pm_unit = (1.0f / (tpcf * tpcf)) * (1.0f + a * a) * (1.0f + bq * bq * bq * bq);
  const float tpfc = 6.283185307179586f * ff / 299792458.0f;
  const float op_unit = tpfc * tpfc * (1.0f + o * o * o * o);
  const float s2 = 8.0f * sx * sx;
  const float p = s2 * 2.0f * pm_unit * (3.0f + 2.0f * cx + c2x);
  const float q = s2 * op_unit * (2.0f + cx);
  rho = p / q;
  iq = (1.0f / q) * 2.9387358770557188e-39f;   // 2^-128
  q64 = (double)q;
}

__global__ void __launch_bounds__(kStThreads)
k_static_part(double tobs, int64_t k0, int64_t nb, const float* __restrict__ R, const double* __restrict__ pp,
              int32_t nwl, double* __restrict__ part) {
  const int chunk = blockIdx.x;
  const int wg = blockIdx.y * kStWalkers;
  const int64_t kbeg = (int64_t)chunk * kStChunk;
  const int64_t kend = min(kbeg + (int64_t)kStChunk, nb);
  const int nchunks = gridDim.x;
  float aw[kStWalkers];
  const float* rw[kStWalkers];
  bool act[kStWalkers];
#pragma unroll
  for (int j = 0; j < kStWalkers; ++j) {
    const int w = wg + j;
    act[j] = w < nwl;
    const int ww = act[j] ? w : 0;
    const double so = pp[2 * ww] * pp[2 * ww], sa = pp[2 * ww + 1] * pp[2 * ww + 1];
    aw[j] = (float)(sa / so);
    rw[j] = R + (int64_t)ww * 2 * nb * 2;
  }
  CompF sq[kStWalkers], sl[kStWalkers];
#pragma unroll
  for (int j = 0; j < kStWalkers; ++j) { sq[j].init(); sl[j].init(); }
  double lnq = 0.0;   // sum of ln Q over this thread's bins (first walker group only)
  const float up = 18446744073709551616.0f;  // 2^64
  for (int64_t k = kbeg + threadIdx.x; k < kend; k += kStThreads) {
    float iq, rh;
    double q64;
    psd_shape_f((double)(k0 + k) / tobs, iq, rh, q64);
    if (blockIdx.y == 0) lnq += log(q64);
#pragma unroll
    for (int j = 0; j < kStWalkers; ++j) {
      if (!act[j]) continue;
      const float2 a = *reinterpret_cast<const float2*>(rw[j] + 2 * k);
      const float2 e = *reinterpret_cast<const float2*>(rw[j] + 2 * (nb + k));
      const float u = fmaf(aw[j], rh, 1.0f);
      const float ax = a.x * up, ay = a.y * up, ex = e.x * up, ey = e.y * up;
      sq[j].add((ax * ax + ay * ay + ex * ex + ey * ey) * iq * __frcp_rn(u));
      sl[j].add(logf(u));
    }
  }
  __shared__ double red[kStThreads / 32][kStWalkers][2];
  __shared__ double redq[kStThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kStWalkers; ++j) {
    const double tq = sq[j].warp_total();
    const double tl = sl[j].warp_total();
    if (lane == 0) { red[wid][j][0] = tq; red[wid][j][1] = tl; }
  }
  for (int o = 16; o > 0; o >>= 1) lnq += __shfl_xor_sync(0xffffffffu, lnq, o);
  if (lane == 0) redq[wid] = lnq;
  __syncthreads();
  if (threadIdx.x < kStWalkers * 2) {
    const int j = threadIdx.x >> 1, which = threadIdx.x & 1;
    if (wg + j < nwl) {
      double s = 0.0;
      for (int w = 0; w < kStThreads / 32; ++w) s += red[w][j][which];
      part[((int64_t)chunk * nwl + wg + j) * 2 + which] = s;
    }
  }
  if (blockIdx.y == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kStThreads / 32; ++w) s += redq[w];
    part[(int64_t)nchunks * nwl * 2 + chunk] = s;
  }
}

__global__ void k_static_final(const double* __restrict__ part, int nchunks, const double* __restrict__ pp,
                               int32_t nwl, int64_t nb, double df, double* __restrict__ logl) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwl) return;
  double q = 0.0, l = 0.0, lq = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    q += part[((int64_t)c * nwl + w) * 2];
    l += part[((int64_t)c * nwl + w) * 2 + 1];
    lq += part[(int64_t)nchunks * nwl * 2 + c];
  }
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
  const int64_t need = nchunks * (int64_t)n_walkers * 2 + nchunks;
  if (need > kStScratchDoubles || nchunks > 65535)
    return set_error(GBK_ERANGE,
                     "total_loglike_noalloc: %lld walkers x %lld bins need %lld scratch doubles, the fixed array holds %lld",
                     (long long)n_walkers, (long long)n_bins, (long long)need, (long long)kStScratchDoubles);
  double* scratch = nullptr;
  gbk_status s = static_scratch(&scratch);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  dim3 grid((unsigned)nchunks, (unsigned)((n_walkers + kStWalkers - 1) / kStWalkers));
  k_static_part<<<grid, kStThreads, 0, st>>>(tobs, k0, n_bins, residual, psd_params, n_walkers, scratch);
  k_static_final<<<(n_walkers + 127) / 128, 128, 0, st>>>(scratch, (int)nchunks, psd_params, n_walkers, n_bins,
                                                          1.0 / tobs, logl);
  return check_launch("total_loglike_noalloc");
}
