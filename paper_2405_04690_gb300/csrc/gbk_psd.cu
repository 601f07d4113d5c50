// Parametric PSD (Eq. psd) and the full log-likelihood pass (Eq. like).
#include <math.h>

#include "gbk_internal.cuh"
#include "gbk_reduce.cuh"

namespace gbk {

constexpr int kTlThreads = 256;
constexpr int kTlWalkers = 4;       // walkers per block
constexpr int kTlMaxW = 4096;       // walkers per launch pair (scratch sizing)

size_t total_loglike_scratch_bytes(int64_t n_bins) {
  const int64_t chunks = (n_bins + kTlChunk - 1) / kTlChunk;
  return (size_t)chunks * kTlMaxW * 2 * sizeof(double);
}

__global__ void k_psd_eval(const double* __restrict__ q, const double* __restrict__ p,
                           const double* __restrict__ pp, int32_t nw, int64_t nb, double* __restrict__ out) {
  const int64_t total = (int64_t)nw * nb;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = i / nb, k = i - w * nb;
    const double so = pp[2 * w] * pp[2 * w], sa = pp[2 * w + 1] * pp[2 * w + 1];
    out[i] = so * q[k] + sa * p[k];
  }
}

// One block: bins [chunk * kTlChunk, +kTlChunk) of walkers wg .. wg + kTlWalkers - 1 (local to
// the launch, wg = (g0 + blockIdx.y) kTlWalkers). Per bin k and walker w (u = 1 + a_w rho_k,
// iq_k = 2^-128 / Q_k): q-term (|R_A|^2 + |R_E|^2) 2^128 iq_k / u, l-term ln u. Writes
// compensated block sums to part[(chunk * nwl + wl) * 2 + {0, 1}].
// FULL: all kTlWalkers walkers present and n_bins even, so each thread takes pairs of bins
// with 16-byte loads, and the two bins of a pair share one reciprocal and one logarithm:
//   m0 iq0 / u0 + m1 iq1 / u1 = (m0 iq0 u1 + m1 iq1 u0) / (u0 u1),  ln u0 + ln u1 = ln(u0 u1).
// Otherwise (the last, partial walker group, or odd n_bins) one bin at a time.
template <bool FULL>
__global__ void __launch_bounds__(kTlThreads, 3)
k_total_loglike_part(const float* __restrict__ R, const float* __restrict__ iq, const float* __restrict__ rho,
                     const double* __restrict__ pp, int32_t w0, int32_t nwl, int32_t g0, int64_t nb,
                     double* __restrict__ part) {
  const int chunk = blockIdx.x;
  const int wg = (g0 + blockIdx.y) * kTlWalkers;
  const int64_t kbeg = (int64_t)chunk * kTlChunk;
  const int64_t kend = min(kbeg + (int64_t)kTlChunk, nb);
  const int nact = FULL ? kTlWalkers : min(kTlWalkers, nwl - wg);
  // per-walker a = S_acc / S_oms as a float pair hi + lo, once per block (see one_plus)
  __shared__ float s_aw[kTlWalkers][2];
  if (threadIdx.x < kTlWalkers) {
    const int wl = wg + threadIdx.x;
    const int w = w0 + (wl < nwl ? wl : 0);
    const double so = pp[2 * w] * pp[2 * w], sa = pp[2 * w + 1] * pp[2 * w + 1];
    const double a = sa / so;
    s_aw[threadIdx.x][0] = (float)a;
    s_aw[threadIdx.x][1] = (float)(a - (double)(float)a);
  }
  __syncthreads();
  float aw[kTlWalkers], awl[kTlWalkers];
#pragma unroll
  for (int j = 0; j < kTlWalkers; ++j) {
    aw[j] = s_aw[j][0];
    awl[j] = s_aw[j][1];
  }
  const float* rbase = R + (int64_t)(w0 + wg) * 2 * nb * 2;
  CompF sq[kTlWalkers], sl[kTlWalkers];
  int ecnt[kTlWalkers];   // sums of the binary exponents of u (ln u = e ln 2 + ln m)
#pragma unroll
  for (int j = 0; j < kTlWalkers; ++j) { sq[j].init(); sl[j].init(); ecnt[j] = 0; }
  const float up = 18446744073709551616.0f;  // 2^64
  if (FULL) {
    for (int64_t k = kbeg + 2 * threadIdx.x; k < kend; k += 2 * kTlThreads) {
      const float2 iq2 = __ldg(reinterpret_cast<const float2*>(iq + k));
      const float2 rh2 = __ldg(reinterpret_cast<const float2*>(rho + k));
      float4 a[kTlWalkers], e[kTlWalkers];
#pragma unroll
      for (int j = 0; j < kTlWalkers; ++j) {
        const float* rw = rbase + (int64_t)j * 2 * nb * 2;
        a[j] = __ldcs(reinterpret_cast<const float4*>(rw + 2 * k));
        e[j] = __ldcs(reinterpret_cast<const float4*>(rw + 2 * (nb + k)));
      }
      // |R|^2 summed unscaled and times 2^64 once, iq times 2^64 once per bin (exact scalings)
      const float iq0 = iq2.x * up, iq1 = iq2.y * up;
#pragma unroll
      for (int j = 0; j < kTlWalkers; ++j) {
        const float u0 = one_plus(aw[j], awl[j], rh2.x);
        const float u1 = one_plus(aw[j], awl[j], rh2.y);
        const float4 A = a[j], E = e[j];
        const float m0 = (A.x * A.x + A.y * A.y + E.x * E.x + E.y * E.y) * up;
        const float m1 = (A.z * A.z + A.w * A.w + E.z * E.z + E.w * E.w) * up;
        const float uu = u0 * u1;
        sq[j].add(fmaf(m0 * iq0, u1, m1 * iq1 * u0) * __frcp_rn(uu));
        sl[j].add(log_split(uu, ecnt[j]));
      }
    }
  } else {
    for (int64_t k = kbeg + threadIdx.x; k < kend; k += kTlThreads) {
      const float iqk = __ldg(iq + k) * up, rhk = __ldg(rho + k);
#pragma unroll
      for (int j = 0; j < kTlWalkers; ++j) {
        if (j >= nact) break;
        const float* rw = rbase + (int64_t)j * 2 * nb * 2;
        const float2 a = *reinterpret_cast<const float2*>(rw + 2 * k);
        const float2 e = *reinterpret_cast<const float2*>(rw + 2 * (nb + k));
        const float u = one_plus(aw[j], awl[j], rhk);
        sq[j].add((a.x * a.x + a.y * a.y + e.x * e.x + e.y * e.y) * up * iqk * __frcp_rn(u));
        sl[j].add(log_split(u, ecnt[j]));
      }
    }
  }
  // warp totals stay float pairs (hi, lo) and integer exponent sums: float64 (a small fraction of
  // the float32 rate) only in the few threads that add up the block
  __shared__ float2 red[kTlThreads / 32][kTlWalkers][2];
  __shared__ int rede[kTlThreads / 32][kTlWalkers];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kTlWalkers; ++j) {
    const float2 tq = sq[j].warp_pair();
    const float2 tl = sl[j].warp_pair();
    const int te = __reduce_add_sync(0xffffffffu, ecnt[j]);
    if (lane == 0) { red[wid][j][0] = tq; red[wid][j][1] = tl; rede[wid][j] = te; }
  }
  __syncthreads();
  if (threadIdx.x < kTlWalkers * 2) {
    const int j = threadIdx.x >> 1, which = threadIdx.x & 1;
    if (j < nact) {
      double s = 0.0;
      int es = 0;
      for (int w = 0; w < kTlThreads / 32; ++w) {
        s += (double)red[w][j][which].x + (double)red[w][j][which].y;
        es += rede[w][j];
      }
      if (which) s += kLn2 * (double)es;
      part[((int64_t)chunk * nwl + wg + j) * 2 + which] = s;
    }
  }
}

// The block passes of nwl walkers (w0 .. w0 + nwl - 1) over n_bins bins into part [chunk][nwl][2]:
// the full walker groups with the pair loop when n_bins is even, the rest one bin at a time.
gbk_status total_loglike_parts(const float* R, const float* iq, const float* rho, const double* pp, int32_t w0,
                               int32_t nwl, int64_t nb, double* part, cudaStream_t st) {
  const int nchunks = (int)((nb + kTlChunk - 1) / kTlChunk);
  const int full = (nb & 1) == 0 && ((uintptr_t)R & 15) == 0 ? nwl / kTlWalkers : 0;
  const int groups = (nwl + kTlWalkers - 1) / kTlWalkers;
  if (full > 0)
    k_total_loglike_part<true><<<dim3(nchunks, full), kTlThreads, 0, st>>>(R, iq, rho, pp, w0, nwl, 0, nb, part);
  if (groups > full)
    k_total_loglike_part<false><<<dim3(nchunks, groups - full), kTlThreads, 0, st>>>(R, iq, rho, pp, w0, nwl, full,
                                                                                     nb, part);
  return check_launch("total_loglike");
}

// Sum the chunk partials of each walker in chunk order and assemble Eq. like.
__global__ void k_total_loglike_final(const double* __restrict__ part, int nchunks, const double* __restrict__ pp,
                                      int32_t w0, int32_t nwl, int64_t nb, double df, double sum_lnq,
                                      double* __restrict__ logl) {
  const int wl = blockIdx.x * blockDim.x + threadIdx.x;
  if (wl >= nwl) return;
  const int w = w0 + wl;
  double q = 0.0, l = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    q += part[((int64_t)c * nwl + wl) * 2];
    l += part[((int64_t)c * nwl + wl) * 2 + 1];
  }
  const double so = pp[2 * w] * pp[2 * w];
  // -1/2 <R|R> = -1/2 (4 df / S_oms) sum |R~|^2 iq / u ; -sum_ch sum_k ln S = -2 (n ln S_oms + sum ln Q + sum ln u)
  logl[w] = -0.5 * (4.0 * df / so) * q - 2.0 * ((double)nb * log(so) + sum_lnq + l);
}

}  // namespace gbk

using namespace gbk;

extern "C" gbk_status psd_eval(gbk_ctx* ctx, const double* psd_params, int32_t n_walkers, double* s_out,
                               void* stream) {
  if (!ctx) return set_error(GBK_EINVAL, "psd_eval: null context");
  if (n_walkers < 0) return set_error(GBK_EINVAL, "psd_eval: n_walkers < 0");
  if (n_walkers == 0 || !s_out) return GBK_OK;
  if (!psd_params) return set_error(GBK_EINVAL, "psd_eval: null psd_params");
  const int64_t total = (int64_t)n_walkers * ctx->grid.n_bins;
  const int threads = 256;
  int64_t blocks = (total + threads - 1) / threads;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_psd_eval<<<(int)blocks, threads, 0, (cudaStream_t)stream>>>(ctx->psd_q, ctx->psd_p, psd_params, n_walkers,
                                                                 ctx->grid.n_bins, s_out);
  return check_launch("psd_eval");
}

extern "C" gbk_status total_loglike(gbk_ctx* ctx, const float* residual, const double* psd_params,
                                    int32_t n_walkers, double* logl, void* stream) {
  if (!ctx) return set_error(GBK_EINVAL, "total_loglike: null context");
  if (n_walkers < 0) return set_error(GBK_EINVAL, "total_loglike: n_walkers < 0");
  if (n_walkers == 0) return GBK_OK;
  if (!residual || !psd_params || !logl) return set_error(GBK_EINVAL, "total_loglike: null device pointer");
  if (((uintptr_t)residual & 7) != 0) return set_error(GBK_EINVAL, "total_loglike: residual must be 8-byte aligned");
  const int64_t nb = ctx->grid.n_bins;
  const int nchunks = (int)((nb + kTlChunk - 1) / kTlChunk);
  cudaStream_t st = (cudaStream_t)stream;
  for (int32_t w0 = 0; w0 < n_walkers; w0 += kTlMaxW) {
    const int32_t nwl = n_walkers - w0 < kTlMaxW ? n_walkers - w0 : kTlMaxW;
    gbk_status s = total_loglike_parts(residual, ctx->iq_f, ctx->rho_f, psd_params, w0, nwl, nb, ctx->scratch, st);
    if (s) return s;
    k_total_loglike_final<<<(nwl + 127) / 128, 128, 0, st>>>(ctx->scratch, nchunks, psd_params, w0, nwl, nb,
                                                            1.0 / ctx->grid.tobs, ctx->sum_lnq, logl);
  }
  return check_launch("total_loglike");
}
