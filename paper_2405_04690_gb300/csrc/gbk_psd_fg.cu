// Per-channel instrument noise plus the Galactic foreground (Sec. III, Eq. psd; Sec. III.A),
// its full log-likelihood pass (Eq. like), and the PSD module's sampler (Sec. V.B): regular
// stretch moves over walkers (Eq. stretch), swaps between neighbouring temperatures of the
// same walker index, which share one residual (Eq. temp-orig).
//
// Parameters of one PSD walker (float64 [9]): sqrt(S_oms,A), sqrt(S_acc,A), sqrt(S_oms,E),
// sqrt(S_acc,E), A_fg, alpha, f_k, s1, s2. Per bin and channel
//   S_ch = S_oms,ch Q (1 + (S_acc,ch / S_oms,ch) rho + g / S_oms,ch),
//   g = S_fg / Q = A_fg exp(ln(6 x^2 sin^2 x / Q) - (7/3) ln f - s1 f^alpha - softplus(2 s2 (f - f_k)))
// (since (1 + tanh(-y)) = 2 / (1 + e^(2y)) and (A_fg / 2) 2 = A_fg), evaluated in base 2 on the
// special-function unit: the context holds log2 f and the bin's constant part in log2 units.
// The exponent (~70 in log2 units) carries the float32 rounding of its table entry, ~4e-6,
// i.e. a relative error of ~3e-6 in S_fg, pseudo-random from bin to bin.
#include <math.h>

#include "gbk_internal.cuh"
#include "gbk_philox.cuh"
#include "gbk_reduce.cuh"

namespace gbk {

constexpr int kFgThreads = 256;
constexpr int kFgChunk = 8192;
constexpr int kFgEntries = 4;   // PSD walkers per block (share one residual load when they share a residual)
constexpr int kPsdDim = 9;

size_t total_loglike_scratch_bytes(int64_t n_bins);

// The walker constants that scale every bin's terms are kept as float pairs (hi = the constant
// rounded to float32, lo = the remainder) and applied as one rounded product x hi + x lo: the
// rounding of a constant would be the same relative error in every bin, ~6e-8 x 2^20 bins = a
// bias of ~0.1 nats in ln L; the product's own rounding is unbiased.
struct FgEntry {
  float iso_a, iso_e, iso_al, iso_el;   // 2^-64 / S_oms per channel (keeps both channels' q-terms in one sum)
  float aw_a, aw_e, aw_al, aw_el;       // S_acc / S_oms per channel
  float k_a, k_e, k_al, k_el;           // A_fg / S_oms per channel (g and S_oms share the 2^128 scale of Q)
  float alpha, s1l, s2l, fk;            // alpha, s1 log2(e), 2 s2 log2(e), f_k
};

__device__ __forceinline__ float mul2(float x, float hi, float lo) { return fmaf(x, hi, x * lo); }
// u = 1 + aw rho + g k
__device__ __forceinline__ float u_of(float awh, float awl, float kh, float kl, float rho, float g) {
  return fmaf(g, kh, fmaf(g, kl, one_plus(awh, awl, rho)));
}

__device__ __forceinline__ float ex2a(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcpa(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2a(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// log2(1 + 2^x) without overflow; for |x| > 25, 1 + 2^-|x| rounds to 1 and the value is
// max(x, 0) (taken without the two special-function evaluations)
__device__ __forceinline__ float softplus2(float x) {
  return fabsf(x) > 25.f ? fmaxf(x, 0.f) : fmaxf(x, 0.f) + lg2a(1.0f + ex2a(-fabsf(x)));
}

__device__ __forceinline__ FgEntry fg_entry(const double* p) {
  FgEntry e;
  const double so_a = p[0] * p[0], sa_a = p[1] * p[1], so_e = p[2] * p[2], sa_e = p[3] * p[3];
  auto pair = [](double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  };
  pair(ldexp(1.0, -64) / so_a, e.iso_a, e.iso_al);
  pair(ldexp(1.0, -64) / so_e, e.iso_e, e.iso_el);
  pair(sa_a / so_a, e.aw_a, e.aw_al);
  pair(sa_e / so_e, e.aw_e, e.aw_el);
  pair(p[4] / so_a, e.k_a, e.k_al);
  pair(p[4] / so_e, e.k_e, e.k_el);
  e.alpha = (float)p[5];
  e.fk = (float)p[6];
  e.s1l = (float)(p[7] * 1.4426950408889634);
  e.s2l = (float)(2.0 * p[8] * 1.4426950408889634);
  return e;
}

// One block: bins [chunk * kFgChunk, +kFgChunk) of entries [eg, eg + kFgEntries).
// part[(chunk * nel + e) * 2 + {0, 1}] = sum_ch |R_ch|^2 2^64 iq / (u_ch S_oms,ch) and
// sum (ln u_A + ln u_E); compensated float32 per thread and (as float pairs) per warp, float64
// only in the threads that add up the block.
__global__ void __launch_bounds__(kFgThreads, 2)
k_fg_part(const float* __restrict__ R, const float* __restrict__ iq, const float* __restrict__ rho,
          const float* __restrict__ lnf, const float* __restrict__ ff, const float* __restrict__ fgc,
          const double* __restrict__ pp, const int32_t* __restrict__ ridx, int32_t n_resid, int32_t e0, int32_t nel,
          int64_t nb, double* __restrict__ part, int* err) {
  const int chunk = blockIdx.x;
  const int eg = blockIdx.y * kFgEntries;
  const int64_t kbeg = (int64_t)chunk * kFgChunk;
  const int64_t kend = min(kbeg + (int64_t)kFgChunk, nb);
  __shared__ FgEntry s_e[kFgEntries];
  __shared__ int s_r[kFgEntries];
  if (threadIdx.x < kFgEntries) {
    const int el = eg + threadIdx.x;
    const int e = e0 + (el < nel ? el : 0);
    s_e[threadIdx.x] = fg_entry(pp + (int64_t)e * kPsdDim);
    int r = ridx ? ridx[e] : e;
    if (r < 0 || r >= n_resid) {   // bad residual index: error bit, read residual 0 instead
      atomicOr(err, kErrWalker);
      r = 0;
    }
    s_r[threadIdx.x] = r;
  }
  __syncthreads();
  const FgEntry* ent = s_e;   // read from shared memory where used (broadcast loads), not held in registers
  const float* rw[kFgEntries];
  bool act[kFgEntries], same[kFgEntries], gsame[kFgEntries];
#pragma unroll
  for (int j = 0; j < kFgEntries; ++j) {
    act[j] = eg + j < nel;
    rw[j] = R + (int64_t)s_r[j] * 2 * nb * 2;
    same[j] = j > 0 && s_r[j] == s_r[j - 1];   // entries of one residual read it once
    // entries whose foreground shape (alpha, f_k, s1, s2) equals the previous entry's share its
    // exponent g (A_fg, which only scales g, may differ)
    gsame[j] = j > 0 && ent[j].alpha == ent[j - 1].alpha && ent[j].fk == ent[j - 1].fk &&
               ent[j].s1l == ent[j - 1].s1l && ent[j].s2l == ent[j - 1].s2l;
  }
  CompF sq[kFgEntries], sl[kFgEntries];
#pragma unroll
  for (int j = 0; j < kFgEntries; ++j) { sq[j].init(); sl[j].init(); }
  const float up = 18446744073709551616.0f;  // 2^64
  // g = 2^(c - log2(e) [s1 f^alpha + softplus(2 s2 (f - f_k))]), f^alpha = 2^(alpha log2 f);
  // far above the knee (softplus > c + 30) g A_fg / S_oms < 2^-30 relative to 1: skipped
  auto fg_g = [&](int j, float lf, float fk, float c) {
    const float y = ent[j].s2l * (fk - ent[j].fk);
    float g = 0.f;
    if (y < c + 30.f) g = ex2a(c - ent[j].s1l * ex2a(ent[j].alpha * lf) - softplus2(y));
    return g;
  };
  // per-bin, per-entry terms; residual values of both channels at bin k given; the two
  // channels share one reciprocal: x / ua + y / ue = (x ue + y ua) / (ua ue)
  auto bin = [&](int j, float g, float iqk, float rhk, float ar, float ai, float er, float ei) {
    const float ua = u_of(ent[j].aw_a, ent[j].aw_al, ent[j].k_a, ent[j].k_al, rhk, g);
    const float ue = u_of(ent[j].aw_e, ent[j].aw_el, ent[j].k_e, ent[j].k_el, rhk, g);
    const float ax = ar * up, ay = ai * up, ex = er * up, ey = ei * up;
    const float uu = ua * ue;
    sq[j].add(iqk * fmaf(mul2(ax * ax + ay * ay, ent[j].iso_a, ent[j].iso_al), ue,
                         mul2(ex * ex + ey * ey, ent[j].iso_e, ent[j].iso_el) * ua) * rcpa(uu));
    sl[j].add(0.6931471805599453f * lg2a(uu));
  };
  // two bins of one entry: one reciprocal of the product of their channel products (separate
  // reciprocals if that product could overflow: windows at very low frequency); the logarithms
  // stay per bin (the approximate log2 of the product added a bias of ~0.035 nats over 2^20 bins)
  auto bin2 = [&](int j, float g0, float g1, float iq0, float iq1, float rh0, float rh1, float4 a, float4 e) {
    const float ua0 = u_of(ent[j].aw_a, ent[j].aw_al, ent[j].k_a, ent[j].k_al, rh0, g0);
    const float ue0 = u_of(ent[j].aw_e, ent[j].aw_el, ent[j].k_e, ent[j].k_el, rh0, g0);
    const float ua1 = u_of(ent[j].aw_a, ent[j].aw_al, ent[j].k_a, ent[j].k_al, rh1, g1);
    const float ue1 = u_of(ent[j].aw_e, ent[j].aw_el, ent[j].k_e, ent[j].k_el, rh1, g1);
    const float ax0 = a.x * up, ay0 = a.y * up, ex0 = e.x * up, ey0 = e.y * up;
    const float ax1 = a.z * up, ay1 = a.w * up, ex1 = e.z * up, ey1 = e.w * up;
    const float uu0 = ua0 * ue0, uu1 = ua1 * ue1;
    const float n0 = iq0 * fmaf(mul2(ax0 * ax0 + ay0 * ay0, ent[j].iso_a, ent[j].iso_al), ue0,
                                mul2(ex0 * ex0 + ey0 * ey0, ent[j].iso_e, ent[j].iso_el) * ua0);
    const float n1 = iq1 * fmaf(mul2(ax1 * ax1 + ay1 * ay1, ent[j].iso_a, ent[j].iso_al), ue1,
                                mul2(ex1 * ex1 + ey1 * ey1, ent[j].iso_e, ent[j].iso_el) * ua1);
    const float pu = uu0 * uu1;
    if (pu < 1e37f) {
      const float r = rcpa(pu);
      sq[j].add(n0 * (uu1 * r));
      sq[j].add(n1 * (uu0 * r));
      sl[j].add(0.6931471805599453f * lg2a(uu0));
      sl[j].add(0.6931471805599453f * lg2a(uu1));
    } else {
      sq[j].add(n0 * rcpa(uu0));
      sq[j].add(n1 * rcpa(uu1));
      sl[j].add(0.6931471805599453f * lg2a(uu0));
      sl[j].add(0.6931471805599453f * lg2a(uu1));
    }
  };
  const bool even = (nb & 1) == 0;
  for (int64_t k = kbeg + 2 * threadIdx.x; k < kend; k += 2 * kFgThreads) {
    if (even && k + 1 < kend) {   // two bins per thread: all entries' residual loads issued first
      const float2 iq2 = __ldg(reinterpret_cast<const float2*>(iq + k));
      const float2 rh2 = __ldg(reinterpret_cast<const float2*>(rho + k));
      const float2 lf2 = __ldg(reinterpret_cast<const float2*>(lnf + k));
      const float2 ff2 = __ldg(reinterpret_cast<const float2*>(ff + k));
      const float2 c2 = __ldg(reinterpret_cast<const float2*>(fgc + k));
      float4 av[kFgEntries], ev[kFgEntries];
#pragma unroll
      for (int j = 0; j < kFgEntries; ++j) {
        if (act[j] && !same[j]) {
          av[j] = __ldcs(reinterpret_cast<const float4*>(rw[j] + 2 * k));
          ev[j] = __ldcs(reinterpret_cast<const float4*>(rw[j] + 2 * (nb + k)));
        }
      }
#pragma unroll
      for (int j = 1; j < kFgEntries; ++j)
        if (same[j]) { av[j] = av[j - 1]; ev[j] = ev[j - 1]; }
      float g0 = 0.f, g1 = 0.f;
#pragma unroll
      for (int j = 0; j < kFgEntries; ++j) {
        if (!act[j]) continue;
        if (!gsame[j]) {
          g0 = fg_g(j, lf2.x, ff2.x, c2.x);
          g1 = fg_g(j, lf2.y, ff2.y, c2.y);
        }
        bin2(j, g0, g1, iq2.x, iq2.y, rh2.x, rh2.y, av[j], ev[j]);
      }
    } else {
      for (int64_t kk = k; kk < min(k + 2, kend); ++kk) {
        const float iqk = __ldg(iq + kk), rhk = __ldg(rho + kk), lf = __ldg(lnf + kk), fk = __ldg(ff + kk),
                    c = __ldg(fgc + kk);
        float g = 0.f;
#pragma unroll
        for (int j = 0; j < kFgEntries; ++j) {
          if (!act[j]) continue;
          const float2 a = *reinterpret_cast<const float2*>(rw[j] + 2 * kk);
          const float2 e = *reinterpret_cast<const float2*>(rw[j] + 2 * (nb + kk));
          if (!gsame[j]) g = fg_g(j, lf, fk, c);
          bin(j, g, iqk, rhk, a.x, a.y, e.x, e.y);
        }
      }
    }
  }
  __shared__ float2 red[kFgThreads / 32][kFgEntries][2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kFgEntries; ++j) {
    const float2 x0 = sq[j].warp_pair(), x1 = sl[j].warp_pair();
    if (lane == 0) { red[wid][j][0] = x0; red[wid][j][1] = x1; }
  }
  __syncthreads();
  if (threadIdx.x < kFgEntries * 2) {
    const int j = threadIdx.x >> 1, which = threadIdx.x & 1;
    if (eg + j < nel) {
      double s = 0.0;
      for (int w = 0; w < kFgThreads / 32; ++w) s += (double)red[w][j][which].x + (double)red[w][j][which].y;
      part[((int64_t)chunk * nel + eg + j) * 2 + which] = s;
    }
  }
}

// Eq. like per entry from the chunk partials (fixed order).
__global__ void k_fg_final(const double* __restrict__ part, int nchunks, const double* __restrict__ pp, int32_t e0,
                           int32_t nel, int64_t nb, double df, double sum_lnq, double* __restrict__ logl) {
  const int el = blockIdx.x * blockDim.x + threadIdx.x;
  if (el >= nel) return;
  const int e = e0 + el;
  double q = 0.0, l = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    q += part[((int64_t)c * nel + el) * 2];
    l += part[((int64_t)c * nel + el) * 2 + 1];
  }
  const double* p = pp + (int64_t)e * kPsdDim;
  const double so_a = p[0] * p[0], so_e = p[2] * p[2];
  // q carries |R|^2 2^128 iq / (u S_oms) x 2^-64: restore the 2^64
  logl[e] = -0.5 * 4.0 * df * ldexp(q, 64) - ((double)nb * (log(so_a) + log(so_e)) + 2.0 * sum_lnq + l);
}

static gbk_status fg_loglike(gbk_ctx* ctx, const float* residual, int32_t n_resid, const double* pp,
                             const int32_t* ridx, int32_t n, double* logl, double* scratch, int64_t max_entries,
                             cudaStream_t st) {
  const int64_t nb = ctx->grid.n_bins;
  const int nchunks = (int)((nb + kFgChunk - 1) / kFgChunk);
  for (int32_t e0 = 0; e0 < n; e0 += (int32_t)max_entries) {
    const int32_t nel = (int32_t)(n - e0 < max_entries ? n - e0 : max_entries);
    dim3 grid(nchunks, (nel + kFgEntries - 1) / kFgEntries);
    k_fg_part<<<grid, kFgThreads, 0, st>>>(residual, ctx->iq_f, ctx->rho_f, ctx->fg_lnf, ctx->fg_f, ctx->fg_c, pp, ridx,
                                           n_resid, e0, nel, nb, scratch, ctx->err);
    k_fg_final<<<(nel + 127) / 128, 128, 0, st>>>(scratch, nchunks, pp, e0, nel, nb, 1.0 / ctx->grid.tobs,
                                                 ctx->sum_lnq, logl);
  }
  return check_launch("total_loglike_fg");
}

// Per-channel PSD values [W][2][n] (float64) of the 9-parameter model.
__global__ void k_psd_eval_fg(const double* __restrict__ q, const double* __restrict__ p, const double* __restrict__ pp,
                              int32_t nw, int64_t k0, int64_t nb, double tobs, double* __restrict__ out) {
  const int64_t total = (int64_t)nw * nb;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = i / nb, k = i - w * nb;
    const double* t = pp + w * kPsdDim;
    const double f = (double)(k0 + k) / tobs;
    const double x = 2.0 * 3.141592653589793 * f * kLc, sx = sin(x);
    const double hfg = 0.5 * t[4] * pow(f, -7.0 / 3.0) * exp(-t[7] * pow(f, t[5])) * (1.0 + tanh(-t[8] * (f - t[6])));
    const double sfg = 6.0 * x * x * sx * sx * hfg;
    out[(w * 2 + 0) * nb + k] = t[0] * t[0] * q[k] + t[1] * t[1] * p[k] + sfg;
    out[(w * 2 + 1) * nb + k] = t[2] * t[2] * q[k] + t[3] * t[3] * p[k] + sfg;
  }
}

// -------------------------------------------------------------- PSD sampler
struct PsdArgs {
  gbk_psd_desc d;
  double* params;        // [T][W][9]
  double* logl;          // [T][W]
  double* prop;          // [T * W/2][9] proposals of one half, entry e = k_local * T + t
  double* prop_logl;     // [T * W/2]
  double* lnz;           // [T * W/2]: ln z, or NaN when outside the prior box
  int32_t* ridx;         // [T * W/2] residual index of each entry
  const double* betas;   // [T]
  uint32_t k0, k1, sweep;
  long long* stats;      // [2][2]: stretch, swap (proposed, accepted)
};

__device__ __forceinline__ void to_v(const double* p, double* v) {
  for (int c = 0; c < 5; ++c) v[c] = log(p[c]);
  for (int c = 5; c < kPsdDim; ++c) v[c] = p[c];
}
__device__ __forceinline__ void from_v(const double* v, double* p) {
  for (int c = 0; c < 5; ++c) p[c] = exp(v[c]);
  for (int c = 5; c < kPsdDim; ++c) p[c] = v[c];
}

// Stretch proposals of half h: Y = X_j + z (X_k - X_j), partner j from the other half.
__global__ void k_psd_propose(PsdArgs a, int h) {
  const int T = a.d.n_temps, W = a.d.n_walkers, half = W / 2;
  const int n = T * half;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int kl = e / T, t = e % T;
  const int k = h * half + kl;
  const U4 wv = philox4x32_10((uint32_t)(t * W + k), (uint32_t)h, 5u, a.sweep, a.k0, a.k1);
  const int j = (1 - h) * half + (int)ranged(wv.x, (uint32_t)half);
  const double zz = (a.d.stretch_a - 1.0) * u32(wv.y) + 1.0;
  const double z = zz * zz / a.d.stretch_a;
  double xk[kPsdDim], xj[kPsdDim], y[kPsdDim];
  to_v(a.params + ((int64_t)t * W + k) * kPsdDim, xk);
  to_v(a.params + ((int64_t)t * W + j) * kPsdDim, xj);
  bool in = true;
  for (int c = 0; c < kPsdDim; ++c) {
    y[c] = xj[c] + z * (xk[c] - xj[c]);
    if (!(y[c] >= a.d.lo[c] && y[c] <= a.d.hi[c])) in = false;
  }
  double* pr = a.prop + (int64_t)e * kPsdDim;
  if (in) {
    from_v(y, pr);
  } else {   // evaluate the current point instead (finite); the move is rejected
    for (int c = 0; c < kPsdDim; ++c) pr[c] = a.params[((int64_t)t * W + k) * kPsdDim + c];
  }
  a.lnz[e] = in ? log(z) : __longlong_as_double(0x7ff8000000000000LL);
  a.ridx[e] = k;
}

// Accept or reject every proposal of half h: ln u < beta_t (lnL_Y - lnL_X) + (d - 1) ln z.
__global__ void k_psd_accept(PsdArgs a, int h) {
  const int T = a.d.n_temps, W = a.d.n_walkers, half = W / 2;
  const int n = T * half;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int kl = e / T, t = e % T;
  const int k = h * half + kl;
  const U4 wv = philox4x32_10((uint32_t)(t * W + k), (uint32_t)h, 5u, a.sweep, a.k0, a.k1);
  const double ul = u53(wv.z, wv.w);
  const double lu = ul > 0.0 ? log(ul) : -INFINITY;
  const double lz = a.lnz[e];
  bool acc = false;
  if (lz == lz) {
    const int64_t i = (int64_t)t * W + k;
    const double la = a.betas[t] * (a.prop_logl[e] - a.logl[i]) + (double)(kPsdDim - 1) * lz;
    acc = lu < la;
    if (acc) {
      for (int c = 0; c < kPsdDim; ++c) a.params[i * kPsdDim + c] = a.prop[(int64_t)e * kPsdDim + c];
      a.logl[i] = a.prop_logl[e];
    }
  }
  if (a.stats) {
    atomicAdd((unsigned long long*)&a.stats[0], 1ull);
    if (acc) atomicAdd((unsigned long long*)&a.stats[1], 1ull);
  }
}

// Swaps between temperatures t and t-1 of walker w (one thread per walker, top down).
__global__ void k_psd_swap(PsdArgs a) {
  const int T = a.d.n_temps, W = a.d.n_walkers;
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  unsigned long long prop = 0, accd = 0;
  for (int t = T - 1; t > 0; --t) {
    const U4 wv = philox4x32_10((uint32_t)t, (uint32_t)w, 6u, a.sweep, a.k0, a.k1);
    const double ul = u53(wv.x, wv.y);
    const double lu = ul > 0.0 ? log(ul) : -INFINITY;
    const int64_t it = (int64_t)t * W + w, im = (int64_t)(t - 1) * W + w;
    const double la = (a.betas[t - 1] - a.betas[t]) * (a.logl[it] - a.logl[im]);
    ++prop;
    if (lu < la) {
      ++accd;
      for (int c = 0; c < kPsdDim; ++c) {
        const double q = a.params[it * kPsdDim + c];
        a.params[it * kPsdDim + c] = a.params[im * kPsdDim + c];
        a.params[im * kPsdDim + c] = q;
      }
      const double q = a.logl[it];
      a.logl[it] = a.logl[im];
      a.logl[im] = q;
    }
  }
  if (a.stats) {
    atomicAdd((unsigned long long*)&a.stats[2], prop);
    atomicAdd((unsigned long long*)&a.stats[3], accd);
  }
}

}  // namespace gbk

using namespace gbk;

struct gbk_psd_plan {
  gbk_ctx* ctx;
  gbk_psd_desc d;
  double* prop;
  double* prop_logl;
  double* lnz;
  int32_t* ridx;
  double* scratch;
  int64_t max_entries;
};

extern "C" gbk_status total_loglike_fg(gbk_ctx* ctx, const float* residual, int32_t n_resid, const double* psd_params,
                                       const int32_t* resid_index, int32_t n, double* logl, void* stream) {
  if (!ctx) return set_error(GBK_EINVAL, "total_loglike_fg: null context");
  if (n < 0 || n_resid < 1) return set_error(GBK_EINVAL, "total_loglike_fg: bad counts");
  if (n == 0) return GBK_OK;
  if (!residual || !psd_params || !logl) return set_error(GBK_EINVAL, "total_loglike_fg: null device pointer");
  if (((uintptr_t)residual & 15) != 0) return set_error(GBK_EINVAL, "total_loglike_fg: residual must be 16-byte aligned");
  if (!resid_index && n > n_resid) return set_error(GBK_EINVAL, "total_loglike_fg: more entries than residuals");
  // the context scratch holds chunks x 4096 walkers x 2 doubles
  const int64_t max_entries = 4096;
  return fg_loglike(ctx, residual, n_resid, psd_params, resid_index, n, logl, ctx->scratch, max_entries,
                    (cudaStream_t)stream);
}

extern "C" gbk_status psd_eval_fg(gbk_ctx* ctx, const double* psd_params, int32_t n_walkers, double* s_out,
                                  void* stream) {
  if (!ctx) return set_error(GBK_EINVAL, "psd_eval_fg: null context");
  if (n_walkers < 0) return set_error(GBK_EINVAL, "psd_eval_fg: n_walkers < 0");
  if (n_walkers == 0 || !s_out) return GBK_OK;
  if (!psd_params) return set_error(GBK_EINVAL, "psd_eval_fg: null psd_params");
  const int64_t total = (int64_t)n_walkers * ctx->grid.n_bins;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_psd_eval_fg<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(ctx->psd_q, ctx->psd_p, psd_params, n_walkers,
                                                               ctx->grid.k0, ctx->grid.n_bins, ctx->grid.tobs, s_out);
  return check_launch("psd_eval_fg");
}

extern "C" gbk_status gbk_psd_plan_create(gbk_ctx* ctx, const gbk_psd_desc* desc, gbk_psd_plan** out) {
  if (!ctx || !desc || !out) return set_error(GBK_EINVAL, "gbk_psd_plan_create: null argument");
  *out = nullptr;
  const gbk_psd_desc& d = *desc;
  if (d.n_temps < 1 || d.n_walkers < 2 || (d.n_walkers & 1) || d.n_temps * (int64_t)d.n_walkers > (1 << 20))
    return set_error(GBK_EINVAL, "gbk_psd_plan_create: need n_temps >= 1 and an even n_walkers >= 2");
  if (!(d.stretch_a > 1.0)) return set_error(GBK_EINVAL, "gbk_psd_plan_create: stretch scale a must exceed 1");
  for (int c = 0; c < kPsdDim; ++c)
    if (!(d.lo[c] < d.hi[c])) return set_error(GBK_EINVAL, "gbk_psd_plan_create: empty prior box in coordinate %d", c);
  gbk_psd_plan* p = new gbk_psd_plan();
  p->ctx = ctx;
  p->d = d;
  const int64_t n = (int64_t)d.n_temps * (d.n_walkers / 2);
  const int64_t nchunks = (ctx->grid.n_bins + kFgChunk - 1) / kFgChunk;
  p->max_entries = n;
  cudaError_t e = cudaMalloc((void**)&p->prop, n * kPsdDim * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->prop_logl, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->lnz, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->ridx, n * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->scratch, nchunks * n * 2 * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    gbk_psd_plan_destroy(p);
    return set_error(GBK_ENOMEM, "gbk_psd_plan_create: %s", cudaGetErrorString(e));
  }
  *out = p;
  return GBK_OK;
}

extern "C" gbk_status gbk_psd_plan_destroy(gbk_psd_plan* p) {
  if (!p) return GBK_OK;
  cudaFree(p->prop);
  cudaFree(p->prop_logl);
  cudaFree(p->lnz);
  cudaFree(p->ridx);
  cudaFree(p->scratch);
  delete p;
  return GBK_OK;
}

extern "C" gbk_status gb_psd_sweep(gbk_psd_plan* plan, double* params, double* logl, const float* residual,
                                   const double* betas, uint64_t key, uint32_t sweep_index, int64_t* stats,
                                   void* stream) {
  if (!plan) return set_error(GBK_EINVAL, "gb_psd_sweep: null plan");
  if (!params || !logl || !residual || !betas) return set_error(GBK_EINVAL, "gb_psd_sweep: null device pointer");
  cudaStream_t st = (cudaStream_t)stream;
  PsdArgs a;
  a.d = plan->d;
  a.params = params;
  a.logl = logl;
  a.prop = plan->prop;
  a.prop_logl = plan->prop_logl;
  a.lnz = plan->lnz;
  a.ridx = plan->ridx;
  a.betas = betas;
  a.k0 = (uint32_t)(key & 0xffffffffu);
  a.k1 = (uint32_t)(key >> 32);
  a.sweep = sweep_index;
  a.stats = (long long*)stats;
  const int n = plan->d.n_temps * (plan->d.n_walkers / 2);
  gbk_status s;
  for (int h = 0; h < 2; ++h) {
    k_psd_propose<<<(n + 127) / 128, 128, 0, st>>>(a, h);
    if ((s = check_launch("gb_psd_sweep(propose)"))) return s;
    if ((s = fg_loglike(plan->ctx, residual, plan->d.n_walkers, plan->prop, plan->ridx, n, plan->prop_logl,
                        plan->scratch, plan->max_entries, st)))
      return s;
    k_psd_accept<<<(n + 127) / 128, 128, 0, st>>>(a, h);
    if ((s = check_launch("gb_psd_sweep(accept)"))) return s;
  }
  if (plan->d.n_temps > 1) {
    k_psd_swap<<<(plan->d.n_walkers + 127) / 128, 128, 0, st>>>(a);
    if ((s = check_launch("gb_psd_sweep(swap)"))) return s;
  }
  return GBK_OK;
}
