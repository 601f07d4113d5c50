// GB waveform, Delta lnL and residual add/sub kernels and their C-ABI entry points.
#include <math.h>
#include <stdio.h>

#include "gbk_internal.cuh"
#include "gbk_wave.cuh"
#include "gbk_reduce.cuh"

namespace gbk {

constexpr int kWarpsPerCta = 4;      // default warps per CTA
constexpr int kMaxWarpsPerCta = 8;   // largest shape the autotuner may pick

template <typename T>
__device__ __forceinline__ const T* orb_table(const gbk_ctx& c, int bi);
template <>
__device__ __forceinline__ const float* orb_table<float>(const gbk_ctx& c, int bi) { return c.orb_f[bi]; }
template <>
__device__ __forceinline__ const double* orb_table<double>(const gbk_ctx& c, int bi) { return c.orb_d[bi]; }
template <typename T>
__device__ __forceinline__ const typename CT<T>::C* tw_table(const gbk_ctx& c, int bi);
template <>
__device__ __forceinline__ const float2* tw_table<float>(const gbk_ctx& c, int bi) { return c.tw_f[bi]; }
template <>
__device__ __forceinline__ const double2* tw_table<double>(const gbk_ctx& c, int bi) { return c.tw_d[bi]; }

// Dispatch a warp to gen_band<T, N> for its runtime N (<= NMAX).
template <typename T, int NMAX>
__device__ __forceinline__ bool gen_any(const gbk_ctx& c, const Src<T>* s, int n,
                                        typename CT<T>::C* b0, typename CT<T>::C* b1, int lane) {
  const double tobs = c.grid.tobs;
  switch (n) {
    case 128: gen_band<T, 128>(s, orb_table<T>(c, 0), tw_table<T>(c, 0), tobs, b0, b1, lane); return true;
    case 256: if (NMAX >= 256) { gen_band<T, 256>(s, orb_table<T>(c, 1), tw_table<T>(c, 1), tobs, b0, b1, lane); return true; } break;
    case 512: if (NMAX >= 512) { gen_band<T, 512>(s, orb_table<T>(c, 2), tw_table<T>(c, 2), tobs, b0, b1, lane); return true; } break;
    case 1024: if (NMAX >= 1024) { gen_band<T, 1024>(s, orb_table<T>(c, 3), tw_table<T>(c, 3), tobs, b0, b1, lane); return true; } break;
    default: break;
  }
  return false;
}

// Shared memory of one warp: `nbuf` waveform buffers [2][NMAX] and a batch of per-source
// constants (lane l of the warp computes the constants of batch item l in float64).
template <typename T>
__host__ __device__ constexpr size_t warp_bytes(int nmax, int nbuf, int nsrc) {
  return (size_t)nbuf * 2 * nmax * sizeof(typename CT<T>::C) + (size_t)nsrc * sizeof(Src<T>) + 64 * sizeof(int) +
         32 * sizeof(double);
}

// ---------------------------------------------------------------- gb_waveform_batch
template <typename T, int NMAX>
__global__ void __launch_bounds__(kMaxWarpsPerCta * 32)
k_waveform(const gbk_ctx c, const double* __restrict__ params, const int32_t* __restrict__ nb,
           int64_t n, int64_t* __restrict__ k_start, typename CT<T>::C* __restrict__ ha,
           typename CT<T>::C* __restrict__ he, const int64_t* __restrict__ off) {
  typedef typename CT<T>::C C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  unsigned char* mine = smem_raw + (size_t)wid * warp_bytes<T>(NMAX, 2, 32);
  C* b0 = reinterpret_cast<C*>(mine);
  C* b1 = b0 + 2 * NMAX;
  Src<T>* srcs = reinterpret_cast<Src<T>*>(b1 + 2 * NMAX);
  int* nbs = reinterpret_cast<int*>(srcs + 32);
  const int wpc = blockDim.x >> 5;
  const int64_t stride_w = (int64_t)gridDim.x * wpc * 32;
  for (int64_t base = ((int64_t)blockIdx.x * wpc + wid) * 32; base < n; base += stride_w) {
    const int64_t me = base + lane;
    if (me < n) {
      const int nbi = nb[me];
      nbs[lane] = nbi;
      if (nbi <= NMAX && band_index(nbi) >= 0) srcs[lane] = make_src<T>(params, n, me, c.grid.tobs, nbi);
    }
    __syncwarp();
    const int cnt = (int)min((int64_t)32, n - base);
    for (int q = 0; q < cnt; ++q) {
      const int64_t i = base + q;
      const int nbi = nbs[q];
      if (nbi > NMAX || band_index(nbi) < 0) {
        if (lane == 0) atomicOr(c.err, kErrBand);
        continue;
      }
      gen_any<T, NMAX>(c, &srcs[q], nbi, b0, b1, lane);
      const T down = (T)5.421010862427522170e-20;  // 2^-64 back to strain units
      const int64_t o = off[i];
      for (int j = lane; j < nbi; j += 32) {
        ha[o + j] = cscale(b0[j], down);
        he[o + j] = cscale(b0[nbi + j], down);
      }
      if (lane == 0) k_start[i] = srcs[q].q - nbi / 2;
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------- Delta lnL
template <typename T> struct Acc;
template <> struct Acc<float> { typedef CompF S; };
template <> struct Acc<double> { typedef PlainD S; };

// Per-walker PSD weight: 4 df / (S_k 2^128) = cw * iq_k / (1 + aw rho_k); the bins
// carry iq_k / (1 + aw rho_k) and cw (float64) multiplies the final sums.
template <typename T>
struct PsdW {
  double cw;
  T aw;
};
template <typename T>
__device__ __forceinline__ PsdW<T> psd_walker(const gbk_ctx& c, const double* __restrict__ pp, int npsd, int w) {
  const int j = (npsd == 1) ? 0 : w;
  const double so = pp[2 * j] * pp[2 * j];
  const double sa = pp[2 * j + 1] * pp[2 * j + 1];
  PsdW<T> r;
  r.cw = 4.0 / c.grid.tobs / so;
  r.aw = (T)(sa / so);
  return r;
}
__device__ __forceinline__ float iq_at(const gbk_ctx& c, int64_t k, float) { return __ldg(&c.iq_f[k]); }
__device__ __forceinline__ double iq_at(const gbk_ctx& c, int64_t k, double) { return __ldg(&c.iq_d[k]); }
__device__ __forceinline__ float rho_at(const gbk_ctx& c, int64_t k, float) { return __ldg(&c.rho_f[k]); }
__device__ __forceinline__ double rho_at(const gbk_ctx& c, int64_t k, double) { return __ldg(&c.rho_d[k]); }
__device__ __forceinline__ float i2r(long long v, float) { return ll_to_float(v); }
__device__ __forceinline__ double i2r(long long v, double) { return __ll2double_rn(v); }
__device__ __forceinline__ float rcp_(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }

// Accumulate |D|^2 w and Re(R* D) w over one bin (both channels).
template <typename T>
__device__ __forceinline__ void acc_bin(const gbk_ctx& c, const long long* __restrict__ rw,
                                        int64_t kloc, typename CT<T>::C da, typename CT<T>::C de,
                                        T aw, T rscale,
                                        typename Acc<T>::S& sdd, typename Acc<T>::S& srd) {
  const int64_t nbins = c.grid.n_bins;
  const longlong2 ra = *reinterpret_cast<const longlong2*>(rw + 2 * kloc);
  const longlong2 re = *reinterpret_cast<const longlong2*>(rw + 2 * (nbins + kloc));
  const T w = iq_at(c, kloc, T()) * rcp_((T)1 + aw * rho_at(c, kloc, T()));
  const T rax = i2r(ra.x, T()) * rscale, ray = i2r(ra.y, T()) * rscale;
  const T rex = i2r(re.x, T()) * rscale, rey = i2r(re.y, T()) * rscale;
  sdd.add(w * (da.x * da.x + da.y * da.y + de.x * de.x + de.y * de.y));
  srd.add(w * (rax * da.x + ray * da.y + rex * de.x + rey * de.y));
}

// Sums <D|D> and <R|D> of proposal (a in ba at window offset ka, r in br at kr; either may be
// absent) against walker w's residual over the band bins [jb, je), by the 32 lanes of one warp:
// lane l sums the bins jb + l, jb + l + 32, ... of each band in order (the same summation in every
// kernel that calls it). Returns the warp totals in dd, rd.
template <typename T>
__device__ __forceinline__ void eval_sums(const gbk_ctx& c, const typename CT<T>::C* ba, const typename CT<T>::C* br,
                                          bool za, bool zr, int64_t ka, int64_t kr, int nbi, int w,
                                          const long long* __restrict__ resid, int32_t frac_bits, T aw, int lane,
                                          int jb, int je, double& dd_out, double& rd_out) {
  typedef typename CT<T>::C C;
  const int64_t nbins = c.grid.n_bins;
  const T rscale = (T)ldexp(1.0, kStrainExp - frac_bits);
  const long long* rw = resid + (int64_t)w * 2 * nbins * 2;
  typename Acc<T>::S sdd, srd;
  sdd.init();
  srd.init();
  const C zero = mkc((T)0, (T)0);
  // bins of a's band: D = a - r (r where the bands overlap)
  if (!za) {
    for (int j = jb + lane; j < je; j += 32) {
      const int64_t k = ka + j;
      C ra = zero, re = zero;
      const int64_t jr = k - kr;
      if (!zr && jr >= 0 && jr < nbi) { ra = br[jr]; re = br[nbi + jr]; }
      acc_bin<T>(c, rw, k, csub(ba[j], ra), csub(ba[nbi + j], re), aw, rscale, sdd, srd);
    }
  }
  // bins of r's band outside a's band: D = -r
  if (!zr) {
    for (int j = jb + lane; j < je; j += 32) {
      const int64_t k = kr + j;
      const int64_t ja = k - ka;
      if (!za && ja >= 0 && ja < nbi) continue;
      const C ra = br[j], re = br[nbi + j];
      acc_bin<T>(c, rw, k, mkc(-ra.x, -ra.y), mkc(-re.x, -re.y), aw, rscale, sdd, srd);
    }
  }
  dd_out = sdd.warp_total();
  rd_out = srd.warp_total();
}

// Delta lnL of the proposal over the whole band by one warp.
template <typename T>
__device__ __forceinline__ void eval_pair(const gbk_ctx& c, const typename CT<T>::C* ba, const typename CT<T>::C* br,
                                          bool za, bool zr, int64_t ka, int64_t kr, int nbi, int w,
                                          const long long* __restrict__ resid, int32_t frac_bits, double cw, T aw,
                                          int lane, double* out) {
  double dd, rd;
  eval_sums<T>(c, ba, br, za, zr, ka, kr, nbi, w, resid, frac_bits, aw, lane, 0, nbi, dd, rd);
  if (lane == 0) *out = cw * (-0.5 * dd + rd);
}

// Batch of 16 proposals per warp: lanes 0-15 set up the new templates, 16-31 the old.
template <typename T, int NMAX>
__global__ void __launch_bounds__(kMaxWarpsPerCta * 32)
k_dlogl(const gbk_ctx c, const double* __restrict__ pnew, const double* __restrict__ pold,
        const int32_t* __restrict__ nb, const int32_t* __restrict__ walker, int64_t n,
        const long long* __restrict__ resid, int32_t n_walkers, int32_t frac_bits,
        const double* __restrict__ psdp, int32_t npsd, double* __restrict__ dlogl) {
  typedef typename CT<T>::C C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  unsigned char* mine = smem_raw + (size_t)wid * warp_bytes<T>(NMAX, 3, 32);
  C* ba = reinterpret_cast<C*>(mine);
  C* br = ba + 2 * NMAX;
  C* bs = br + 2 * NMAX;
  Src<T>* srcs = reinterpret_cast<Src<T>*>(bs + 2 * NMAX);   // [0,16) new, [16,32) old
  int* meta = reinterpret_cast<int*>(srcs + 32);            // [0,16) N, [16,32) walker
  double* s_cw = reinterpret_cast<double*>(meta + 64);       // [16] PSD weights of the batch's walkers
  T* s_aw = reinterpret_cast<T*>(s_cw + 16);                 // [16]
  const int wpc = blockDim.x >> 5;
  const int64_t stride_w = (int64_t)gridDim.x * wpc * 16;
  const int64_t nbins = c.grid.n_bins;
  for (int64_t base = ((int64_t)blockIdx.x * wpc + wid) * 16; base < n; base += stride_w) {
    {
      const int l = lane & 15;
      const int64_t me = base + l;
      if (me < n) {
        const int nbi = nb[me];
        if (lane < 16) {
          const int w = walker[me];
          meta[l] = nbi;
          meta[16 + l] = w;
          if (w >= 0 && w < n_walkers && (npsd == 1 || w < npsd)) {   // once per proposal, lane-parallel
            const PsdW<T> pw = psd_walker<T>(c, psdp, npsd, w);
            s_cw[l] = pw.cw;
            s_aw[l] = pw.aw;
          }
        }
        if (nbi <= NMAX && band_index(nbi) >= 0)
          srcs[lane] = make_src<T>(lane < 16 ? pnew : pold, n, me, c.grid.tobs, nbi);
      }
    }
    __syncwarp();
    const int cnt = (int)min((int64_t)16, n - base);
    for (int q = 0; q < cnt; ++q) {
      const int64_t i = base + q;
      const int nbi = meta[q];
      const int w = meta[16 + q];
      if (nbi > NMAX || band_index(nbi) < 0 || w < 0 || w >= n_walkers || (npsd != 1 && w >= npsd)) {
        if (lane == 0) {
          atomicOr(c.err, (w < 0 || w >= n_walkers || (npsd != 1 && w >= npsd)) ? kErrWalker : kErrBand);
          dlogl[i] = __longlong_as_double(0x7ff8000000000000LL);
        }
        continue;
      }
      const Src<T>* sa = &srcs[q];
      const Src<T>* sr = &srcs[16 + q];
      const bool za = sa->zero, zr = sr->zero;
      const int64_t ka = sa->q - nbi / 2 - c.grid.k0;
      const int64_t kr = sr->q - nbi / 2 - c.grid.k0;
      const bool bad = (!za && (ka < 0 || ka + nbi > nbins)) || (!zr && (kr < 0 || kr + nbi > nbins));
      if (bad) {
        if (lane == 0) {
          atomicOr(c.err, kErrRange);
          dlogl[i] = __longlong_as_double(0x7ff8000000000000LL);
        }
        continue;
      }
      if (!za) gen_any<T, NMAX>(c, sa, nbi, ba, bs, lane);
      if (!zr) gen_any<T, NMAX>(c, sr, nbi, br, bs, lane);
      eval_pair<T>(c, ba, br, za, zr, ka, kr, nbi, w, resid, frac_bits, s_cw[q], s_aw[q], lane, dlogl + i);
      __syncwarp();
    }
    __syncwarp();
  }
}

// Delta lnL for long bands with each waveform generated by a whole block of NT threads: one
// warp's three band buffers of 1024 bins (48 KB) would leave an SM four warps, the block shares
// them among NT / 32 warps. Batches of 16 proposals as in k_dlogl: warp 0 sets up the source
// constants and evaluates the sums with eval_pair, so every result has the same bits as
// k_dlogl's for the same proposal.
template <typename T, int NMAX, int NT>
__device__ __forceinline__ bool gen_any_block(const gbk_ctx& c, const Src<T>* s, int n, typename CT<T>::C* b0,
                                              typename CT<T>::C* b1, int tid) {
  const double tobs = c.grid.tobs;
  switch (n) {
    case 128: gen_band_block<T, 128, NT>(s, orb_table<T>(c, 0), tw_table<T>(c, 0), tobs, b0, b1, tid); return true;
    case 256: gen_band_block<T, 256, NT>(s, orb_table<T>(c, 1), tw_table<T>(c, 1), tobs, b0, b1, tid); return true;
    case 512: gen_band_block<T, 512, NT>(s, orb_table<T>(c, 2), tw_table<T>(c, 2), tobs, b0, b1, tid); return true;
    case 1024: if (NMAX >= 1024) { gen_band_block<T, 1024, NT>(s, orb_table<T>(c, 3), tw_table<T>(c, 3), tobs, b0, b1, tid); return true; } break;
    default: break;
  }
  return false;
}

template <typename T, int NMAX>
constexpr int block_threads() { return NMAX / 8; }   // 8 coarse samples per thread

template <typename T, int NMAX, int NT>
__global__ void __launch_bounds__(NT, 512 / NT)
k_dlogl_block(const gbk_ctx c, const double* __restrict__ pnew, const double* __restrict__ pold,
              const int32_t* __restrict__ nb, const int32_t* __restrict__ walker, int64_t n,
              const long long* __restrict__ resid, int32_t n_walkers, int32_t frac_bits,
              const double* __restrict__ psdp, int32_t npsd, double* __restrict__ dlogl) {
  typedef typename CT<T>::C C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int wid = tid >> 5;
  C* ba = reinterpret_cast<C*>(smem_raw);
  C* br = ba + 2 * NMAX;
  C* bs = br + 2 * NMAX;
  Src<T>* srcs = reinterpret_cast<Src<T>*>(bs + 2 * NMAX);   // [0,16) new, [16,32) old
  int* meta = reinterpret_cast<int*>(srcs + 32);            // [0,16) N, [16,32) walker
  __shared__ double part[NT / 32][2];                        // per-warp sums of one proposal
  const int64_t nbins = c.grid.n_bins;
  for (int64_t base = (int64_t)blockIdx.x * 16; base < n; base += (int64_t)gridDim.x * 16) {
    if (wid == 0) {
      const int l = lane & 15;
      const int64_t me = base + l;
      if (me < n) {
        const int nbi = nb[me];
        if (lane < 16) { meta[l] = nbi; meta[16 + l] = walker[me]; }
        if (nbi <= NMAX && band_index(nbi) >= 0)
          srcs[lane] = make_src<T>(lane < 16 ? pnew : pold, n, me, c.grid.tobs, nbi);
      }
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)16, n - base);
    for (int q = 0; q < cnt; ++q) {
      const int64_t i = base + q;
      const int nbi = meta[q];
      const int w = meta[16 + q];
      if (nbi > NMAX || band_index(nbi) < 0 || w < 0 || w >= n_walkers || (npsd != 1 && w >= npsd)) {
        if (tid == 0) {
          atomicOr(c.err, (w < 0 || w >= n_walkers || (npsd != 1 && w >= npsd)) ? kErrWalker : kErrBand);
          dlogl[i] = __longlong_as_double(0x7ff8000000000000LL);
        }
        continue;
      }
      const Src<T>* sa = &srcs[q];
      const Src<T>* sr = &srcs[16 + q];
      const bool za = sa->zero, zr = sr->zero;
      const int64_t ka = sa->q - nbi / 2 - c.grid.k0;
      const int64_t kr = sr->q - nbi / 2 - c.grid.k0;
      const bool bad = (!za && (ka < 0 || ka + nbi > nbins)) || (!zr && (kr < 0 || kr + nbi > nbins));
      if (bad) {
        if (tid == 0) {
          atomicOr(c.err, kErrRange);
          dlogl[i] = __longlong_as_double(0x7ff8000000000000LL);
        }
        continue;
      }
      if (!za) gen_any_block<T, NMAX, NT>(c, sa, nbi, ba, bs, tid);
      if (!zr) gen_any_block<T, NMAX, NT>(c, sr, nbi, br, bs, tid);
      // the sums over 256-bin quarters of the band by as many warps (a partition fixed by the band
      // length alone, so any block shape gives the same bits), added in quarter order
      const int ne = nbi > 256 ? nbi / 256 : 1;
      if (wid < ne) {
        const int jb = wid * (nbi / ne);
        double dd, rd;
        // the PSD weight per warp (from a per-batch table, as in k_dlogl, this kernel ran 8 % slower)
        eval_sums<T>(c, ba, br, za, zr, ka, kr, nbi, w, resid, frac_bits, psd_walker<T>(c, psdp, npsd, w).aw, lane, jb,
                     jb + nbi / ne, dd, rd);
        if (lane == 0) { part[wid][0] = dd; part[wid][1] = rd; }
      }
      __syncthreads();
      if (tid == 0) {
        double dd = part[0][0], rd = part[0][1];
        for (int v = 1; v < ne; ++v) { dd += part[v][0]; rd += part[v][1]; }
        dlogl[i] = psd_walker<T>(c, psdp, npsd, w).cw * (-0.5 * dd + rd);
      }
      __syncthreads();   // the buffers are reused by the next proposal
    }
    __syncthreads();     // the batch's constants are rewritten
  }
}

// ---------------------------------------------------------------- residual add/sub
__device__ __forceinline__ long long to_grid(float v, float s) { return float_to_ll(v * s); }
__device__ __forceinline__ long long to_grid(double v, double s) { return __double2ll_rn(v * s); }

template <typename T, int NMAX>
__global__ void __launch_bounds__(kMaxWarpsPerCta * 32)
k_addsub(const gbk_ctx c, const double* __restrict__ params, const int32_t* __restrict__ nb,
         const int32_t* __restrict__ walker, int64_t n, long long* __restrict__ resid,
         int32_t n_walkers, int32_t frac_bits, int sign) {
  typedef typename CT<T>::C C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  unsigned char* mine = smem_raw + (size_t)wid * warp_bytes<T>(NMAX, 2, 32);
  C* b0 = reinterpret_cast<C*>(mine);
  C* b1 = b0 + 2 * NMAX;
  Src<T>* srcs = reinterpret_cast<Src<T>*>(b1 + 2 * NMAX);
  int* meta = reinterpret_cast<int*>(srcs + 32);   // N in [0,32); walker kept in registers of lane q
  const int wpc = blockDim.x >> 5;
  const int64_t stride_w = (int64_t)gridDim.x * wpc * 32;
  const int64_t nbins = c.grid.n_bins;
  const T gs = (T)ldexp(1.0, frac_bits - kStrainExp);
  for (int64_t base = ((int64_t)blockIdx.x * wpc + wid) * 32; base < n; base += stride_w) {
    const int64_t me = base + lane;
    int my_w = -1;
    if (me < n) {
      const int nbi = nb[me];
      meta[lane] = nbi;
      my_w = walker[me];
      if (nbi <= NMAX && band_index(nbi) >= 0) srcs[lane] = make_src<T>(params, n, me, c.grid.tobs, nbi);
    }
    __syncwarp();
    const int cnt = (int)min((int64_t)32, n - base);
    for (int q = 0; q < cnt; ++q) {
      const int nbi = meta[q];
      const int w = __shfl_sync(0xffffffffu, my_w, q);
      if (nbi > NMAX || band_index(nbi) < 0 || w < 0 || w >= n_walkers) {
        if (lane == 0) atomicOr(c.err, (w < 0 || w >= n_walkers) ? kErrWalker : kErrBand);
        continue;
      }
      const Src<T>* s = &srcs[q];
      if (s->zero) continue;
      const int64_t k = s->q - nbi / 2 - c.grid.k0;
      if (k < 0 || k + nbi > nbins) {
        if (lane == 0) atomicOr(c.err, kErrRange);
        continue;
      }
      gen_any<T, NMAX>(c, s, nbi, b0, b1, lane);
      unsigned long long* rw = reinterpret_cast<unsigned long long*>(resid) + (int64_t)w * 2 * nbins * 2;
      for (int j = lane; j < nbi; j += 32) {
        for (int ch = 0; ch < 2; ++ch) {
          const C h = b0[ch * nbi + j];
          long long hx = to_grid(h.x, gs), hy = to_grid(h.y, gs);
          if (sign > 0) { hx = -hx; hy = -hy; }   // template enters the model: R -= h
          unsigned long long* dst = rw + 2 * (ch * nbins + k + j);
          atomicAdd(dst, (unsigned long long)hx);
          atomicAdd(dst + 1, (unsigned long long)hy);
        }
      }
      __syncwarp();
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- launch helpers

// Warps per CTA: up to kWarpsPerCta, fewer when a warp's buffers are large.
static int warps_for(size_t per_warp) {
  const size_t cap = 220 * 1024;
  int w = (int)(cap / per_warp);
  return w < 1 ? 1 : (w > kWarpsPerCta ? kWarpsPerCta : w);
}

template <typename K>
static gbk_status launch_cfg(K kernel, size_t per_warp, int64_t items, int* grid_out, int* threads_out,
                             size_t* smem_out, int want_wpc = 0, int want_bps = 0) {
  int wpc = warps_for(per_warp);
  if (want_wpc > 0 && (size_t)want_wpc * per_warp <= 220 * 1024) wpc = want_wpc;
  const size_t smem = per_warp * wpc;
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return set_error(GBK_ECUDA, "cudaFuncSetAttribute(smem=%zu) failed", smem);
    }
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, wpc * 32, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return set_error(GBK_ECUDA, "kernel does not fit on an SM (smem=%zu)", smem);
  }
  if (want_bps > 0 && want_bps < per_sm) per_sm = want_bps;
  int64_t need = (items + wpc - 1) / wpc;
  int64_t cap = (int64_t)sms * per_sm;   // a multiple of the SM count: one persistent wave
  *grid_out = (int)(need < cap ? (need > 0 ? need : 1) : cap);
  *threads_out = wpc * 32;
  *smem_out = smem;
  return GBK_OK;
}

static bool valid_nmax(int nmax) { return band_index(nmax) >= 0; }

template <typename T>
static gbk_status waveform_t(gbk_ctx* ctx, const double* params, const int32_t* nb, int nmax, int64_t n,
                             int64_t* ks, void* ha, void* he, const int64_t* off, cudaStream_t st) {
  typedef typename CT<T>::C C;
  const size_t pw = warp_bytes<T>(nmax, 2, 32);
  int grid = 0, thr = 0;
  size_t smem = 0;
  gbk_status s = GBK_OK;
#define GBK_WF(NM)                                                                              \
  case NM:                                                                                      \
    s = launch_cfg(k_waveform<T, NM>, pw, (n + 31) / 32, &grid, &thr, &smem);                               \
    if (s) return s;                                                                            \
    k_waveform<T, NM><<<grid, thr, smem, st>>>(*ctx, params, nb, n, ks, (C*)ha, (C*)he, off);   \
    break;
  switch (nmax) { GBK_WF(128) GBK_WF(256) GBK_WF(512) GBK_WF(1024) }
#undef GBK_WF
  return check_launch("gb_waveform_batch");
}

// Block shape of k_dlogl_block: its shared memory, and blocks per SM (the autotuned cap, if any).
template <typename T, int NMAX>
static gbk_status dlogl_block(gbk_ctx* ctx, const double* pn, const double* po, const int32_t* nb,
                              const int32_t* walker, int64_t n, const gbk_residual* R, const gbk_psd* psd,
                              double* out, cudaStream_t st) {
  constexpr int NT = block_threads<T, NMAX>();
  const size_t smem = 3 * 2 * NMAX * sizeof(typename CT<T>::C) + 32 * sizeof(Src<T>) + 32 * sizeof(int);
  auto kernel = k_dlogl_block<T, NMAX, NT>;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return set_error(GBK_ECUDA, "cudaFuncSetAttribute(smem=%zu) failed", smem);
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return set_error(GBK_ECUDA, "k_dlogl_block does not fit on an SM (smem=%zu)", smem);
  }
  const int pi = sizeof(T) == sizeof(float) ? GBK_MIXED : GBK_FP64;
  const int cap_bps = ctx->tune_bps[pi][band_index(NMAX)];
  if (cap_bps > 0 && cap_bps < per_sm) per_sm = cap_bps;
  const int64_t need = (n + 15) / 16;
  const int64_t cap = (int64_t)sms * per_sm;
  const int grid = (int)(need < cap ? need : cap);
  kernel<<<grid, NT, smem, st>>>(*ctx, pn, po, nb, walker, n, (const long long*)R->data, R->n_walkers, R->frac_bits,
                                 psd->params, psd->n_psd, out);
  return check_launch("gb_delta_loglike_batch");
}

template <typename T>
static gbk_status dlogl_t(gbk_ctx* ctx, const double* pn, const double* po, const int32_t* nb, int nmax,
                          const int32_t* walker, int64_t n, const gbk_residual* R, const gbk_psd* psd,
                          double* out, cudaStream_t st) {
  // long bands: waveforms generated by a block (512: 2 warps, 1024: 4 warps)
  if (nmax == 512) return dlogl_block<T, 512>(ctx, pn, po, nb, walker, n, R, psd, out, st);
  if (nmax == 1024) return dlogl_block<T, 1024>(ctx, pn, po, nb, walker, n, R, psd, out, st);
  const size_t pw = warp_bytes<T>(nmax, 3, 32);
  const int pi = sizeof(T) == sizeof(float) ? GBK_MIXED : GBK_FP64;
  int grid = 0, thr = 0;
  size_t smem = 0;
  gbk_status s = GBK_OK;
#define GBK_DL(NM)                                                                                      \
  case NM:                                                                                              \
    s = launch_cfg(k_dlogl<T, NM>, pw, (n + 15) / 16, &grid, &thr, &smem, ctx->tune_wpc[pi][band_index(NM)],     \
                   ctx->tune_bps[pi][band_index(NM)]);                                          \
    if (s) return s;                                                                                    \
    k_dlogl<T, NM><<<grid, thr, smem, st>>>(*ctx, pn, po, nb, walker, n,                                \
                                                          (const long long*)R->data, R->n_walkers,      \
                                                          R->frac_bits, psd->params, psd->n_psd, out);  \
    break;
  switch (nmax) { GBK_DL(128) GBK_DL(256) GBK_DL(512) GBK_DL(1024) }
#undef GBK_DL
  return check_launch("gb_delta_loglike_batch");
}

template <typename T>
static gbk_status addsub_t(gbk_ctx* ctx, const gbk_residual* R, const double* params, const int32_t* nb,
                           int nmax, const int32_t* walker, int64_t n, int sign, cudaStream_t st) {
  const size_t pw = warp_bytes<T>(nmax, 2, 32);
  int grid = 0, thr = 0;
  size_t smem = 0;
  gbk_status s = GBK_OK;
#define GBK_AS(NM)                                                                               \
  case NM:                                                                                       \
    s = launch_cfg(k_addsub<T, NM>, pw, (n + 31) / 32, &grid, &thr, &smem);                                  \
    if (s) return s;                                                                             \
    k_addsub<T, NM><<<grid, thr, smem, st>>>(*ctx, params, nb, walker, n,                        \
                                                           (long long*)R->data, R->n_walkers,    \
                                                           R->frac_bits, sign);                  \
    break;
  switch (nmax) { GBK_AS(128) GBK_AS(256) GBK_AS(512) GBK_AS(1024) }
#undef GBK_AS
  return check_launch("residual_add_sub");
}

}  // namespace gbk

using namespace gbk;

extern "C" gbk_status gb_waveform_batch(gbk_ctx* ctx, const double* params, const int32_t* n_band,
                                        int32_t n_band_max, int64_t n, int64_t* k_start, void* h_a,
                                        void* h_e, const int64_t* out_off, gbk_precision precision,
                                        void* stream) {
  if (!ctx) return set_error(GBK_EINVAL, "gb_waveform_batch: null context");
  if (n < 0) return set_error(GBK_EINVAL, "gb_waveform_batch: n < 0");
  if (n == 0) return GBK_OK;
  if (!params || !n_band || !k_start || !h_a || !h_e || !out_off)
    return set_error(GBK_EINVAL, "gb_waveform_batch: null device pointer");
  if (!valid_nmax(n_band_max)) return set_error(GBK_EINVAL, "gb_waveform_batch: n_band_max %d not in {128,256,512,1024}", n_band_max);
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == GBK_MIXED) return waveform_t<float>(ctx, params, n_band, n_band_max, n, k_start, h_a, h_e, out_off, st);
  if (precision == GBK_FP64) return waveform_t<double>(ctx, params, n_band, n_band_max, n, k_start, h_a, h_e, out_off, st);
  return set_error(GBK_EINVAL, "gb_waveform_batch: bad precision %d", (int)precision);
}

extern "C" gbk_status gb_delta_loglike_batch(gbk_ctx* ctx, const double* params_new,
                                             const double* params_old, const int32_t* n_band,
                                             int32_t n_band_max, const int32_t* walker, int64_t n,
                                             const gbk_residual* residual, const gbk_psd* psd,
                                             double* dlogl, gbk_precision precision, void* stream) {
  if (!ctx || !residual || !psd) return set_error(GBK_EINVAL, "gb_delta_loglike_batch: null context/struct");
  if (n < 0) return set_error(GBK_EINVAL, "gb_delta_loglike_batch: n < 0");
  if (n == 0) return GBK_OK;
  if (!params_new || !params_old || !n_band || !walker || !dlogl || !residual->data || !psd->params)
    return set_error(GBK_EINVAL, "gb_delta_loglike_batch: null device pointer");
  if (!valid_nmax(n_band_max)) return set_error(GBK_EINVAL, "gb_delta_loglike_batch: bad n_band_max %d", n_band_max);
  if (residual->n_walkers < 1 || residual->frac_bits < 40 || residual->frac_bits > 120 || psd->n_psd < 1)
    return set_error(GBK_EINVAL, "gb_delta_loglike_batch: bad residual/psd description");
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == GBK_MIXED) return dlogl_t<float>(ctx, params_new, params_old, n_band, n_band_max, walker, n, residual, psd, dlogl, st);
  if (precision == GBK_FP64) return dlogl_t<double>(ctx, params_new, params_old, n_band, n_band_max, walker, n, residual, psd, dlogl, st);
  return set_error(GBK_EINVAL, "gb_delta_loglike_batch: bad precision %d", (int)precision);
}

extern "C" gbk_status residual_add_sub(gbk_ctx* ctx, const gbk_residual* residual, const double* params,
                                       const int32_t* n_band, int32_t n_band_max, const int32_t* walker,
                                       int64_t n, int32_t sign, gbk_precision precision, void* stream) {
  if (!ctx || !residual) return set_error(GBK_EINVAL, "residual_add_sub: null context/struct");
  if (n < 0) return set_error(GBK_EINVAL, "residual_add_sub: n < 0");
  if (sign != 1 && sign != -1) return set_error(GBK_EINVAL, "residual_add_sub: sign must be +1 or -1");
  if (n == 0) return GBK_OK;
  if (!params || !n_band || !walker || !residual->data) return set_error(GBK_EINVAL, "residual_add_sub: null device pointer");
  if (!valid_nmax(n_band_max)) return set_error(GBK_EINVAL, "residual_add_sub: bad n_band_max %d", n_band_max);
  if (residual->n_walkers < 1 || residual->frac_bits < 40 || residual->frac_bits > 120)
    return set_error(GBK_EINVAL, "residual_add_sub: bad residual description");
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == GBK_MIXED) return addsub_t<float>(ctx, residual, params, n_band, n_band_max, walker, n, sign, st);
  if (precision == GBK_FP64) return addsub_t<double>(ctx, residual, params, n_band, n_band_max, walker, n, sign, st);
  return set_error(GBK_EINVAL, "residual_add_sub: bad precision %d", (int)precision);
}

// Time gb_delta_loglike_batch on the caller's sample batch for every launch shape (warps per
// CTA 1, 2, 4, 8 that fit; CTAs per SM 1, 2, 4 or as many as fit) and keep the fastest for
// this precision and band length in the context.
extern "C" gbk_status gbk_autotune_dlogl(gbk_ctx* ctx, const double* params_new, const double* params_old,
                                         const int32_t* n_band, int32_t n_band_max, const int32_t* walker, int64_t n,
                                         const gbk_residual* residual, const gbk_psd* psd, double* dlogl,
                                         gbk_precision precision, int32_t* best_out, void* stream) {
  if (!ctx) return set_error(GBK_EINVAL, "gbk_autotune_dlogl: null context");
  if (!valid_nmax(n_band_max) || (precision != GBK_MIXED && precision != GBK_FP64) || n < 1)
    return set_error(GBK_EINVAL, "gbk_autotune_dlogl: bad arguments");
  const int bi = band_index(n_band_max);
  const int pi = (int)precision;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return set_error(GBK_ECUDA, "gbk_autotune_dlogl: cudaEventCreate failed");
  }
  float best = 1e30f;
  int bw = 0, bb = 0;
  const int wpcs[4] = {1, 2, 4, 8};
  const int bpss[4] = {1, 2, 4, 0};
  gbk_status s = GBK_OK;
  const int n_wpc = n_band_max >= 512 ? 1 : 4;   // long bands: fixed block shape, only its count per SM
  for (int i = 0; i < n_wpc && !s; ++i)
    for (int j = 0; j < 4 && !s; ++j) {
      ctx->tune_wpc[pi][bi] = wpcs[i];
      ctx->tune_bps[pi][bi] = bpss[j];
      s = gb_delta_loglike_batch(ctx, params_new, params_old, n_band, n_band_max, walker, n, residual, psd, dlogl,
                                 precision, stream);
      if (s) break;
      cudaEventRecord(e0, st);
      for (int r = 0; r < 3 && !s; ++r)
        s = gb_delta_loglike_batch(ctx, params_new, params_old, n_band, n_band_max, walker, n, residual, psd, dlogl,
                                   precision, stream);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (!s && ms < best) { best = ms; bw = wpcs[i]; bb = bpss[j]; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->tune_wpc[pi][bi] = bw;
  ctx->tune_bps[pi][bi] = bb;
  if (s) return s;
  if (n_band_max >= 512) bw = n_band_max / 256;   // warps of the block shape
  if (best_out) { best_out[0] = bw; best_out[1] = bb; }
  return GBK_OK;
}
