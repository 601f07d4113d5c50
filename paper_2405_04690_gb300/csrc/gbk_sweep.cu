// Ensemble sweep of the GB sampler: band windows, in-model + flip-all RJ per band
// (Alg. 1, App. C), ensemble-permuted tempering swaps (Alg. 2, Eq. temp-final).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "gbk_internal.cuh"
#include "gbk_mix.cuh"
#include "gbk_philox.cuh"
#include "gbk_reduce.cuh"
#include "gbk_wave.cuh"

struct gbk_sweep {
  gbk_ctx* ctx;
  gbk_sweep_desc d;
  int n_bp_max;         // bands of the larger parity
  long long* rsnap;     // residual snapshot [W][2][n_bins][2]
  void* rho;            // opened windows [W][n_bp_max][2][3N], complex of the sweep precision
  void* wcache;         // current waveform of every slot [T][W][B][n_max][2][N]
  void* hsum;           // sum of the present templates of every band on its window [T][W][B][2][3N]
  int32_t* setid;       // cache block of band (t, w, b) [T][W][B]; tempering swaps exchange ids
  void* rwbuf;          // band windows of the band kernel's warps [SMs x 64][3N][2]
  size_t rwbuf_bytes;
  size_t rho_bytes, cache_bytes, hsum_bytes;
  cudaEvent_t ev[2][4][2];  // [parity][refresh, open, band, swap][begin, end] when timing
  bool timed, have_ev;
  bool refreshed;           // the caches have been filled (a gb_sweep with GBK_SWEEP_REFRESH ran)
  // learned proposal (gbk_sweep_set_proposal)
  bool mdn_set;
  gbk_mdn* net;             // network run on each half sweep's opened windows, or
  const float* raw_table;   // fixed mixture outputs [W][B][272]
  double mdn_eps, mdn_inmodel;
  uint16_t* xfeat;          // BF16 features [W][n_bp_max][1024]
  float* rawbuf;            // network outputs [W][n_bp_max][272]
  void* mix;                // mixture rows [W][n_bp_max] (MixRow of the sweep precision)
  // group stretch (gbk_sweep_update_group): stationary group of every band, sorted by f0
  double* grp_f0;           // [B][gmax]
  double* grp_par;          // [B][gmax][8]
  int32_t* grp_n;           // [B]
  int gmax;
  double grp_frac;
  int n_friends;
  int32_t* swap_acc;        // accepted swaps of the last sweep per band and rung [B][T]
  int32_t* xfer_dest;       // ownership transfer: destination (band n_max + slot) of every cold slot, or -1
  unsigned long long* task_ctr;   // next band task of the band kernel, one counter per parity
};

namespace gbk {

constexpr int kSwWarps = 4;
// band kernel: 4 warps per CTA, 3 CTAs per SM (15 KB of shared memory per warp, 168
// registers per thread). Capping registers for 14 warps per SM spilled and ran 6 % slower.
constexpr int kBandWarps = 4, kBandMinCtas = 3;
constexpr int kSwapMinCtas = 5;
constexpr int kMaxSlots = 64;

struct SweepArgs {
  gbk_ctx c;
  gbk_sweep_desc d;
  double* params;
  uint8_t* exists;
  const double* betas;
  long long* resid;       // live cold-chain residual (updated)
  const long long* rsnap; // snapshot taken at the start of the half sweep
  void* rho;
  void* wcache;
  void* hsum;
  int32_t* setid;
  int n_bp_max;
  int32_t n_walkers_r;
  int32_t frac_bits;
  const double* psdp;
  int32_t npsd;
  uint32_t k0, k1, sweep;
  int parity;
  gbk_trace_rec* trace;
  int32_t trace_cap;
  int32_t* trace_count;
  long long* stats;
  // band windows r' of the band kernel's warps (global, L1-cached): [warps][3N][2]
  void* rwbuf;
  // learned proposal: mixture row of every opened (walker, band) or NULL
  const void* mix;
  double mdn_eps, mdn_inmodel;
  // group stretch: stationary group (NULL when off)
  const double* grp_f0;
  const double* grp_par;
  const int32_t* grp_n;
  int gmax, n_friends;
  double grp_frac;
  int32_t* swap_acc;      // [B][T] accepted swaps between rungs t-1 and t
  unsigned long long* task_ctr;   // [2] next band task of the band kernel (zeroed before each launch)
};

template <typename T> __device__ __forceinline__ const T* orb_of(const gbk_ctx& c, int bi);
template <> __device__ __forceinline__ const float* orb_of<float>(const gbk_ctx& c, int bi) { return c.orb_f[bi]; }
template <> __device__ __forceinline__ const double* orb_of<double>(const gbk_ctx& c, int bi) { return c.orb_d[bi]; }
template <typename T> __device__ __forceinline__ const typename CT<T>::C* tw_of(const gbk_ctx& c, int bi);
template <> __device__ __forceinline__ const float2* tw_of<float>(const gbk_ctx& c, int bi) { return c.tw_f[bi]; }
template <> __device__ __forceinline__ const double2* tw_of<double>(const gbk_ctx& c, int bi) { return c.tw_d[bi]; }
__device__ __forceinline__ float iqv(const gbk_ctx& c, int64_t k, float) { return __ldg(&c.iq_f[k]); }
__device__ __forceinline__ double iqv(const gbk_ctx& c, int64_t k, double) { return __ldg(&c.iq_d[k]); }
__device__ __forceinline__ float rhov(const gbk_ctx& c, int64_t k, float) { return __ldg(&c.rho_f[k]); }
__device__ __forceinline__ double rhov(const gbk_ctx& c, int64_t k, double) { return __ldg(&c.rho_d[k]); }
__device__ __forceinline__ const float* tab_iq(const gbk_ctx& c, float) { return c.iq_f; }
__device__ __forceinline__ const double* tab_iq(const gbk_ctx& c, double) { return c.iq_d; }
__device__ __forceinline__ const float* tab_rho(const gbk_ctx& c, float) { return c.rho_f; }
__device__ __forceinline__ const double* tab_rho(const gbk_ctx& c, double) { return c.rho_d; }
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float i2t(long long v, float) { return ll_to_float(v); }
__device__ __forceinline__ double i2t(long long v, double) { return __ll2double_rn(v); }
__device__ __forceinline__ long long t2grid(float v, float s) { return float_to_ll(v * s); }
__device__ __forceinline__ long long t2grid(double v, double s) { return __double2ll_rn(v * s); }
template <typename T> struct SAcc;
template <> struct SAcc<float> { typedef CompF S; };
template <> struct SAcc<double> { typedef PlainD S; };

__device__ __forceinline__ double nan_d() { return __longlong_as_double(0x7ff8000000000000LL); }

// -------------------------------------------------------------- prior and proposals
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

__device__ __forceinline__ void allowance(const gbk_sweep_desc& d, double tobs, int b, double& lo, double& hi) {
  const long long lob = d.band_k0 + (long long)b * d.band_bins;
  const long long hib = lob + d.band_bins;
  const double half = 0.5 * d.band_bins;
  lo = __ddiv_rn(dsub((double)lob, half), tobs);
  hi = __ddiv_rn(dadd((double)hib, half), tobs);
  if (lo < d.f_min) lo = d.f_min;
  if (hi > d.f_max) hi = d.f_max;
}

// f0 range [lo, hi) of band b's sources, computed once per band task.
struct BandGeom {
  double lo, hi, inv_span;
};
__device__ __forceinline__ BandGeom band_geom(const gbk_sweep_desc& d, double tobs, int b) {
  BandGeom g;
  allowance(d, tobs, b, g.lo, g.hi);
  g.inv_span = 1.0 / (g.hi - g.lo);
  return g;
}

// Prior support of a source of band b (lo <= f0 < hi over the band's allowance;
// A_min <= A <= A_max; |cos i|, |sin b| <= 1; chirp mass in [mc_min, mc_max] written as
// c_lo f0^(11/3) <= fdot <= c_hi f0^(11/3) with c = 96/5 pi^(8/3) (mc G M_sun / c^3)^(5/3)).
struct PriorK {
  double a_min, a_max, c_lo, c_hi;
  float inv_lna, inv_mc;   // 1 / (ln A_max - ln A_min), 1 / (Mc_max - Mc_min)
};
constexpr double kKChirp = 96.0 / 5.0 * 21.170591578193026;   // 96/5 pi^(8/3)
constexpr double kGmSun = 4.925490947e-6;                       // G M_sun / c^3 [s]
__device__ __forceinline__ PriorK prior_consts(const gbk_sweep_desc& d) {
  PriorK p;
  p.a_min = exp(d.ln_a_min);
  p.a_max = exp(d.ln_a_max);
  p.c_lo = kKChirp * pow(d.mc_min * kGmSun, 5.0 / 3.0);
  p.c_hi = kKChirp * pow(d.mc_max * kGmSun, 5.0 / 3.0);
  p.inv_lna = (float)(1.0 / (d.ln_a_max - d.ln_a_min));
  p.inv_mc = (float)(1.0 / (d.mc_max - d.mc_min));
  return p;
}

// f0^(11/3): float64 pow for the float64 sweep; in the mixed sweep exp/log in float32
// (relative error ~1e-6, which moves the chirp-mass bounds by as much).
__device__ __forceinline__ double f0_113(double f0, double) { return pow(f0, 11.0 / 3.0); }
__device__ __forceinline__ double f0_113(double f0, float) {
  return (double)expf((float)(11.0 / 3.0) * logf((float)f0));
}

template <typename T>
__device__ __forceinline__ bool in_support(const PriorK& pk, const BandGeom& bg, const double* th) {
  if (!(th[1] >= bg.lo && th[1] < bg.hi)) return false;
  if (!(th[0] >= pk.a_min && th[0] <= pk.a_max)) return false;
  if (!(th[5] >= -1.0 && th[5] <= 1.0 && th[6] >= -1.0 && th[6] <= 1.0)) return false;
  const double f113 = f0_113(th[1], T());
  return th[2] >= dmul(pk.c_lo, f113) && th[2] <= dmul(pk.c_hi, f113);
}

// ln p(theta') - ln p(theta) of the non-uniform prior factor p(fdot | f0) ~ fdot^-2/5 f0^-11/5,
// from logarithms of ratios (precision of the sweep's arithmetic type).
__device__ __forceinline__ double dlog_prior(const double* nw, const double* th, float) {
  return (double)(-0.4f * logf((float)(nw[2] / th[2])) - 2.2f * logf((float)(nw[1] / th[1])));
}
__device__ __forceinline__ double dlog_prior(const double* nw, const double* th, double) {
  return dsub(dmul(-0.4, log(nw[2] / th[2])), dmul(2.2, log(nw[1] / th[1])));
}
__device__ __forceinline__ double log_u(double u, float) { return u > 0.0 ? (double)logf((float)u) : -INFINITY; }
__device__ __forceinline__ double log_u(double u, double) { return u > 0.0 ? log(u) : -INFINITY; }

__device__ __forceinline__ double wrap(double x, double period) {
  if (x >= period) return dsub(x, period);
  if (x < 0.0) return dadd(x, period);
  return x;
}

// In-model proposal from the 48 words of proposal j (word 0 picks the source). The
// float64 sweep computes every step in float64; the mixed sweep forms the steps
// sigma_c z_c (and the amplitude factor exp(sigma_A z)) in float32 and adds them in
// float64, so the move stays symmetric (rounding to nearest is odd-symmetric).
__device__ __forceinline__ void propose(const gbk_sweep_desc& d, const double* th, const uint32_t* w, double* nw,
                                        double) {
  double z[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const double s4 = dadd(dadd(dadd(u24(w[1 + 4 * c]), u24(w[2 + 4 * c])), u24(w[3 + 4 * c])), u24(w[4 + 4 * c]));
    z[c] = dmul(dsub(s4, 2.0), 1.7320508075688772);
  }
  const double TWO_PI = 6.283185307179586, PI = 3.141592653589793;
  nw[0] = dmul(th[0], exp(dmul(d.sigma[0], z[0])));
  nw[1] = dadd(th[1], dmul(d.sigma[1], z[1]));
  nw[2] = dadd(th[2], dmul(d.sigma[2], z[2]));
  nw[3] = wrap(dadd(th[3], dmul(d.sigma[3], z[3])), TWO_PI);
  nw[4] = wrap(dadd(th[4], dmul(d.sigma[4], z[4])), PI);
  nw[5] = dadd(th[5], dmul(d.sigma[5], z[5]));
  nw[6] = dadd(th[6], dmul(d.sigma[6], z[6]));
  nw[7] = wrap(dadd(th[7], dmul(d.sigma[7], z[7])), TWO_PI);
}
__device__ __forceinline__ void propose(const gbk_sweep_desc& d, const double* th, const uint32_t* w, double* nw,
                                        float) {
  float z[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {   // (sum of four 24-bit uniforms - 2) sqrt3, centred in integers first
    const int ic = (int)((w[1 + 4 * c] >> 8) + (w[2 + 4 * c] >> 8) + (w[3 + 4 * c] >> 8) + (w[4 + 4 * c] >> 8)) -
                   (1 << 25);
    z[c] = (float)ic * (float)(1.7320508075688772 / 16777216.0);
  }
  const double TWO_PI = 6.283185307179586, PI = 3.141592653589793;
  // A' = A e^x, x = sigma_A z formed in float32 as above; e^x = 1 + expm1f(x) keeps the float64
  // precision of A' (|expm1f error| ~1e-7 |x|, |x| ~ 0.05: |Delta lnL| scales with A^2) with
  // one float64 fma in place of a float64 exp
  nw[0] = fma(th[0], (double)expm1f((float)d.sigma[0] * z[0]), th[0]);
  nw[1] = th[1] + (double)((float)d.sigma[1] * z[1]);
  nw[2] = th[2] + (double)((float)d.sigma[2] * z[2]);
  nw[3] = wrap(th[3] + (double)((float)d.sigma[3] * z[3]), TWO_PI);
  nw[4] = wrap(th[4] + (double)((float)d.sigma[4] * z[4]), PI);
  nw[5] = th[5] + (double)((float)d.sigma[5] * z[5]);
  nw[6] = th[6] + (double)((float)d.sigma[6] * z[6]);
  nw[7] = wrap(th[7] + (double)((float)d.sigma[7] * z[7]), TWO_PI);
}

// fdot = K f0^(11/3) (Mc G M_sun)^(5/3): float64 pow, or float32 exp/log (~1e-6 relative).
__device__ __forceinline__ double fdot_of(double f0, double mc, double) {
  return kKChirp * pow(f0, 11.0 / 3.0) * pow(mc * kGmSun, 5.0 / 3.0);
}
__device__ __forceinline__ double fdot_of(double f0, double mc, float) {
  const float l = (float)(11.0 / 3.0) * logf((float)f0) + (float)(5.0 / 3.0) * logf((float)(mc * kGmSun));
  return kKChirp * (double)expf(l);
}
// chirp mass of (f0, fdot)
__device__ __forceinline__ double mc_of(double f0, double fdot, double) {
  return pow(fdot / (kKChirp * pow(f0, 11.0 / 3.0)), 0.6) / kGmSun;
}
__device__ __forceinline__ double mc_of(double f0, double fdot, float) {
  const float l = 0.6f * (logf((float)(fdot / kKChirp)) - (float)(11.0 / 3.0) * logf((float)f0));
  return (double)expf(l) * (1.0 / kGmSun);
}
__device__ __forceinline__ double exp_t(double x, double) { return exp(x); }
__device__ __forceinline__ double exp_t(double x, float) { return (double)expf((float)x); }
__device__ __forceinline__ double log_t(double x, double) { return log(x); }
__device__ __forceinline__ double log_t(double x, float) { return (double)logf((float)x); }

// Amplitude of a prior draw, A = exp(ln A_min + (ln A_max - ln A_min) u): the float64 sweep in
// float64; the mixed sweep as A_min (float64) times expf of the float32 offset (relative error
// ~1e-7: a fixed map of u, which the stored parameters and the template then both follow).
__device__ __forceinline__ double prior_amp(const gbk_sweep_desc& d, const PriorK&, double u, double) {
  return exp(dadd(d.ln_a_min, dmul(dsub(d.ln_a_max, d.ln_a_min), u)));
}
__device__ __forceinline__ double prior_amp(const gbk_sweep_desc& d, const PriorK& pk, double u, float) {
  return pk.a_min * (double)expf((float)(d.ln_a_max - d.ln_a_min) * (float)u);
}

// Prior draw of a new source in band b from 8 words (f0 always in float64: the likelihood of a
// loud source is sensitive to it at the 1e-7 level).
template <typename T>
__device__ __forceinline__ void draw_birth(const gbk_sweep_desc& d, const PriorK& pk, const BandGeom& bg,
                                           const uint32_t* w, double* nw) {
  const double TWO_PI = 6.283185307179586, PI = 3.141592653589793;
  const double f0 = dadd(bg.lo, dmul(dsub(bg.hi, bg.lo), u32(w[0])));
  nw[1] = f0;
  nw[0] = prior_amp(d, pk, u32(w[1]), T());
  const double mc = dadd(d.mc_min, dmul(dsub(d.mc_max, d.mc_min), u32(w[2])));
  nw[2] = fdot_of(f0, mc, T());
  nw[3] = dmul(TWO_PI, u32(w[3]));
  nw[4] = dmul(PI, u32(w[4]));
  nw[5] = dsub(dmul(2.0, u32(w[5])), 1.0);
  nw[6] = dsub(dmul(2.0, u32(w[6])), 1.0);
  nw[7] = dmul(TWO_PI, u32(w[7]));
}

// Unit-box coordinates of band b, where the prior is uniform (the learned proposal's
// space): ln A, f0 over the allowance, chirp mass, phi0 / 2pi, psi / pi, (cos i + 1) / 2,
// (sin beta + 1) / 2, lambda / 2pi. The f0 coordinate is always formed in float64.
template <typename T>
__device__ __forceinline__ void to_unit(const gbk_sweep_desc& d, const PriorK&, const BandGeom& bg, const double* th,
                                       double* u) {
  const double mc = mc_of(th[1], th[2], T());
  u[0] = (log_t(th[0], T()) - d.ln_a_min) / (d.ln_a_max - d.ln_a_min);
  u[1] = (th[1] - bg.lo) / (bg.hi - bg.lo);
  u[2] = (mc - d.mc_min) / (d.mc_max - d.mc_min);
  u[3] = th[3] / 6.283185307179586;
  u[4] = th[4] / 3.141592653589793;
  u[5] = (th[5] + 1.0) / 2.0;
  u[6] = (th[6] + 1.0) / 2.0;
  u[7] = th[7] / 6.283185307179586;
}
// Mixed sweep: float32 except the f0 coordinate (float64 difference times 1 / span).
template <>
__device__ __forceinline__ void to_unit<float>(const gbk_sweep_desc& d, const PriorK& pk, const BandGeom& bg,
                                              const double* th, double* u) {
  const float mc = (float)mc_of(th[1], th[2], float());
  u[0] = (double)((logf((float)th[0]) - (float)d.ln_a_min) * pk.inv_lna);
  u[1] = (th[1] - bg.lo) * bg.inv_span;
  u[2] = (double)((mc - (float)d.mc_min) * pk.inv_mc);
  u[3] = (double)((float)th[3] * 0.15915494f);
  u[4] = (double)((float)th[4] * 0.31830989f);
  u[5] = (double)(((float)th[5] + 1.0f) * 0.5f);
  u[6] = (double)(((float)th[6] + 1.0f) * 0.5f);
  u[7] = (double)((float)th[7] * 0.15915494f);
}
template <typename T>
__device__ __forceinline__ void from_unit(const gbk_sweep_desc& d, const BandGeom& bg, const double* u, double* nw) {
  const double f0 = bg.lo + (bg.hi - bg.lo) * u[1];
  const double mc = d.mc_min + (d.mc_max - d.mc_min) * u[2];
  nw[0] = exp_t(d.ln_a_min + (d.ln_a_max - d.ln_a_min) * u[0], T());
  nw[1] = f0;
  nw[2] = fdot_of(f0, mc, T());
  nw[3] = 6.283185307179586 * u[3];
  nw[4] = 3.141592653589793 * u[4];
  nw[5] = 2.0 * u[5] - 1.0;
  nw[6] = 2.0 * u[6] - 1.0;
  nw[7] = 6.283185307179586 * u[7];
}

// Draw from eps prior + (1 - eps) mixture: the prior branch is draw_birth on the same 8 words.
template <typename T>
__device__ __forceinline__ void mdn_draw(const SweepArgs& a, const PriorK& pk, const MixRow<T>& m, const BandGeom& bg,
                                         uint32_t w_def, uint32_t w_comp, const uint32_t* w_dims, double* nw) {
  if (mix_u32(w_def) < a.mdn_eps) {
    draw_birth<T>(a.d, pk, bg, w_dims, nw);
    return;
  }
  T u[kMixDim];
  mix_draw<T>(m, w_comp, w_dims, u);
  double ud[kMixDim];
#pragma unroll
  for (int c = 0; c < kMixDim; ++c) ud[c] = (double)u[c];
  from_unit<T>(a.d, bg, ud, nw);
}
template <typename T>
__device__ __forceinline__ double mdn_logq(const SweepArgs& a, const PriorK& pk, const MixRow<T>& m,
                                           const BandGeom& bg, const double* th) {
  double ud[kMixDim];
  to_unit<T>(a.d, pk, bg, th, ud);
  T u[kMixDim];
#pragma unroll
  for (int c = 0; c < kMixDim; ++c) u[c] = (T)ud[c];
  return (double)mix_logq<T>(m, u, (T)a.mdn_eps);
}

// -------------------------------------------------------------- group stretch
// Start of the window of the nf stationary-group members nearest in f0 to f (fs sorted, G
// members, nf <= G): lower bound, then nf steps taking the nearer side (ties to the lower).
__device__ __forceinline__ int friends_start(const double* fs, int G, double f, int nf) {
  int lo = 0, hi = G;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (fs[mid] < f) lo = mid + 1; else hi = mid;
  }
  int l = lo - 1, h = lo;
  for (int i = 0; i < nf; ++i) {
    if (h >= G || (l >= 0 && f - fs[l] <= fs[h] - f)) --l; else ++h;
  }
  return l + 1;
}
__device__ __forceinline__ double wrap_sym(double d, double period) {
  if (d >= 0.5 * period) return d - period;
  if (d < -0.5 * period) return d + period;
  return d;
}
// Stretch move Y = X_j + z (X - X_j) (Eq. stretch) with X_j one of the nf nearest members of
// band b's stationary group, in the coordinates (ln A, f0, fdot, phi0, psi, cos i, sin b,
// lambda), periodic differences in [-P/2, P/2). Returns ln z, or NaN when the move is not
// reversible as drawn (a stretched periodic difference leaves [-P/2, P/2), or X_j is not
// among the nf nearest members of Y).
__device__ __noinline__ double group_stretch(const SweepArgs& a, int b, const double* th, uint32_t w_j, uint32_t w_z,
                                             double* nw) {
  const double* fs = a.grp_f0 + (int64_t)b * a.gmax;
  const double* gp = a.grp_par + (int64_t)b * a.gmax * 8;
  const int G = a.grp_n[b];
  const int nf = a.n_friends < G ? a.n_friends : G;
  const int j = friends_start(fs, G, th[1], nf) + (int)ranged(w_j, (uint32_t)nf);
  const double* xj = gp + (int64_t)j * 8;
  const double sa = 2.0;   // stretch scale a
  const double zz = (sa - 1.0) * u32(w_z) + 1.0;
  const double z = zz * zz / sa;
  const double TWO_PI = 6.283185307179586, PI = 3.141592653589793;
  bool ok = true;
  const double lx = log(th[0]), lj = log(xj[0]);
  nw[0] = exp(lj + z * (lx - lj));
  nw[1] = xj[1] + z * (th[1] - xj[1]);
  nw[2] = xj[2] + z * (th[2] - xj[2]);
  nw[5] = xj[5] + z * (th[5] - xj[5]);
  nw[6] = xj[6] + z * (th[6] - xj[6]);
  const int pc[3] = {3, 4, 7};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int c = pc[q];
    const double per = c == 4 ? PI : TWO_PI;
    const double dlt = z * wrap_sym(th[c] - xj[c], per);
    if (!(dlt >= -0.5 * per && dlt < 0.5 * per)) ok = false;
    nw[c] = wrap(xj[c] + dlt, per);
  }
  if (ok) {
    const int s1 = friends_start(fs, G, nw[1], nf);
    ok = s1 <= j && j < s1 + nf;
  }
  return ok ? log(z) : nan_d();
}

// Lanes compute Philox blocks c0 = base + m (m < nblk) into words[4m .. 4m+3].
__device__ __forceinline__ void fill_words(uint32_t* words, int nblk, uint32_t base, uint32_t c1, uint32_t c2,
                                           uint32_t c3, uint32_t k0, uint32_t k1, int lane) {
  for (int m = lane; m < nblk; m += 32) {
    const U4 v = philox4x32_10(base + m, c1, c2, c3, k0, k1);
    words[4 * m] = v.x; words[4 * m + 1] = v.y; words[4 * m + 2] = v.z; words[4 * m + 3] = v.w;
  }
  __syncwarp();
}

// Move statistics are counted per warp (lane 0) and added to the global counters once
// per kernel: same-address atomics from every proposal would serialise in L2.
struct WarpStats {
  unsigned long long c[10];  // rows 0-3 (proposed, accepted) per kind, row 4 (waveforms, evaluations)
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int i = 0; i < 10; ++i) c[i] = 0ull;
  }
  __device__ __forceinline__ void flush(const long long* stats) {
    if (!stats) return;
#pragma unroll
    for (int i = 0; i < 10; ++i)
      if (c[i]) atomicAdd((unsigned long long*)&stats[i], c[i]);
  }
};

__device__ __forceinline__ void record(const SweepArgs& a, WarpStats& ws, int kind, int t, int w, int b, int slot,
                                       int seq, bool acc, double dll, double la, const double* th, int wf, int ev) {
  ws.c[2 * kind] += 1ull;
  if (acc) ws.c[2 * kind + 1] += 1ull;
  ws.c[8] += (unsigned long long)wf;
  ws.c[9] += (unsigned long long)ev;
  if (a.trace_count) {
    const int i = atomicAdd(a.trace_count, 1);
    if (a.trace && i < a.trace_cap) {
      gbk_trace_rec& r = a.trace[i];
      r.kind = kind; r.t = t; r.w = w; r.b = b; r.slot = slot; r.seq = seq; r.accepted = acc ? 1 : 0;
      r.parity = a.parity; r.dlogl = dll; r.log_alpha = la;
      for (int c = 0; c < 8; ++c) r.params[c] = th ? th[c] : 0.0;
    }
  }
}

// -------------------------------------------------------------- band-window pieces
template <typename T>
struct PsdWt {
  double cw;
  T aw;
};
template <typename T>
__device__ __forceinline__ PsdWt<T> walker_psd(const SweepArgs& a, int w) {
  const int j = (a.npsd == 1) ? 0 : w;
  const double so = a.psdp[2 * j] * a.psdp[2 * j], sa = a.psdp[2 * j + 1] * a.psdp[2 * j + 1];
  PsdWt<T> r;
  r.cw = 4.0 / a.c.grid.tobs / so;
  r.aw = (T)(sa / so);
  return r;
}

__device__ __forceinline__ int64_t slot_index(const gbk_sweep_desc& d, int t, int w, int b) {
  return (((int64_t)t * d.n_walkers + w) * d.n_bands + b) * d.n_max;
}
// The waveform and set-sum caches of band (t, w, b) live in block setid[t][w][b]; a
// tempering swap exchanges the two blocks' ids instead of copying their contents.
__device__ __forceinline__ int64_t cache_base(const SweepArgs& a, int t, int w, int b) {
  return (int64_t)a.setid[((int64_t)t * a.d.n_walkers + w) * a.d.n_bands + b] * a.d.n_max;
}
template <typename T>
__device__ __forceinline__ typename CT<T>::C* cache_ptr(const SweepArgs& a, int64_t cslot) {
  return reinterpret_cast<typename CT<T>::C*>(a.wcache) + cslot * 2 * a.d.band_bins;
}
template <typename T>
__device__ __forceinline__ typename CT<T>::C* hsum_ptr(const SweepArgs& a, int t, int w, int b) {
  return reinterpret_cast<typename CT<T>::C*>(a.hsum) +
         (int64_t)a.setid[((int64_t)t * a.d.n_walkers + w) * a.d.n_bands + b] * 2 * 3 * a.d.band_bins;
}
template <typename T>
__device__ __forceinline__ const MixRow<T>* mix_ptr(const SweepArgs& a, int w, int j) {
  return a.mix ? reinterpret_cast<const MixRow<T>*>(a.mix) + ((int64_t)w * a.n_bp_max + j) : nullptr;
}
template <typename T>
__device__ __forceinline__ typename CT<T>::C* rho_ptr(const SweepArgs& a, int w, int j) {
  typedef typename CT<T>::C C;
  return reinterpret_cast<C*>(a.rho) + ((int64_t)w * a.n_bp_max + j) * 2 * 3 * a.d.band_bins;
}
// window offset of a template's band: bins [q - N/2, q + N/2) relative to window start gw
template <int N>
__device__ __forceinline__ int band_off(long long q, int64_t gw, const gbk_ctx& c) {
  return (int)(q - N / 2 - (gw + c.grid.k0));
}
// window offset of a cached template (its q from its f0)
template <int N>
__device__ __forceinline__ int cached_off(const double* th, int64_t gw, const gbk_ctx& c) {
  return band_off<N>((long long)floor(th[1] * c.grid.tobs), gw, c);
}

__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// The band kernel's window keeps both channels of a bin together ([3N][A, E]) and the PSD
// tables' (iq, rho) pairs are read together: per evaluated bin one 16-byte window load and one
// 8-byte table load in float32 where there were four loads (band kernel -5 %: its evaluations
// wait on load latency). The search sampler's windows, read by 128 chains each, keep [2][3N]
// with separate table loads: interleaved, its sweep took 16 % longer; so did the swap kernel's
// pass with the paired table loads (+9 %).
__device__ __forceinline__ void ld_win(const float2* p, float2& x, float2& y) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  x = make_float2(v.x, v.y);
  y = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld_win(const double2* p, double2& x, double2& y) { x = p[0]; y = p[1]; }
__device__ __forceinline__ void st_win(float2* p, float2 x, float2 y) {
  *reinterpret_cast<float4*>(p) = make_float4(x.x, x.y, y.x, y.y);
}
__device__ __forceinline__ void st_win(double2* p, double2 x, double2 y) { p[0] = x; p[1] = y; }
// (iq, rho) of bin k: one 8-byte load in float32
__device__ __forceinline__ float2 iqrho(const gbk_ctx& c, int64_t k, float) { return __ldg(&c.iqrho_f[k]); }
__device__ __forceinline__ double2 iqrho(const gbk_ctx& c, int64_t k, double) { return make_double2(__ldg(&c.iq_d[k]), __ldg(&c.rho_d[k])); }

// Delta lnL of swapping template r (br, window offset orr) for a (ba, offset oa) against
// the window residual rw: [3N][2] if IL (the band kernel's window), [2][3N] otherwise; either
// template may be absent. Window bin i is grid bin gw + i.
template <typename T, int N, bool IL>
__device__ __noinline__ double window_dll(const SweepArgs& a, const typename CT<T>::C* rw, const typename CT<T>::C* ba, int oa,
                             const typename CT<T>::C* br, int orr, int64_t gw, const PsdWt<T>& pw, int lane) {
  typedef typename CT<T>::C C;
  constexpr int W3 = 3 * N;
  typename SAcc<T>::S sdd, srd;
  sdd.init();
  srd.init();
  {   // the lines this evaluation reads (window, old template, PSD tables) towards L1: their
      // loads then meet L1 instead of L2 in the latency-bound loops below
    const int o0 = ba ? oa : orr;
    constexpr int kPer = 128 / (int)sizeof(C);          // complex bins per 128-byte line
    if (IL) {   // N bins of both channels: 2N complex values from bin o0 on
      const int nl = (2 * N + kPer - 1) / kPer + 1;
      for (int i = lane; i < nl; i += 32) {
        const int idx = ((2 * o0) & ~(kPer - 1)) + i * kPer;
        if (idx < 2 * W3) prefetch_l1(rw + idx);
      }
    } else {
      const int nl = (N + kPer - 1) / kPer + 1;           // lines of N bins (unaligned start)
      for (int i = lane; i < 2 * nl; i += 32) {
        const int ch = i / nl, li = i % nl;
        const int idx = (o0 & ~(kPer - 1)) + li * kPer;      // stays inside this warp's window
        if (idx < W3) prefetch_l1(rw + ch * W3 + idx);
      }
    }
    constexpr int nt = N / kPer;                          // lines of one channel of a template
    if (br)
      for (int i = lane; i < 2 * nt; i += 32) prefetch_l1(br + i * kPer);
    if (IL && sizeof(T) == 4) {   // lines of the (iq, rho) pairs of the evaluated bins
      constexpr int kT = 128 / 8;
      const int64_t k0 = (gw + o0) & ~(int64_t)(kT - 1);
      constexpr int nq = N / kT + 1;
      const int64_t kend = a.c.grid.n_bins;
      for (int i = lane; i < nq; i += 32) {
        const int64_t k = k0 + (int64_t)kT * i;
        if (k < kend) prefetch_l1(a.c.iqrho_f + k);
      }
    } else {   // PSD-table lines of the evaluated bins
      constexpr int kT = 128 / (int)sizeof(T);           // table entries per line
      const int64_t k0 = (gw + o0) & ~(int64_t)(kT - 1);
      constexpr int nq = N / kT + 1;
      const int64_t kend = a.c.grid.n_bins;
      const T* iq = tab_iq(a.c, T());
      const T* rh = tab_rho(a.c, T());
      for (int i = lane; i < 2 * nq; i += 32) {
        const int64_t k = k0 + (int64_t)kT * (i % nq);
        if (k < kend) prefetch_l1(i < nq ? iq + k : rh + k);
      }
    }
  }
  auto bin = [&](int i, C da, C de) {
    const int64_t k = gw + i;
    T wt;
    if (IL) {
      const C q = iqrho(a.c, k, T());
      wt = q.x * recip((T)1 + pw.aw * q.y);
    } else {
      wt = iqv(a.c, k, T()) * recip((T)1 + pw.aw * rhov(a.c, k, T()));
    }
    C ra, re;
    if (IL) {
      ld_win(rw + 2 * i, ra, re);
    } else {
      ra = rw[i];
      re = rw[W3 + i];
    }
    sdd.add(wt * (da.x * da.x + da.y * da.y + de.x * de.x + de.y * de.y));
    srd.add(wt * (ra.x * da.x + ra.y * da.y + re.x * de.x + re.y * de.y));
  };
  if (ba) {
    for (int j = lane; j < N; j += 32) {
      const int i = oa + j;
      C xa = ba[j], xe = ba[N + j];
      const int jr = i - orr;
      if (br && jr >= 0 && jr < N) { xa = csub(xa, br[jr]); xe = csub(xe, br[N + jr]); }
      bin(i, xa, xe);
    }
  }
  if (br) {
    for (int j = lane; j < N; j += 32) {
      const int i = orr + j;
      const int ja = i - oa;
      if (ba && ja >= 0 && ja < N) continue;
      const C xa = br[j], xe = br[N + j];
      bin(i, mkc(-xa.x, -xa.y), mkc(-xe.x, -xe.y));
    }
  }
  const double dd = sdd.warp_total();
  const double rd = srd.warp_total();
  return pw.cw * (-0.5 * dd + rd);
}

// r' <- r' - a + r over the window; for the cold chain also R <- R - round(a) + round(r).
template <typename T, int N>
__device__ __noinline__ void apply_change(const SweepArgs& a, typename CT<T>::C* rw, const typename CT<T>::C* ba, int oa,
                             const typename CT<T>::C* br, int orr, bool cold, long long* rglob, int64_t gw, T gs,
                             int lane) {
  typedef typename CT<T>::C C;
  const int64_t nb = a.c.grid.n_bins;
  if (ba) {
    for (int j = lane; j < N; j += 32) {
      C x, y;
      ld_win(rw + 2 * (oa + j), x, y);
      st_win(rw + 2 * (oa + j), csub(x, ba[j]), csub(y, ba[N + j]));
    }
    __syncwarp();
  }
  if (br) {
    for (int j = lane; j < N; j += 32) {
      C x, y;
      ld_win(rw + 2 * (orr + j), x, y);
      st_win(rw + 2 * (orr + j), cadd(x, br[j]), cadd(y, br[N + j]));
    }
    __syncwarp();
  }
  if (cold) {
    unsigned long long* R = reinterpret_cast<unsigned long long*>(rglob);
    for (int j = lane; j < N; j += 32) {
      for (int ch = 0; ch < 2; ++ch) {
        if (ba) {
          const typename CT<T>::C h = ba[ch * N + j];
          unsigned long long* dst = R + 2 * (ch * nb + gw + oa + j);
          atomicAdd(dst, (unsigned long long)(-t2grid(h.x, gs)));
          atomicAdd(dst + 1, (unsigned long long)(-t2grid(h.y, gs)));
        }
        if (br) {
          const typename CT<T>::C h = br[ch * N + j];
          unsigned long long* dst = R + 2 * (ch * nb + gw + orr + j);
          atomicAdd(dst, (unsigned long long)t2grid(h.x, gs));
          atomicAdd(dst + 1, (unsigned long long)t2grid(h.y, gs));
        }
      }
    }
  }
}

template <typename C>
__device__ __forceinline__ void copy_band(C* dst, const C* src, int n2, int lane) {
  for (int i = lane; i < n2; i += 32) dst[i] = src[i];
}

// H(t, w, b) <- sum of the band's present cached templates on its window, summed in slot
// order (deterministic), written to global memory. Templates and sums pass through once
// (evict-first loads and stores).
template <typename T, int N>
__device__ __noinline__ void write_hsum(const SweepArgs& a, int t, int w, int b, int lane) {
  typedef typename CT<T>::C C;
  constexpr int W3 = 3 * N;
  const gbk_sweep_desc& d = a.d;
  C* H = hsum_ptr<T>(a, t, w, b);
  const int64_t gw = d.band_k0 + (int64_t)(b - 1) * N - a.c.grid.k0;
  const int64_t base = slot_index(d, t, w, b);
  const int64_t cb = cache_base(a, t, w, b);
  // lane-parallel offsets of the present slots (slot lane and slot lane + 32)
  int off0 = -1, off1 = -1;
  if (lane < d.n_max && a.exists[base + lane]) off0 = cached_off<N>(a.params + (base + lane) * 8, gw, a.c);
  if (lane + 32 < d.n_max && a.exists[base + lane + 32]) off1 = cached_off<N>(a.params + (base + lane + 32) * 8, gw, a.c);
  const unsigned p0 = __ballot_sync(0xffffffffu, off0 >= 0);
  const unsigned p1 = __ballot_sync(0xffffffffu, off1 >= 0);
  // G window bins per lane at a time: for each slot (in slot order) the loads of all G bins
  // are issued together, then added
  constexpr int G = 4;
#pragma unroll 1
  for (int i0 = lane; i0 < W3; i0 += 32 * G) {
    C xa[G], xe[G];
#pragma unroll
    for (int u = 0; u < G; ++u) xa[u] = xe[u] = mkc((T)0, (T)0);
    for (int half = 0; half < 2; ++half) {
      for (unsigned m = half ? p1 : p0; m; m &= m - 1) {
        const int sl = __ffs(m) - 1;
        const int o = __shfl_sync(0xffffffffu, half ? off1 : off0, sl);
        const C* h = cache_ptr<T>(a, cb + sl + 32 * half);
#pragma unroll
        for (int u = 0; u < G; ++u) {
          const int j = i0 + 32 * u - o;
          if (j >= 0 && j < N) {
            xa[u] = cadd(xa[u], __ldcs(h + j));
            xe[u] = cadd(xe[u], __ldcs(h + N + j));
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < G; ++u) {
      __stcs(H + i0 + 32 * u, xa[u]);
      __stcs(H + W3 + i0 + 32 * u, xe[u]);
    }
  }
  __syncwarp();
}

// (temperatures [0, n_t): all of them after a refresh, the cold chain after a transfer)
template <typename T, int N>
__global__ void __launch_bounds__(kSwWarps * 32) k_hsum(const SweepArgs a, int n_t) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const gbk_sweep_desc& d = a.d;
  const int64_t ntask = (int64_t)n_t * d.n_walkers * d.n_bands;
  for (int64_t x = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid; x < ntask; x += (int64_t)gridDim.x * (blockDim.x >> 5)) {
    const int t = (int)(x / ((int64_t)d.n_walkers * d.n_bands));
    const int rem = (int)(x % ((int64_t)d.n_walkers * d.n_bands));
    write_hsum<T, N>(a, t, rem / d.n_bands, rem % d.n_bands, lane);
  }
}

// -------------------------------------------------------------- cache refresh
// Regenerate the cached waveform of every present slot (32 slots per warp batch).
__global__ void k_identity_ids(int32_t* ids, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    ids[i] = (int32_t)i;
}

template <typename T, int N>
__global__ void __launch_bounds__(kSwWarps * 32) k_refresh(const SweepArgs a) {
  typedef typename CT<T>::C C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char* mine = smem_raw + (size_t)wid * (4 * N * sizeof(C) + 32 * sizeof(Src<T>) + 128);  // refresh_warp_bytes
  C* b0 = reinterpret_cast<C*>(mine);
  C* b1 = b0 + 2 * N;
  Src<T>* srcs = reinterpret_cast<Src<T>*>(b1 + 2 * N);
  int* ok = reinterpret_cast<int*>(srcs + 32);
  const gbk_sweep_desc& d = a.d;
  const int64_t nslot = (int64_t)d.n_temps * d.n_walkers * d.n_bands * d.n_max;
  const T* orb = orb_of<T>(a.c, band_index(N));
  const C* tw = tw_of<T>(a.c, band_index(N));
  const int wpc = blockDim.x >> 5;
  for (int64_t base = ((int64_t)blockIdx.x * wpc + wid) * 32; base < nslot;
       base += (int64_t)gridDim.x * wpc * 32) {
    const int64_t me = base + lane;
    ok[lane] = (me < nslot && a.exists[me]) ? 1 : 0;
    if (ok[lane]) srcs[lane] = make_src<T>(a.params + me * 8, 1, 0, a.c.grid.tobs, N);
    __syncwarp();
    for (int q = 0; q < 32; ++q) {
      if (!ok[q]) continue;
      gen_band<T, N>(&srcs[q], orb, tw, a.c.grid.tobs, b0, b1, lane);
      copy_band(cache_ptr<T>(a, base + q), b0, 2 * N, lane);
      __syncwarp();
    }
    __syncwarp();
  }
}

// -------------------------------------------------------------- open pass
// rho_{w,b} = snapshot residual on b's window + band b's cold-chain sources (cached).
template <typename T, int N>
__global__ void __launch_bounds__(kSwWarps * 32) k_open(const SweepArgs a) {
  typedef typename CT<T>::C C;
  constexpr int W3 = 3 * N;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const gbk_sweep_desc& d = a.d;
  const int nbp = (d.n_bands - a.parity + 1) / 2;
  const int64_t ntask = (int64_t)d.n_walkers * nbp;
  const int64_t nb = a.c.grid.n_bins;
  const T rs = (T)ldexp(1.0, kStrainExp - a.frac_bits);
  for (int64_t x = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid; x < ntask; x += (int64_t)gridDim.x * (blockDim.x >> 5)) {
    const int w = (int)(x / nbp), j = (int)(x % nbp);
    const int b = a.parity + 2 * j;
    const int64_t gw = d.band_k0 + (int64_t)(b - 1) * N - a.c.grid.k0;
    C* rho = rho_ptr<T>(a, w, j);
    const long long* rs_w = a.rsnap + (int64_t)w * 2 * nb * 2;
    for (int i = lane; i < W3; i += 32)
      for (int ch = 0; ch < 2; ++ch) {
        const longlong2 v = *reinterpret_cast<const longlong2*>(rs_w + 2 * (ch * nb + gw + i));
        rho[ch * W3 + i] = mkc(i2t(v.x, T()) * rs, i2t(v.y, T()) * rs);
      }
    __syncwarp();
    const C* H = hsum_ptr<T>(a, 0, w, b);
    for (int i = lane; i < 2 * W3; i += 32) rho[i] = cadd(rho[i], H[i]);
  }
}

// -------------------------------------------------------------- learned-proposal inputs
// Whitened residual of band b's own sub-band from its opened window:
// x[ch 512 + 2 i + {0, 1}] = (Re, Im) rho[ch][N + i] sqrt(4 df / S_n), rounded to BF16.
// Row (w, j) of the parity's bands goes to x + (w * w_stride + j * j_stride + j_off) * 4N
// (j_off, j_stride = 0, 1 for the sweep's compact rows; parity, 2 for [W][n_bands] rows).
template <typename T, int N>
__global__ void __launch_bounds__(kSwWarps * 32) k_features(const SweepArgs a, uint16_t* __restrict__ x,
                                                            int64_t w_stride, int j_stride, int j_off) {
  typedef typename CT<T>::C C;
  constexpr int W3 = 3 * N;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const gbk_sweep_desc& d = a.d;
  const int nbp = (d.n_bands - a.parity + 1) / 2;
  const int64_t ntask = (int64_t)d.n_walkers * nbp;
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid; t < ntask; t += (int64_t)gridDim.x * (blockDim.x >> 5)) {
    const int w = (int)(t / nbp), j = (int)(t % nbp);
    const int b = a.parity + 2 * j;
    const int64_t gw = d.band_k0 + (int64_t)(b - 1) * N - a.c.grid.k0;
    const PsdWt<T> pw = walker_psd<T>(a, w);
    const C* rho = rho_ptr<T>(a, w, j);
    __nv_bfloat162* out = reinterpret_cast<__nv_bfloat162*>(x + (w * w_stride + (int64_t)j * j_stride + j_off) * 4 * N);
    for (int i = lane; i < N; i += 32) {
      const int64_t k = gw + N + i;
      const T wt = sqrt((T)pw.cw * iqv(a.c, k, T()) * recip((T)1 + pw.aw * rhov(a.c, k, T())));
#pragma unroll
      for (int ch = 0; ch < 2; ++ch) {
        const C r = rho[ch * W3 + N + i];
        out[ch * N + i] = __floats2bfloat162_rn((float)(r.x * wt), (float)(r.y * wt));
      }
    }
  }
}

// Mixture rows of the parity's bands from network outputs (raw row (w, j)) or from the
// caller's table (raw row (w, b) of [W][n_bands]).
template <typename T>
__global__ void k_mixrows(const SweepArgs a, const float* __restrict__ raw, int table, MixRow<T>* __restrict__ rows) {
  const gbk_sweep_desc& d = a.d;
  const int nbp = (d.n_bands - a.parity + 1) / 2;
  const int64_t n = (int64_t)d.n_walkers * nbp;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int w = (int)(t / nbp), j = (int)(t % nbp);
    const int64_t src = table ? (int64_t)w * d.n_bands + a.parity + 2 * j : (int64_t)w * a.n_bp_max + j;
    mix_build<T>(raw + src * kMixOut, rows[(int64_t)w * a.n_bp_max + j]);
  }
}

// Unit-box coordinates of every cold-chain slot [W][n_bands][n_max][8] (NaN where empty).
__global__ void k_cold_unit(const SweepArgs a, float* __restrict__ u) {
  const gbk_sweep_desc& d = a.d;
  const int64_t n = (int64_t)d.n_walkers * d.n_bands * d.n_max;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)((i / d.n_max) % d.n_bands);
    double ud[8];
    if (a.exists[i]) {
      to_unit<double>(d, prior_consts(d), band_geom(d, a.c.grid.tobs, b), a.params + i * 8, ud);
    } else {
      for (int c = 0; c < 8; ++c) ud[c] = nan_d();
    }
    for (int c = 0; c < 8; ++c) u[i * 8 + c] = (float)ud[c];
  }
}

// -------------------------------------------------------------- stationary group
// Band b's group: every cold-chain source of bands b-1, b, b+1 of all walkers, sorted by
// (f0, slot index) with a bitonic sort in shared memory (p2 = power of two >= members).
__global__ void k_group_build(const double* __restrict__ params, const uint8_t* __restrict__ exists,
                              gbk_sweep_desc d, int gmax, int p2, double* __restrict__ gf0, double* __restrict__ gpar,
                              int32_t* __restrict__ gn) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* key = reinterpret_cast<double*>(smem_raw);
  int32_t* idx = reinterpret_cast<int32_t*>(key + p2);
  __shared__ int count;
  const int b = blockIdx.x;
  if (threadIdx.x == 0) count = 0;
  __syncthreads();
  const int per_band = d.n_walkers * d.n_max;
  for (int c = threadIdx.x; c < 3 * per_band; c += blockDim.x) {
    const int bb = b - 1 + c / per_band;
    if (bb < 0 || bb >= d.n_bands) continue;
    const int w = (c % per_band) / d.n_max, s = c % d.n_max;
    const int64_t slot = ((int64_t)w * d.n_bands + bb) * d.n_max + s;   // cold chain: t = 0
    if (!exists[slot]) continue;
    const int i = atomicAdd(&count, 1);
    if (i < gmax) {
      key[i] = params[slot * 8 + 1];
      idx[i] = (int32_t)slot;
    }
  }
  __syncthreads();
  const int n = count < gmax ? count : gmax;
  for (int i = n + threadIdx.x; i < p2; i += blockDim.x) {
    key[i] = INFINITY;
    idx[i] = 0x7fffffff;
  }
  __syncthreads();
  for (int k = 2; k <= p2; k <<= 1)
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < p2; i += blockDim.x) {
        const int l = i ^ jj;
        if (l > i) {
          const bool up = (i & k) == 0;
          const bool gt = key[i] > key[l] || (key[i] == key[l] && idx[i] > idx[l]);
          if (gt == up) {
            const double tk = key[i]; key[i] = key[l]; key[l] = tk;
            const int32_t ti = idx[i]; idx[i] = idx[l]; idx[l] = ti;
          }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    gf0[(int64_t)b * gmax + i] = key[i];
    for (int c = 0; c < 8; ++c) gpar[((int64_t)b * gmax + i) * 8 + c] = params[(int64_t)idx[i] * 8 + c];
  }
  if (threadIdx.x == 0) gn[b] = n;
}

// -------------------------------------------------------------- band task
// Per-warp shared memory of k_band.
template <typename T, int N>
struct BandSmem {
  typename CT<T>::C ba[2 * N], bs[2 * N];
  Src<T> src[32];                      // constants of the batch's new templates
  double th[32][8];                    // proposed parameters
  double lpn[32], lu[32];              // prior log-ratio of the proposal, ln u
  int k[32], supp[32];
  int list[kMaxSlots];
};

// Set up proposal j (lane-parallel): words, source, perturbation, support, prior, constants.
// __noinline__ and not unrolled over blocks: this set-up runs on a few lanes between
// waveform generations, and its code must not crowd the instruction cache.
template <typename T, int N>
__device__ __noinline__ void prep_inmodel(const SweepArgs& a, const PriorK& pk, BandSmem<T, N>& S, int l, int jp,
                                          uint32_t tid, int g, const double* P, int b, const BandGeom& bg,
                                          const MixRow<T>* mrow) {
  const gbk_sweep_desc& d = a.d;
  uint32_t w[48];
#pragma unroll 1
  for (int m = 0; m < 12; ++m) {
    const U4 v = philox4x32_10(12u * jp + m, tid, 0u | ((uint32_t)a.parity << 4), a.sweep, a.k0, a.k1);
    w[4 * m] = v.x; w[4 * m + 1] = v.y; w[4 * m + 2] = v.z; w[4 * m + 3] = v.w;
  }
  const int k = S.list[ranged(w[0], (uint32_t)g)];
  double th[8], nw[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) th[c] = P[k * 8 + c];
  const bool indep = mrow && mix_u32(w[35]) < a.mdn_inmodel;   // independence move from the learned mixture
  const bool grp = !indep && a.grp_f0 && a.grp_n[b] > 0 && mix_u32(w[46]) < a.grp_frac;   // group stretch
  double lnz = 0.0;
  if (indep)
    mdn_draw<T>(a, pk, *mrow, bg, w[36], w[37], w + 38, nw);
  else if (grp)
    lnz = group_stretch(a, b, th, w[1], w[2], nw);
  else
    propose(d, th, w, nw, T());
  S.lu[l] = log_u(u53(w[33], w[34]), T());
  S.k[l] = k;
  const bool ok = !(lnz != lnz) && in_support<T>(pk, bg, nw);   // NaN ln z: not reversible as drawn
  S.supp[l] = ok ? 1 : 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) S.th[l][c] = nw[c];
  if (ok) {
    // unit coordinates: prior density 1, so q(theta) / q(theta') is the whole Hastings factor;
    // the stretch adds its Jacobian z^(d-1), d = 8
    S.lpn[l] = indep ? mdn_logq<T>(a, pk, *mrow, bg, th) - mdn_logq<T>(a, pk, *mrow, bg, nw)
                     : dlog_prior(nw, th, T()) + (grp ? 7.0 * lnz : 0.0);
    S.src[l] = make_src<T>(nw, 1, 0, a.c.grid.tobs, N);
  }
}

template <typename T, int N>
__device__ __noinline__ void prep_rj(const SweepArgs& a, const PriorK& pk, BandSmem<T, N>& S, int l, int jp,
                                     uint32_t tid, const uint8_t* E, const double* P, const BandGeom& bg,
                                     const MixRow<T>* mrow) {
  const int s = S.list[jp];
  uint32_t wv[16];
#pragma unroll 1
  for (int m = 0; m < 4; ++m) {
    const U4 v = philox4x32_10(4u * jp + m, tid, 2u | ((uint32_t)a.parity << 4), a.sweep, a.k0, a.k1);
    wv[4 * m] = v.x; wv[4 * m + 1] = v.y; wv[4 * m + 2] = v.z; wv[4 * m + 3] = v.w;
  }
  S.lu[l] = log_u(u53(wv[8], wv[9]), T());
  S.k[l] = s;
  S.supp[l] = 1;
  S.lpn[l] = 0.0;
  if (!E[s]) {
    double nw[8];
    if (mrow) {
      mdn_draw<T>(a, pk, *mrow, bg, wv[10], wv[11], wv, nw);
      S.supp[l] = in_support<T>(pk, bg, nw) ? 1 : 0;
      if (S.supp[l]) S.lpn[l] = -mdn_logq<T>(a, pk, *mrow, bg, nw);
    } else {
      draw_birth<T>(a.d, pk, bg, wv, nw);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) S.th[l][c] = nw[c];
    if (S.supp[l]) S.src[l] = make_src<T>(nw, 1, 0, a.c.grid.tobs, N);
  } else if (mrow) {
    S.lpn[l] = mdn_logq<T>(a, pk, *mrow, bg, P + s * 8);
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(kBandWarps * 32, kBandMinCtas) k_band(const SweepArgs a, int flags) {
  typedef typename CT<T>::C C;
  constexpr int W3 = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  BandSmem<T, N>& S = reinterpret_cast<BandSmem<T, N>*>(smem_raw)[wid];
  // the band window lives in a per-warp global slot: cached in L1 (which takes the shared
  // memory it would have used), so more warps fit per SM
  C* const rw = reinterpret_cast<C*>(a.rwbuf) + ((size_t)blockIdx.x * (blockDim.x >> 5) + wid) * 2 * W3;
  const gbk_sweep_desc& d = a.d;
  const int nbp = (d.n_bands - a.parity + 1) / 2;
  const int64_t ntask = (int64_t)d.n_temps * d.n_walkers * nbp;
  const int64_t nb = a.c.grid.n_bins;
  const double tobs = a.c.grid.tobs;
  const T rs = (T)ldexp(1.0, kStrainExp - a.frac_bits);
  const T gs = (T)ldexp(1.0, a.frac_bits - kStrainExp);
  const T* orb = orb_of<T>(a.c, band_index(N));
  const C* tw = tw_of<T>(a.c, band_index(N));
  WarpStats ws;
  ws.init();
  const PriorK pk = prior_consts(d);
  // band tasks taken one at a time from a counter: tasks differ in cost (sources, accepted
  // moves), and a fixed share per warp leaves the launch waiting for its slowest warps
  for (;;) {
    int64_t x = 0;
    if (lane == 0) x = (int64_t)atomicAdd(a.task_ctr + a.parity, 1ull);
    x = __shfl_sync(0xffffffffu, x, 0);
    if (x >= ntask) break;
    const int t = (int)(x / ((int64_t)d.n_walkers * nbp));
    const int rem = (int)(x % ((int64_t)d.n_walkers * nbp));
    const int w = rem / nbp, j = rem % nbp;
    const int b = a.parity + 2 * j;
    const int64_t gw = d.band_k0 + (int64_t)(b - 1) * N - a.c.grid.k0;
    const int64_t base = slot_index(d, t, w, b);
    const int64_t cb = cache_base(a, t, w, b);
    double* P = a.params + base * 8;
    uint8_t* E = a.exists + base;
    const double beta = a.betas[(int64_t)b * d.n_temps + t];
    const uint32_t tid = (uint32_t)(((int64_t)t * d.n_walkers + w) * d.n_bands + b);
    const PsdWt<T> pw = walker_psd<T>(a, w);
    const bool cold = (t == 0);
    const MixRow<T>* mrow = mix_ptr<T>(a, w, j);
    const BandGeom bg = band_geom(d, tobs, b);
    long long* Rw = a.resid + (int64_t)w * 2 * nb * 2;
    // r' for the band: cold chain from the snapshot; hotter chains from the opened window
    // minus their own (cached) templates. These inputs are read once per task: evict-first
    // loads keep L1 for the window, the templates and the tables the proposals reuse.
    if (cold) {
      const long long* rs_w = a.rsnap + (int64_t)w * 2 * nb * 2;
#pragma unroll 4
      for (int i = lane; i < W3; i += 32) {
        const longlong2 va = __ldcs(reinterpret_cast<const longlong2*>(rs_w + 2 * (gw + i)));
        const longlong2 ve = __ldcs(reinterpret_cast<const longlong2*>(rs_w + 2 * (nb + gw + i)));
        st_win(rw + 2 * i, mkc(i2t(va.x, T()) * rs, i2t(va.y, T()) * rs), mkc(i2t(ve.x, T()) * rs, i2t(ve.y, T()) * rs));
      }
      __syncwarp();
    } else {
      const C* rho = rho_ptr<T>(a, w, j);
      const C* H = hsum_ptr<T>(a, t, w, b);
#pragma unroll 4
      for (int i = lane; i < W3; i += 32)
        st_win(rw + 2 * i, csub(__ldcs(rho + i), __ldcs(H + i)), csub(__ldcs(rho + W3 + i), __ldcs(H + W3 + i)));
      __syncwarp();
    }
    // ---- in-model proposals (Alg. 1)
    if (flags & GBK_SWEEP_INMODEL) {
      if (lane == 0) {
        int g = 0;
        for (int s = 0; s < d.n_max; ++s)
          if (E[s]) S.list[g++] = s;
        S.list[kMaxSlots - 1] = g;
      }
      __syncwarp();
      const int g = S.list[kMaxSlots - 1];
      const int n_prop = (int)rint(d.props_per_source * (double)g);
      for (int j0 = 0; j0 < n_prop; j0 += 32) {
        const int cnt = min(32, n_prop - j0);
        if (lane < cnt) prep_inmodel<T, N>(a, pk, S, lane, j0 + lane, tid, g, P, b, bg, mrow);
        __syncwarp();
        for (int q = 0; q < cnt; ++q) {
          const int jp = j0 + q;
          const int k = S.k[q];
          if (!S.supp[q]) {
            if (lane == 0) record(a, ws, 0, t, w, b, k, jp, false, nan_d(), -INFINITY, S.th[q], 0, 0);
            continue;
          }
          gen_band<T, N>(&S.src[q], orb, tw, tobs, S.ba, S.bs, lane);
          const C* hr = cache_ptr<T>(a, cb + k);
          const int oa = band_off<N>(S.src[q].q, gw, a.c);
          const int orr = cached_off<N>(P + k * 8, gw, a.c);
          const double dll = window_dll<T, N, true>(a, rw, S.ba, oa, hr, orr, gw, pw, lane);
          const double la = beta * dll + S.lpn[q];
          const bool acc = __shfl_sync(0xffffffffu, (int)(S.lu[q] < la), 0) != 0;
          if (lane == 0) record(a, ws, 0, t, w, b, k, jp, acc, dll, la, S.th[q], 1, 1);
          if (acc) {
            apply_change<T, N>(a, rw, S.ba, oa, hr, orr, cold, Rw, gw, gs, lane);
            __syncwarp();
            copy_band(cache_ptr<T>(a, cb + k), S.ba, 2 * N, lane);
            if (lane < 8) P[k * 8 + lane] = S.th[q][lane];
            __syncwarp();
            // later proposals of this batch that move the same source start from the new state
            if (lane > q && lane < cnt && S.k[lane] == k)
              prep_inmodel<T, N>(a, pk, S, lane, j0 + lane, tid, g, P, b, bg, mrow);
          }
          __syncwarp();
        }
      }
    }
    // ---- flip-all reversible jump (App. C)
    if ((flags & GBK_SWEEP_RJ) && d.n_max > 0) {
      if (lane == 0) {
        uint32_t buf[4];
        int wi = 4, blk = 0;
        for (int s = 0; s < d.n_max; ++s) S.list[s] = s;
        for (int i = d.n_max - 1; i > 0; --i) {
          if (wi == 4) {
            const U4 v = philox4x32_10((uint32_t)blk++, tid, 1u | ((uint32_t)a.parity << 4), a.sweep, a.k0, a.k1);
            buf[0] = v.x; buf[1] = v.y; buf[2] = v.z; buf[3] = v.w;
            wi = 0;
          }
          const int jx = (int)ranged(buf[wi++], (uint32_t)(i + 1));
          const int tmp = S.list[i]; S.list[i] = S.list[jx]; S.list[jx] = tmp;
        }
      }
      __syncwarp();
      for (int j0 = 0; j0 < d.n_max; j0 += 32) {
        const int cnt = min(32, d.n_max - j0);
        // lane-parallel set-up: uniform for the decision and, for empty slots, the prior draw
        if (lane < cnt) prep_rj<T, N>(a, pk, S, lane, j0 + lane, tid, E, P, bg, mrow);
        __syncwarp();
        for (int q = 0; q < cnt; ++q) {
          const int jp = j0 + q;
          const int s = S.k[q];
          if (E[s]) {
            const C* hr = cache_ptr<T>(a, cb + s);
            const int orr = cached_off<N>(P + s * 8, gw, a.c);
            const double dll = window_dll<T, N, true>(a, rw, (const C*)nullptr, 0, hr, orr, gw, pw, lane);
            const double la = beta * dll - d.log_occ_odds + S.lpn[q];
            const bool acc = __shfl_sync(0xffffffffu, (int)(S.lu[q] < la), 0) != 0;
            if (lane == 0) record(a, ws, 2, t, w, b, s, jp, acc, dll, la, P + s * 8, 0, 1);
            if (acc) {
              apply_change<T, N>(a, rw, (const C*)nullptr, 0, hr, orr, cold, Rw, gw, gs, lane);
              __syncwarp();
              if (lane == 0) E[s] = 0;
            }
          } else if (!S.supp[q]) {   // learned-proposal draw on the box edge outside the support
            if (lane == 0) record(a, ws, 1, t, w, b, s, jp, false, nan_d(), -INFINITY, S.th[q], 0, 0);
          } else {
            gen_band<T, N>(&S.src[q], orb, tw, tobs, S.ba, S.bs, lane);
            const int oa = band_off<N>(S.src[q].q, gw, a.c);
            const double dll = window_dll<T, N, true>(a, rw, S.ba, oa, (const C*)nullptr, 0, gw, pw, lane);
            const double la = beta * dll + d.log_occ_odds + S.lpn[q];
            const bool acc = __shfl_sync(0xffffffffu, (int)(S.lu[q] < la), 0) != 0;
            if (lane == 0) record(a, ws, 1, t, w, b, s, jp, acc, dll, la, S.th[q], 1, 1);
            if (acc) {
              apply_change<T, N>(a, rw, S.ba, oa, (const C*)nullptr, 0, cold, Rw, gw, gs, lane);
              copy_band(cache_ptr<T>(a, cb + s), S.ba, 2 * N, lane);
              if (lane < 8) P[s * 8 + lane] = S.th[q][lane];
              __syncwarp();
              if (lane == 0) E[s] = 1;
            }
          }
          __syncwarp();
        }
      }
    }
    __syncwarp();
    write_hsum<T, N>(a, t, w, b, lane);   // the band's template sum for openings and swaps
  }
  if (lane == 0) ws.flush(a.stats);
}

// -------------------------------------------------------------- tempering (Alg. 2)
// <rho - Hx|rho - Hx> - <rho - Hy|rho - Hy> = cw sum_k w_k Re[(Hy - Hx) conj(2 rho - Hx - Hy)],
// formed bin by bin so the large common parts cancel before summation.
// Both set differences of one swap proposal in one pass over the window, the two template
// sums read once: D1 = diff(rho_t; hx, hy) with walker t's PSD weights and D2 = diff(rho_m;
// hy, hx) with walker m's, where diff(rho; x, y) = <rho - x|rho - x> - <rho - y|rho - y>.
template <typename T, int N>
__device__ __noinline__ void set_diff2(const SweepArgs& a, const typename CT<T>::C* __restrict__ rt,
                                       const typename CT<T>::C* __restrict__ rm, const typename CT<T>::C* __restrict__ hx,
                                       const typename CT<T>::C* __restrict__ hy, int64_t gw, const PsdWt<T>& pt,
                                       const PsdWt<T>& pm, int lane, double& d1, double& d2) {
  typedef typename CT<T>::C C;
  constexpr int W3 = 3 * N;
  typename SAcc<T>::S a1, a2;
  a1.init();
  a2.init();
#pragma unroll 4
  for (int i = lane; i < W3; i += 32) {
    const int64_t k = gw + i;
    const T iq = iqv(a.c, k, T()), rh = rhov(a.c, k, T());
    const T w1 = iq * recip((T)1 + pt.aw * rh);
    const T w2 = iq * recip((T)1 + pm.aw * rh);
    T s1 = (T)0, s2 = (T)0;
#pragma unroll
    for (int ch = 0; ch < 2; ++ch) {
      const C x = hx[ch * W3 + i], y = hy[ch * W3 + i];
      const C r1 = rt[ch * W3 + i], r2 = rm[ch * W3 + i];
      const C dl1 = csub(y, x), dl2 = csub(x, y);
      const C sm1 = csub(cscale(r1, (T)2), cadd(x, y));
      const C sm2 = csub(cscale(r2, (T)2), cadd(y, x));
      s1 += dl1.x * sm1.x + dl1.y * sm1.y;
      s2 += dl2.x * sm2.x + dl2.y * sm2.y;
    }
    a1.add(w1 * s1);
    a2.add(w2 * s2);
  }
  d1 = pt.cw * a1.warp_total();
  d2 = pm.cw * a2.warp_total();
}

// Move the cached templates of one band into (sign +1: R -= h) or out of (sign -1:
// R += h) the cold-chain residual, each rounded to the fixed-point grid.
template <typename T, int N>
__device__ __noinline__ void cold_update(const SweepArgs& a, int64_t base, int64_t cb, int sign, long long* Rw,
                                         int lane) {
  typedef typename CT<T>::C C;
  const int64_t nb = a.c.grid.n_bins;
  const T gs = (T)ldexp(1.0, a.frac_bits - kStrainExp);
  unsigned long long* R = reinterpret_cast<unsigned long long*>(Rw);
  for (int s = 0; s < a.d.n_max; ++s) {
    if (!a.exists[base + s]) continue;
    const C* h = cache_ptr<T>(a, cb + s);
    const int64_t o = (long long)floor(a.params[(base + s) * 8 + 1] * a.c.grid.tobs) - N / 2 - a.c.grid.k0;
    for (int i = lane; i < N; i += 32)
      for (int ch = 0; ch < 2; ++ch) {
        const C v = h[ch * N + i];
        long long hx = t2grid(v.x, gs), hy = t2grid(v.y, gs);
        if (sign > 0) { hx = -hx; hy = -hy; }
        unsigned long long* dst = R + 2 * (ch * nb + o + i);
        atomicAdd(dst, (unsigned long long)hx);
        atomicAdd(dst + 1, (unsigned long long)hy);
      }
  }
  __syncwarp();
}

template <typename T, int N>
__host__ __device__ constexpr size_t swap_warp_bytes(int nt, int nw) {
  return ((size_t)nt * nw * sizeof(short) + 15) / 16 * 16;
}
template <typename T, int N>
__host__ __device__ constexpr size_t refresh_warp_bytes() {
  return 4 * N * sizeof(typename CT<T>::C) + 32 * sizeof(Src<T>) + 128;
}

// One warp per (band, chain): walkers permuted per temperature, swaps from the top
// temperature down; the band's template sums come from the set-sum cache. Each warp's swaps
// are a chain of latency-bound window passes: 5 CTAs per SM (96 registers, no spills; 128
// registers gave 4) hide more of the latency, and the bench's 5920 tasks per parity then fit
// in two waves of 3040 warps instead of three of 2432 (-29 % per sweep). The float64 kernel
// would spill at 96 registers and keeps 4 CTAs.
template <typename T, int N>
__global__ void __launch_bounds__(kSwWarps * 32, sizeof(T) == 4 ? kSwapMinCtas : 4) k_swap(const SweepArgs a) {
  typedef typename CT<T>::C C;
  constexpr int W3 = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const gbk_sweep_desc& d = a.d;
  const int T_ = d.n_temps, W = d.n_walkers;
  short* perm = reinterpret_cast<short*>(smem_raw + (size_t)wid * swap_warp_bytes<T, N>(T_, W));   // [T][W]
  const int nbp = (d.n_bands - a.parity + 1) / 2;
  const int64_t ntask = (int64_t)nbp * W;
  const int nslotc = 2 * N;
  WarpStats ws;
  ws.init();
  for (int64_t x = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid; x < ntask; x += (int64_t)gridDim.x * (blockDim.x >> 5)) {
    const int j = (int)(x / W), c = (int)(x % W);
    const int b = a.parity + 2 * j;
    const int64_t gw = d.band_k0 + (int64_t)(b - 1) * N - a.c.grid.k0;
    // walker permutation of every temperature (Fisher-Yates on Philox words)
    for (int t = lane; t < T_; t += 32) {
      short* pt = perm + t * W;
      for (int i = 0; i < W; ++i) pt[i] = (short)i;
      uint32_t buf[4];
      int wi = 4, blk = 0;
      for (int i = W - 1; i > 0; --i) {
        if (wi == 4) {
          const U4 v = philox4x32_10((uint32_t)blk++, (uint32_t)(b * T_ + t), 3u | ((uint32_t)a.parity << 4), a.sweep,
                                     a.k0, a.k1);
          buf[0] = v.x; buf[1] = v.y; buf[2] = v.z; buf[3] = v.w;
          wi = 0;
        }
        const int jx = (int)ranged(buf[wi++], (uint32_t)(i + 1));
        const short tmp = pt[i]; pt[i] = pt[jx]; pt[jx] = tmp;
      }
    }
    __syncwarp();
    for (int t = T_ - 1; t > 0; --t) {
      const int wt = perm[t * W + c];
      const int wm = perm[(t - 1) * W + c];
      const int64_t bt = slot_index(d, t, wt, b), bm = slot_index(d, t - 1, wm, b);
      C* Ht = hsum_ptr<T>(a, t, wt, b);
      C* Hm = hsum_ptr<T>(a, t - 1, wm, b);
      const PsdWt<T> pt_ = walker_psd<T>(a, wt), pm_ = walker_psd<T>(a, wm);
      // l_t(m) - l_t(t) = -1/2 D1, l_m(t) - l_m(m) = -1/2 D2 (band-local likelihoods)
      double D1, D2;
      set_diff2<T, N>(a, rho_ptr<T>(a, wt, j), rho_ptr<T>(a, wm, j), Hm, Ht, gw, pt_, pm_, lane, D1, D2);
      const double la = a.betas[(int64_t)b * T_ + t] * (-0.5 * D1) + a.betas[(int64_t)b * T_ + t - 1] * (-0.5 * D2);
      const U4 v = philox4x32_10((uint32_t)t, (uint32_t)(b * W + c), 4u | ((uint32_t)a.parity << 4), a.sweep, a.k0, a.k1);
      const double lu = log_u(u53(v.x, v.y), T());
      const bool acc = __shfl_sync(0xffffffffu, (int)(lu < la), 0) != 0;
      if (acc) {
        double* Pt = a.params + bt * 8;
        double* Pm = a.params + bm * 8;
        for (int i = lane; i < d.n_max * 8; i += 32) {
          const double q = Pt[i]; Pt[i] = Pm[i]; Pm[i] = q;
        }
        for (int i = lane; i < d.n_max; i += 32) {
          const uint8_t q = a.exists[bt + i]; a.exists[bt + i] = a.exists[bm + i]; a.exists[bm + i] = q;
        }
        if (lane == 0) {
          int32_t* it = a.setid + ((int64_t)t * W + wt) * d.n_bands + b;
          int32_t* im = a.setid + ((int64_t)(t - 1) * W + wm) * d.n_bands + b;
          const int32_t q = *it; *it = *im; *im = q;
        }
        __syncwarp();
        if (t == 1) {
          long long* Rw = a.resid + (int64_t)wm * 2 * a.c.grid.n_bins * 2;
          cold_update<T, N>(a, bt, cache_base(a, t, wt, b), -1, Rw, lane);       // old cold set leaves the model
          cold_update<T, N>(a, bm, cache_base(a, t - 1, wm, b), +1, Rw, lane);   // new cold set enters
        }
      }
      if (lane == 0) {
        record(a, ws, 3, t, wt, b, c, t, acc, la, la, nullptr, 0, 0);
        if (acc) atomicAdd(&a.swap_acc[(int64_t)b * T_ + t], 1);
      }
      __syncwarp();
    }
  }
  if (lane == 0) ws.flush(a.stats);
}

// -------------------------------------------------------------- host side
static int sms_of_device() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// Warps per CTA (<= kSwWarps) so that the CTA's shared memory fits the SM.
static int sweep_warps(size_t per_warp, int max_warps) {
  int w = (int)((220 * 1024) / (per_warp > 0 ? per_warp : 1));
  return w < 1 ? 1 : (w > max_warps ? max_warps : w);
}

template <typename K>
static gbk_status prep(K kernel, size_t per_warp, int64_t items, int* grid, int* threads, size_t* smem,
                       int max_warps = kSwWarps, int64_t* resident_warps = nullptr) {
  const int wpc = sweep_warps(per_warp, max_warps);
  *threads = wpc * 32;
  *smem = per_warp * wpc;
  if (*smem > 48 * 1024 && cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem) != cudaSuccess) {
    cudaGetLastError();
    return set_error(GBK_ECUDA, "sweep kernel needs %zu bytes of shared memory", *smem);
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, *threads, *smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return set_error(GBK_ECUDA, "sweep kernel does not fit on an SM (%zu bytes of shared memory)", *smem);
  }
  const int64_t need = (items + wpc - 1) / wpc;
  const int64_t cap = (int64_t)sms_of_device() * per_sm;
  *grid = (int)(need < cap ? (need > 0 ? need : 1) : cap);
  if (resident_warps) *resident_warps = cap * wpc;
  return GBK_OK;
}

static thread_local gbk_sweep* g_timing_plan = nullptr;  // plan whose kernels are being timed (per host thread)
static void ev_rec(int parity, int which, int edge, cudaStream_t st) {
  if (g_timing_plan && g_timing_plan->timed) cudaEventRecord(g_timing_plan->ev[parity][which][edge], st);
}

template <typename T, int N>
static gbk_status run_refresh(SweepArgs& a, cudaStream_t st) {
  const int64_t nslot = (int64_t)a.d.n_temps * a.d.n_walkers * a.d.n_bands * a.d.n_max;
  if (nslot == 0) return GBK_OK;
  int grid = 0, thr = 0;
  size_t sm = 0;
  gbk_status s;
  if ((s = prep(k_refresh<T, N>, refresh_warp_bytes<T, N>(), (nslot + 31) / 32, &grid, &thr, &sm))) return s;
  ev_rec(1, 0, 0, st);
  const int64_t nsets = (int64_t)a.d.n_temps * a.d.n_walkers * a.d.n_bands;
  k_identity_ids<<<(int)((nsets + 255) / 256 < 4096 ? (nsets + 255) / 256 : 4096), 256, 0, st>>>(a.setid, nsets);
  k_refresh<T, N><<<grid, thr, sm, st>>>(a);
  if ((s = check_launch("gb_sweep(refresh)"))) return s;
  const int64_t ntask = (int64_t)a.d.n_temps * a.d.n_walkers * a.d.n_bands;
  if ((s = prep(k_hsum<T, N>, 0, ntask, &grid, &thr, &sm))) return s;
  k_hsum<T, N><<<grid, kSwWarps * 32, 0, st>>>(a, a.d.n_temps);
  ev_rec(1, 0, 1, st);
  return check_launch("gb_sweep(refresh)");
}

// -------------------------------------------------------------- band-edge ownership transfer
// Sec. V.D: a cold-chain source of band b whose f0 lies in the own bins of a neighbour moves
// there. Decided on the state at the call: destination band b' (one thread per (w, b'))
// takes its candidates from b' - 1, then b' + 1, in slot order, into its free slots in slot
// order; candidates beyond its free slots stay. Every cold slot has at most one destination
// (its owner), so each entry of dest is written by one thread at most.
__device__ __forceinline__ long long owner_of(double f0, double tobs, const gbk_sweep_desc& d) {
  return (long long)floor(__ddiv_rn(dsub(dmul(f0, tobs), (double)d.band_k0), (double)d.band_bins));
}

__global__ void k_xfer_assign(const double* __restrict__ params, const uint8_t* __restrict__ exists,
                              const gbk_sweep_desc d, double tobs, int32_t* __restrict__ dest,
                              int32_t* __restrict__ counts) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= d.n_walkers * d.n_bands) return;
  const int w = x / d.n_bands, b = x % d.n_bands;
  const int64_t base = ((int64_t)w * d.n_bands + b) * d.n_max;   // temperature 0
  int free_s[kMaxSlots];
  int nfree = 0;
  for (int s = 0; s < d.n_max; ++s)
    if (!exists[base + s]) free_s[nfree++] = s;
  int k = 0, moved = 0, blocked = 0;
  for (int side = 0; side < 2; ++side) {
    const int sb = side == 0 ? b - 1 : b + 1;
    if (sb < 0 || sb >= d.n_bands) continue;
    const int64_t sbase = ((int64_t)w * d.n_bands + sb) * d.n_max;
    for (int s = 0; s < d.n_max; ++s) {
      if (!exists[sbase + s] || owner_of(params[(sbase + s) * 8 + 1], tobs, d) != b) continue;
      if (k < nfree) {
        dest[sbase + s] = b * d.n_max + free_s[k];
        ++moved;
      } else {
        ++blocked;
      }
      ++k;
    }
  }
  if (counts && (moved | blocked)) {
    atomicAdd(&counts[0], moved);
    atomicAdd(&counts[1], blocked);
  }
}

// One warp per cold slot with a destination: parameters, occupancy and the cached template
// (tmpl16 16-byte words) move; reads only dest and the moving slot, writes only the moving
// slot and its (free) destination.
__global__ void k_xfer_apply(const SweepArgs a, const int32_t* __restrict__ dest, int tmpl16) {
  const int lane = threadIdx.x & 31;
  const gbk_sweep_desc& d = a.d;
  const int64_t nslot = (int64_t)d.n_walkers * d.n_bands * d.n_max;
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < nslot;
       x += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t to = dest[x];
    if (to < 0) continue;
    const int w = (int)(x / ((int64_t)d.n_bands * d.n_max));
    const int b = (int)((x / d.n_max) % d.n_bands), s = (int)(x % d.n_max);
    const int db = to / d.n_max, ds = to % d.n_max;
    const int64_t y = ((int64_t)w * d.n_bands + db) * d.n_max + ds;
    if (lane < 8) a.params[y * 8 + lane] = a.params[x * 8 + lane];
    const int64_t cs = (int64_t)a.setid[(int64_t)w * d.n_bands + b] * d.n_max + s;
    const int64_t cd = (int64_t)a.setid[(int64_t)w * d.n_bands + db] * d.n_max + ds;
    const uint4* src = reinterpret_cast<const uint4*>(a.wcache) + cs * tmpl16;
    uint4* dst = reinterpret_cast<uint4*>(a.wcache) + cd * tmpl16;
    for (int i = lane; i < tmpl16; i += 32) dst[i] = src[i];
    if (lane == 0) {
      a.exists[y] = 1;
      a.exists[x] = 0;
    }
  }
}

template <typename T, int N>
static gbk_status run_transfer(gbk_sweep* plan, SweepArgs& a, int32_t* counts, cudaStream_t st) {
  const gbk_sweep_desc& d = a.d;
  const int64_t nslot = (int64_t)d.n_walkers * d.n_bands * d.n_max;
  if (nslot == 0) return GBK_OK;
  if (cudaMemsetAsync(plan->xfer_dest, 0xff, nslot * sizeof(int32_t), st) != cudaSuccess)
    return set_error(GBK_ECUDA, "gbk_sweep_transfer: cannot clear the destinations");
  const int wb = d.n_walkers * d.n_bands;
  k_xfer_assign<<<(wb + 127) / 128, 128, 0, st>>>(a.params, a.exists, d, a.c.grid.tobs, plan->xfer_dest, counts);
  gbk_status s;
  if ((s = check_launch("gbk_sweep_transfer(assign)"))) return s;
  const int tmpl16 = (int)(2 * N * sizeof(typename CT<T>::C) / 16);
  const int64_t blocks = (nslot + 7) / 8;
  k_xfer_apply<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(a, plan->xfer_dest, tmpl16);
  if ((s = check_launch("gbk_sweep_transfer(apply)"))) return s;
  int grid = 0, thr = 0;
  size_t sm = 0;
  if ((s = prep(k_hsum<T, N>, 0, wb, &grid, &thr, &sm))) return s;
  k_hsum<T, N><<<grid, kSwWarps * 32, 0, st>>>(a, 1);   // the cold chain's template sums
  return check_launch("gbk_sweep_transfer(template sums)");
}

template <typename T>
static gbk_status transfer_n(gbk_sweep* plan, SweepArgs& a, int32_t* counts, cudaStream_t st) {
  switch (a.d.band_bins) {
    case 128: return run_transfer<T, 128>(plan, a, counts, st);
    case 256: return run_transfer<T, 256>(plan, a, counts, st);
    case 512: return run_transfer<T, 512>(plan, a, counts, st);
    case 1024: return run_transfer<T, 1024>(plan, a, counts, st);
    default: return set_error(GBK_EINVAL, "gbk_sweep_transfer: band_bins %d", a.d.band_bins);
  }
}

static thread_local gbk_sweep* g_active_plan = nullptr;   // plan of the gb_sweep call in progress (per host thread)

// Learned proposal of one half sweep: features of the opened windows -> network ->
// mixture rows (or mixture rows straight from the caller's table).
template <typename T, int N>
static gbk_status run_proposal(gbk_sweep* plan, SweepArgs& a, cudaStream_t st) {
  const int nbp = (a.d.n_bands - a.parity + 1) / 2;
  const int rows = a.d.n_walkers * nbp;
  gbk_status s;
  const float* raw = plan->raw_table;
  if (!raw) {
    if (N != 256) return set_error(GBK_ENOTIMPL, "gb_sweep: the network takes 256-bin bands");
    int grid = 0, thr = 0;
    size_t sm = 0;
    if ((s = prep(k_features<T, N>, 0, rows, &grid, &thr, &sm))) return s;
    k_features<T, N><<<grid, kSwWarps * 32, 0, st>>>(a, plan->xfeat, plan->n_bp_max, 1, 0);
    if ((s = check_launch("gb_sweep(features)"))) return s;
    // rows (w, j) are compact per walker: run the network on the full [W][n_bp_max] block
    if ((s = mdn_forward(plan->net, plan->xfeat, a.d.n_walkers * plan->n_bp_max, plan->rawbuf, st))) return s;
    raw = plan->rawbuf;
  }
  k_mixrows<T><<<(rows + 127) / 128, 128, 0, st>>>(a, raw, plan->raw_table ? 1 : 0,
                                                   reinterpret_cast<MixRow<T>*>(plan->mix));
  return check_launch("gb_sweep(mixture rows)");
}

template <typename T, int N>
static gbk_status run_half(SweepArgs& a, int flags, cudaStream_t st) {
  const gbk_sweep_desc& d = a.d;
  const int nbp = (d.n_bands - a.parity + 1) / 2;
  if (nbp <= 0) return GBK_OK;
  gbk_status s;
  int grid = 0, thr = 0;
  size_t sm = 0;
  if ((s = prep(k_open<T, N>, 0, (int64_t)d.n_walkers * nbp, &grid, &thr, &sm))) return s;
  ev_rec(a.parity, 1, 0, st);
  k_open<T, N><<<grid, kSwWarps * 32, 0, st>>>(a);
  if ((s = check_launch("gb_sweep(open)"))) return s;
  if (a.mix && (s = run_proposal<T, N>(g_active_plan, a, st))) return s;
  ev_rec(a.parity, 1, 1, st);
  if (flags & (GBK_SWEEP_INMODEL | GBK_SWEEP_RJ)) {
    if ((s = prep(k_band<T, N>, sizeof(BandSmem<T, N>), (int64_t)d.n_temps * d.n_walkers * nbp, &grid, &thr, &sm,
                  kBandWarps)))
      return s;
    ev_rec(a.parity, 2, 0, st);
    if (cudaMemsetAsync(a.task_ctr + a.parity, 0, sizeof(unsigned long long), st) != cudaSuccess)
      return set_error(GBK_ECUDA, "gb_sweep: task counter reset failed");
    k_band<T, N><<<grid, thr, sm, st>>>(a, flags);
    ev_rec(a.parity, 2, 1, st);
    if ((s = check_launch("gb_sweep(band)"))) return s;
  }
  if (flags & GBK_SWEEP_SWAP) {
    if ((s = prep(k_swap<T, N>, swap_warp_bytes<T, N>(d.n_temps, d.n_walkers), (int64_t)d.n_walkers * nbp, &grid,
                  &thr, &sm)))
      return s;
    ev_rec(a.parity, 3, 0, st);
    k_swap<T, N><<<grid, thr, sm, st>>>(a);
    ev_rec(a.parity, 3, 1, st);
    if ((s = check_launch("gb_sweep(swap)"))) return s;
  }
  return GBK_OK;
}

template <typename T, int N>
static gbk_status run_sweep_n(gbk_sweep* plan, SweepArgs& a, int flags, cudaStream_t st) {
  gbk_status s;
  if (flags & GBK_SWEEP_REFRESH)
    if ((s = run_refresh<T, N>(a, st))) return s;
  const size_t rbytes = (size_t)a.d.n_walkers * 2 * plan->ctx->grid.n_bins * 2 * sizeof(long long);
  for (int parity = 1; parity >= 0; --parity) {
    a.parity = parity;
    if (cudaMemcpyAsync(plan->rsnap, a.resid, rbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return set_error(GBK_ECUDA, "gb_sweep: residual snapshot copy failed");
    if ((s = run_half<T, N>(a, flags, st))) return s;
  }
  return GBK_OK;
}

template <typename T>
static gbk_status run_sweep(gbk_sweep* plan, SweepArgs& a, int flags, cudaStream_t st) {
  switch (a.d.band_bins) {
    case 128: return run_sweep_n<T, 128>(plan, a, flags, st);
    case 256: return run_sweep_n<T, 256>(plan, a, flags, st);
    case 512: return run_sweep_n<T, 512>(plan, a, flags, st);
    case 1024: return run_sweep_n<T, 1024>(plan, a, flags, st);
    default: return set_error(GBK_EINVAL, "gb_sweep: band_bins %d", a.d.band_bins);
  }
}

}  // namespace gbk

using namespace gbk;

extern "C" gbk_status gbk_sweep_create(gbk_ctx* ctx, const gbk_sweep_desc* desc, gbk_sweep** out_plan) {
  if (!ctx || !desc || !out_plan) return set_error(GBK_EINVAL, "gbk_sweep_create: null argument");
  *out_plan = nullptr;
  const gbk_sweep_desc& d = *desc;
  if (d.n_temps < 1 || d.n_temps > 64 || d.n_walkers < 1 || d.n_walkers > 64 || d.n_bands < 1 || d.n_max < 0 ||
      d.n_max > kMaxSlots - 1 || band_index(d.band_bins) < 0 || d.props_per_source < 0)
    return set_error(GBK_EINVAL, "gbk_sweep_create: bad sizes (T=%d W=%d B=%d n_max=%d N=%d)", d.n_temps,
                     d.n_walkers, d.n_bands, d.n_max, d.band_bins);
  if (d.precision != GBK_MIXED && d.precision != GBK_FP64) return set_error(GBK_EINVAL, "gbk_sweep_create: bad precision");
  const int64_t lo = d.band_k0 - d.band_bins - ctx->grid.k0;
  const int64_t hi = d.band_k0 + (int64_t)(d.n_bands + 1) * d.band_bins - ctx->grid.k0;
  if (lo < 0 || hi > ctx->grid.n_bins)
    return set_error(GBK_ERANGE, "gbk_sweep_create: band windows [%lld, %lld) leave the grid", (long long)lo,
                     (long long)hi);
  if (!(d.f_min < d.f_max) || !(d.mc_min < d.mc_max) || !(d.ln_a_min < d.ln_a_max))
    return set_error(GBK_EINVAL, "gbk_sweep_create: bad prior bounds");
  gbk_sweep* p = (gbk_sweep*)calloc(1, sizeof(gbk_sweep));
  if (!p) return set_error(GBK_ENOMEM, "gbk_sweep_create: host allocation failed");
  p->ctx = ctx;
  p->d = d;
  p->n_bp_max = (d.n_bands + 1) / 2;
  const size_t csz = d.precision == GBK_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t rbytes = (size_t)d.n_walkers * 2 * ctx->grid.n_bins * 2 * sizeof(long long);
  p->rho_bytes = (size_t)d.n_walkers * p->n_bp_max * 2 * 3 * d.band_bins * csz;
  p->cache_bytes = (size_t)d.n_temps * d.n_walkers * d.n_bands * (d.n_max > 0 ? d.n_max : 1) * 2 * d.band_bins * csz;
  p->hsum_bytes = (size_t)d.n_temps * d.n_walkers * d.n_bands * 2 * 3 * d.band_bins * csz;
  cudaError_t e = cudaMalloc((void**)&p->rsnap, rbytes);
  if (e == cudaSuccess) e = cudaMalloc(&p->rho, p->rho_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&p->wcache, p->cache_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&p->hsum, p->hsum_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->setid, (size_t)d.n_temps * d.n_walkers * d.n_bands * sizeof(int32_t));
  p->rwbuf_bytes = (size_t)sms_of_device() * 64 * 2 * 3 * d.band_bins * csz;   // every warp an SM can hold
  if (e == cudaSuccess) e = cudaMalloc(&p->rwbuf, p->rwbuf_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->swap_acc, (size_t)d.n_bands * d.n_temps * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(p->swap_acc, 0, (size_t)d.n_bands * d.n_temps * sizeof(int32_t));
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&p->xfer_dest, (size_t)d.n_walkers * d.n_bands * (d.n_max > 0 ? d.n_max : 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->task_ctr, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    cudaFree(p->rsnap);
    cudaFree(p->rho);
    cudaFree(p->wcache);
    cudaFree(p->hsum);
    cudaFree(p->setid);
    cudaFree(p->rwbuf);
    cudaFree(p->swap_acc);
    cudaFree(p->xfer_dest);
    cudaFree(p->xfer_dest);
    free(p);
    cudaGetLastError();
    return set_error(e == cudaErrorMemoryAllocation ? GBK_ENOMEM : GBK_ECUDA, "gbk_sweep_create: %s",
                     cudaGetErrorString(e));
  }
  *out_plan = p;
  return GBK_OK;
}

extern "C" gbk_status gbk_sweep_destroy(gbk_sweep* plan) {
  if (!plan) return set_error(GBK_EINVAL, "gbk_sweep_destroy: null plan");
  cudaDeviceSynchronize();
  cudaFree(plan->rsnap);
  cudaFree(plan->rho);
  cudaFree(plan->wcache);
  cudaFree(plan->hsum);
  cudaFree(plan->setid);
  cudaFree(plan->rwbuf);
  cudaFree(plan->swap_acc);
  cudaFree(plan->xfer_dest);
  cudaFree(plan->task_ctr);
  cudaFree(plan->mix);
  cudaFree(plan->grp_f0);
  cudaFree(plan->grp_par);
  cudaFree(plan->grp_n);
  cudaFree(plan->xfeat);
  cudaFree(plan->rawbuf);
  if (plan->have_ev)
    for (int p = 0; p < 2; ++p)
      for (int k = 0; k < 4; ++k)
        for (int e = 0; e < 2; ++e) cudaEventDestroy(plan->ev[p][k][e]);
  free(plan);
  return GBK_OK;
}

extern "C" gbk_status gbk_sweep_kernel_ms(gbk_sweep* plan, double* ms_out) {
  if (!plan || !ms_out) return set_error(GBK_EINVAL, "gbk_sweep_kernel_ms: null argument");
  if (!plan->have_ev) return set_error(GBK_EINVAL, "gbk_sweep_kernel_ms: no timed sweep yet");
  for (int k = 0; k < 4; ++k) {
    ms_out[k] = 0.0;
    for (int p = 0; p < 2; ++p) {
      float ms = 0.f;
      if (cudaEventSynchronize(plan->ev[p][k][1]) == cudaSuccess &&
          cudaEventElapsedTime(&ms, plan->ev[p][k][0], plan->ev[p][k][1]) == cudaSuccess)
        ms_out[k] += ms;
      else
        cudaGetLastError();
    }
  }
  return GBK_OK;
}

static gbk_status check_state(gbk_sweep* plan, const double* params, const uint8_t* exists,
                              const gbk_residual* residual, const gbk_psd* psd, const char* what) {
  if (!plan || !residual || !psd) return set_error(GBK_EINVAL, "%s: null plan/struct", what);
  if (!params || !exists || !residual->data || !psd->params) return set_error(GBK_EINVAL, "%s: null device pointer", what);
  if (residual->n_walkers != plan->d.n_walkers || residual->frac_bits < 40 || residual->frac_bits > 120)
    return set_error(GBK_EINVAL, "%s: residual must hold n_walkers = %d walkers", what, plan->d.n_walkers);
  if (psd->n_psd != 1 && psd->n_psd < plan->d.n_walkers) return set_error(GBK_EINVAL, "%s: psd covers too few walkers", what);
  return GBK_OK;
}

static SweepArgs make_args(gbk_sweep* plan, double* params, uint8_t* exists, const double* betas,
                           const gbk_residual* residual, const gbk_psd* psd, uint64_t key, uint32_t sweep_index) {
  SweepArgs a;
  a.c = *plan->ctx;
  a.d = plan->d;
  a.params = params;
  a.exists = exists;
  a.betas = betas;
  a.resid = (long long*)residual->data;
  a.rsnap = plan->rsnap;
  a.rho = plan->rho;
  a.wcache = plan->wcache;
  a.hsum = plan->hsum;
  a.setid = plan->setid;
  a.rwbuf = plan->rwbuf;
  a.task_ctr = plan->task_ctr;
  a.n_bp_max = plan->n_bp_max;
  a.n_walkers_r = residual->n_walkers;
  a.frac_bits = residual->frac_bits;
  a.psdp = psd->params;
  a.npsd = psd->n_psd;
  a.k0 = (uint32_t)(key & 0xffffffffu);
  a.k1 = (uint32_t)(key >> 32);
  a.sweep = sweep_index;
  a.parity = 1;
  a.trace = nullptr;
  a.trace_cap = 0;
  a.trace_count = nullptr;
  a.stats = nullptr;
  a.mix = nullptr;
  a.mdn_eps = plan->mdn_eps;
  a.mdn_inmodel = plan->mdn_inmodel;
  const bool grp = plan->grp_f0 && plan->grp_frac > 0.0;
  a.grp_f0 = grp ? plan->grp_f0 : nullptr;
  a.grp_par = grp ? plan->grp_par : nullptr;
  a.grp_n = grp ? plan->grp_n : nullptr;
  a.gmax = plan->gmax;
  a.n_friends = plan->n_friends;
  a.grp_frac = plan->grp_frac;
  a.swap_acc = plan->swap_acc;
  return a;
}

extern "C" gbk_status gb_sweep(gbk_sweep* plan, double* params, uint8_t* exists, const double* betas,
                               const gbk_residual* residual, const gbk_psd* psd, uint64_t key, uint32_t sweep_index,
                               int32_t flags, const gbk_trace* trace, int64_t* stats, void* stream) {
  gbk_status s0 = check_state(plan, params, exists, residual, psd, "gb_sweep");
  if (s0) return s0;
  if (!betas) return set_error(GBK_EINVAL, "gb_sweep: null betas");
  if (flags & ~(GBK_SWEEP_INMODEL | GBK_SWEEP_RJ | GBK_SWEEP_SWAP | GBK_SWEEP_REFRESH | GBK_SWEEP_TIMING | GBK_SWEEP_MDN))
    return set_error(GBK_EINVAL, "gb_sweep: unknown flags 0x%x", flags);
  if ((flags & GBK_SWEEP_MDN) && !plan->mdn_set)
    return set_error(GBK_EINVAL, "gb_sweep: GBK_SWEEP_MDN without a proposal (gbk_sweep_set_proposal)");
  if (!(flags & GBK_SWEEP_REFRESH) && !plan->refreshed)
    return set_error(GBK_EINVAL, "gb_sweep: the plan's caches are empty (the first call needs GBK_SWEEP_REFRESH)");
  SweepArgs a = make_args(plan, params, exists, betas, residual, psd, key, sweep_index);
  a.trace = trace ? trace->records : nullptr;
  a.trace_cap = trace ? trace->capacity : 0;
  a.trace_count = trace ? trace->count : nullptr;
  a.stats = (long long*)stats;
  a.mix = (flags & GBK_SWEEP_MDN) ? plan->mix : nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  plan->timed = (flags & GBK_SWEEP_TIMING) != 0;
  if (plan->timed && !plan->have_ev) {
    for (int p = 0; p < 2; ++p)
      for (int k = 0; k < 4; ++k)
        for (int e = 0; e < 2; ++e) cudaEventCreate(&plan->ev[p][k][e]);
    plan->have_ev = true;
  }
  if (plan->timed) {   // kernels that do not run this call report 0 ms
    for (int p = 0; p < 2; ++p)
      for (int k = 0; k < 4; ++k) {
        cudaEventRecord(plan->ev[p][k][0], st);
        cudaEventRecord(plan->ev[p][k][1], st);
      }
  }
  if ((flags & GBK_SWEEP_SWAP) &&
      cudaMemsetAsync(plan->swap_acc, 0, (size_t)plan->d.n_bands * plan->d.n_temps * sizeof(int32_t), st) != cudaSuccess)
    return set_error(GBK_ECUDA, "gb_sweep: cannot clear the swap counters");
  g_timing_plan = plan;
  g_active_plan = plan;
  const int fl = flags & ~(GBK_SWEEP_TIMING | GBK_SWEEP_MDN);
  gbk_status s = (plan->d.precision == GBK_MIXED) ? run_sweep<float>(plan, a, fl, st) : run_sweep<double>(plan, a, fl, st);
  if (s == GBK_OK && (flags & GBK_SWEEP_REFRESH)) plan->refreshed = true;
  g_timing_plan = nullptr;
  g_active_plan = nullptr;
  return s;
}

extern "C" gbk_status gbk_sweep_set_proposal(gbk_sweep* plan, gbk_mdn* net, const float* raw_table, double eps,
                                             double inmodel_frac) {
  if (!plan) return set_error(GBK_EINVAL, "gbk_sweep_set_proposal: null plan");
  if (!(eps >= 0.0 && eps <= 1.0) || !(inmodel_frac >= 0.0 && inmodel_frac <= 1.0))
    return set_error(GBK_EINVAL, "gbk_sweep_set_proposal: eps and inmodel_frac must lie in [0, 1]");
  plan->mdn_set = false;
  plan->net = nullptr;
  plan->raw_table = nullptr;
  if (!net && !raw_table) return GBK_OK;   // learned proposal off
  const int64_t rows = (int64_t)plan->d.n_walkers * plan->n_bp_max;
  if (!raw_table) {
    if (plan->d.band_bins != 256)
      return set_error(GBK_ENOTIMPL, "gbk_sweep_set_proposal: the network takes 256-bin bands (band_bins %d)",
                       plan->d.band_bins);
    if (net->max_batch < rows)
      return set_error(GBK_EINVAL, "gbk_sweep_set_proposal: network max_batch %d < %lld windows per half sweep",
                       net->max_batch, (long long)rows);
    if (!net->have_params) return set_error(GBK_EINVAL, "gbk_sweep_set_proposal: network parameters not set");
  }
  const size_t mixb = (size_t)rows * (plan->d.precision == GBK_FP64 ? sizeof(MixRow<double>) : sizeof(MixRow<float>));
  cudaError_t e = cudaSuccess;
  if (!plan->mix) e = cudaMalloc(&plan->mix, mixb);
  if (e == cudaSuccess && !raw_table && !plan->xfeat) {
    e = cudaMalloc((void**)&plan->xfeat, (size_t)rows * 1024 * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMemset(plan->xfeat, 0, (size_t)rows * 1024 * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&plan->rawbuf, (size_t)rows * kMixOut * sizeof(float));
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(GBK_ENOMEM, "gbk_sweep_set_proposal: %s", cudaGetErrorString(e));
  }
  plan->net = raw_table ? nullptr : net;
  plan->raw_table = raw_table;
  plan->mdn_eps = eps;
  plan->mdn_inmodel = inmodel_frac;
  plan->mdn_set = true;
  return GBK_OK;
}

template <typename T>
static gbk_status features_impl(gbk_sweep* plan, SweepArgs& a, uint16_t* x_out, float* u_out, cudaStream_t st) {
  gbk_status s;
  int grid = 0, thr = 0;
  size_t sm = 0;
  a.rsnap = a.resid;   // nothing changes the residual during this call
  for (int parity = 1; parity >= 0; --parity) {
    a.parity = parity;
    const int nbp = (a.d.n_bands - parity + 1) / 2;
    if (nbp <= 0) continue;
    if ((s = prep(k_open<T, 256>, 0, (int64_t)a.d.n_walkers * nbp, &grid, &thr, &sm))) return s;
    k_open<T, 256><<<grid, kSwWarps * 32, 0, st>>>(a);
    if ((s = check_launch("gb_sweep_features(open)"))) return s;
    if (x_out) {
      k_features<T, 256><<<grid, kSwWarps * 32, 0, st>>>(a, x_out, a.d.n_bands, 2, parity);
      if ((s = check_launch("gb_sweep_features(features)"))) return s;
    }
  }
  if (u_out && a.d.n_max > 0) {
    const int64_t n = (int64_t)a.d.n_walkers * a.d.n_bands * a.d.n_max;
    k_cold_unit<<<(int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, st>>>(a, u_out);
    if ((s = check_launch("gb_sweep_features(unit)"))) return s;
  }
  return GBK_OK;
}

extern "C" gbk_status gb_sweep_features(gbk_sweep* plan, const double* params, const uint8_t* exists,
                                        const gbk_residual* residual, const gbk_psd* psd, uint16_t* x_out,
                                        float* u_out, void* stream) {
  gbk_status s = check_state(plan, params, exists, residual, psd, "gb_sweep_features");
  if (s) return s;
  if (plan->d.band_bins != 256)
    return set_error(GBK_ENOTIMPL, "gb_sweep_features: features are defined for 256-bin bands (band_bins %d)",
                     plan->d.band_bins);
  if (x_out && ((uintptr_t)x_out & 3)) return set_error(GBK_EINVAL, "gb_sweep_features: x_out must be 4-byte aligned");
  if (!plan->refreshed)
    return set_error(GBK_EINVAL, "gb_sweep_features: the plan's caches are empty (run gb_sweep with GBK_SWEEP_REFRESH)");
  SweepArgs a = make_args(plan, const_cast<double*>(params), const_cast<uint8_t*>(exists), nullptr, residual, psd, 0, 0);
  cudaStream_t st = (cudaStream_t)stream;
  return plan->d.precision == GBK_MIXED ? features_impl<float>(plan, a, x_out, u_out, st)
                                        : features_impl<double>(plan, a, x_out, u_out, st);
}

extern "C" gbk_status gbk_sweep_update_group(gbk_sweep* plan, const double* params, const uint8_t* exists,
                                             double frac, int32_t n_friends, void* stream) {
  if (!plan) return set_error(GBK_EINVAL, "gbk_sweep_update_group: null plan");
  if (!(frac >= 0.0 && frac <= 1.0) || n_friends < 1)
    return set_error(GBK_EINVAL, "gbk_sweep_update_group: frac must lie in [0, 1] and n_friends >= 1");
  plan->grp_frac = frac;
  plan->n_friends = n_friends;
  if (frac == 0.0) return GBK_OK;
  if (!params || !exists) return set_error(GBK_EINVAL, "gbk_sweep_update_group: null device pointer");
  const gbk_sweep_desc& d = plan->d;
  const int gmax = 3 * d.n_walkers * (d.n_max > 0 ? d.n_max : 1);
  int p2 = 1;
  while (p2 < gmax) p2 <<= 1;
  const size_t smem = (size_t)p2 * (sizeof(double) + sizeof(int32_t));
  if (smem > 200 * 1024)
    return set_error(GBK_ENOTIMPL, "gbk_sweep_update_group: group of %d members exceeds the sort's shared memory", gmax);
  if (!plan->grp_f0) {
    cudaError_t e = cudaMalloc((void**)&plan->grp_f0, (size_t)d.n_bands * gmax * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&plan->grp_par, (size_t)d.n_bands * gmax * 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&plan->grp_n, (size_t)d.n_bands * sizeof(int32_t));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(GBK_ENOMEM, "gbk_sweep_update_group: %s", cudaGetErrorString(e));
    }
    plan->gmax = gmax;
  }
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_group_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return set_error(GBK_ECUDA, "gbk_sweep_update_group: cannot set shared memory size");
  }
  k_group_build<<<d.n_bands, 256, smem, (cudaStream_t)stream>>>(params, exists, d, gmax, p2, plan->grp_f0,
                                                                plan->grp_par, plan->grp_n);
  return check_launch("gbk_sweep_update_group");
}

// Ladder of band b (one thread): Vousden, Farr & Mandel (2016) update from the last sweep's
// swap acceptance A_i = accepted(i-1 <-> i) / W.
__global__ void k_adapt_ladder(double* __restrict__ betas, const int32_t* __restrict__ acc, int nb, int nt, int nw,
                               double kappa) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double* bt = betas + (int64_t)b * nt;
  const bool top_inf = bt[nt - 1] == 0.0;
  const int last = top_inf ? nt - 2 : nt - 1;
  if (last < 1) return;
  double t_prev = 1.0, t_old_prev = 1.0;
  for (int i = 1; i <= last; ++i) {
    const double t_old = 1.0 / bt[i];
    const double ai = (double)acc[(int64_t)b * nt + i] / nw;
    const double an = i + 1 < nt ? (double)acc[(int64_t)b * nt + i + 1] / nw : 0.0;
    const double s = log(t_old - t_old_prev) + kappa * (ai - an);
    t_old_prev = t_old;
    t_prev = t_prev + exp(s);
    bt[i] = 1.0 / t_prev;
  }
}

extern "C" gbk_status gbk_sweep_adapt_temps(gbk_sweep* plan, double* betas, int32_t iteration, double nu, double t0,
                                            void* stream) {
  if (!plan || !betas) return set_error(GBK_EINVAL, "gbk_sweep_adapt_temps: null argument");
  if (!(nu > 0.0) || !(t0 > 0.0) || iteration < 0) return set_error(GBK_EINVAL, "gbk_sweep_adapt_temps: bad schedule");
  const double kappa = t0 / (nu * ((double)iteration + t0));
  const int nb = plan->d.n_bands;
  k_adapt_ladder<<<(nb + 127) / 128, 128, 0, (cudaStream_t)stream>>>(betas, plan->swap_acc, nb, plan->d.n_temps,
                                                                     plan->d.n_walkers, kappa);
  return check_launch("gbk_sweep_adapt_temps");
}

extern "C" gbk_status gbk_sweep_transfer(gbk_sweep* plan, double* params, uint8_t* exists, int32_t* counts,
                                         void* stream) {
  if (!plan) return set_error(GBK_EINVAL, "gbk_sweep_transfer: null plan");
  if (!params || !exists) return set_error(GBK_EINVAL, "gbk_sweep_transfer: null device pointer");
  if (!plan->refreshed)
    return set_error(GBK_EINVAL, "gbk_sweep_transfer: the plan's caches are empty (run gb_sweep with GBK_SWEEP_REFRESH)");
  SweepArgs a;
  memset(&a, 0, sizeof(a));
  a.c = *plan->ctx;
  a.d = plan->d;
  a.params = params;
  a.exists = exists;
  a.wcache = plan->wcache;
  a.hsum = plan->hsum;
  a.setid = plan->setid;
  a.n_bp_max = plan->n_bp_max;
  cudaStream_t st = (cudaStream_t)stream;
  return plan->d.precision == GBK_MIXED ? transfer_n<float>(plan, a, counts, st) : transfer_n<double>(plan, a, counts, st);
}

// ==================================================================== per-band search sampler
// The search-RJ proposal's sampler (Sec. V.E, App. G): for every sub-band an independent,
// parallel-tempered ensemble of single sources with stretch moves in the band's own-bin prior
// box, looking for the highest-likelihood source left in one walker's residual. n_sets such
// searches run side by side, set s on the residual of walker w0 + s; their bands are
// flattened, fb = s n_bands + b (band geometry b = fb mod n_bands).
struct gbk_search {
  gbk_ctx* ctx;
  gbk_search_desc d;   // n_sets >= 1
  void* rw;            // residual windows [n_sets B][2][3N] of the sampler's precision
  bool have_windows;
};

namespace gbk {

constexpr int kSearchWarps = 4;

struct SearchArgs {
  SweepArgs sa;        // context, PSD and the residual windows (sa.rho) for the shared helpers
  gbk_search_desc d;
  int nbt;             // n_sets x n_bands (flattened index fb)
  double* u;           // [nbt][T][W][8]
  double* ell;         // [nbt][T][W]
  const double* betas; // [nbt][T]
  int psd_walker;      // PSD row of set 0; set s uses psd_walker + s (a one-row PSD: row 0)
  long long* stats;    // [2][2]: stretch proposals, accepted; swaps, accepted
  const int32_t* stall;  // [nbt] sweeps without a better point (NULL: no convergence test)
  int stall_limit;       // a band with stall >= stall_limit has converged: left as it is
};

// Has band fb's search converged (App. G: n_it,max sweeps without a better point)?
__device__ __forceinline__ bool search_frozen(const SearchArgs& a, int fb) {
  return a.stall && a.stall_limit > 0 && a.stall[fb] >= a.stall_limit;
}

// per warp: the FFT buffers and the set-up of a batch of 32 chains (one lane each)
template <typename T, int N>
struct SearchSmem {
  typename CT<T>::C ba[2 * N], bs[2 * N];
  Src<T> src[32];
  double y[32][8];
  double lz[32];
  int inb[32];
};

// Source parameters of unit coordinates u in band b's own-bin box (f0 over [lo_b, hi_b)),
// rounded step by step as written (no contraction).
__device__ __forceinline__ void search_from_unit(const gbk_search_desc& d, double tobs, int b, const double* u,
                                                 double* th) {
  const long long lob = d.band_k0 + (long long)b * d.band_bins;
  const double lo = __ddiv_rn((double)lob, tobs), hi = __ddiv_rn((double)(lob + d.band_bins), tobs);
  const double f0 = dadd(lo, dmul(dsub(hi, lo), u[1]));
  const double mc = dadd(d.mc_min, dmul(dsub(d.mc_max, d.mc_min), u[2]));
  th[0] = exp(dadd(d.ln_a_min, dmul(dsub(d.ln_a_max, d.ln_a_min), u[0])));
  th[1] = f0;
  th[2] = fdot_of(f0, mc, double());
  th[3] = dmul(6.283185307179586, u[3]);
  th[4] = dmul(3.141592653589793, u[4]);
  th[5] = dsub(dmul(2.0, u[5]), 1.0);
  th[6] = dsub(dmul(2.0, u[6]), 1.0);
  th[7] = dmul(6.283185307179586, u[7]);
}

template <typename T, int N>
__device__ __forceinline__ const typename CT<T>::C* search_window(const SearchArgs& a, int fb) {
  return reinterpret_cast<const typename CT<T>::C*>(a.sa.rho) + (int64_t)fb * 2 * 3 * N;
}

// Set-up of one source (one lane): parameters of u in band fb's box and the waveform constants.
template <typename T, int N>
__device__ __forceinline__ void search_prep(const SearchArgs& a, SearchSmem<T, N>& S, int q, int fb, const double* u) {
  double th[8];
  search_from_unit(a.d, a.sa.c.grid.tobs, fb % a.d.n_bands, u, th);
  S.src[q] = make_src<T>(th, 1, 0, a.sa.c.grid.tobs, N);
}

// l = <R|h> - 1/2 <h|h> on band fb's window for the prepared source q (the birth Delta lnL,
// Eq. addsource), with the PSD of the set's walker; whole warp.
template <typename T, int N>
__device__ double search_ell(const SearchArgs& a, SearchSmem<T, N>& S, int q, int fb, int lane) {
  gen_band<T, N>(&S.src[q], orb_of<T>(a.sa.c, band_index(N)), tw_of<T>(a.sa.c, band_index(N)), a.sa.c.grid.tobs,
                 S.ba, S.bs, lane);
  const int b = fb % a.d.n_bands;
  const int64_t gw = a.d.band_k0 + (int64_t)(b - 1) * N - a.sa.c.grid.k0;
  const int oa = band_off<N>(S.src[q].q, gw, a.sa.c);
  const PsdWt<T> pw = walker_psd<T>(a.sa, a.psd_walker + (a.sa.npsd > 1 ? fb / a.d.n_bands : 0));
  const double l = window_dll<T, N, false>(a.sa, search_window<T, N>(a, fb), S.ba, oa, (const typename CT<T>::C*)nullptr, 0,
                                    gw, pw, lane);
  __syncwarp();
  return l;
}

// residual windows: R of walker w0 + s on the three sub-bands of every band of set s
template <typename T, int N>
__global__ void __launch_bounds__(kSearchWarps * 32) k_search_windows(const SearchArgs a, const long long* resid,
                                                                      int64_t n_bins, int walker, int frac_bits) {
  typedef typename CT<T>::C C;
  constexpr int W3 = 3 * N;
  const int lane = threadIdx.x & 31;
  const int fb = blockIdx.x * kSearchWarps + (threadIdx.x >> 5);
  if (fb >= a.nbt) return;
  const int b = fb % a.d.n_bands;
  const T rs = (T)ldexp(1.0, kStrainExp - frac_bits);
  const int64_t gw = a.d.band_k0 + (int64_t)(b - 1) * N - a.sa.c.grid.k0;
  const long long* rw = resid + (int64_t)(walker + fb / a.d.n_bands) * 2 * n_bins * 2;
  C* out = reinterpret_cast<C*>(a.sa.rho) + (int64_t)fb * 2 * W3;
  for (int i = lane; i < W3; i += 32)
    for (int ch = 0; ch < 2; ++ch) {
      const longlong2 v = *reinterpret_cast<const longlong2*>(rw + 2 * (ch * n_bins + gw + i));
      out[ch * W3 + i] = mkc(i2t(v.x, T()) * rs, i2t(v.y, T()) * rs);
    }
}

// walkers from the prior: u = u32 of 8 Philox words at (chain, m, 9, seed), m = 0, 1
__global__ void k_search_init(double* u, int n, uint32_t seed, uint32_t k0, uint32_t k1) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int m = 0; m < 2; ++m) {
    const U4 v = philox4x32_10((uint32_t)c, (uint32_t)m, 9u, seed, k0, k1);
    u[(int64_t)c * 8 + 4 * m] = u32(v.x);
    u[(int64_t)c * 8 + 4 * m + 1] = u32(v.y);
    u[(int64_t)c * 8 + 4 * m + 2] = u32(v.z);
    u[(int64_t)c * 8 + 4 * m + 3] = u32(v.w);
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(kSearchWarps * 32) k_search_eval(const SearchArgs a, int bs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  SearchSmem<T, N>& S = reinterpret_cast<SearchSmem<T, N>*>(smem_raw)[wid];
  const int n = a.nbt * a.d.n_temps * a.d.n_walkers;
  const int per = a.d.n_temps * a.d.n_walkers;
  // batches of bs <= 32 chains per warp: the float64 set-up lane-parallel, then one waveform at a time
  for (int g0 = (blockIdx.x * wpc + wid) * bs; g0 < n; g0 += gridDim.x * wpc * bs) {
    const int cnt = min(bs, n - g0);
    if (lane < cnt) search_prep<T, N>(a, S, lane, (g0 + lane) / per, a.u + (int64_t)(g0 + lane) * 8);
    __syncwarp();
    for (int q = 0; q < cnt; ++q) {
      const double l = search_ell<T, N>(a, S, q, (g0 + q) / per, lane);
      if (lane == 0) a.ell[g0 + q] = l;
    }
    __syncwarp();
  }
}

// Stretch moves of half h (one warp per batch of 32 chains of the half): partner from the other half, z
// from g(z) ~ 1/sqrt(z) on [1/a, a], Y = X_j + z (X_k - X_j) in the unit box, acceptance
// ln u < beta (l_Y - l_X) + 7 ln z; a Y outside [0, 1]^8 is rejected without a likelihood.
template <typename T, int N>
__global__ void __launch_bounds__(kSearchWarps * 32) k_search_half(const SearchArgs a, int h, uint32_t sweep,
                                                                   uint32_t k0, uint32_t k1, int bs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  SearchSmem<T, N>& S = reinterpret_cast<SearchSmem<T, N>*>(smem_raw)[wid];
  const int T_ = a.d.n_temps, W = a.d.n_walkers, half = W / 2;
  const int n = a.nbt * T_ * half;
  // batches of bs <= 32 chains of the half per warp: words, partner, z, Y, box test and the
  // float64 source set-up lane-parallel, then the waveforms and decisions one chain at a time
  for (int g0 = (blockIdx.x * wpc + wid) * bs; g0 < n; g0 += gridDim.x * wpc * bs) {
    const int cnt = min(bs, n - g0);
    bool live = false;
    if (lane < cnt) {
      const int e = g0 + lane;
      const int fb = e / (T_ * half), r = e % (T_ * half);
      const int t = r / half, k = h * half + r % half;
      const int64_t ck = ((int64_t)fb * T_ + t) * W + k;
      live = !search_frozen(a, fb);
      const U4 wv = philox4x32_10((uint32_t)ck, (uint32_t)h, 7u, sweep, k0, k1);
      const int j = (1 - h) * half + (int)ranged(wv.x, (uint32_t)half);
      const double zz = dadd(dmul(dsub(a.d.stretch_a, 1.0), u32(wv.y)), 1.0);
      const double z = __ddiv_rn(dmul(zz, zz), a.d.stretch_a);
      const double* xk = a.u + ck * 8;
      const double* xj = a.u + (ck - k + j) * 8;
      int inb = 1;
      for (int c = 0; c < 8; ++c) {
        const double y = dadd(xj[c], dmul(z, dsub(xk[c], xj[c])));
        S.y[lane][c] = y;
        if (!(y >= 0.0 && y <= 1.0)) inb = 0;
      }
      if (!live) inb = 0;   // a converged band: no move (and not counted)
      S.inb[lane] = inb;
      S.lz[lane] = log(z);
      if (inb) search_prep<T, N>(a, S, lane, fb, S.y[lane]);
    }
    const int n_live = __popc(__ballot_sync(0xffffffffu, live));
    __syncwarp();
    int n_acc = 0;
    for (int q = 0; q < cnt; ++q) {
      const int e = g0 + q;
      const int fb = e / (T_ * half), r = e % (T_ * half);
      const int t = r / half, k = h * half + r % half;
      const int64_t ck = ((int64_t)fb * T_ + t) * W + k;
      if (!S.inb[q]) continue;
      const double ly = search_ell<T, N>(a, S, q, fb, lane);
      const U4 wv = philox4x32_10((uint32_t)ck, (uint32_t)h, 7u, sweep, k0, k1);
      const double ul = u53(wv.z, wv.w);
      const double lu = ul > 0.0 ? log(ul) : -INFINITY;
      const double la = a.betas[(int64_t)fb * T_ + t] * (ly - a.ell[ck]) + 7.0 * S.lz[q];
      const bool acc = __shfl_sync(0xffffffffu, (int)(lu < la), 0) != 0;
      if (acc) {
        if (lane == 0) a.ell[ck] = ly;
        if (lane < 8) a.u[ck * 8 + lane] = S.y[q][lane];
        ++n_acc;
      }
    }
    if (lane == 0 && a.stats) {
      atomicAdd((unsigned long long*)&a.stats[0], (unsigned long long)n_live);
      if (n_acc) atomicAdd((unsigned long long*)&a.stats[1], (unsigned long long)n_acc);
    }
    __syncwarp();
  }
}

// Tempering swaps of walker index w between t and t-1, from the top down (one thread per (fb, w)).
__global__ void k_search_swap(const SearchArgs a, uint32_t sweep, uint32_t k0, uint32_t k1) {
  const int T_ = a.d.n_temps, W = a.d.n_walkers;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= a.nbt * W) return;
  const int b = x / W, w = x % W;   // b: the flattened band index fb
  if (search_frozen(a, b)) return;
  int n = 0, na = 0;
  for (int t = T_ - 1; t > 0; --t) {
    const U4 wv = philox4x32_10((uint32_t)x, (uint32_t)t, 8u, sweep, k0, k1);
    const double ul = u53(wv.x, wv.y);
    const double lu = ul > 0.0 ? log(ul) : -INFINITY;
    const int64_t i1 = ((int64_t)b * T_ + t) * W + w, i0 = i1 - W;
    const double la = (a.betas[(int64_t)b * T_ + t - 1] - a.betas[(int64_t)b * T_ + t]) * (a.ell[i1] - a.ell[i0]);
    ++n;
    if (lu < la) {
      ++na;
      const double tl = a.ell[i1];
      a.ell[i1] = a.ell[i0];
      a.ell[i0] = tl;
      for (int c = 0; c < 8; ++c) {
        const double tu = a.u[i1 * 8 + c];
        a.u[i1 * 8 + c] = a.u[i0 * 8 + c];
        a.u[i0 * 8 + c] = tu;
      }
    }
  }
  if (a.stats && n) {
    atomicAdd((unsigned long long*)&a.stats[2], (unsigned long long)n);
    atomicAdd((unsigned long long*)&a.stats[3], (unsigned long long)na);
  }
}

// best point of every band: the largest cold-chain l (first walker on ties) if it improves
// (b: the flattened band index fb)
__global__ void k_search_best(const SearchArgs a, double* best_ell, double* best_u, int32_t* stall) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.nbt || search_frozen(a, b)) return;
  const int W = a.d.n_walkers;
  const double* l = a.ell + (int64_t)b * a.d.n_temps * W;
  int k = 0;
  for (int i = 1; i < W; ++i)
    if (l[i] > l[k]) k = i;
  if (l[k] > best_ell[b]) {
    best_ell[b] = l[k];
    for (int c = 0; c < 8; ++c) best_u[(int64_t)b * 8 + c] = a.u[((int64_t)b * a.d.n_temps * W + k) * 8 + c];
    stall[b] = 0;
  } else {
    stall[b] += 1;
  }
}

// Relaunch around the best points: every chain of a band with a best point becomes
// clip(best + sigma z, 0, 1), z standard normal by Box-Muller on the Philox words of counters
// (chain, m, 10, seed), m = 0, 1 (word pairs (2i, 2i + 1) -> z_2i, z_2i+1). One thread per chain.
__global__ void k_search_ball(double* __restrict__ u, const double* __restrict__ best_ell,
                              const double* __restrict__ best_u, int n_bands, int per_band, double sigma,
                              uint32_t seed, uint32_t k0, uint32_t k1) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_bands * per_band) return;
  const int b = c / per_band;
  if (!(best_ell[b] > -INFINITY)) return;
  uint32_t w[8];
  for (int m = 0; m < 2; ++m) {
    const U4 v = philox4x32_10((uint32_t)c, (uint32_t)m, 10u, seed, k0, k1);
    w[4 * m] = v.x; w[4 * m + 1] = v.y; w[4 * m + 2] = v.z; w[4 * m + 3] = v.w;
  }
  for (int i = 0; i < 4; ++i) {
    const double r = sqrt(-2.0 * log(u32(w[2 * i])));
    const double an = 2.0 * 3.141592653589793 * u32(w[2 * i + 1]);
    const double z[2] = {dmul(r, cos(an)), dmul(r, sin(an))};
    for (int j = 0; j < 2; ++j) {
      const int d = 2 * i + j;
      const double x = dadd(best_u[(int64_t)b * 8 + d], dmul(sigma, z[j]));
      u[(int64_t)c * 8 + d] = x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
    }
  }
}

// Training points of the search-RJ mixtures: the cold walkers of every band in the sampler's
// unit coordinates (f0 over the band's allowance, clipped to [f_min, f_max]), NaN rows for a
// band whose best point has sqrt(2 l_best) < snr_min. One thread per (band, walker).
__global__ void k_search_samples(const SearchArgs a, const double* __restrict__ best_ell, double snr_min,
                                 double f_min, double f_max, float* __restrict__ x, int n_rows, int row0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int W = a.d.n_walkers;
  if (i >= a.nbt * W) return;
  const int fb = i / W, k = i % W, b = fb % a.d.n_bands;
  float* o = x + ((int64_t)fb * n_rows + row0 + k) * 8;
  const double be = best_ell[fb];
  if (!(be > 0.0 && sqrt(2.0 * be) >= snr_min)) {
    for (int c = 0; c < 8; ++c) o[c] = __int_as_float(0x7fc00000);
    return;
  }
  const double* u = a.u + ((int64_t)fb * a.d.n_temps * W + k) * 8;
  const double tobs = a.sa.c.grid.tobs;
  const long long lob = a.d.band_k0 + (long long)b * a.d.band_bins;
  const double lo = __ddiv_rn((double)lob, tobs), hi = __ddiv_rn((double)(lob + a.d.band_bins), tobs);
  const double f0 = dadd(lo, dmul(dsub(hi, lo), u[1]));
  const double half = 0.5 * a.d.band_bins;
  double alo = __ddiv_rn(dsub((double)lob, half), tobs), ahi = __ddiv_rn(dadd((double)(lob + a.d.band_bins), half), tobs);
  if (alo < f_min) alo = f_min;
  if (ahi > f_max) ahi = f_max;
  for (int c = 0; c < 8; ++c) o[c] = (float)u[c];
  o[1] = (float)__ddiv_rn(dsub(f0, alo), dsub(ahi, alo));
}

// chains per warp batch: the fewest that let one wave of the resident warps take all n chains,
// at most 32 (one lane each), at least 4. (Sized for ~12 warps per SM and rounded down, the
// bench's 23,616 chains per half made 1968 batches for 1824 resident warps: two waves, and the
// sweep took 32 % longer.)
static int search_batch(int64_t n, int64_t resident_warps) {
  const int64_t slots = resident_warps > 0 ? resident_warps : 1;
  const int64_t per = (n + slots - 1) / slots;
  return per < 4 ? 4 : (per > 32 ? 32 : (int)per);
}

// launch shapes from prep(): warps per CTA fitted to the per-warp shared memory (float64 at
// N = 1024 takes 64 KB per warp), grid capped at the resident CTAs
template <typename T, int N>
static gbk_status search_launch(SearchArgs& a, int what, uint32_t sweep, uint32_t k0, uint32_t k1, cudaStream_t st) {
  int grid = 0, thr = 0;
  size_t sm = 0;
  gbk_status s;
  int64_t slots = 0;
  if (what == 0) {
    const int64_t n = (int64_t)a.nbt * a.d.n_temps * a.d.n_walkers;
    if ((s = prep(k_search_eval<T, N>, sizeof(SearchSmem<T, N>), 1, &grid, &thr, &sm, kSearchWarps, &slots))) return s;
    const int bs = search_batch(n, slots);
    if ((s = prep(k_search_eval<T, N>, sizeof(SearchSmem<T, N>), (n + bs - 1) / bs, &grid, &thr, &sm, kSearchWarps)))
      return s;
    k_search_eval<T, N><<<grid, thr, sm, st>>>(a, bs);
    return check_launch("gb_search_eval");
  }
  const int64_t n = (int64_t)a.nbt * a.d.n_temps * (a.d.n_walkers / 2);
  if ((s = prep(k_search_half<T, N>, sizeof(SearchSmem<T, N>), 1, &grid, &thr, &sm, kSearchWarps, &slots))) return s;
  const int bs = search_batch(n, slots);
  if ((s = prep(k_search_half<T, N>, sizeof(SearchSmem<T, N>), (n + bs - 1) / bs, &grid, &thr, &sm, kSearchWarps)))
    return s;
  for (int h = 0; h < 2; ++h) {
    k_search_half<T, N><<<grid, thr, sm, st>>>(a, h, sweep, k0, k1, bs);
    if ((s = check_launch("gb_search_sweep(stretch)"))) return s;
  }
  return GBK_OK;
}

template <typename T>
static gbk_status search_dispatch(SearchArgs& a, int what, uint32_t sweep, uint32_t k0, uint32_t k1, cudaStream_t st) {
  switch (a.d.band_bins) {
    case 128: return search_launch<T, 128>(a, what, sweep, k0, k1, st);
    case 256: return search_launch<T, 256>(a, what, sweep, k0, k1, st);
    case 512: return search_launch<T, 512>(a, what, sweep, k0, k1, st);
    case 1024: return search_launch<T, 1024>(a, what, sweep, k0, k1, st);
    default: return set_error(GBK_EINVAL, "gb_search: band_bins %d", a.d.band_bins);
  }
}

static SearchArgs search_args(gbk_search* p, double* u, double* ell, const double* betas, const gbk_psd* psd,
                              int psd_walker) {
  SearchArgs a;
  memset(&a, 0, sizeof(a));
  a.sa.c = *p->ctx;
  a.sa.rho = p->rw;
  if (psd) {
    a.sa.psdp = psd->params;
    a.sa.npsd = psd->n_psd;
  }
  a.d = p->d;
  a.nbt = p->d.n_sets * p->d.n_bands;
  a.u = u;
  a.ell = ell;
  a.betas = betas;
  a.psd_walker = psd_walker;
  return a;
}

}  // namespace gbk

extern "C" gbk_status gbk_search_create(gbk_ctx* ctx, const gbk_search_desc* desc, gbk_search** out) {
  if (!ctx || !desc || !out) return set_error(GBK_EINVAL, "gbk_search_create: null argument");
  *out = nullptr;
  gbk_search_desc d = *desc;
  if (d.n_sets == 0) d.n_sets = 1;
  if (d.n_bands < 1 || d.n_temps < 1 || d.n_walkers < 4 || (d.n_walkers & 1) || band_index(d.band_bins) < 0 ||
      d.n_sets < 1 || (int64_t)d.n_sets * d.n_bands * d.n_temps * d.n_walkers > (1 << 26))
    return set_error(GBK_EINVAL, "gbk_search_create: bad sizes (S=%d B=%d T=%d W=%d N=%d; W even, >= 4)", d.n_sets,
                     d.n_bands, d.n_temps, d.n_walkers, d.band_bins);
  if (d.precision != GBK_MIXED && d.precision != GBK_FP64) return set_error(GBK_EINVAL, "gbk_search_create: bad precision");
  if (d.stall_limit < 0) return set_error(GBK_EINVAL, "gbk_search_create: stall_limit < 0");
  if (!(d.stretch_a > 1.0) || !(d.ln_a_min < d.ln_a_max) || !(d.mc_min < d.mc_max) || !(d.mc_min > 0.0))
    return set_error(GBK_EINVAL, "gbk_search_create: bad prior bounds or stretch scale");
  const int64_t lo = d.band_k0 - d.band_bins - ctx->grid.k0;
  const int64_t hi = d.band_k0 + (int64_t)(d.n_bands + 1) * d.band_bins - ctx->grid.k0;
  if (lo < 0 || hi > ctx->grid.n_bins)
    return set_error(GBK_ERANGE, "gbk_search_create: band windows [%lld, %lld) leave the grid", (long long)lo,
                     (long long)hi);
  gbk_search* p = (gbk_search*)calloc(1, sizeof(gbk_search));
  if (!p) return set_error(GBK_ENOMEM, "gbk_search_create: host allocation");
  p->ctx = ctx;
  p->d = d;
  const size_t csz = d.precision == GBK_MIXED ? sizeof(float2) : sizeof(double2);
  if (cudaMalloc(&p->rw, (size_t)d.n_sets * d.n_bands * 2 * 3 * d.band_bins * csz) != cudaSuccess) {
    cudaGetLastError();
    free(p);
    return set_error(GBK_ENOMEM, "gbk_search_create: device allocation");
  }
  *out = p;
  return GBK_OK;
}

extern "C" gbk_status gbk_search_destroy(gbk_search* p) {
  if (!p) return set_error(GBK_EINVAL, "gbk_search_destroy: null plan");
  cudaDeviceSynchronize();
  cudaFree(p->rw);
  free(p);
  return GBK_OK;
}

extern "C" gbk_status gb_search_init(gbk_search* p, double* u, uint64_t key, uint32_t seed, void* stream) {
  if (!p || !u) return set_error(GBK_EINVAL, "gb_search_init: null argument");
  const int n = p->d.n_sets * p->d.n_bands * p->d.n_temps * p->d.n_walkers;
  k_search_init<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(u, n, seed, (uint32_t)(key & 0xffffffffu),
                                                                   (uint32_t)(key >> 32));
  return check_launch("gb_search_init");
}

extern "C" gbk_status gb_search_windows(gbk_search* p, const gbk_residual* residual, int32_t walker, void* stream) {
  if (!p || !residual || !residual->data) return set_error(GBK_EINVAL, "gb_search_windows: null argument");
  if (walker < 0 || walker + p->d.n_sets > residual->n_walkers || residual->frac_bits < 40 || residual->frac_bits > 120)
    return set_error(GBK_EINVAL, "gb_search_windows: walkers [%d, %d) outside the residual's %d", walker,
                     walker + p->d.n_sets, residual->n_walkers);
  SearchArgs a = search_args(p, nullptr, nullptr, nullptr, nullptr, 0);
  const int grid = (a.nbt + kSearchWarps - 1) / kSearchWarps;
  cudaStream_t st = (cudaStream_t)stream;
  const long long* r = (const long long*)residual->data;
  const int64_t nb = p->ctx->grid.n_bins;
#define GBK_SW(TT, NN) k_search_windows<TT, NN><<<grid, kSearchWarps * 32, 0, st>>>(a, r, nb, walker, residual->frac_bits)
  const bool mixed = p->d.precision == GBK_MIXED;
  switch (p->d.band_bins) {
    case 128: if (mixed) GBK_SW(float, 128); else GBK_SW(double, 128); break;
    case 256: if (mixed) GBK_SW(float, 256); else GBK_SW(double, 256); break;
    case 512: if (mixed) GBK_SW(float, 512); else GBK_SW(double, 512); break;
    default: if (mixed) GBK_SW(float, 1024); else GBK_SW(double, 1024); break;
  }
#undef GBK_SW
  p->have_windows = true;
  return check_launch("gb_search_windows");
}

extern "C" gbk_status gb_search_eval(gbk_search* p, const double* u, double* ell, const gbk_psd* psd, int32_t psd_walker,
                                     void* stream) {
  if (!p || !u || !ell || !psd || !psd->params) return set_error(GBK_EINVAL, "gb_search_eval: null argument");
  if (!p->have_windows) return set_error(GBK_EINVAL, "gb_search_eval: no residual windows (gb_search_windows)");
  if (psd_walker < 0 || (psd->n_psd != 1 && psd_walker + p->d.n_sets > psd->n_psd))
    return set_error(GBK_EINVAL, "gb_search_eval: PSD rows [%d, %d) outside the PSD's %d", psd_walker,
                     psd_walker + p->d.n_sets, psd->n_psd);
  SearchArgs a = search_args(p, const_cast<double*>(u), ell, nullptr, psd, psd_walker);
  cudaStream_t st = (cudaStream_t)stream;
  return p->d.precision == GBK_MIXED ? search_dispatch<float>(a, 0, 0, 0, 0, st) : search_dispatch<double>(a, 0, 0, 0, 0, st);
}

extern "C" gbk_status gb_search_sweep(gbk_search* p, double* u, double* ell, const double* betas, const gbk_psd* psd,
                                      int32_t psd_walker, uint64_t key, uint32_t sweep_index, double* best_ell,
                                      double* best_u, int32_t* stall, int64_t* stats, void* stream) {
  if (!p || !u || !ell || !betas || !psd || !psd->params) return set_error(GBK_EINVAL, "gb_search_sweep: null argument");
  if (!p->have_windows) return set_error(GBK_EINVAL, "gb_search_sweep: no residual windows (gb_search_windows)");
  if (psd_walker < 0 || (psd->n_psd != 1 && psd_walker + p->d.n_sets > psd->n_psd))
    return set_error(GBK_EINVAL, "gb_search_sweep: PSD rows [%d, %d) outside the PSD's %d", psd_walker,
                     psd_walker + p->d.n_sets, psd->n_psd);
  if ((best_ell || best_u || stall) && !(best_ell && best_u && stall))
    return set_error(GBK_EINVAL, "gb_search_sweep: best_ell, best_u and stall go together");
  if (p->d.stall_limit > 0 && !stall)
    return set_error(GBK_EINVAL, "gb_search_sweep: a plan with a stall limit needs best_ell, best_u and stall");
  SearchArgs a = search_args(p, u, ell, betas, psd, psd_walker);
  a.stats = (long long*)stats;
  a.stall = stall;
  a.stall_limit = p->d.stall_limit;
  const uint32_t k0 = (uint32_t)(key & 0xffffffffu), k1 = (uint32_t)(key >> 32);
  cudaStream_t st = (cudaStream_t)stream;
  gbk_status s = p->d.precision == GBK_MIXED ? search_dispatch<float>(a, 1, sweep_index, k0, k1, st)
                                             : search_dispatch<double>(a, 1, sweep_index, k0, k1, st);
  if (s) return s;
  if (p->d.n_temps > 1) {
    const int n = a.nbt * p->d.n_walkers;
    k_search_swap<<<(n + 127) / 128, 128, 0, st>>>(a, sweep_index, k0, k1);
    if ((s = check_launch("gb_search_sweep(swap)"))) return s;
  }
  if (best_ell) {
    k_search_best<<<(a.nbt + 127) / 128, 128, 0, st>>>(a, best_ell, best_u, stall);
    if ((s = check_launch("gb_search_sweep(best)"))) return s;
  }
  return GBK_OK;
}

extern "C" gbk_status gb_search_samples(gbk_search* p, const double* u, const double* best_ell, double snr_min,
                                        double f_min, double f_max, float* x, int32_t n_rows, int32_t row0,
                                        void* stream) {
  if (!p || !u || !best_ell || !x) return set_error(GBK_EINVAL, "gb_search_samples: null argument");
  if (row0 < 0 || (int64_t)row0 + p->d.n_walkers > n_rows)
    return set_error(GBK_EINVAL, "gb_search_samples: rows [%d, %d) outside %d", row0, row0 + p->d.n_walkers, n_rows);
  if (!(f_min < f_max)) return set_error(GBK_EINVAL, "gb_search_samples: f_min >= f_max");
  SearchArgs a = search_args(p, const_cast<double*>(u), nullptr, nullptr, nullptr, 0);
  const int n = a.nbt * p->d.n_walkers;
  k_search_samples<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(a, best_ell, snr_min, f_min, f_max, x, n_rows,
                                                                       row0);
  return check_launch("gb_search_samples");
}

extern "C" gbk_status gb_search_ball(gbk_search* p, double* u, const double* best_ell, const double* best_u,
                                     double sigma, uint64_t key, uint32_t seed, void* stream) {
  if (!p || !u || !best_ell || !best_u) return set_error(GBK_EINVAL, "gb_search_ball: null argument");
  if (!(sigma > 0.0)) return set_error(GBK_EINVAL, "gb_search_ball: sigma must be > 0");
  const int per = p->d.n_temps * p->d.n_walkers;
  const int nbt = p->d.n_sets * p->d.n_bands;
  const int n = nbt * per;
  k_search_ball<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(u, best_ell, best_u, nbt, per, sigma, seed,
                                                                  (uint32_t)(key & 0xffffffffu), (uint32_t)(key >> 32));
  return check_launch("gb_search_ball");
}
