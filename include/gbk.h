/*
 * gbk.h -- C ABI of the GB300 Galactic-Binary likelihood library (libgbk.so).
 *
 * The library computes the hot path of the GPU global fit of arXiv:2405.04690 for
 * Galactic binaries (GBs): the TDI A/E frequency-domain waveform of each source over its
 * local band by the fast/slow decomposition (Sec. II.A, App. F), the noise-weighted
 * inner products against a residual and PSD (Eq. inner), the change in log-likelihood
 * for in-model, birth/death and swap moves (Eq. addsource, Eq. swapsource), the
 * residual update when templates enter or leave the model (Alg. 1, Alg. 2), the
 * parametric noise PSD (Eq. psd) and the full log-likelihood (Eq. like).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every pointer argument whose name is not `ctx`, `out_ctx` or a host struct is a
 *   DEVICE pointer owned by the caller. The library reads or writes it only during the
 *   stream-ordered execution of the call and never frees or keeps it.
 * - Host structs (gbk_grid, gbk_residual, gbk_psd) are read during the call only.
 * - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the legacy default
 *   stream) and returns a gbk_status for argument and launch errors, with a message in
 *   gbk_last_error(). Errors found by a kernel (a band outside the residual window, an
 *   unsupported band length, a walker index out of range) set a device error word that
 *   gbk_sync_status() reads after synchronising the stream; the offending item is
 *   skipped, nothing out of bounds is touched.
 * - Source parameters are SoA float64 [8][n] in the order
 *   A (strain amplitude, >= 0; 0 gives an identically zero template), f0 [Hz],
 *   fdot [Hz/s], phi0 [rad], psi [rad], cos(iota), sin(beta) (ecliptic latitude),
 *   lambda [rad] (ecliptic longitude).
 * - Band lengths N are 128, 256, 512 or 1024 bins; the band of a source covers absolute
 *   frequency bins [q - N/2, q + N/2) with q = floor(f0 * Tobs) (bin k is f = k / Tobs).
 * - Frequency-domain values are complex, stored as interleaved (re, im) pairs, in the
 *   physical normalisation x~(f_k) = dt * sum_n x(t_n) exp(-2 pi i k n / N_t).
 * - A and E share one PSD per walker, given by its two amplitudes
 *   (sqrt(S_oms) [m/sqrt(Hz)], sqrt(S_acc) [m s^-2/sqrt(Hz)]) through Eq. psd.
 */
#ifndef GBK_H
#define GBK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gbk_status {
  GBK_OK = 0,
  GBK_EINVAL = 1,    /* bad argument (null pointer, size, enum value) */
  GBK_ERANGE = 2,    /* a band fell outside the residual window, or an index out of range */
  GBK_ENOMEM = 3,    /* device allocation failed (only the create calls and the plan set-up
                        calls gbk_sweep_set_proposal / gbk_sweep_update_group allocate) */
  GBK_ECUDA = 4,     /* a CUDA runtime call or kernel launch failed */
  GBK_ETIMEOUT = 5,  /* a device-side wait gave up after its iteration limit */
  GBK_ENOTIMPL = 6   /* combination not implemented */
} gbk_status;

/* Arithmetic of the waveform and inner-product steps.
 * GBK_FP64: everything in float64 (the plain method).
 * GBK_MIXED: float64 only for the carrier-bin offset delta = f0 T - q, fdot T^2 and the
 *            final per-result sums; slow-part response, band FFT and per-bin products in
 *            float32 with compensated float32 accumulation. */
typedef enum gbk_precision { GBK_FP64 = 0, GBK_MIXED = 1 } gbk_precision;

/* Observation grid and residual window. */
typedef struct gbk_grid {
  double tobs;     /* observation time T [s]; df = 1 / T (Eq. inner's Delta f) */
  double dt;       /* sampling cadence [s]; T / dt must be a multiple of 1024 */
  int64_t k0;      /* first absolute frequency bin of the residual window, >= 1 */
  int64_t n_bins;  /* bins in the window, >= 1; (k0 + n_bins) / tobs < c / (2L) */
} gbk_grid;

/* Residual d - H of every walker as int64 fixed point: value = integer * 2^-frac_bits.
 * Layout [n_walkers][2 channels (A, E)][n_bins][2 (re, im)], row-major, on the device.
 * Fixed point makes adding and then removing a template restore the residual bit for
 * bit (each template value is rounded to the grid, half to even, before the add). */
typedef struct gbk_residual {
  int64_t* data;
  int32_t n_walkers;
  int32_t frac_bits;  /* 40 .. 120 */
} gbk_residual;

/* Per-walker parametric PSD: params[n_psd][2] = (sqrt(S_oms), sqrt(S_acc)), float64,
 * device. n_psd == 1 shares one PSD by all walkers; otherwise n_psd must cover every
 * walker index used. */
typedef struct gbk_psd {
  const double* params;
  int32_t n_psd;
} gbk_psd;

typedef struct gbk_ctx gbk_ctx;

/* Create a context on the current CUDA device: orbit tables for every band length,
 * FFT twiddles, PSD shape tables over the window and scratch. Allocates device memory,
 * as do the other create calls (gbk_sweep_create, mdn_create, gbk_psd_plan_create,
 * gbk_search_create) and, on first use, the plan set-up calls gbk_sweep_set_proposal and
 * gbk_sweep_update_group; no other call allocates. Returns GBK_ENOMEM / GBK_ECUDA on
 * failure. */
gbk_status gbk_create(gbk_ctx** out_ctx, const gbk_grid* grid);

/* Free everything the context owns. Synchronises the device first. */
gbk_status gbk_destroy(gbk_ctx* ctx);

/* Message describing the last error returned on the calling host thread ("" if none). */
const char* gbk_last_error(void);

/* Synchronise `stream`, then read and clear the context's device error word.
 * GBK_OK if no kernel reported an error since the last call. */
gbk_status gbk_sync_status(gbk_ctx* ctx, void* stream);

/* Library ABI version (major * 100 + minor). */
int gbk_version(void);

/*
 * gb_waveform_batch -- TDI A and E band of n sources (Sec. II.A, App. F).
 * Fast/slow decomposition: slow-part response on N coarse samples t_p = p T / N, band
 * FFT, heterodyne of offset m in [-N/2, N/2) to bin q + m; scaled by T / (2 N) so the
 * result is the positive-frequency DFT of the real TDI signal.
 *   params    [8][n] float64
 *   n_band    [n] int32, each in {128, 256, 512, 1024}, <= n_band_max
 *   k_start   [n] int64, out: q - N/2 (first bin of each band)
 *   h_a, h_e  out: complex bands, source i at complex element offset out_off[i];
 *             float32 pairs for GBK_MIXED, float64 pairs for GBK_FP64
 *   out_off   [n] int64
 */
gbk_status gb_waveform_batch(gbk_ctx* ctx, const double* params, const int32_t* n_band,
                             int32_t n_band_max, int64_t n, int64_t* k_start, void* h_a,
                             void* h_e, const int64_t* out_off, gbk_precision precision,
                             void* stream);

/*
 * gb_delta_loglike_batch -- Delta ln L of n independent proposals (Eq. swapsource).
 * Proposal i swaps template r = h(params_old[:, i]) for a = h(params_new[:, i]) in
 * walker walker[i]'s model, whose current residual d - H (H including r) is R:
 *   Delta ln L = -1/2 [<a|a> + <r|r> - 2<a|r> - 2<d-H|a> + 2<d-H|r>]
 * evaluated in the equivalent form -1/2 <a-r|a-r> + <d-H|a-r> over the union of the two
 * bands. Amplitude 0 in params_old gives a birth (Eq. addsource), 0 in params_new a
 * death. Both bands must lie inside the window (else GBK_ERANGE via gbk_sync_status and
 * dlogl[i] = NaN).
 *   params_new, params_old [8][n] float64;  n_band [n] int32 (both templates use it)
 *   walker [n] int32;  dlogl [n] float64 out
 */
gbk_status gb_delta_loglike_batch(gbk_ctx* ctx, const double* params_new,
                                  const double* params_old, const int32_t* n_band,
                                  int32_t n_band_max, const int32_t* walker, int64_t n,
                                  const gbk_residual* residual, const gbk_psd* psd,
                                  double* dlogl, gbk_precision precision, void* stream);

/*
 * gbk_autotune_dlogl -- pick the launch shape of gb_delta_loglike_batch for one band
 * length and precision by timing the caller's sample batch (same arguments as that call)
 * with every candidate (warps per CTA in {1, 2, 4, 8}, CTAs per SM in {1, 2, 4, as many as
 * fit}); the fastest is kept in the context and used by later calls with the same
 * n_band_max and precision. Synchronises `stream`. best_out (host, 2 ints, or NULL)
 * receives (warps per CTA, CTAs per SM; 0 = as many as fit). dlogl is overwritten.
 */
gbk_status gbk_autotune_dlogl(gbk_ctx* ctx, const double* params_new, const double* params_old,
                              const int32_t* n_band, int32_t n_band_max, const int32_t* walker, int64_t n,
                              const gbk_residual* residual, const gbk_psd* psd, double* dlogl,
                              gbk_precision precision, int32_t* best_out, void* stream);

/*
 * residual_add_sub -- move n templates into or out of the model (Alg. 1 write-back).
 * sign = +1: the templates enter the model, R <- R - h; sign = -1: they leave, R <- R + h.
 * Each template value is rounded to the fixed-point grid before the integer update, so
 * residual_add_sub(+1) followed by residual_add_sub(-1) with the same arguments restores
 * R bit for bit, in any order and with any overlap (int64 atomics).
 *   params [8][n] float64; n_band [n] int32; walker [n] int32
 */
gbk_status residual_add_sub(gbk_ctx* ctx, const gbk_residual* residual, const double* params,
                            const int32_t* n_band, int32_t n_band_max, const int32_t* walker,
                            int64_t n, int32_t sign, gbk_precision precision, void* stream);

/*
 * psd_eval -- Eq. psd on the context window for W walkers.
 *   psd_params [W][2] float64 (sqrt(S_oms), sqrt(S_acc))
 *   s_out      [W][n_bins] float64 out, or NULL (then nothing is written)
 * S_n(x) = 8 sin^2 x [2 S_pm (3 + 2 cos x + cos 2x) + S_op (2 + cos x)], x = 2 pi f L / c.
 */
gbk_status psd_eval(gbk_ctx* ctx, const double* psd_params, int32_t n_walkers, double* s_out,
                    void* stream);

/*
 * total_loglike -- Eq. like over the window for W walkers, both channels:
 *   ln L_w = -1/2 <R_w|R_w> - sum_{A,E} sum_k ln S_w(f_k)
 *   residual   [W][2][n_bins][2] float32 (physical units)
 *   psd_params [W][2] float64;  logl [W] float64 out
 * Per-bin terms in float32, per-block sums compensated, cross-block sums in float64 in a
 * fixed order (deterministic). Uses context scratch: concurrent calls on one context
 * must be ordered on one stream.
 */
gbk_status total_loglike(gbk_ctx* ctx, const float* residual, const double* psd_params,
                         int32_t n_walkers, double* logl, void* stream);


/* ------------------------------------------------------------------ noise PSD and foreground
 * Per-channel instrument noise plus the Galactic foreground (Sec. III, Eq. psd; Sec. III.A) and
 * the PSD module's sampler (Sec. V.B). A PSD walker has 9 float64 parameters:
 *   sqrt(S_oms,A), sqrt(S_acc,A), sqrt(S_oms,E), sqrt(S_acc,E), A_fg, alpha, f_k [Hz], s1, s2
 * and channel ch has S_ch = S_n(sqrt(S_oms,ch), sqrt(S_acc,ch)) + S_fg with
 *   S_fg = 6 x^2 sin^2 x (A_fg / 2) f^(-7/3) exp(-s1 f^alpha) [1 + tanh(-s2 (f - f_k))],
 * shared by both channels (the paper's parametrisation).
 */

/* Per-channel PSD values s_out [W][2][n_bins] float64 (or NULL) for psd_params [W][9]. */
gbk_status psd_eval_fg(gbk_ctx* ctx, const double* psd_params, int32_t n_walkers, double* s_out, void* stream);

/* Eq. like with the per-channel PSD of psd_params [n][9] for n entries: entry i uses residual
 * resid_index[i] of residual [n_resid][2][n_bins][2] float32, 16-byte aligned (resid_index
 * NULL: entry i uses residual i). Entries that share a residual and sit next to each other (groups of 4) read it
 * once. Per-bin terms in float32 (the foreground factor as one base-2 exponential on the
 * special-function unit; bins where it is below 2^-30 of the instrument term skip it), sums as
 * in total_loglike. Uses the context scratch (order concurrent calls on one stream). */
gbk_status total_loglike_fg(gbk_ctx* ctx, const float* residual, int32_t n_resid, const double* psd_params,
                            const int32_t* resid_index, int32_t n, double* logl, void* stream);

/* PSD sampler: n_temps x n_walkers PSD walkers; walker w at every temperature uses residual w.
 * Sampled coordinates v = (ln of the 4 noise amplitudes, ln A_fg, alpha, f_k, s1, s2) with a
 * uniform prior on the box [lo, hi]. */
typedef struct gbk_psd_desc {
  int32_t n_temps, n_walkers;  /* n_walkers even */
  double lo[9], hi[9];         /* prior box in v */
  double stretch_a;            /* stretch scale a > 1 (2 in the paper's sampler library) */
} gbk_psd_desc;

/* PSD-sampler plan: allocates the proposal, likelihood and partial-sum buffers of T x W
 * walkers (GBK_ENOMEM on failure); destroy frees them (a NULL plan is a no-op). */
typedef struct gbk_psd_plan gbk_psd_plan;
gbk_status gbk_psd_plan_create(gbk_ctx* ctx, const gbk_psd_desc* desc, gbk_psd_plan** out_plan);
gbk_status gbk_psd_plan_destroy(gbk_psd_plan* plan);

/* One sweep: stretch moves (Eq. stretch) of walkers [0, W/2) then [W/2, W) at every
 * temperature, the partner drawn from the other half, z ~ 1/sqrt(z) on [1/a, a], acceptance
 * z^8 (L_Y / L_X)^beta (box prior); then swaps between temperatures t and t-1 of the same
 * walker from the top down (Eq. temp-orig: the residual is shared). Philox4x32-10 counters:
 * stretch of walker k at temperature t in half h: (t W + k, h, 5, sweep_index), words 0
 * partner, 1 z, 2-3 ln u; swap (t, w, 6, sweep_index), words 0-1 ln u.
 *   params [T][W][9], logl [T][W] (the current ln L of each walker, kept up to date) in/out;
 *   residual [W][2][n_bins][2] float32; betas [T]; stats [2][2] int64 added to (stretch,
 *   swap) x (proposed, accepted), or NULL. Allocates nothing. */
gbk_status gb_psd_sweep(gbk_psd_plan* plan, double* params, double* logl, const float* residual,
                        const double* betas, uint64_t key, uint32_t sweep_index, int64_t* stats, void* stream);

/* ------------------------------------------------------------------ ensemble sweep
 * One sweep of the GB sampler over an ensemble of n_temps x n_walkers chains whose
 * sources are grouped by sub-band (Sec. V.D): odd sub-bands first, then even ones;
 * for each half: (1) the residual window of every band (three sub-bands, Alg. 1) is
 * opened from a snapshot of the cold-chain residual, (2) every band (t, w, b) runs
 * n_prop in-model proposals with accept/reject inside the band (Alg. 1) and then the
 * flip-all reversible jump over its n_max slots in random order (App. C, Eq.
 * rj-acceptance), (3) every band runs ensemble-permuted tempering swaps from the top
 * temperature down (Alg. 2, Eq. temp-final). Accepted changes of the cold chain are
 * written to the residual exactly (fixed point, int64 atomics).
 *
 * Readings where the paper is silent: sources of band b may hold f0 in b's bins widened
 * by half a band on each side; births draw from the band's prior over that range
 * (p / q = 1); each slot is occupied with prior probability pi (log_occ_odds =
 * ln(pi / (1 - pi)), 0 gives Eq. rj-acceptance unchanged); priors uniform in ln A,
 * chirp mass, phi0, psi, cos iota, sin beta, lambda; in-model moves perturb ln A and
 * the other seven parameters by sigma * z with z the centred unit-variance Irwin-Hall(4)
 * variable (sum of four uniforms); n_prop = rint(props_per_source * g) with g the
 * band's source count at the start of its task. Every random number comes from
 * Philox4x32-10 (Salmon et al. 2011) at fixed counters derived from
 * (key, sweep_index, band, temperature, walker, proposal).
 */
typedef struct gbk_sweep_desc {
  int32_t n_temps, n_walkers, n_bands, n_max;  /* n_max <= 64, n_temps <= 64, n_walkers <= 64 */
  int32_t band_bins;       /* sub-band width = template length N, 128 .. 1024 */
  int64_t band_k0;         /* absolute first bin of band 0; windows [band_k0 + (b-1) N, +3N) must lie in the grid */
  double sigma[8];         /* in-model widths: ln A, f0, fdot, phi0, psi, cos iota, sin beta, lambda */
  double log_occ_odds;
  double props_per_source;
  double ln_a_min, ln_a_max, mc_min, mc_max, f_min, f_max;  /* prior bounds (chirp mass in M_sun) */
  int32_t precision;       /* gbk_precision of every waveform and inner product of the sweep */
} gbk_sweep_desc;

/* One record per proposal when tracing (debugging and parity tests). kind: 0 in-model,
 * 1 birth, 2 death, 3 swap; slot is the chain index for swaps; seq the proposal index
 * within the band task (the temperature for swaps); dlogl is NaN for a proposal outside
 * the prior support (rejected without a likelihood). */
typedef struct gbk_trace_rec {
  int32_t kind, t, w, b, slot, seq, accepted, parity;
  double dlogl, log_alpha;
  double params[8];
} gbk_trace_rec;

typedef struct gbk_trace {
  gbk_trace_rec* records;  /* device, capacity records, or NULL */
  int32_t capacity;
  int32_t* count;          /* device counter (records wanted; may exceed capacity) */
} gbk_trace;

typedef struct gbk_sweep gbk_sweep;

/* Sweep plan: validates the description against the context grid and allocates the
 * sweep's device memory: a residual snapshot, the opened band windows, a cache of the
 * current waveform of every slot ([T][W][B][n_max][2][N] complex, 15.5 GB in float32
 * for 16 x 32 x 369 bands x 20 slots at N = 256) and a cache of every band's template
 * sum on its window ([T][W][B][2][3N] complex, 1.2 GB), so that deaths, band openings
 * and tempering swaps reuse waveforms instead of regenerating them. The caches must be
 * refreshed (GBK_SWEEP_REFRESH) whenever params/exists are changed outside gb_sweep; until
 * the first successful call with GBK_SWEEP_REFRESH they are empty, and gb_sweep without that
 * flag, gbk_sweep_transfer and gb_sweep_features return GBK_EINVAL. */
gbk_status gbk_sweep_create(gbk_ctx* ctx, const gbk_sweep_desc* desc, gbk_sweep** out_plan);
gbk_status gbk_sweep_destroy(gbk_sweep* plan);

/* flags */
#define GBK_SWEEP_INMODEL 1
#define GBK_SWEEP_RJ 2
#define GBK_SWEEP_SWAP 4
#define GBK_SWEEP_REFRESH 8   /* regenerate the waveform cache from params/exists first */
#define GBK_SWEEP_TIMING 16   /* record CUDA events around each kernel (see gbk_sweep_kernel_ms) */
#define GBK_SWEEP_MDN 32      /* use the learned proposal set by gbk_sweep_set_proposal */

/*
 * gb_sweep -- one sweep (both parities) on `stream`; allocates nothing.
 *   params   [n_temps][n_walkers][n_bands][n_max][8] float64, in/out
 *   exists   [n_temps][n_walkers][n_bands][n_max] uint8 (0/1), in/out
 *   betas    [n_bands][n_temps] float64 inverse temperatures (0 allowed: T = infinity)
 *   residual cold-chain residual of every walker (d - H of the t = 0 sources), in/out
 *   psd      per-walker PSD
 *   stats    [5][2] int64, added to, or NULL: rows 0-3 (proposed, accepted) for in-model,
 *            birth, death, swap; row 4 (waveforms generated, likelihood evaluations) of
 *            the band kernel
 *   trace    or NULL
 */
gbk_status gb_sweep(gbk_sweep* plan, double* params, uint8_t* exists, const double* betas,
                    const gbk_residual* residual, const gbk_psd* psd, uint64_t key,
                    uint32_t sweep_index, int32_t flags, const gbk_trace* trace, int64_t* stats,
                    void* stream);

/* Device time in ms of the last sweep run with GBK_SWEEP_TIMING, per kernel kind:
 * ms_out[0] cache refresh, [1] band opening (with the learned proposal's features,
 * network and mixture rows under GBK_SWEEP_MDN), [2] band kernel (in-model + RJ), [3]
 * tempering swaps, each summed over both parities. Synchronises with those events. */
gbk_status gbk_sweep_kernel_ms(gbk_sweep* plan, double* ms_out);

/* ------------------------------------------------------------------ learned proposal
 * A mixture-density network (MDN) proposes births and independence in-model moves. The
 * paper proposes births from Gaussian mixtures fitted to earlier sampler output (Sec.
 * V.E, App. G) and names learned density estimators as the next step (App. G). Here an
 * MLP maps the whitened residual of a band to a 16-component diagonal Gaussian mixture
 * truncated to the unit box of the band's prior coordinates
 *   u = ((ln A - ln A_min) / (ln A_max - ln A_min), (f0 - lo_b) / (hi_b - lo_b),
 *        (Mc - Mc_min) / (Mc_max - Mc_min), phi0 / 2pi, psi / pi, (cos i + 1) / 2,
 *        (sin beta + 1) / 2, lambda / 2pi)
 * ([lo_b, hi_b) the f0 range of band b's sources, Mc the chirp mass of (f0, fdot)), where
 * the prior density is 1. Each component is renormalised on the box (erf), so q is an
 * exact density and Eq. rj-acceptance uses it as it stands: birth ratio
 * L'^beta pi_occ / ((1 - pi_occ) q_eps(u')), death its inverse, independence in-model
 * move (L'/L)^beta q_eps(u) / q_eps(u'), with q_eps = eps + (1 - eps) q (a fraction eps of
 * the draws from the prior).
 *
 * The network's input for band b of walker w is the band's opened window rho (the cold
 * residual with b's own cold sources added back), which does not change while band b's
 * tasks run, so q is one fixed density for every move of that pass (detailed balance
 * holds move by move); its 256 central bins, whitened, are the 1024 inputs
 *   x[ch 512 + 2 i + {0, 1}] = (Re, Im) rho_ch(f_i) sqrt(4 df / S_n(f_i)),  ch = A, E.
 *
 * Network: 1024 -> 512 -> 512 -> 512 (ReLU) -> 272 = 16 x (weight logit, 8 mean logits,
 * 8 width logits); weights [out][in] row-major, flat parameter vector
 *   W1[512][1024] b1[512] W2[512][512] b2[512] W3[512][512] b3[512] W4[272][512] b4[272]
 * (mdn_param_count() = 1,189,648 float32). Mixture: pi = softmax(weight logits),
 * mu = sigmoid(mean logits), ln s = -10 + 10 sigmoid(width logits).
 * Products run on the BF16 tensor cores (tcgen05, TMA, accumulators in tensor memory) with
 * float32 accumulation; weights and hidden activations are rounded to BF16 (that rounded
 * network is the model). The float32 master parameters and Adam moments belong to the
 * caller. Every wait inside the tensor-core kernels is bounded; one that gives up skips the
 * rest of its tile and is reported by mdn_status.
 */
typedef struct gbk_mdn gbk_mdn;

int64_t mdn_param_count(void);

/* Workspace for batches of up to max_batch rows (activations, gradient partials, BF16
 * weight copies, transposed operand copies). Allocates device memory (about 12 KB per row
 * + 45 MB). */
gbk_status mdn_create(gbk_mdn** out, int32_t max_batch);
gbk_status mdn_destroy(gbk_mdn* net);

/* Synchronise `stream`, then read and clear the workspace's device error word: GBK_ETIMEOUT
 * if a tensor-core product gave up a bounded wait since the last call, else GBK_OK. */
gbk_status mdn_status(gbk_mdn* net, void* stream);

/* Load float32 parameters [mdn_param_count()] (device) into the workspace's copies. */
gbk_status mdn_set_params(gbk_mdn* net, const float* params, void* stream);

/* raw [batch][272] float32 out = network(x), x [batch][1024] BF16 bit patterns; both
 * 16-byte aligned. */
gbk_status mdn_forward(gbk_mdn* net, const uint16_t* x, int32_t batch, float* raw, void* stream);

/* Gradient of the mean negative log density -1/batch sum_i ln q(u_i | x_i) with respect
 * to the parameters: grad [mdn_param_count()] float32 out; loss (device double, or NULL)
 * out. u [batch][8] float32 unit coordinates. Weight gradients are summed over batch
 * splits in a fixed order (deterministic). */
gbk_status mdn_backward(gbk_mdn* net, const uint16_t* x, const float* u, int32_t batch, float* grad,
                        double* loss, void* stream);

/* One Adam step (Kingma & Ba 2015): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
 * params <- params - lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps); also
 * reloads the workspace's copies. step counts from 1. */
gbk_status mdn_adam(gbk_mdn* net, float* params, float* m, float* v, const float* grad, int32_t step,
                    float lr, float beta1, float beta2, float eps, void* stream);

/* mdn_backward followed by Adam (b1 0.9, b2 0.999, eps 1e-8) without the reduced
 * gradient leaving the device workspace. */
gbk_status mdn_train_step(gbk_mdn* net, float* params, float* m, float* v, const uint16_t* x,
                          const float* u, int32_t batch, int32_t step, float lr, double* loss,
                          void* stream);

/* n_steps Adam steps (as mdn_train_step) over minibatches gathered on the device:
 * step k trains on rows order[k batch .. (k+1) batch) of x [n_rows][1024] (BF16) and
 * u [n_rows][8]; Adam step numbers step0 + 1 .. step0 + n_steps; loss (device double, or
 * NULL) receives the last minibatch's mean -ln q. An index outside [0, n_rows) trains on a
 * zero row and is reported by mdn_status. */
gbk_status mdn_train_epoch(gbk_mdn* net, float* params, float* m, float* v, const uint16_t* x,
                           const float* u, int64_t n_rows, const int32_t* order, int32_t batch,
                           int32_t n_steps, int32_t step0, float lr, double* loss, void* stream);

/* Draws from and densities of the eps-defensive mixture given raw outputs [batch][272]
 * (the sampler's own arithmetic, in `precision`):
 *   words  [batch][9] uint32 or NULL: word 0 picks the component (first k whose
 *          cumulative weight exceeds (w + 1/2) 2^-32), words 1-8 give the dimensions by
 *          the inverse CDF of the truncated normal; u_out [batch][8] (or NULL) receives u
 *   u_in   [batch][8], used when words is NULL
 *   logq   [batch] out (or NULL): ln q_eps at the drawn or given u. */
gbk_status mdn_sample_logpdf(const float* raw, int32_t batch, double eps, const uint32_t* words,
                             float* u_out, const float* u_in, float* logq, int32_t precision,
                             void* stream);

/* ------------------------------------------------------------------ Gaussian-mixture refit
 * gmm_fit -- the paper's GMM-based reversible-jump proposals (Sec. V.E, App. G) fit Gaussian
 * mixtures to sampler output (scikit-learn on CPUs in the paper, which names batched GPU
 * fitting as the desirable form). One CTA per group fits a diagonal-covariance mixture of
 * K = min(n_comp, n) components to the group's n present points by EM (Dempster, Laird &
 * Rubin 1977): start from the points sorted by the second coordinate (f0; ties by
 * position), means at ranks floor((k + 1/2) n / K), every variance the group's
 * per-dimension variance + reg, weights 1/K; then n_iter (E, M) iterations with
 * N_k = sum_i r_ik + 10 DBL_EPSILON, w_k = N_k / sum_j N_j, mu_k = sum_i r_ik x_i / N_k,
 * var_k = sum_i r_ik (x_i - mu_k)^2 / N_k + reg. The result is written as the sampler's
 * 272 mixture outputs (the learned-proposal raw layout: 16 x (weight logit, 8 logit(mu),
 * 8 logit((ln sigma + 10) / 10)), logits clamped to p in [1e-9, 1 - 1e-9]): components
 * with w_k >= min_weight share equal probability (the paper weights each fitted group
 * equally), the others get weight logit -30, missing components (K < 16) are broad
 * (mu 0.5, sigma 1), and an empty group is 16 broad components of equal weight. Feed it to
 * gbk_sweep_set_proposal as raw_table for RJ births (and in-model independence moves).
 *   x          [n_groups][n_points][8] float32 (device): points in the unit coordinates of the
 *              learned proposal; a row with a NaN is absent; the first gmm_max_points()
 *              present rows of a group are used
 *   n_comp     1..16;  n_iter >= 0;  reg > 0 (1e-6 typical);  min_weight in [0, 1]
 *   precision  GBK_MIXED: float32 E-step and per-lane sums (centred on the current means),
 *              float64 combination and M-step; GBK_FP64: float64 throughout
 *   raw_out    [n_copies][n_groups][272] float32 (device): the same rows n_copies times
 *              (n_copies = n_walkers gives a sweep table [W][n_bands][272])
 *   fit_out    optional [n_groups][16][17] float64: w, mu[8], var[8] (zero beyond K)
 *   loglike    optional [n_groups] float64: sum_i ln sum_k w_k N(x_i) of the result
 * One launch, ~98 KB of shared memory per CTA; no allocation. */
int32_t gmm_max_points(void);
gbk_status gmm_fit(const float* x, int32_t n_groups, int32_t n_points, int32_t n_comp, int32_t n_iter, double reg,
                   double min_weight, int32_t precision, int32_t n_copies, float* raw_out, double* fit_out,
                   double* loglike, void* stream);

/* Attach the learned proposal to a sweep plan (used by gb_sweep with GBK_SWEEP_MDN):
 *   net        network evaluated on each half sweep's opened windows (band_bins 256;
 *              max_batch >= n_walkers * ceil(n_bands / 2)), its parameters as last set, or
 *   raw_table  [n_walkers][n_bands][272] float32 device: fixed mixture outputs used as
 *              given (any band_bins; net is then ignored)
 *   eps        prior fraction of the defensive mixture, in [0, 1] (1: the plain prior)
 *   inmodel_frac  fraction of in-model moves that are independence draws, in [0, 1]
 * Both NULL turns the proposal off. Allocates the plan's feature / mixture buffers
 * (about 12 KB per window) on first use. The table, or the network object, must stay
 * alive while the plan uses it. */
gbk_status gbk_sweep_set_proposal(gbk_sweep* plan, gbk_mdn* net, const float* raw_table, double eps,
                                  double inmodel_frac);

/* Temperature-ladder adaptation (Vousden, Farr & Mandel 2016; the paper adapts every ladder,
 * App. D): for every band independently, with T_0 = 1 and S_i = ln(T_i - T_{i-1}),
 * S_i += kappa (A_i - A_{i+1}), kappa = t0 / (nu (iteration + t0)), where A_i is the fraction
 * of walkers whose swap between rungs i-1 and i was accepted in the last gb_sweep (counted on
 * the device); T_i = T_{i-1} + e^{S_i}. An infinite top rung (beta = 0) stays; a finite one
 * adapts with A_N = 0. betas [n_bands][n_temps] (device) is updated in place. */
gbk_status gbk_sweep_adapt_temps(gbk_sweep* plan, double* betas, int32_t iteration, double nu, double t0,
                                 void* stream);

/* Band-edge ownership transfer (Sec. V.D): sources may wander half a band into each
 * neighbour while their band is sampled; afterwards a cold-chain source of band b whose f0
 * lies in the own bins of a neighbour b' = b -+ 1 (floor((f0 Tobs - band_k0) / band_bins)
 * = b') moves to a free slot of b'. Decided on the state at the call, every move at once:
 * band b' takes candidates from b' - 1, then from b' + 1, each in ascending slot order, into
 * its free slots in ascending order; candidates beyond its free slots stay (blocked), as do
 * sources whose owner is outside [0, n_bands) and all hotter chains. The model does not
 * change (the residual is untouched): only which band's slots hold a source. The plan's
 * template caches move with the sources, so params/exists must be the state left by the
 * last gb_sweep (caches current), and the next gb_sweep needs no refresh.
 *   params, exists  the sweep state (device), updated in place
 *   counts          optional device int32[2]: moved and blocked sources are ADDED (NULL: none)
 * Three small kernels plus the cold chain's template sums (n_walkers x n_bands warps). */
gbk_status gbk_sweep_transfer(gbk_sweep* plan, double* params, uint8_t* exists, int32_t* counts, void* stream);

/* ------------------------------------------------------------------ per-band search sampler
 * The search-RJ proposal's sampler (Sec. V.E, App. G): for every sub-band b an independent,
 * parallel-tempered ensemble (n_temps x n_walkers single sources) with stretch moves,
 * looking for the highest-likelihood source still in one walker's residual R. A walker is a
 * point u of the unit box of band b's prior with f0 narrowed to the band's own bins:
 *   u0 = (ln A - ln_a_min) / (ln_a_max - ln_a_min), u1 = (f0 T - band_k0 - b N) / N,
 *   u2 = (Mc - mc_min) / (mc_max - mc_min), u3 = phi0 / 2 pi, u4 = psi / pi,
 *   u5 = (cos iota + 1) / 2, u6 = (sin beta + 1) / 2, u7 = lambda / 2 pi,
 * and its likelihood is l(u) = <R|h> - 1/2 <h|h> on the band's window b-1..b+1 (the birth
 * Delta lnL, Eq. addsource). A sweep: stretch moves of walker half 0, then half 1, at every
 * temperature (partner from the other half, z ~ 1/sqrt(z) on [1/a, a], Y = X_j + z (X_k -
 * X_j); a Y outside [0, 1]^8 is rejected; acceptance ln u < beta (l_Y - l_X) + 7 ln z), then
 * tempering swaps of each walker index from the top temperature down (Eq. temp-orig), then
 * (optionally) the best point of every band: the largest cold l, kept if it improves
 * (stall = 0) else stall += 1. Random numbers: Philox4x32-10 with the 64-bit key; start of
 * chain c = (b T + t) W + k from counters (c, m, 9, seed), m = 0, 1; stretch of chain c in
 * half h of sweep s from (c, h, 7, s) (words: partner, z, ln u); swap of (b, w) between t and
 * t - 1 from (b W + w, t, 8, s). SNR of a band's best point: sqrt(2 l_best).
 * A plan runs n_sets such searches side by side (the paper keeps one search per walker): set s
 * searches the residual of walker w0 + s (gb_search_windows) with that walker's PSD row
 * (psd_walker + s; a one-row PSD serves every set). Every per-band array then carries the sets
 * first: band b of set s is the flattened band fb = s n_bands + b (u [n_sets][n_bands][T][W][8],
 * betas [n_sets][n_bands][T], ...), and fb takes b's place in the counters above; with n_sets = 1
 * fb = b. */
typedef struct gbk_search_desc {
  int32_t n_bands, band_bins, n_temps, n_walkers;  /* n_walkers even, >= 4 */
  int64_t band_k0;        /* absolute first bin of band 0; windows [band_k0 + (b-1) N, +3N) in the grid */
  double ln_a_min, ln_a_max, mc_min, mc_max;        /* prior bounds (chirp mass in M_sun) */
  double stretch_a;       /* stretch scale a > 1 (2 in the paper's sampler) */
  int32_t precision;      /* GBK_MIXED or GBK_FP64 (waveforms and inner products) */
  int32_t stall_limit;    /* n_it,max: a band whose best point has not improved for this many sweeps
                             has converged and is frozen (no moves, swaps or best-point updates in
                             later sweeps until its stall count is reset); 0: never */
  int32_t n_sets;         /* searches side by side, one per residual walker (0 means 1) */
} gbk_search_desc;

typedef struct gbk_search gbk_search;

/* Plan: validates the description against the context grid; allocates the residual windows
 * ([n_bands][2][3N] complex of the precision). */
gbk_status gbk_search_create(gbk_ctx* ctx, const gbk_search_desc* desc, gbk_search** out);
gbk_status gbk_search_destroy(gbk_search* plan);
/* u [n_sets][n_bands][n_temps][n_walkers][8] float64 (device) drawn from the prior (uniform
 * box). */
gbk_status gb_search_init(gbk_search* plan, double* u, uint64_t key, uint32_t seed, void* stream);
/* Copies the fixed-point residual (gbk_residual, device) of walker `walker` + s onto the window of
 * every band of set s (walker + n_sets <= the residual's walkers); the windows stay until the
 * next call. */
gbk_status gb_search_windows(gbk_search* plan, const gbk_residual* residual, int32_t walker, void* stream);
/* ell [n_sets][n_bands][n_temps][n_walkers] float64 (device) = l(u) of every walker, with set s
 * taking the PSD row psd_walker + s (its residual's walker; row 0 of a one-row PSD). */
gbk_status gb_search_eval(gbk_search* plan, const double* u, double* ell, const gbk_psd* psd, int32_t psd_walker,
                          void* stream);
/* One sweep; u and ell (consistent, e.g. from gb_search_eval) are updated in place.
 *   betas     [n_sets][n_bands][n_temps] float64 (device)
 *   best_ell  [n_sets][n_bands] float64, best_u [n_sets][n_bands][8], stall [n_sets][n_bands]
 *             int32 (device, in/out; start best_ell at -inf); all three or none, and all three
 *             with a stall_limit: the
 *             bands whose stall count has reached it at the start of the sweep are left as they are
 *   stats     optional int64[2][2] (device): stretch proposals, accepted; swaps, accepted (added) */
gbk_status gb_search_sweep(gbk_search* plan, double* u, double* ell, const double* betas, const gbk_psd* psd,
                           int32_t psd_walker, uint64_t key, uint32_t sweep_index, double* best_ell, double* best_u,
                           int32_t* stall, int64_t* stats, void* stream);
/* Relaunch around the best points (App. G: a new ball of points around the maximum-likelihood
 * point, then the same search again): every chain of a band whose best_ell is finite becomes
 * clip(best_u + sigma z, 0, 1) with z standard normal (Box-Muller on Philox words at counters
 * (chain, m, 10, seed), m = 0, 1); other bands keep their walkers. Follow with gb_search_eval.
 *   u [n_sets][n_bands][n_temps][n_walkers][8] (device, updated); best_ell [n_sets][n_bands],
 *   best_u [n_sets][n_bands][8] */
gbk_status gb_search_ball(gbk_search* plan, double* u, const double* best_ell, const double* best_u, double sigma,
                          uint64_t key, uint32_t seed, void* stream);
/* Training points of the search-RJ mixtures from the current state: for every band b the cold
 * walkers' u in the sweep's unit coordinates (the learned proposal's: f0 over the band's
 * allowance, own bins +- half a band clipped to [f_min, f_max]; the other coordinates
 * unchanged) into x[fb][row0 + k][8] (float32, device, [n_sets][n_bands][n_rows][8]),
 * k < n_walkers;
 * rows of a band whose best point has sqrt(2 best_ell) < snr_min are NaN. Fit them with
 * gmm_fit (one group per band) for the sweep's mixture table. */
gbk_status gb_search_samples(gbk_search* plan, const double* u, const double* best_ell, double snr_min, double f_min,
                             double f_max, float* x, int32_t n_rows, int32_t row0, void* stream);

/* Group stretch in-model moves (the paper's in-model proposal, Eq. stretch with a stationary
 * group): builds every band's stationary group from the current cold chain -- the sources of
 * bands b-1, b, b+1 of all walkers, sorted by f0 -- and makes a fraction `frac` of the
 * in-model moves of later gb_sweep calls stretch moves Y = X_j + z (X_k - X_j) in the
 * coordinates (ln A, f0, fdot, phi0, psi, cos iota, sin beta, lambda), X_j drawn uniformly
 * from the n_friends group members nearest in f0 to X_k, z from g(z) ~ 1/sqrt(z) on
 * [1/2, 2], acceptance z^7 (L'/L)^beta p'/p. A draw whose X_j is not also among the
 * n_friends nearest members of Y (or whose stretched phase difference leaves half a period)
 * is rejected without a likelihood: the friend choice is then symmetric and the move exact.
 * The group stays fixed until the next call (the paper rebuilds it every ~30 sweeps).
 * frac = 0 turns the moves off. Allocates the group on first use (B x 3 W n_max x 72 bytes).
 *   params, exists  the sweep state (device), as for gb_sweep */
gbk_status gbk_sweep_update_group(gbk_sweep* plan, const double* params, const uint8_t* exists, double frac,
                                  int32_t n_friends, void* stream);

/* Training pairs from the current cold chain (band_bins 256): x_out [n_walkers][n_bands]
 * [1024] BF16 features of every band's opened window (as above), u_out [n_walkers]
 * [n_bands][n_max][8] float32 unit coordinates of every cold slot (NaN where empty);
 * either may be NULL. Reads the plan's template-sum cache, so params/exists must be the
 * state left by the last gb_sweep (or a sweep with GBK_SWEEP_REFRESH). */
gbk_status gb_sweep_features(gbk_sweep* plan, const double* params, const uint8_t* exists,
                             const gbk_residual* residual, const gbk_psd* psd, uint16_t* x_out,
                             float* u_out, void* stream);

/* ------------------------------------------------------------------ no-allocation variant
 * total_loglike_noalloc -- the total Gaussian log-likelihood of W walkers over both channels
 * (what total_loglike returns), for callers that cannot allocate device memory: code that
 * runs inside another framework's allocator or memory budget, or that must not grow the
 * device footprint after start-up. It needs no gbk_ctx (whose creation allocates): the grid
 * is passed directly and the PSD shape is evaluated in float64 by a kernel of the call. The
 * paper has no counterpart: this is a deployment variant of the total-likelihood pass.
 *   tobs, k0, n_bins  the window, as in gbk_grid; (k0 + n_bins) / tobs < c / (2L)
 *   residual          [W][2][n_bins][2] float32, 8-byte aligned
 *   psd_params        [W][2] float64;  logl [W] float64 out
 * Its scratch (the float32 shape tables and the cross-block partial sums) is a fixed array
 * of total_loglike_noalloc_capacity() doubles (16 MiB) in the library's device memory, held
 * on every device that loads the library until the process exits. A call needs
 * n_bins + 2 W ceil(n_bins / 8192) + ceil(n_bins / 4096) doubles and W <= 262140; larger
 * requests return GBK_ERANGE. Every call overwrites all the scratch it reads, so earlier
 * contents do not matter; but all calls share the one array, so calls that overlap on the
 * GPU (different streams, or host threads without ordering) race and give wrong results:
 * order them on one stream. The first call on each device looks up the array's device
 * address and keeps it for the process; make that first call before any stream capture. A
 * device reset (cudaDeviceReset) invalidates the kept address: do not call this entry
 * point after one. Allocates nothing (no cudaMalloc, no library calls that allocate).
 */
int64_t total_loglike_noalloc_capacity(void);
gbk_status total_loglike_noalloc(double tobs, int64_t k0, int64_t n_bins, const float* residual,
                                 const double* psd_params, int32_t n_walkers, double* logl, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GBK_H */
