// Context of libgbk: orbit tables, FFT twiddles, PSD shape tables, error handling.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "gbk_internal.cuh"

namespace gbk {

static thread_local char g_last_error[512] = "";

gbk_status set_error(gbk_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return st;
}

gbk_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GBK_ECUDA, "%s: launch failed: %s", what, cudaGetErrorString(e));
  return GBK_OK;
}

// Analytic orbits: first order in the eccentricity e = L / (2 sqrt3 AU), orbital phase
// alpha = 2 pi t / year and constellation orientation zero at t = 0:
//   x_n = AU cos a + (e AU / 2)(cos(2a - b_n) - 3 cos b_n)
//   y_n = AU sin a + (e AU / 2)(sin(2a - b_n) - 3 sin b_n)
//   z_n = -sqrt3 e AU cos(a - b_n),   b_n = 2 pi (n - 1) / 3.
static void craft_position(double t, int n, double out[3]) {
  const double ecc = kLArm / (2.0 * sqrt(3.0) * kAU);
  const double a = 2.0 * M_PI * t / kYear;
  const double b = 2.0 * M_PI * n / 3.0;
  out[0] = kAU * cos(a) + 0.5 * ecc * kAU * (cos(2.0 * a - b) - 3.0 * cos(b));
  out[1] = kAU * sin(a) + 0.5 * ecc * kAU * (sin(2.0 * a - b) - 3.0 * sin(b));
  out[2] = -sqrt(3.0) * ecc * kAU * cos(a - b);
}

// Rows (SoA [kOrbRows][N]): 0-1 guiding-centre direction (cos a, sin a); 2-10 craft
// offsets from the guiding centre / c; 11-19 arm unit vectors n12, n23, n31;
// 20-21 remainders of rows 0-1 after rounding to the table's type (0 in float64).
static void build_orbit_table(double tobs, int n, std::vector<double>& tab) {
  tab.assign((size_t)kOrbRows * n, 0.0);
  for (int p = 0; p < n; ++p) {
    const double t = p * (tobs / n);
    const double a = 2.0 * M_PI * t / kYear;
    const double gc[3] = {kAU * cos(a), kAU * sin(a), 0.0};
    double x[3][3];
    for (int c = 0; c < 3; ++c) craft_position(t, c, x[c]);
    tab[0 * n + p] = cos(a);
    tab[1 * n + p] = sin(a);
    // rows 20-21: float remainders of cos a, sin a (filled by the caller for float tables)
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) tab[(size_t)(2 + 3 * c + d) * n + p] = (x[c][d] - gc[d]) / kC;
    const int from[3] = {0, 1, 2}, to[3] = {1, 2, 0};
    for (int arm = 0; arm < 3; ++arm) {
      double v[3], nn = 0.0;
      for (int d = 0; d < 3; ++d) {
        v[d] = x[to[arm]][d] - x[from[arm]][d];
        nn += v[d] * v[d];
      }
      nn = sqrt(nn);
      for (int d = 0; d < 3; ++d) tab[(size_t)(11 + 3 * arm + d) * n + p] = v[d] / nn;
    }
  }
}

// Eq. psd split by noise power: S_n = S_oms Q(f) + S_acc P(f).
static void psd_shape(double f, double* p_acc, double* q_oms) {
  const double x = 2.0 * M_PI * f * kLc;
  const double sx = sin(x);
  const double pm_unit = pow(2.0 * M_PI * kC * f, -2.0) * (1.0 + pow(0.4e-3 / f, 2.0)) * (1.0 + pow(f / 8e-3, 4.0));
  const double op_unit = pow(2.0 * M_PI * f / kC, 2.0) * (1.0 + pow(2e-3 / f, 4.0));
  *p_acc = 8.0 * sx * sx * 2.0 * pm_unit * (3.0 + 2.0 * cos(x) + cos(2.0 * x));
  *q_oms = 8.0 * sx * sx * op_unit * (2.0 + cos(x));
}

template <typename P>
static cudaError_t upload(P** dst, const void* src, size_t bytes) {
  cudaError_t e = cudaMalloc((void**)dst, bytes);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
}

size_t total_loglike_scratch_bytes(int64_t n_bins);

}  // namespace gbk

using namespace gbk;

extern "C" int gbk_version(void) { return 100; }

extern "C" const char* gbk_last_error(void) { return g_last_error; }

extern "C" gbk_status gbk_destroy(gbk_ctx* ctx) {
  if (!ctx) return set_error(GBK_EINVAL, "gbk_destroy: null context");
  cudaDeviceSynchronize();
  for (int i = 0; i < kNumBandSizes; ++i) {
    cudaFree(ctx->orb_f[i]);
    cudaFree(ctx->orb_d[i]);
    cudaFree(ctx->tw_f[i]);
    cudaFree(ctx->tw_d[i]);
  }
  cudaFree(ctx->psd_q);
  cudaFree(ctx->psd_p);
  cudaFree(ctx->iq_f);
  cudaFree(ctx->rho_f);
  cudaFree(ctx->iqrho_f);
  cudaFree(ctx->iq_d);
  cudaFree(ctx->rho_d);
  cudaFree(ctx->fg_lnf);
  cudaFree(ctx->fg_f);
  cudaFree(ctx->fg_c);
  cudaFree(ctx->err);
  cudaFree(ctx->scratch);
  free(ctx);
  return GBK_OK;
}

extern "C" gbk_status gbk_create(gbk_ctx** out_ctx, const gbk_grid* grid) {
  if (!out_ctx || !grid) return set_error(GBK_EINVAL, "gbk_create: null argument");
  *out_ctx = nullptr;
  if (!(grid->tobs > 0) || !(grid->dt > 0) || grid->k0 < 1 || grid->n_bins < 1)
    return set_error(GBK_EINVAL, "gbk_create: bad grid (tobs=%g dt=%g k0=%lld n_bins=%lld)", grid->tobs,
                     grid->dt, (long long)grid->k0, (long long)grid->n_bins);
  const double nt = grid->tobs / grid->dt;
  if (fabs(nt - rint(nt)) > 1e-9 * nt || fmod(rint(nt), 1024.0) != 0.0)
    return set_error(GBK_EINVAL, "gbk_create: tobs/dt = %g is not a multiple of 1024", nt);
  // Eq. psd vanishes at x = pi (f = c / 2L); windows must stay below it. A window may pass
  // the Nyquist bin N_t/2 (a synthetic total-likelihood pass over 2^20 bins from 0.1 mHz
  // does), where only the PSD model, not the waveform, is evaluated.
  if ((double)(grid->k0 + grid->n_bins) / grid->tobs >= 0.5 / kLc)
    return set_error(GBK_EINVAL, "gbk_create: window reaches f = c/(2L), where the PSD vanishes");
  gbk_ctx* c = (gbk_ctx*)calloc(1, sizeof(gbk_ctx));
  if (!c) return set_error(GBK_ENOMEM, "gbk_create: host allocation failed");
  c->grid = *grid;
  cudaGetDevice(&c->device);
  cudaError_t e = cudaSuccess;
  std::vector<double> tab;
  for (int bi = 0; bi < kNumBandSizes && e == cudaSuccess; ++bi) {
    const int n = 128 << bi;
    build_orbit_table(grid->tobs, n, tab);
    std::vector<float> tabf(tab.begin(), tab.end());
    for (int p = 0; p < n; ++p) {
      tabf[(size_t)20 * n + p] = (float)(tab[(size_t)0 * n + p] - (double)tabf[(size_t)0 * n + p]);
      tabf[(size_t)21 * n + p] = (float)(tab[(size_t)1 * n + p] - (double)tabf[(size_t)1 * n + p]);
    }
    e = upload(&c->orb_d[bi], tab.data(), tab.size() * sizeof(double));
    if (e == cudaSuccess) e = upload(&c->orb_f[bi], tabf.data(), tabf.size() * sizeof(float));
    std::vector<double2> twd(n);
    std::vector<float2> twf(n);
    for (int m = 0; m < n; ++m) {
      twd[m] = make_double2(cos(2.0 * M_PI * m / n), -sin(2.0 * M_PI * m / n));
      twf[m] = make_float2((float)twd[m].x, (float)twd[m].y);
    }
    if (e == cudaSuccess) e = upload(&c->tw_d[bi], twd.data(), n * sizeof(double2));
    if (e == cudaSuccess) e = upload(&c->tw_f[bi], twf.data(), n * sizeof(float2));
  }
  const int64_t nb = grid->n_bins;
  std::vector<double> q(nb), pa(nb), iq(nb), rho(nb);
  std::vector<float> iqf(nb), rhof(nb), lnff(nb), ff(nb), fgc(nb);
  std::vector<float2> iqrf(nb);
  double s = 0.0, comp = 0.0;  // compensated sum of ln Q
  for (int64_t i = 0; i < nb; ++i) {
    const double f = (double)(grid->k0 + i) / grid->tobs;
    psd_shape(f, &pa[i], &q[i]);
    rho[i] = pa[i] / q[i];
    iq[i] = ldexp(1.0 / q[i], -2 * kStrainExp);
    iqf[i] = (float)iq[i];
    rhof[i] = (float)rho[i];
    iqrf[i] = make_float2(iqf[i], rhof[i]);
    const double x = 2.0 * M_PI * f * kLc, sx = sin(x);
    lnff[i] = (float)log2(f);
    ff[i] = (float)f;
    fgc[i] = (float)((log(6.0 * x * x * sx * sx) - log(q[i]) - (7.0 / 3.0) * log(f)) * 1.4426950408889634);
    const double y = log(q[i]) - comp;
    const double t = s + y;
    comp = (t - s) - y;
    s = t;
  }
  c->sum_lnq = s;
  if (e == cudaSuccess) e = upload(&c->psd_q, q.data(), nb * sizeof(double));
  if (e == cudaSuccess) e = upload(&c->psd_p, pa.data(), nb * sizeof(double));
  if (e == cudaSuccess) e = upload(&c->iq_d, iq.data(), nb * sizeof(double));
  if (e == cudaSuccess) e = upload(&c->rho_d, rho.data(), nb * sizeof(double));
  if (e == cudaSuccess) e = upload(&c->iq_f, iqf.data(), nb * sizeof(float));
  if (e == cudaSuccess) e = upload(&c->rho_f, rhof.data(), nb * sizeof(float));
  if (e == cudaSuccess) e = upload(&c->iqrho_f, iqrf.data(), nb * sizeof(float2));
  if (e == cudaSuccess) e = upload(&c->fg_lnf, lnff.data(), nb * sizeof(float));
  if (e == cudaSuccess) e = upload(&c->fg_f, ff.data(), nb * sizeof(float));
  if (e == cudaSuccess) e = upload(&c->fg_c, fgc.data(), nb * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(int));
  if (e == cudaSuccess) {
    c->scratch_bytes = total_loglike_scratch_bytes(nb);
    e = cudaMalloc((void**)&c->scratch, c->scratch_bytes);
  }
  if (e != cudaSuccess) {
    gbk_status st = (e == cudaErrorMemoryAllocation) ? GBK_ENOMEM : GBK_ECUDA;
    set_error(st, "gbk_create: %s", cudaGetErrorString(e));
    gbk_destroy(c);
    return st;
  }
  *out_ctx = c;
  return GBK_OK;
}

extern "C" gbk_status gbk_sync_status(gbk_ctx* ctx, void* stream) {
  if (!ctx) return set_error(GBK_EINVAL, "gbk_sync_status: null context");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return set_error(GBK_ECUDA, "gbk_sync_status: %s", cudaGetErrorString(e));
  int h = 0;
  e = cudaMemcpy(&h, ctx->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_error(GBK_ECUDA, "gbk_sync_status: %s", cudaGetErrorString(e));
  if (h == 0) return GBK_OK;
  cudaMemset(ctx->err, 0, sizeof(int));
  if (h & kErrTimeout) return set_error(GBK_ETIMEOUT, "device wait gave up (error bits 0x%x)", h);
  if (h & (kErrRange | kErrWalker)) return set_error(GBK_ERANGE, "band or walker out of range (error bits 0x%x)", h);
  return set_error(GBK_EINVAL, "device reported bad input (error bits 0x%x)", h);
}
