// Internal definitions of libgbk: context, constants, device helpers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gbk.h"

namespace gbk {

// Physical constants (standard LISA / LDC values; the paper fixes only f* = c / L).
constexpr double kC = 299792458.0;          // m/s
constexpr double kLArm = 2.5e9;             // m
constexpr double kAU = 1.495978707e11;      // m
constexpr double kYear = 31557600.0;        // s
constexpr double kLc = kLArm / kC;          // s, one-arm light time

// Internal strain scale: strain-like values are carried as value * 2^64 and PSDs as
// S * 2^128 so that float32 never meets denormals (S_n ~ 1e-42 in these units is
// below float32's normal range). Powers of two: the rescaling is exact.
constexpr int kStrainExp = 64;

// Conversions between the fixed-point residual (int64) and float32 without the 64-bit
// conversion instructions, which run at the reduced float64 rate on this part. Values that fit
// in 32 bits (most residual samples: |v| ~ 2^27 for a 1e-21 strain at 98 fraction bits) take one
// 32-bit conversion, rounded exactly as the 64-bit one; larger ones split into 32-bit halves:
// ll_to_float = RN(hi 2^32 + RN(lo)), at most one unit in the last place from the single
// rounding (the rounding of lo moves the sum by up to 2^7). float_to_ll is exact: a float of
// magnitude >= 2^31 is an integer, and both of its 32-bit halves are exact floats.
__device__ __forceinline__ float ll_to_float(long long v) {
  const int lo = (int)v;
  if ((long long)lo == v) return (float)lo;
  return fmaf((float)(int)(v >> 32), 4294967296.0f, (float)(unsigned)v);
}
__device__ __forceinline__ long long float_to_ll(float x) {
  if (fabsf(x) < 2147483648.0f) return (long long)__float2int_rn(x);
  const float h = floorf(x * 2.3283064365386963e-10f);   // x / 2^32, exact
  const float l = fmaf(h, -4294967296.0f, x);            // x - h 2^32 in [0, 2^32), exact
  return (long long)(((unsigned long long)(unsigned)(int)h << 32) | (unsigned long long)(unsigned)l);
}

// Band lengths: 128 << i for i = 0..3.
constexpr int kNumBandSizes = 4;
inline __host__ __device__ int band_index(int n) {
  return n == 128 ? 0 : n == 256 ? 1 : n == 512 ? 2 : n == 1024 ? 3 : -1;
}

// Orbit table rows, SoA [kOrbRows][N] per band length: guiding-centre direction
// (cos alpha, sin alpha), spacecraft offsets from the guiding centre in
// light-seconds (3 craft x 3), arm unit vectors n12, n23, n31 (3 x 3), and the
// rounding remainders of the two direction rows (2).
constexpr int kOrbRows = 22;

// Device error bits (OR-ed into the context's error word).
constexpr int kErrRange = 1;
constexpr int kErrBand = 2;
constexpr int kErrWalker = 4;
constexpr int kErrTimeout = 8;

}  // namespace gbk

struct gbk_ctx {
  gbk_grid grid;
  int device;
  // per band length: orbit tables and FFT twiddles W_N^k = exp(-2 pi i k / N)
  float* orb_f[gbk::kNumBandSizes];
  double* orb_d[gbk::kNumBandSizes];
  float2* tw_f[gbk::kNumBandSizes];
  double2* tw_d[gbk::kNumBandSizes];
  // PSD shape over the window: S = S_oms * Q_k + S_acc * P_k (physical),
  // rho = P / Q, iq = 2^-128 / Q, lnq = ln Q.
  double* psd_q;
  double* psd_p;
  float* iq_f;
  float* rho_f;
  float2* iqrho_f;     // (iq, rho) per bin, float32, for loads of both at once
  double* iq_d;
  double* rho_d;
  double sum_lnq;      // sum_k ln Q_k over the window, float64
  // Galactic-foreground shape over the window (Sec. III.A), in base-2 logarithms: log2 f, the
  // float32 frequency and fgc = log2(6 x^2 sin^2 x / Q) - (7/3) log2 f, so that
  // S_fg / Q = A_fg 2^(fgc - log2(e) [s1 f^alpha + softplus(2 s2 (f - f_k))])
  float* fg_lnf;
  float* fg_f;
  float* fg_c;
  int* err;            // device error word
  // scratch for cross-block partial sums of total_loglike
  double* scratch;
  size_t scratch_bytes;
  // launch shapes chosen by gbk_autotune_dlogl: [precision][band index] warps per CTA
  // and CTAs per SM (0 = library default)
  int tune_wpc[2][4];
  int tune_bps[2][4];
};

// Mixture-density network workspace (gbk_mdn.cu).
struct gbk_mdn {
  int32_t max_batch;
  int64_t ldt;           // row length of the transposed copies (2 x max_batch rounded up to 8)
  float* pf;             // float32 copy of the parameters (biases of the forward pass)
  __nv_bfloat16* pb;     // BF16 copy (weights, [out][in])
  __nv_bfloat16* pbT;    // BF16 [W^T | W^T] [in][2 out] of layers 2-4
  __nv_bfloat16* h[3];   // hidden activations [max_batch][512]
  __nv_bfloat16* hT[3];  // and transposed twice, [h^T | h^T] [512][ldt]
  float* raw;            // [max_batch][272]
  __nv_bfloat16* g4;     // d loss / d raw as BF16 pairs [max_batch][hi 272 | lo 272]
  __nv_bfloat16* g4T;    // and transposed [272][hi B | lo B] (pitch ldt)
  __nv_bfloat16* g[2];   // back-propagated signals [max_batch][hi 512 | lo 512]
  __nv_bfloat16* gT[2];  // and transposed [512][hi B | lo B] (pitch ldt)
  __nv_bfloat16* xT;     // input features transposed twice, [x^T | x^T] [1024][ldt]
  float* nll;            // [max_batch]
  float* part;           // split-K gradient partials [8][n_params]
  int* err;              // device error word (bounded waits of the tensor-core products)
  __nv_bfloat16* xb;     // gathered training rows [max_batch][1024]
  float* ub;             // and their targets [max_batch][8]
  bool have_params;
  // encoded TMA maps of the operands seen so far (pointers and shapes repeat every step)
  struct MapEntry {
    const void* p;
    int64_t rows, k, ld;
    int box;
    alignas(64) unsigned char map[128];
  };
  MapEntry maps[48];
  int n_maps, next_map;
};

namespace gbk {

// Record an error message for gbk_last_error() and return the status.
gbk_status set_error(gbk_status st, const char* fmt, ...);
gbk_status check_launch(const char* what);
// Block passes of the total log-likelihood over the float32 shape tables iq, rho: per chunk of
// kTlChunk bins and walker, the sums of |R|^2 2^128 iq / u and of ln u into part [chunk][nwl][2]
// (gbk_psd.cu; shared with the no-allocation variant).
constexpr int kTlChunk = 8192;
gbk_status total_loglike_parts(const float* R, const float* iq, const float* rho, const double* pp, int32_t w0,
                               int32_t nwl, int64_t nb, double* part, cudaStream_t st);

}  // namespace gbk
