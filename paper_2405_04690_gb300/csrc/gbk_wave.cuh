// Warp-level GB waveform generator: slow-part TDI response, shared-memory Stockham
// FFT and heterodyne, in float32 (mixed) or float64 (plain) arithmetic.
//
// Model (arXiv:2405.04690 Sec. II.A and App. F name FastGB; the response below is the
// standard equal-arm one: the link response n.H.n / (2 (1 - k.n)) [H(t_emit) - H(t_recv)]
// with the carrier phase expanded to first order in the light times, Phi(t - tau) =
// Phi(t) - 2 pi f(t) tau, and the geometry taken at each coarse sample):
//   H(t) = Re[Hc e^{i Phi(t)}], Hc = A(1+cos^2 i) e+(psi) + 2i A cos i ex(psi),
//   Phi(t) = phi0 + 2 pi f0 t + pi fdot t^2.
//   Link i->j (unit vector n from craft i to j, receiver position x_j), slow part:
//   Y_ij = n.Hc.n (-i pi f L/c) sinc(pi f L/c (1 - k.n)) e^{-i pi f L/c (1 - k.n)}
//          e^{-2 pi i f k.x_j / c},  f = f0 + fdot t.
//   X = (1 - D^2)[(Y31 - Y21) + D (Y13 - Y12)], D = e^{-2 pi i f L/c}; Y, Z cyclic.
//   A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6 (Sec. II, A_1/E_1).
//   Band: (T / 2N) FFT_N[ slow(t_p) e^{i(phi0 + 2 pi delta p/N + pi fdot t_p^2)} ],
//   offset m in [-N/2, N/2) -> bin q + m, q = floor(f0 T), delta = f0 T - q.
//
// One warp computes one band from per-source constants (Src) that the lanes of a warp
// compute for up to 32 sources at once (make_src holds the float64 work, which runs at a
// small fraction of the float32 rate on GB300, so it is spread over lanes, not repeated
// by every lane). Every kernel that needs a waveform calls gen_band<T, N>,
// which is __noinline__ so that all call sites run the same machine code: the same
// parameters then give bit-identical bands in every kernel, which the fixed-point
// residual bookkeeping relies on (a template removed by one kernel cancels the one
// another kernel added).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbk_internal.cuh"

#ifndef GBK_SAMPLE_UNROLL
#define GBK_SAMPLE_UNROLL 1
#endif

namespace gbk {

constexpr int kSampleUnroll = GBK_SAMPLE_UNROLL;

template <typename T> struct CT;
template <> struct CT<float> { typedef float2 C; };
template <> struct CT<double> { typedef double2 C; };

__device__ __forceinline__ float2 mkc(float r, float i) { return make_float2(r, i); }
__device__ __forceinline__ double2 mkc(double r, double i) { return make_double2(r, i); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// multiply by -i
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }
__device__ __forceinline__ double2 cmul_mi(double2 a) { return make_double2(a.y, -a.x); }

// (cos, sin) of 2 pi x for x in cycles: reduce to [-1/2, 1/2] first.
__device__ __forceinline__ float2 expi_cycles(float x) {
  float r = x - rintf(x);
  float s, c;
  __sincosf(6.283185307179586f * r, &s, &c);
  return make_float2(c, s);
}
__device__ __forceinline__ double2 expi_cycles(double x) {
  double r = x - rint(x);
  double s, c;
  sincospi(2.0 * r, &s, &c);
  return make_double2(c, s);
}

// exp(i x) for |x| <= 1.1 rad by Taylor series (truncation < 2e-10): used for the
// slowly varying link and arm-delay phases, whose errors would otherwise be the same
// in every sample of a band and add up coherently. float64 uses sincos.
__device__ __forceinline__ float2 expi_small(float x) {
  const float z = x * x;
  float sp = 1.0f / 39916800.0f;
  sp = sp * -z + 1.0f / 362880.0f;
  sp = sp * -z + 1.0f / 5040.0f;
  sp = sp * -z + 1.0f / 120.0f;
  sp = sp * -z + 1.0f / 6.0f;
  sp = sp * -z + 1.0f;
  float cp = 1.0f / 479001600.0f;
  cp = cp * -z + 1.0f / 3628800.0f;
  cp = cp * -z + 1.0f / 40320.0f;
  cp = cp * -z + 1.0f / 720.0f;
  cp = cp * -z + 1.0f / 24.0f;
  cp = cp * -z + 0.5f;
  cp = cp * -z + 1.0f;
  return make_float2(cp, x * sp);
}
__device__ __forceinline__ double2 expi_small(double x) {
  double s, c;
  sincos(x, &s, &c);
  return make_double2(c, s);
}
// The same for sources whose series arguments are small (the shorter-series path, see
// Src::lo): the series cut after x^7 (sin) and x^8 (cos). Its largest argument there is a link
// phase, (1/2 + 1/sqrt3) x kLoArg = 0.27 rad, where the first dropped terms are below 1e-10
// relative. float64 keeps sincos.
constexpr double kLoArg = 0.25;
__device__ __forceinline__ float2 expi_small_lo(float x) {
  const float z = x * x;
  float sp = 1.0f / 5040.0f;
  sp = sp * -z + 1.0f / 120.0f;
  sp = sp * -z + 1.0f / 6.0f;
  sp = sp * -z + 1.0f;
  float cp = 1.0f / 40320.0f;
  cp = cp * -z + 1.0f / 720.0f;
  cp = cp * -z + 1.0f / 24.0f;
  cp = cp * -z + 0.5f;
  cp = cp * -z + 1.0f;
  return make_float2(cp, x * sp);
}
__device__ __forceinline__ double2 expi_small_lo(double x) { return expi_small(x); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ void fma_err(float a, float b, float p, float& e) { e = fmaf(a, b, -p); }
__device__ __forceinline__ void fma_err(double a, double b, double p, double& e) { e = fma(a, b, -p); }

__device__ __forceinline__ float fmaf_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaf_(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float rint_(float x) { return rintf(x); }
__device__ __forceinline__ double rint_(double x) { return rint(x); }
__device__ __forceinline__ void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_(double x, double* s, double* c) { sincos(x, s, c); }

// sin(pi s) / (pi s) by its Taylor series in z = (pi s)^2 (truncation < 1e-9 for
// float, < 2e-15 for double, for |pi s| <= 1.8, i.e. f up to the 1/30 Hz Nyquist).
__device__ __forceinline__ float sincpi_poly(float s) {
  float x = 3.14159265358979f * s;
  float z = x * x;
  float p = -1.0f / 1307674368000.0f;
  p = p * z + 1.0f / 6227020800.0f;
  p = p * z - 1.0f / 39916800.0f;
  p = p * z + 1.0f / 362880.0f;
  p = p * z - 1.0f / 5040.0f;
  p = p * z + 1.0f / 120.0f;
  p = p * z - 1.0f / 6.0f;
  p = p * z + 1.0f;
  return p;
}
__device__ __forceinline__ double sincpi_poly(double s) {
  double x = 3.141592653589793 * s;
  double z = x * x;
  double p = 1.0 / 51090942171709440000.0;
  p = p * z - 1.0 / 121645100408832000.0;
  p = p * z + 1.0 / 355687428096000.0;
  p = p * z - 1.0 / 1307674368000.0;
  p = p * z + 1.0 / 6227020800.0;
  p = p * z - 1.0 / 39916800.0;
  p = p * z + 1.0 / 362880.0;
  p = p * z - 1.0 / 5040.0;
  p = p * z + 1.0 / 120.0;
  p = p * z - 1.0 / 6.0;
  p = p * z + 1.0;
  return p;
}
// sin(pi s) / (pi s) for |pi s| <= kLoArg, cut after (pi s)^6 (first dropped term < 5e-11).
__device__ __forceinline__ float sincpi_poly_lo(float s) {
  float x = 3.14159265358979f * s;
  float z = x * x;
  float p = -1.0f / 5040.0f;
  p = p * z + 1.0f / 120.0f;
  p = p * z - 1.0f / 6.0f;
  p = p * z + 1.0f;
  return p;
}
__device__ __forceinline__ double sincpi_poly_lo(double s) { return sincpi_poly(s); }
template <bool LO, typename T> __device__ __forceinline__ typename CT<T>::C expi_sm(T x) {
  return LO ? expi_small_lo(x) : expi_small(x);
}
template <bool LO, typename T> __device__ __forceinline__ T sincpi_sm(T s) {
  return LO ? sincpi_poly_lo(s) : sincpi_poly(s);
}

// Per-source constants, computed in float64 and rounded once. Phases are in cycles.
// Every phase coefficient that multiplies an O(1) quantity is split into a float hi
// part and the float remainder lo, so that its rounding error does not become a
// systematic phase error of the band (the guiding-centre Doppler phase is ~2 cycles at
// 4 mHz and must be right to ~1e-7 cycles for Delta lnL to 1e-2 at SNR ~ 200).
template <typename T>
struct Src {
  long long q;     // carrier bin
  T dhi, dlo;      // delta = f0 T - q in [0, 1)
  T fdh, fdl;      // fdot T^2 / 2 (up to ~100 cycles at 20 mHz: split as well)
  T phh, phl;      // phi0 / (2 pi)
  T dxh, dxl, dyh, dyl;  // f0 k_x AU/c, f0 k_y AU/c: guiding-centre Doppler amplitudes
  T fkx, fky;      // fdot k_x AU/c, fdot k_y AU/c
  T f0, fdot;
  T kx, ky, kz;    // propagation direction
  T ux, uy, uz, vx, vy, vz;
  T c2p, s2p;      // cos 2psi, sin 2psi
  T hp, hc;        // A (1 + cos^2 i) S, 2 A cos i S with S = 2^64 (T / 2N) pi L / c
  bool zero;       // amplitude exactly zero
  bool lo;         // every series argument of the slow part within kLoArg (float path)
};

template <typename T> __device__ __forceinline__ void split(double x, T& hi, T& lo) {
  hi = (T)x;
  lo = (T)(x - (double)hi);
}

// __noinline__: one compiled body for every kernel (see gen_band).
template <typename T>
__device__ __noinline__ Src<T> make_src(const double* __restrict__ prm, int64_t stride,
                                           int64_t i, double tobs, int n) {
  Src<T> s;
  const double amp = prm[0 * stride + i];
  const double f0 = prm[1 * stride + i];
  const double fdot = prm[2 * stride + i];
  const double phi0 = prm[3 * stride + i];
  const double psi = prm[4 * stride + i];
  const double cosi = prm[5 * stride + i];
  const double sinb = prm[6 * stride + i];
  const double lam = prm[7 * stride + i];
  const double ft = f0 * tobs;
  const double qd = floor(ft);
  s.q = (long long)qd;
  split<T>(ft - qd, s.dhi, s.dlo);
  split<T>(0.5 * fdot * tobs * tobs, s.fdh, s.fdl);
  {
    double ph = phi0 * 0.15915494309189535;
    ph -= rint(ph);
    split<T>(ph, s.phh, s.phl);
  }
  const double cbd = sqrt(1.0 - sinb * sinb);
  double sld, cld;
  sincos(lam, &sld, &cld);
  const double aoc = kAU / kC;
  split<T>(-cbd * cld * f0 * aoc, s.dxh, s.dxl);
  split<T>(-cbd * sld * f0 * aoc, s.dyh, s.dyl);
  s.fkx = (T)(-cbd * cld * fdot * aoc);
  s.fky = (T)(-cbd * sld * fdot * aoc);
  s.f0 = (T)f0;
  s.fdot = (T)fdot;
  const T sb = (T)sinb;
  const T cb = (T)cbd;
  const T sl = (T)sld, cl = (T)cld;
  // sky position in float64: its rounding would move the antenna pattern (an amplitude
  // error, which <a|a> feels directly) by ~1e-7, too much for Delta lnL ~ 1e4 to 1e-2
  double s2d, c2d;
  sincos(2.0 * psi, &s2d, &c2d);
  const T s2 = (T)s2d, c2 = (T)c2d;
  s.kx = -cb * cl; s.ky = -cb * sl; s.kz = -sb;
  s.ux = sb * cl; s.uy = sb * sl; s.uz = -cb;
  s.vx = sl; s.vy = -cl; s.vz = (T)0;
  s.c2p = c2; s.s2p = s2;
  const double scale = 18446744073709551616.0 * (0.5 * tobs / n) * 3.141592653589793 * kLc;  // 2^64 (T/2N) pi L/c
  s.hp = (T)(amp * (1.0 + cosi * cosi) * scale);
  s.hc = (T)(2.0 * amp * cosi * scale);
  s.zero = (amp == 0.0);
  // x = 2 pi |f| L/c over the observation bounds the slow part's series arguments: the sincs'
  // pi s and the doubled arm delay reach x, a link phase pi f L/c k.n +- 2 pi f k.dx/c
  // (craft offsets |dx| = L/sqrt3) (1/2 + 1/sqrt3) x
  s.lo = 6.283185307179586 * fmax(fabs(f0), fabs(f0 + fdot * tobs)) * kLc <= kLoArg;
  return s;
}

// Radix-4 and radix-2 Stockham stages over both channels of the buffers (layout [2][N]),
// shared by NT threads (thread index tid); twiddles tw[m] = exp(-2 pi i m / N). Every
// butterfly is the same arithmetic whatever NT, so a warp and a block give the same bits.
template <typename C, int N, int NT>
__device__ __forceinline__ void stage_r4(const C* __restrict__ in, C* __restrict__ out,
                                         const C* __restrict__ tw, int ns, int lane) {
  constexpr int NB = N / 4;
  const int step = N / (ns * 4);
#pragma unroll 2
  for (int b = lane; b < 2 * NB; b += NT) {
    const int ch = b / NB;
    const int j = b - ch * NB;
    const C* x = in + ch * N;
    C* y = out + ch * N;
    const int k = j & (ns - 1);
    C v0 = x[j], v1 = x[j + NB], v2 = x[j + 2 * NB], v3 = x[j + 3 * NB];
    if (ns > 1) {
      v1 = cmul(v1, __ldg(&tw[k * step]));
      v2 = cmul(v2, __ldg(&tw[2 * k * step]));
      v3 = cmul(v3, __ldg(&tw[3 * k * step]));
    }
    // 4-point DFT with w = -i
    const C s02 = cadd(v0, v2), d02 = csub(v0, v2);
    const C s13 = cadd(v1, v3), d13 = cmul_mi(csub(v1, v3));
    const int d = (j - k) * 4 + k;
    y[d] = cadd(s02, s13);
    y[d + ns] = cadd(d02, d13);
    y[d + 2 * ns] = csub(s02, s13);
    y[d + 3 * ns] = csub(d02, d13);
  }
}

template <typename C, int N, int NT>
__device__ __forceinline__ void stage_r2_first(const C* __restrict__ in, C* __restrict__ out,
                                               int lane) {
  constexpr int NB = N / 2;
  for (int b = lane; b < 2 * NB; b += NT) {
    const int ch = b / NB;
    const int j = b - ch * NB;
    const C* x = in + ch * N;
    C* y = out + ch * N;
    const C v0 = x[j], v1 = x[j + NB];
    y[2 * j] = cadd(v0, v1);
    y[2 * j + 1] = csub(v0, v1);
  }
}

// Slow-part sample p of one source (band FFT input of the A and E channels): the TDI response
// at the coarse time t_p = p T / N times the heterodyned carrier.
template <typename T, int N, bool LO>
__device__ __forceinline__ void slow_sample(const Src<T>& src, const T* __restrict__ orb, int p, T dtp, T inv_n,
                                            typename CT<T>::C& outA, typename CT<T>::C& outE) {
  typedef typename CT<T>::C C;
  const T lc = (T)kLc;
  const T rs2 = (T)0.70710678118654752440;
  const T rs6 = (T)0.40824829046386301637;
  const T* o = orb + p;
  const T cah = o[0 * N], sah = o[1 * N], cal = o[20 * N], sal = o[21 * N];
  T dx[3][3], na[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      dx[c][d] = o[(2 + 3 * c + d) * N];
      na[c][d] = o[(11 + 3 * c + d) * N];
    }
  const T tp = (T)p * dtp;
  const T f = src.f0 + src.fdot * tp;
  const T flc = f * lc;
  const T pif = (T)3.14159265358979323846 * flc;
  // exponentials with small arguments: E0 = e^{-i pi f L/c}, Ea = e^{i pi f L/c k.n_a},
  // Ej = e^{-2 pi i f k.dx_j / c}; D = E0^2
  C ea[3], ej[3];
  T kn[3], jd[3];
  C nhn[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T kd = src.kx * dx[c][0] + src.ky * dx[c][1] + src.kz * dx[c][2];
    jd[c] = (T)-6.28318530717958647692 * f * kd;
    if (!LO) ej[c] = expi_sm<LO>(jd[c]);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T un = src.ux * na[a][0] + src.uy * na[a][1] + src.uz * na[a][2];
    const T vn = src.vx * na[a][0] + src.vy * na[a][1] + src.vz * na[a][2];
    kn[a] = src.kx * na[a][0] + src.ky * na[a][1] + src.kz * na[a][2];
    const T xp = un * un - vn * vn;
    const T xc = (T)2 * un * vn;
    nhn[a] = mkc(src.hp * (src.c2p * xp - src.s2p * xc), src.hc * (src.s2p * xp + src.c2p * xc));
    if (!LO) ea[a] = expi_sm<LO>(pif * kn[a]);
  }
  // link i->j (arm a, direction sign sg, receiver j), common factor E0 removed:
  //   y_ij = n.Hc.n sinc(pi f L/c (1 - sg k.n_a)) Ea^sg Ej
  // 12: (0,+,1) 21: (0,-,0) 23: (1,+,2) 32: (1,-,1) 31: (2,+,0) 13: (2,-,2)
  C y[6];
  const int arm[6] = {0, 0, 1, 1, 2, 2};
  const int rcv[6] = {1, 0, 2, 1, 0, 2};
#pragma unroll
  for (int l = 0; l < 6; ++l) {
    const bool plus = (l & 1) == 0;
    const T sarg = flc * ((T)1 - (plus ? kn[arm[l]] : -kn[arm[l]]));
    const T sc = sincpi_sm<LO>(sarg);
    // shorter series: the link phase from its summed argument (one series instead of two and
    // a complex product)
    const C ph = LO ? expi_sm<LO>(fmaf_(pif, plus ? kn[arm[l]] : -kn[arm[l]], jd[rcv[l]]))
                    : cmul(plus ? ea[arm[l]] : cconj(ea[arm[l]]), ej[rcv[l]]);
    y[l] = cmul(mkc(nhn[arm[l]].x * sc, nhn[arm[l]].y * sc), ph);
  }
  // y index: 0=12 1=21 2=23 3=32 4=31 5=13
  const C dd = LO ? expi_sm<LO>((T)-2 * pif) : [&] { const C e0 = expi_sm<LO>(-pif); return cmul(e0, e0); }();
  const C X = cadd(csub(y[4], y[1]), cmul(dd, csub(y[5], y[0])));
  const C Y = cadd(csub(y[0], y[3]), cmul(dd, csub(y[1], y[2])));
  const C Z = cadd(csub(y[2], y[5]), cmul(dd, csub(y[3], y[4])));
  const C As = cscale(csub(Z, X), rs2);
  const C Es = cscale(cadd(csub(X, cscale(Y, (T)2)), Z), rs6);
  // common factor: (-i f)(1 - D^2) E0 e^{2 pi i cyc0} = 2 f sin(2 pi f L/c) e^{2 pi i (cyc0 - 3/2 f L/c)},
  // cyc0 = phi0/2pi + delta p/N + fdot T^2 (p/N)^2 / 2 - f k.R_gc/c. The guiding-centre
  // Doppler phase (O(f0 AU/c) cycles) is formed in double-float and reduced exactly.
  T dop_h, dop_l;
  {
    const T p1 = src.dxh * cah, p2 = src.dyh * sah;
    T e1, e2;
    fma_err(src.dxh, cah, p1, e1);
    fma_err(src.dyh, sah, p2, e2);
    dop_h = p1 + p2;
    const T bp = dop_h - p1;
    const T es = (p1 - (dop_h - bp)) + (p2 - bp);
    dop_l = es + e1 + e2 + (src.dxh * cal + src.dyh * sal) + (src.dxl * cah + src.dyl * sah);
  }
  const T pn = (T)p * inv_n;
  const T pn2 = pn * pn;  // exact: p^2 < 2^24
  T xd = src.dhi * pn;
  xd -= rint_(xd);
  const T q1 = src.fdh * pn2;
  T q1e;
  fma_err(src.fdh, pn2, q1, q1e);
  T big = (src.phh - (dop_h - rint_(dop_h))) + (xd + (q1 - rint_(q1)));
  big -= rint_(big);
  const T small = (src.dlo * pn + src.phl) + (q1e + src.fdl * pn2) - dop_l
                  - tp * (src.fkx * cah + src.fky * sah) - (T)1.5 * flc;
  const C car = expi_cycles(big + small);
  const T amp = (T)2 * f * ((T)6.28318530717958647692 * flc) * sincpi_sm<LO>((T)2 * flc);
  const C com = cscale(car, amp);
  outA = cmul(com, As);
  outE = cmul(com, Es);
}

// Band FFT of buf0 ([2][N] slow-part samples) by NT threads, then the rotation by N/2 into
// band order in buf0; buf1 is scratch. `sync` orders the threads between passes.
template <typename C, int N, int NT, typename Sync>
__device__ __forceinline__ void band_fft(C* buf0, C* buf1, const C* __restrict__ tw, int tid, Sync sync) {
  // Stockham FFT: optional radix-2 first stage, then radix-4 stages.
  C* in = buf0;
  C* out = buf1;
  int ns = 1;
  if (N == 128 || N == 512) {
    stage_r2_first<C, N, NT>(in, out, tid);
    sync();
    C* t = in; in = out; out = t;
    ns = 2;
  }
  for (; ns < N; ns *= 4) {
    stage_r4<C, N, NT>(in, out, tw, ns, tid);
    sync();
    C* t = in; in = out; out = t;
  }
  // result is in `in`; rotate by N/2 into buf0 (band order)
  if (in == buf0) {
    for (int i = tid; i < N; i += NT) {   // swap halves, one thread per pair
      const int ch = i / (N / 2);
      const int ii = i - ch * (N / 2);
      C* b = buf0 + ch * N;
      const C lo = b[ii], hi = b[ii + N / 2];
      b[ii] = hi;
      b[ii + N / 2] = lo;
    }
  } else {
    for (int i = tid; i < 2 * N; i += NT) {
      const int ch = i / N;
      const int ii = i - ch * N;
      buf0[i] = in[ch * N + ((ii + N / 2) & (N - 1))];
    }
  }
  sync();
}

struct WarpSync {
  __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Generate the A/E band of one source into buf0 ([2][N], band order: element i is bin
// q - N/2 + i), in strain units times 2^64. buf1 is scratch of the same size.
// Called by all 32 lanes of a warp; returns with the warp synchronised.
template <typename T, int N>
__device__ __noinline__ void gen_band(const Src<T>* __restrict__ srcp, const T* __restrict__ orb,
                                      const typename CT<T>::C* __restrict__ tw, double tobs,
                                      typename CT<T>::C* buf0, typename CT<T>::C* buf1,
                                      int lane) {
  typedef typename CT<T>::C C;
  const Src<T> src = *srcp;
  const T dtp = (T)(tobs / N);
  const T inv_n = (T)1 / (T)N;
  // The per-sample body is long; unrolling the sample loop multiplies the code that
  // every warp must fetch (GBK_SAMPLE_UNROLL, chosen by measurement).
  if (sizeof(T) == 4 && src.lo) {   // the shorter series (one branch per warp: one source)
#pragma unroll (kSampleUnroll)
    for (int p = lane; p < N; p += 32) {
      C sa, se;
      slow_sample<T, N, true>(src, orb, p, dtp, inv_n, sa, se);
      buf0[p] = sa;
      buf0[N + p] = se;
    }
  } else {
#pragma unroll (kSampleUnroll)
    for (int p = lane; p < N; p += 32) {
      C sa, se;
      slow_sample<T, N, false>(src, orb, p, dtp, inv_n, sa, se);
      buf0[p] = sa;
      buf0[N + p] = se;
    }
  }
  __syncwarp();
  band_fft<C, N, 32>(buf0, buf1, tw, lane, WarpSync());
}

// The same band generated by all NT threads of a block (thread index tid): the samples and
// butterflies are shared out, each computed exactly as in gen_band (the same bits). Called by
// every thread of the block; returns with the block synchronised.
template <typename T, int N, int NT>
__device__ __noinline__ void gen_band_block(const Src<T>* __restrict__ srcp, const T* __restrict__ orb,
                                            const typename CT<T>::C* __restrict__ tw, double tobs,
                                            typename CT<T>::C* buf0, typename CT<T>::C* buf1, int tid) {
  typedef typename CT<T>::C C;
  const Src<T> src = *srcp;
  const T dtp = (T)(tobs / N);
  const T inv_n = (T)1 / (T)N;
  // two samples per thread at a time (a CTA has registers to spare here: -1.4 % at N = 1024);
  // each sample's arithmetic is the warp generator's, so both give the same bits
  if (sizeof(T) == 4 && src.lo) {
#pragma unroll 2
    for (int p = tid; p < N; p += NT) {
      C sa, se;
      slow_sample<T, N, true>(src, orb, p, dtp, inv_n, sa, se);
      buf0[p] = sa;
      buf0[N + p] = se;
    }
  } else {
#pragma unroll 2
    for (int p = tid; p < N; p += NT) {
      C sa, se;
      slow_sample<T, N, false>(src, orb, p, dtp, inv_n, sa, se);
      buf0[p] = sa;
      buf0[N + p] = se;
    }
  }
  __syncthreads();
  band_fft<C, N, NT>(buf0, buf1, tw, tid, BlockSync());
}

}  // namespace gbk
