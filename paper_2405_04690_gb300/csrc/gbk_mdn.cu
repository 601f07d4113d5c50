// Mixture-density network of the learned proposal: forward, loss and gradient, backward,
// Adam, all on BF16 tensor cores with float32 accumulation.
//
// The paper draws births from Gaussian mixtures fitted to earlier sampler output
// (Sec. V.E, App. G) and names learned density estimators as the next step (App. G).
// Here a small MLP maps a band's whitened residual (1024 values) to a 16-component
// truncated diagonal mixture over the band's unit-box coordinates (gbk_mix.cuh):
//   1024 -> 512 -> 512 -> 512 (ReLU) -> 272,  weights [out][in], float32 master copy.
// Every matrix product is one launch of k_gemm: mma.sync m16n8k16 BF16 x BF16 -> FP32,
// 3-stage cp.async pipeline through shared memory, operands of either orientation read
// with ldmatrix (.trans where the contraction index is the strided one), a fused
// epilogue (bias + ReLU -> BF16, bias -> FP32, ReLU-mask -> BF16, or split-K partials).
// Weight gradients are split over the batch into fixed partial slots and summed in a
// fixed order by the Adam / reduce kernel, so training is deterministic.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include "gbk_internal.cuh"
#include "gbk_mix.cuh"

namespace gbk {

constexpr int kIn = 1024, kHid = 512, kOut = kMixOut;
// flat parameter offsets (oracle order): W1 b1 W2 b2 W3 b3 W4 b4
constexpr int64_t kOffW1 = 0, kOffB1 = kOffW1 + (int64_t)kHid * kIn;
constexpr int64_t kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + (int64_t)kHid * kHid;
constexpr int64_t kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + (int64_t)kHid * kHid;
constexpr int64_t kOffW4 = kOffB3 + kHid, kOffB4 = kOffW4 + (int64_t)kOut * kHid;
constexpr int64_t kNParams = kOffB4 + kOut;
constexpr int kMaxSplit = 16;

typedef __nv_bfloat16 bf16;

// -------------------------------------------------------------- GEMM
enum { EPI_BIAS_RELU_BF16 = 0, EPI_BIAS_F32 = 1, EPI_MASK_BF16 = 2, EPI_PART_F32 = 3 };

struct GemmArgs {
  const bf16* A; int64_t lda;      // A(m, k) = AK ? A[m lda + k] : A[k lda + m]
  const bf16* B; int64_t ldb;      // B(k, n) = BK ? B[n ldb + k] : B[k ldb + n]
  int M, N, K, kps;                // kps: K range of one split (multiple of 32)
  const float* bias;               // [N]
  const bf16* mask; int64_t ldm;   // EPI_MASK: keep (m, n) where mask[m ldm + n] > 0
  void* C; int64_t ldc;            // C(m, n) = C[m ldc + n]
  int64_t split_stride;            // EPI_PART: split z writes C + z split_stride
};

constexpr int kBN = 128, kBK = 32, kStages = 3, kGemmThreads = 256;
constexpr int kPitchK = kBK + 8;       // [rows][k] tiles: 80-byte rows
constexpr int kPitchMN = 128 + 8;      // [k][rows] tiles: 272-byte rows

template <int BM, bool AK, bool BK>
struct GemmSmem {
  static constexpr int a_elems = AK ? BM * kPitchK : kBK * (BM + 8);
  static constexpr int b_elems = BK ? kBN * kPitchK : kBK * kPitchMN;
  static constexpr int stage_elems = a_elems + b_elems;
  static constexpr size_t bytes = (size_t)kStages * stage_elems * sizeof(bf16);
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool ok) {
  const int n = ok ? 16 : 0;   // src-size 0: fill the 16 bytes with zeros, read nothing
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Copy k-tile [k0, k0 + 32) of A and B into one pipeline stage (zero outside the matrix
// or the split's K range; every 16-byte chunk lies wholly inside or outside, since
// the contiguous extents are multiples of 8 elements).
template <int BM, bool AK, bool BK>
__device__ __forceinline__ void gemm_load(const GemmArgs& g, bf16* sa, bf16* sb, int m0, int n0, int k0, int kend) {
  const int tid = threadIdx.x;
  if (AK) {   // [BM][32]: BM x 4 chunks
    for (int c = tid; c < BM * 4; c += kGemmThreads) {
      const int r = c >> 2, kc = (c & 3) * 8;
      const int m = m0 + r, k = k0 + kc;
      const bool ok = m < g.M && k < kend;
      cp_async16(sa + r * kPitchK + kc, ok ? g.A + (int64_t)m * g.lda + k : g.A, ok);
    }
  } else {    // [32][BM]: 32 x BM/8 chunks
    constexpr int cpr = BM / 8;
    for (int c = tid; c < kBK * cpr; c += kGemmThreads) {
      const int r = c / cpr, mc = (c % cpr) * 8;
      const int k = k0 + r, m = m0 + mc;
      const bool ok = k < kend && m < g.M;
      cp_async16(sa + r * (BM + 8) + mc, ok ? g.A + (int64_t)k * g.lda + m : g.A, ok);
    }
  }
  if (BK) {   // [128][32]
    for (int c = tid; c < kBN * 4; c += kGemmThreads) {
      const int r = c >> 2, kc = (c & 3) * 8;
      const int n = n0 + r, k = k0 + kc;
      const bool ok = n < g.N && k < kend;
      cp_async16(sb + r * kPitchK + kc, ok ? g.B + (int64_t)n * g.ldb + k : g.B, ok);
    }
  } else {    // [32][128]
    for (int c = tid; c < kBK * 16; c += kGemmThreads) {
      const int r = c >> 4, nc = (c & 15) * 8;
      const int k = k0 + r, n = n0 + nc;
      const bool ok = k < kend && n < g.N;
      cp_async16(sb + r * kPitchMN + nc, ok ? g.B + (int64_t)k * g.ldb + n : g.B, ok);
    }
  }
}

// C tile [BM][128] per CTA; 8 warps as 2 (m) x 4 (n), each (BM/2) x 32.
template <int BM, bool AK, bool BK, int EPI>
__global__ void __launch_bounds__(kGemmThreads) k_gemm(const GemmArgs g) {
  constexpr int MI = BM / 32;   // m16 tiles per warp
  typedef GemmSmem<BM, AK, BK> SM;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  bf16* smem = reinterpret_cast<bf16*>(smem_raw);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int wm = wid >> 2, wn = wid & 3;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * kBN;
  const int kbeg = blockIdx.z * g.kps;
  const int kend = min(g.K, kbeg + g.kps);
  const int nk = kend > kbeg ? (kend - kbeg + kBK - 1) / kBK : 0;

  float acc[MI][4][4];
#pragma unroll
  for (int i = 0; i < MI; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) {
    if (s < nk) gemm_load<BM, AK, BK>(g, smem + s * SM::stage_elems, smem + s * SM::stage_elems + SM::a_elems, m0, n0,
                                      kbeg + s * kBK, kend);
    cp_commit();
  }
  const int r8 = lane & 7, mat = lane >> 3;
  for (int kt = 0; kt < nk; ++kt) {
    cp_wait<kStages - 2>();
    __syncthreads();
    {   // refill the stage consumed in the previous iteration
      const int nt = kt + kStages - 1;
      if (nt < nk) {
        const int st = nt % kStages;
        gemm_load<BM, AK, BK>(g, smem + st * SM::stage_elems, smem + st * SM::stage_elems + SM::a_elems, m0, n0,
                              kbeg + nt * kBK, kend);
      }
      cp_commit();
    }
    const bf16* sa = smem + (kt % kStages) * SM::stage_elems;
    const bf16* sb = sa + SM::a_elems;
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 16) {
      uint32_t af[MI][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < MI; ++i) {
        const int mb = wm * (BM / 2) + i * 16;
        if (AK) {   // matrix j: rows mb + (j & 1) 8, k kk + (j >> 1) 8
          ldsm_x4(af[i], sa + (mb + (mat & 1) * 8 + r8) * kPitchK + kk + (mat >> 1) * 8);
        } else {    // stored [k][m]: rows k = kk + (j >> 1) 8 + r, cols m = mb + (j & 1) 8
          ldsm_x4_t(af[i], sa + (kk + (mat >> 1) * 8 + r8) * (BM + 8) + mb + (mat & 1) * 8);
        }
      }
#pragma unroll
      for (int jp = 0; jp < 2; ++jp) {   // two n16 pairs -> four n8 tiles
        const int nb = wn * 32 + jp * 16;
        uint32_t r[4];
        if (BK) {   // stored [n][k]: matrix j: n = nb + (j >> 1) 8 + r, k = kk + (j & 1) 8
          ldsm_x4(r, sb + (nb + (mat >> 1) * 8 + r8) * kPitchK + kk + (mat & 1) * 8);
        } else {    // stored [k][n]: rows k = kk + (j & 1) 8 + r, cols n = nb + (j >> 1) 8
          ldsm_x4_t(r, sb + (kk + (mat & 1) * 8 + r8) * kPitchMN + nb + (mat >> 1) * 8);
        }
        bfr[2 * jp][0] = r[0]; bfr[2 * jp][1] = r[1];
        bfr[2 * jp + 1][0] = r[2]; bfr[2 * jp + 1][1] = r[3];
      }
#pragma unroll
      for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
    }
  }
  cp_wait<0>();

  // epilogue: acc[i][j] = rows m (e 0, 1) and m + 8 (e 2, 3), columns n, n + 1
  const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int i = 0; i < MI; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + wn * 32 + j * 8 + 2 * tq;
      if (n >= g.N) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = m0 + wm * (BM / 2) + i * 16 + gq + 8 * h;
        if (m >= g.M) continue;
        float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
        if (EPI == EPI_BIAS_RELU_BF16) {
          v0 = fmaxf(v0 + g.bias[n], 0.f);
          v1 = fmaxf(v1 + g.bias[n + 1], 0.f);
          *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<bf16*>(g.C) + (int64_t)m * g.ldc + n) =
              __floats2bfloat162_rn(v0, v1);
        } else if (EPI == EPI_BIAS_F32) {
          *reinterpret_cast<float2*>(reinterpret_cast<float*>(g.C) + (int64_t)m * g.ldc + n) =
              make_float2(v0 + g.bias[n], v1 + g.bias[n + 1]);
        } else if (EPI == EPI_MASK_BF16) {
          const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(g.mask + (int64_t)m * g.ldm + n);
          if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
          if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
          *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<bf16*>(g.C) + (int64_t)m * g.ldc + n) =
              __floats2bfloat162_rn(v0, v1);
        } else {
          *reinterpret_cast<float2*>(reinterpret_cast<float*>(g.C) + blockIdx.z * g.split_stride +
                                     (int64_t)m * g.ldc + n) = make_float2(v0, v1);
        }
      }
    }
}

template <int BM, bool AK, bool BK, int EPI>
static gbk_status gemm(const GemmArgs& g, int splits, cudaStream_t st) {
  typedef GemmSmem<BM, AK, BK> SM;
  static bool attr = false;   // per instantiation; same value on every device
  if (!attr) {
    if (cudaFuncSetAttribute(k_gemm<BM, AK, BK, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes) !=
        cudaSuccess) {
      cudaGetLastError();
      return set_error(GBK_ECUDA, "mdn: cannot set GEMM shared memory size");
    }
    attr = true;
  }
  dim3 grid((g.N + kBN - 1) / kBN, (g.M + BM - 1) / BM, splits);
  k_gemm<BM, AK, BK, EPI><<<grid, kGemmThreads, SM::bytes, st>>>(g);
  return check_launch("mdn gemm");
}

// -------------------------------------------------------------- loss and its gradient
// One warp per sample; lane k + 16 h handles component k, dimensions 4h .. 4h + 3.
// -ln q and d(-ln q)/d raw (the same formulas as the float64 oracle), gradient scaled
// by 1/B and stored as BF16 for the backward products; per-sample losses to nll[m].
__global__ void k_mdn_loss(const float* __restrict__ raw, const float* __restrict__ u, int B, float inv_b,
                           bf16* __restrict__ graw, float* __restrict__ nll) {
  const int lane = threadIdx.x & 31;
  const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (m >= B) return;
  const int k = lane & 15, h = lane >> 4;
  const float* r = raw + (int64_t)m * kOut + k * 17;
  const float lg = r[0];
  float mx = lg;
  for (int o = 8; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  float se = expf(lg - mx);
  for (int o = 8; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
  const float lpi = lg - (mx + logf(se));
  float mu[4], sg[4], ls[4], s[4], a[4], bb[4], z[4], pa[4], pb[4], uu[4];
  float part = 0.f;
  const float inv_sqrt2pi = 0.3989422804014327f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int d = 4 * h + i;
    mu[i] = 1.f / (1.f + expf(-r[1 + d]));
    sg[i] = 1.f / (1.f + expf(-r[9 + d]));
    ls[i] = (float)kMixSMin + (float)(kMixSMax - kMixSMin) * sg[i];
    s[i] = expf(ls[i]);
    a[i] = (1.f - mu[i]) / s[i];
    bb[i] = -mu[i] / s[i];
    z[i] = normcdff(a[i]) - normcdff(bb[i]);
    pa[i] = inv_sqrt2pi * expf(-0.5f * a[i] * a[i]);
    pb[i] = inv_sqrt2pi * expf(-0.5f * bb[i] * bb[i]);
    uu[i] = u[(int64_t)m * kMixDim + d];
    const float x = (uu[i] - mu[i]) / s[i];
    part += -0.5f * x * x - ls[i] - (float)kLogSqrt2Pi - logf(z[i]);
  }
  const float comp = lpi + part + __shfl_xor_sync(0xffffffffu, part, 16);
  float cm = comp;
  for (int o = 8; o > 0; o >>= 1) cm = fmaxf(cm, __shfl_xor_sync(0xffffffffu, cm, o));
  float ce = expf(comp - cm);
  for (int o = 8; o > 0; o >>= 1) ce += __shfl_xor_sync(0xffffffffu, ce, o);
  const float lq = cm + logf(ce);
  const float resp = expf(comp - lq);
  bf16* gr = graw + (int64_t)m * kOut + k * 17;
  if (h == 0) gr[0] = __float2bfloat16_rn((expf(lpi) - resp) * inv_b);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int d = 4 * h + i;
    const float dx = uu[i] - mu[i];
    const float dmu = dx / (s[i] * s[i]) - (pb[i] - pa[i]) / (s[i] * z[i]);
    const float dls = (dx / s[i]) * (dx / s[i]) - 1.f - (-a[i] * pa[i] + bb[i] * pb[i]) / z[i];
    gr[1 + d] = __float2bfloat16_rn(-resp * dmu * mu[i] * (1.f - mu[i]) * inv_b);
    gr[9 + d] = __float2bfloat16_rn(-resp * dls * (float)(kMixSMax - kMixSMin) * sg[i] * (1.f - sg[i]) * inv_b);
  }
  if (lane == 0) nll[m] = -lq;
}

// Mean of the per-sample losses, one block, fixed order.
__global__ void k_mean(const float* __restrict__ x, int n, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += (double)x[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] / (double)n;
}

// Bias gradients: column sums of g [B][N] over split z's rows, into part + z stride + off.
__global__ void k_colsum(const bf16* __restrict__ g, int B, int N, int kps, float* __restrict__ part,
                         int64_t stride, int64_t off) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int z = blockIdx.y;
  const int r1 = min(B, (z + 1) * kps);
  float s = 0.f;
  for (int r = z * kps; r < r1; ++r) s += __bfloat162float(g[(int64_t)r * N + n]);
  part[(int64_t)z * stride + off + n] = s;
}

// grad = sum over splits (fixed order).
__global__ void k_reduce(const float* __restrict__ part, int S, int64_t n, float* __restrict__ grad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < S; ++z) s += part[(int64_t)z * n + i];
    grad[i] = s;
  }
}

// Adam (Kingma & Ba 2015) on the float32 master parameters, gradient summed from the
// split partials (S > 0) or read directly (S == 0); refreshes the network's float32 and
// BF16 copies. c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t).
__global__ void k_adam(const float* __restrict__ part, int S, const float* __restrict__ grad, int64_t n,
                       float* __restrict__ p, float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                       float b2, float eps, float c1, float c2, float* __restrict__ pf, bf16* __restrict__ pb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float gi;
    if (S > 0) {
      gi = 0.f;
      for (int z = 0; z < S; ++z) gi += part[(int64_t)z * n + i];
    } else {
      gi = grad[i];
    }
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    p[i] = pi;
    pf[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void k_copy_params(const float* __restrict__ p, int64_t n, float* __restrict__ pf, bf16* __restrict__ pb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    pf[i] = p[i];
    pb[i] = __float2bfloat16_rn(p[i]);
  }
}

// Mixture rows, log densities and draws for the mdn_sample_logpdf entry point.
template <typename T>
__global__ void k_mix_eval(const float* __restrict__ raw, int B, double eps, const uint32_t* __restrict__ words,
                           float* __restrict__ u_out, const float* __restrict__ u_in, float* __restrict__ logq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  MixRow<T> m;
  mix_build<T>(raw + (int64_t)i * kMixOut, m);
  T u[kMixDim];
  if (words) {
    mix_draw<T>(m, words[(int64_t)i * 9], words + (int64_t)i * 9 + 1, u);
    if (u_out)
      for (int d = 0; d < kMixDim; ++d) u_out[(int64_t)i * kMixDim + d] = (float)u[d];
  } else {
    for (int d = 0; d < kMixDim; ++d) u[d] = (T)u_in[(int64_t)i * kMixDim + d];
  }
  if (logq) logq[i] = (float)mix_logq<T>(m, u, (T)eps);
}

}  // namespace gbk

using namespace gbk;


namespace {

int splits_for(int B, int* kps) {
  int S = (B + 255) / 256;
  if (S < 1) S = 1;
  if (S > kMaxSplit) S = kMaxSplit;
  int per = (B + S - 1) / S;
  per = (per + kBK - 1) / kBK * kBK;
  *kps = per;
  return S;
}

GemmArgs ga(const bf16* A, int64_t lda, const bf16* B, int64_t ldb, int M, int N, int K, void* C, int64_t ldc) {
  GemmArgs g;
  g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.M = M; g.N = N; g.K = K; g.kps = K;
  g.bias = nullptr; g.mask = nullptr; g.ldm = 0; g.C = C; g.ldc = ldc; g.split_stride = 0;
  return g;
}

// Forward through the four layers; raw outputs to out (float32 [B][272]).
gbk_status forward(gbk_mdn* net, const bf16* x, int B, float* out, cudaStream_t st) {
  const int64_t offw[4] = {kOffW1, kOffW2, kOffW3, kOffW4}, offb[4] = {kOffB1, kOffB2, kOffB3, kOffB4};
  const bf16* in = x;
  int64_t ldin = kIn;
  gbk_status s;
  for (int l = 0; l < 3; ++l) {
    GemmArgs g = ga(in, ldin, net->pb + offw[l], ldin, B, kHid, (int)ldin, net->h[l], kHid);
    g.bias = net->pf + offb[l];
    if ((s = (B >= 4096 ? gemm<128, true, true, EPI_BIAS_RELU_BF16>(g, 1, st)
                        : gemm<64, true, true, EPI_BIAS_RELU_BF16>(g, 1, st))))
      return s;
    in = net->h[l];
    ldin = kHid;
  }
  GemmArgs g = ga(in, kHid, net->pb + kOffW4, kHid, B, kOut, kHid, out, kOut);
  g.bias = net->pf + kOffB4;
  return gemm<64, true, true, EPI_BIAS_F32>(g, 1, st);
}

// Loss, gradient and backward pass; weight / bias gradient partials to net->part.
gbk_status backward(gbk_mdn* net, const bf16* x, const float* u, int B, double* loss, int* S_out, cudaStream_t st) {
  gbk_status s;
  if ((s = forward(net, x, B, net->raw, st))) return s;
  k_mdn_loss<<<(B + 7) / 8, 256, 0, st>>>(net->raw, u, B, 1.0f / (float)B, net->g4, net->nll);
  if ((s = check_launch("mdn loss"))) return s;
  if (loss) {
    k_mean<<<1, 256, 0, st>>>(net->nll, B, loss);
    if ((s = check_launch("mdn loss mean"))) return s;
  }
  int kps;
  const int S = splits_for(B, &kps);
  *S_out = S;
  const int64_t offw[4] = {kOffW1, kOffW2, kOffW3, kOffW4}, offb[4] = {kOffB1, kOffB2, kOffB3, kOffB4};
  const int nout[4] = {kHid, kHid, kHid, kOut}, nin[4] = {kIn, kHid, kHid, kHid};
  const bf16* gcur = net->g4;
  for (int l = 3; l >= 0; --l) {
    const bf16* hin = l == 0 ? x : net->h[l - 1];
    // dW_l[o][i] = sum_m g[m][o] hin[m][i]: A = g^T (M = out, contiguous in M), B = hin (contiguous in N)
    GemmArgs gw = ga(gcur, nout[l], hin, nin[l], nout[l], nin[l], B, net->part + offw[l], nin[l]);
    gw.kps = kps;
    gw.split_stride = kNParams;
    if ((s = gemm<128, false, false, EPI_PART_F32>(gw, S, st))) return s;
    k_colsum<<<dim3((nout[l] + 255) / 256, S), 256, 0, st>>>(gcur, B, nout[l], kps, net->part, kNParams, offb[l]);
    if ((s = check_launch("mdn bias gradient"))) return s;
    if (l == 0) break;
    // g_prev[m][i] = sum_o g[m][o] W[o][i], kept where the forward activation was positive
    bf16* gn = net->g[l & 1];
    GemmArgs gx = ga(gcur, nout[l], net->pb + offw[l], nin[l], B, nin[l], nout[l], gn, nin[l]);
    gx.mask = net->h[l - 1];
    gx.ldm = kHid;
    if ((s = (B >= 4096 ? gemm<128, true, false, EPI_MASK_BF16>(gx, 1, st)
                        : gemm<64, true, false, EPI_MASK_BF16>(gx, 1, st))))
      return s;
    gcur = gn;
  }
  return GBK_OK;
}

gbk_status check_batch(gbk_mdn* net, int B, const char* what) {
  if (!net) return set_error(GBK_EINVAL, "%s: null network", what);
  if (B < 1 || B > net->max_batch) return set_error(GBK_EINVAL, "%s: batch %d outside [1, %d]", what, B, net->max_batch);
  if (!net->have_params) return set_error(GBK_EINVAL, "%s: parameters not set (call mdn_set_params)", what);
  return GBK_OK;
}

int blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b > 152 * 16 ? 152 * 16 : b);
}

}  // namespace

extern "C" int64_t mdn_param_count(void) { return kNParams; }

extern "C" gbk_status mdn_create(gbk_mdn** out, int32_t max_batch) {
  if (!out) return set_error(GBK_EINVAL, "mdn_create: null output pointer");
  *out = nullptr;
  if (max_batch < 1 || max_batch > (1 << 22)) return set_error(GBK_EINVAL, "mdn_create: max_batch out of range");
  gbk_mdn* n = new gbk_mdn();
  n->max_batch = max_batch;
  const size_t B = (size_t)max_batch;
  bool ok = cudaMalloc(&n->pf, kNParams * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->pb, kNParams * sizeof(bf16)) == cudaSuccess &&
            cudaMalloc(&n->raw, B * kOut * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->g4, B * kOut * sizeof(bf16)) == cudaSuccess &&
            cudaMalloc(&n->nll, B * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->part, (size_t)kMaxSplit * kNParams * sizeof(float)) == cudaSuccess;
  for (int i = 0; i < 3 && ok; ++i) ok = cudaMalloc(&n->h[i], B * kHid * sizeof(bf16)) == cudaSuccess;
  for (int i = 0; i < 2 && ok; ++i) ok = cudaMalloc(&n->g[i], B * kHid * sizeof(bf16)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    mdn_destroy(n);
    return set_error(GBK_ENOMEM, "mdn_create: device allocation failed (max_batch %d)", max_batch);
  }
  *out = n;
  return GBK_OK;
}

extern "C" gbk_status mdn_destroy(gbk_mdn* n) {
  if (!n) return GBK_OK;
  cudaFree(n->pf); cudaFree(n->pb); cudaFree(n->raw); cudaFree(n->g4); cudaFree(n->nll); cudaFree(n->part);
  for (int i = 0; i < 3; ++i) cudaFree(n->h[i]);
  for (int i = 0; i < 2; ++i) cudaFree(n->g[i]);
  delete n;
  return GBK_OK;
}

extern "C" gbk_status mdn_set_params(gbk_mdn* net, const float* params, void* stream) {
  if (!net || !params) return set_error(GBK_EINVAL, "mdn_set_params: null argument");
  k_copy_params<<<blocks_for(kNParams), 256, 0, (cudaStream_t)stream>>>(params, kNParams, net->pf, net->pb);
  net->have_params = true;
  return check_launch("mdn_set_params");
}

extern "C" gbk_status mdn_forward(gbk_mdn* net, const uint16_t* x, int32_t batch, float* raw, void* stream) {
  gbk_status s = check_batch(net, batch, "mdn_forward");
  if (s) return s;
  if (!x || !raw) return set_error(GBK_EINVAL, "mdn_forward: null device pointer");
  if (((uintptr_t)x & 15) || ((uintptr_t)raw & 7)) return set_error(GBK_EINVAL, "mdn_forward: misaligned buffer");
  return forward(net, reinterpret_cast<const bf16*>(x), batch, raw, (cudaStream_t)stream);
}

extern "C" gbk_status mdn_backward(gbk_mdn* net, const uint16_t* x, const float* u, int32_t batch, float* grad,
                                   double* loss, void* stream) {
  gbk_status s = check_batch(net, batch, "mdn_backward");
  if (s) return s;
  if (!x || !u || !grad) return set_error(GBK_EINVAL, "mdn_backward: null device pointer");
  if ((uintptr_t)x & 15) return set_error(GBK_EINVAL, "mdn_backward: x must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  int S = 0;
  if ((s = backward(net, reinterpret_cast<const bf16*>(x), u, batch, loss, &S, st))) return s;
  k_reduce<<<blocks_for(kNParams), 256, 0, st>>>(net->part, S, kNParams, grad);
  return check_launch("mdn_backward");
}

extern "C" gbk_status mdn_adam(gbk_mdn* net, float* params, float* m, float* v, const float* grad, int32_t step,
                               float lr, float beta1, float beta2, float eps, void* stream) {
  if (!net || !params || !m || !v || !grad) return set_error(GBK_EINVAL, "mdn_adam: null argument");
  if (step < 1) return set_error(GBK_EINVAL, "mdn_adam: step counts from 1");
  const float c1 = (float)(1.0 / (1.0 - pow((double)beta1, step)));
  const float c2 = (float)(1.0 / (1.0 - pow((double)beta2, step)));
  k_adam<<<blocks_for(kNParams), 256, 0, (cudaStream_t)stream>>>(nullptr, 0, grad, kNParams, params, m, v, lr, beta1,
                                                                  beta2, eps, c1, c2, net->pf, net->pb);
  net->have_params = true;
  return check_launch("mdn_adam");
}

extern "C" gbk_status mdn_train_step(gbk_mdn* net, float* params, float* m, float* v, const uint16_t* x,
                                     const float* u, int32_t batch, int32_t step, float lr, double* loss,
                                     void* stream) {
  gbk_status s = check_batch(net, batch, "mdn_train_step");
  if (s) return s;
  if (!params || !m || !v || !x || !u) return set_error(GBK_EINVAL, "mdn_train_step: null device pointer");
  if ((uintptr_t)x & 15) return set_error(GBK_EINVAL, "mdn_train_step: x must be 16-byte aligned");
  if (step < 1) return set_error(GBK_EINVAL, "mdn_train_step: step counts from 1");
  cudaStream_t st = (cudaStream_t)stream;
  int S = 0;
  if ((s = backward(net, reinterpret_cast<const bf16*>(x), u, batch, loss, &S, st))) return s;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 / (1.0 - pow(b1, step))), c2 = (float)(1.0 / (1.0 - pow(b2, step)));
  k_adam<<<blocks_for(kNParams), 256, 0, st>>>(net->part, S, nullptr, kNParams, params, m, v, lr, (float)b1, (float)b2,
                                              1e-8f, c1, c2, net->pf, net->pb);
  return check_launch("mdn_train_step");
}

extern "C" gbk_status mdn_sample_logpdf(const float* raw, int32_t batch, double eps, const uint32_t* words,
                                        float* u_out, const float* u_in, float* logq, int precision, void* stream) {
  if (batch < 0) return set_error(GBK_EINVAL, "mdn_sample_logpdf: batch < 0");
  if (batch == 0) return GBK_OK;
  if (!raw || (!words && !u_in)) return set_error(GBK_EINVAL, "mdn_sample_logpdf: null device pointer");
  if (!(eps >= 0.0 && eps <= 1.0)) return set_error(GBK_EINVAL, "mdn_sample_logpdf: eps outside [0, 1]");
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = (batch + 63) / 64;
  if (precision == GBK_FP64)
    k_mix_eval<double><<<blocks, 64, 0, st>>>(raw, batch, eps, words, u_out, u_in, logq);
  else if (precision == GBK_MIXED)
    k_mix_eval<float><<<blocks, 64, 0, st>>>(raw, batch, eps, words, u_out, u_in, logq);
  else
    return set_error(GBK_EINVAL, "mdn_sample_logpdf: bad precision");
  return check_launch("mdn_sample_logpdf");
}
