// Mixture-density network of the learned proposal: forward, loss and gradient, backward,
// Adam, all on BF16 tensor cores with float32 accumulation.
//
// The paper draws births from Gaussian mixtures fitted to earlier sampler output
// (Sec. V.E, App. G) and names learned density estimators as the next step (App. G).
// Here a small MLP maps a band's whitened residual (1024 values) to a 16-component
// truncated diagonal mixture over the band's unit-box coordinates (gbk_mix.cuh):
//   1024 -> 512 -> 512 -> 512 (ReLU) -> 272,  weights [out][in], float32 master copy.
// Every matrix product is one launch of the tcgen05 kernel of gbk_umma.cuh (TMA tiles,
// 128 x 128 accumulator in tensor memory, fused epilogue). Both of its operands are
// K-contiguous, so the backward products read transposed copies that the producing kernels
// write alongside: hidden activations h^T and back-propagated signals g^T (by the GEMM
// epilogues and the loss kernel), W^T of layers 2-4 (by the parameter update), x^T (by a
// transpose kernel). The back-propagated signal is kept as a BF16 pair g = hi + lo (about 16
// significant bits): every backward product contracts over [hi | lo] against a doubled copy
// of its other operand ([W^T | W^T], [h^T | h^T]), so it sums hi and lo terms in one
// accumulator. Weight gradients are split over the batch into fixed partial slots
// and summed in a fixed order by the Adam / reduce kernel, so training is deterministic.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <string.h>

#include <mutex>

#include "gbk_internal.cuh"
#include "gbk_mix.cuh"
#include "gbk_umma.cuh"

namespace gbk {

constexpr int kIn = 1024, kHid = 512, kOut = kMixOut;
// flat parameter offsets (oracle order): W1 b1 W2 b2 W3 b3 W4 b4
constexpr int64_t kOffW1 = 0, kOffB1 = kOffW1 + (int64_t)kHid * kIn;
constexpr int64_t kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + (int64_t)kHid * kHid;
constexpr int64_t kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + (int64_t)kHid * kHid;
constexpr int64_t kOffW4 = kOffB3 + kHid, kOffB4 = kOffW4 + (int64_t)kOut * kHid;
constexpr int64_t kNParams = kOffB4 + kOut;
constexpr int kMaxSplit = 8;

typedef __nv_bfloat16 bf16;

// transposed weight copies W^T [in][out] of layers 2-4 (the input-gradient products' B)
// (each row doubled: [in][2 out] = [W^T | W^T])
constexpr int64_t kOffT2 = 0, kOffT3 = 2 * (int64_t)kHid * kHid, kOffT4 = 4 * (int64_t)kHid * kHid;
constexpr int64_t kNT = kOffT4 + 2 * (int64_t)kHid * kOut;

// Launch with programmatic stream serialization (see griddep_wait): every kernel launched this
// way calls griddep_wait() before it touches global memory.
template <typename... KArgs, typename... Args>
static gbk_status launch_pdl(const char* what, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k, args...);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(GBK_ECUDA, "%s: launch failed: %s", what, cudaGetErrorString(e));
  }
  return GBK_OK;
}

// -------------------------------------------------------------- tensor-core products
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// TMA map of a row-major BF16 matrix [rows][ld] read as [rows][K] tiles of box_rows x 64,
// from the workspace's cache when the same operand was seen before.
static gbk_status tmap(gbk_mdn* net, CUtensorMap* m, const bf16* p, int64_t rows, int64_t K, int64_t ld,
                       int box_rows) {
  for (int i = 0; i < net->n_maps; ++i) {
    const gbk_mdn::MapEntry& e = net->maps[i];
    if (e.p == p && e.rows == rows && e.k == K && e.ld == ld && e.box == box_rows) {
      memcpy(m, e.map, sizeof(CUtensorMap));
      return GBK_OK;
    }
  }
  EncodeTiledFn fn = encode_fn();
  if (!fn) return set_error(GBK_ECUDA, "mdn: cuTensorMapEncodeTiled unavailable");
  if (((uintptr_t)p & 15) || ((ld * 2) & 15)) return set_error(GBK_EINVAL, "mdn: operand not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)umma::kBK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(p), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(GBK_ECUDA, "mdn: tensor map encoding failed (%d)", (int)r);
  const int slot = net->n_maps < 48 ? net->n_maps++ : (net->next_map++ % 48);
  gbk_mdn::MapEntry& e = net->maps[slot];
  e.p = p; e.rows = rows; e.k = K; e.ld = ld; e.box = box_rows;
  memcpy(e.map, m, sizeof(CUtensorMap));
  return GBK_OK;
}

constexpr int kBN = 128;

// C[M][N] = A[M][K] . B[N][K]^T (+ epilogue); A, B row-major BF16 with leading dimensions.
template <int EPI>
static gbk_status mm(gbk_mdn* net, const bf16* A, int64_t lda, const bf16* B, int64_t ldb, int M, int N, int K,
                     umma::Args g, int splits, cudaStream_t st) {
  typedef umma::Smem<kBN> SM;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(umma::k_umma<kBN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes) !=
        cudaSuccess) {
      cudaGetLastError();
      return set_error(GBK_ECUDA, "mdn: cannot set the tensor-core kernel's shared memory size");
    }
    attr = true;
  }
  CUtensorMap ma, mb;
  gbk_status s;
  if ((s = tmap(net, &ma, A, M, K, lda, umma::kBM))) return s;
  if ((s = tmap(net, &mb, B, N, K, ldb, kBN))) return s;
  g.M = M;
  g.N = N;
  g.K = K;
  if (splits <= 1) g.kps = K;
  dim3 grid((N + kBN - 1) / kBN, (M + umma::kBM - 1) / umma::kBM, splits > 1 ? splits : 1);
  return launch_pdl("mdn tensor-core product", umma::k_umma<kBN, EPI>, grid, dim3(umma::kThreads), SM::bytes, st, ma,
                    mb, g);
}

static umma::Args margs(gbk_mdn* net, void* C, int64_t ldc) {
  umma::Args g;
  g.M = g.N = g.K = g.kps = 0;
  g.bias = nullptr;
  g.mask = nullptr;
  g.ldm = 0;
  g.C = C;
  g.ldc = ldc;
  g.split_stride = 0;
  g.CT = nullptr;
  g.ldct = 0;
  g.ct_dup = 0;
  g.err = net->err;
  return g;
}

// Transposes x [B][cols] through 32 x 32 shared-memory tiles into [x^T | x^T]: xt[c][r] and
// xt[c][B + r].
__global__ void k_transpose(const bf16* __restrict__ x, int B, int cols, bf16* __restrict__ xt, int64_t ldt) {
  umma::griddep_wait();
  umma::griddep_launch();
  __shared__ bf16 t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < B && c < cols) t[i][threadIdx.x] = x[(int64_t)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < B && c < cols) {
      xt[(int64_t)c * ldt + r] = t[threadIdx.x][i];
      xt[(int64_t)c * ldt + B + r] = t[threadIdx.x][i];
    }
  }
}

// Training rows of one minibatch and their transposed copy in one pass: a block takes 64 rows x
// 64 features, x[order[r]] -> xb[r] (16-byte chunks), and through a shared-memory tile
// xT[c][r] = xT[c][B + r] = x[order[r]][c] ([x^T | x^T], the weight-gradient product's B
// operand). u[order[r]] -> ub[r] by the blocks of the first feature column.
__global__ void __launch_bounds__(256) k_gather_t(const bf16* __restrict__ x, const float* __restrict__ u,
                                                  const int32_t* __restrict__ order, int B, int64_t n_rows,
                                                  bf16* __restrict__ xb, float* __restrict__ ub,
                                                  bf16* __restrict__ xT, int64_t ldt, int* err) {
  umma::griddep_wait();
  umma::griddep_launch();
  __shared__ uint32_t t[64][33];   // 64 rows x 64 BF16 (pairs), odd pitch: column reads hit 32 banks
  const int c0 = blockIdx.x * 64, r0 = blockIdx.y * 64;
  for (int idx = threadIdx.x; idx < 64 * 8; idx += 256) {
    const int r = idx >> 3, c8 = idx & 7;
    const int row = r0 + r;
    if (row >= B) continue;
    const int32_t src = order[row];
    uint4 q = make_uint4(0, 0, 0, 0);
    if (src < 0 || src >= n_rows) {   // bad index: zero row, error bit, nothing read
      if (c8 == 0) atomicOr(err, 4);
      if (blockIdx.x == 0 && c8 == 0)
        for (int d = 0; d < kMixDim; ++d) ub[(int64_t)row * kMixDim + d] = 0.5f;
    } else {
      q = reinterpret_cast<const uint4*>(x + (int64_t)src * kIn + c0)[c8];
      if (blockIdx.x == 0 && c8 == 0)
        for (int d = 0; d < kMixDim; ++d) ub[(int64_t)row * kMixDim + d] = u[(int64_t)src * kMixDim + d];
    }
    reinterpret_cast<uint4*>(xb + (int64_t)row * kIn + c0)[c8] = q;
    t[r][4 * c8] = q.x;
    t[r][4 * c8 + 1] = q.y;
    t[r][4 * c8 + 2] = q.z;
    t[r][4 * c8 + 3] = q.w;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < 64; c += 8) {
    bf16* dst = xT + (int64_t)(c0 + c) * ldt;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = lane + 32 * h;
      if (r0 + r >= B) continue;
      const uint32_t w = t[r][c >> 1];
      const unsigned short bits = (c & 1) ? (unsigned short)(w >> 16) : (unsigned short)(w & 0xffffu);
      const bf16 v = __ushort_as_bfloat16(bits);
      dst[r0 + r] = v;
      dst[B + r0 + r] = v;
    }
  }
}

// -------------------------------------------------------------- loss and its gradient
// -ln q of sample m and d(-ln q)/d raw (the same formulas as the float64 oracle), the gradient
// scaled by 1/B as BF16 pairs into grow = [hi 272 | lo 272]; one warp, lane k + 16 h handles
// component k, dimensions 4h .. 4h + 3.
__device__ __forceinline__ void loss_row(const float* __restrict__ raw, const float* __restrict__ u, int m, int lane,
                                         float inv_b, bf16* grow, float* __restrict__ nll) {
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
  bf16* gr = grow + k * 17;   // [hi | lo] pairs, row of 2 x 272
  auto put = [&](int j, float v) {
    const bf16 hi = __float2bfloat16_rn(v);
    gr[j] = hi;
    gr[kOut + j] = __float2bfloat16_rn(v - __bfloat162float(hi));
  };
  if (h == 0) put(0, (expf(lpi) - resp) * inv_b);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int d = 4 * h + i;
    const float dx = uu[i] - mu[i];
    const float dmu = dx / (s[i] * s[i]) - (pb[i] - pa[i]) / (s[i] * z[i]);
    const float dls = (dx / s[i]) * (dx / s[i]) - 1.f - (-a[i] * pa[i] + bb[i] * pb[i]) / z[i];
    put(1 + d, -resp * dmu * mu[i] * (1.f - mu[i]) * inv_b);
    put(9 + d, -resp * dls * (float)(kMixSMax - kMixSMin) * sg[i] * (1.f - sg[i]) * inv_b);
  }
  if (lane == 0) nll[m] = -lq;
}

// A block of 16 warps takes 16 samples, one per warp (loss_row into a shared-memory tile), then
// writes the gradient rows graw[m] = [hi 272 | lo 272] and their transposed copy gT[j][m] = hi,
// gT[j][B + m] = lo (the weight-gradient product's A operand); per-sample losses to nll[m].
constexpr int kLossRows = 16, kLossPitch = 2 * kMixOut + 2;   // odd word pitch: column reads hit distinct banks
__global__ void __launch_bounds__(kLossRows * 32, 2)
k_mdn_loss(const float* __restrict__ raw, const float* __restrict__ u, int B, float inv_b, bf16* __restrict__ graw,
           bf16* __restrict__ gT, int64_t ldt, float* __restrict__ nll) {
  umma::griddep_wait();
  umma::griddep_launch();
  __shared__ __align__(16) bf16 tile[kLossRows][kLossPitch];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m0 = blockIdx.x * kLossRows;
  if (m0 + warp < B) loss_row(raw, u, m0 + warp, lane, inv_b, &tile[warp][0], nll);
  __syncthreads();
  const int nr = min(kLossRows, B - m0);
  for (int idx = threadIdx.x; idx < nr * kOut; idx += kLossRows * 32) {   // rows, as 32-bit words
    const int r = idx / kOut, wd = idx % kOut;
    reinterpret_cast<uint32_t*>(graw + (int64_t)(m0 + r) * 2 * kOut)[wd] =
        reinterpret_cast<const uint32_t*>(&tile[r][0])[wd];
  }
  const int r = lane & 15;   // a warp writes two columns of 16 samples at a time
  if (r < nr)
    for (int j = 2 * warp + (lane >> 4); j < 2 * kOut; j += 2 * kLossRows) {
      const int jj = j < kOut ? j : j - kOut;
      gT[(int64_t)jj * ldt + (j < kOut ? 0 : B) + m0 + r] = tile[r][j];
    }
}

// Mean of the per-sample losses, one block, fixed order.
__global__ void k_mean(const float* __restrict__ x, int n, double* __restrict__ out) {
  umma::griddep_wait();
  umma::griddep_launch();
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

// Bias gradients: row sums of the transposed signal gT [N][hi B | lo B] (pitch ldt), one warp per
// row (16-byte loads, lanes in a fixed order, then a fixed shuffle tree), into partial slot 0 at
// part + off; slots 1 .. S-1 of those entries get 0 (the parameter update sums every slot).
__global__ void __launch_bounds__(256) k_bias_grad(const bf16* __restrict__ gT, int64_t ldt, int n2, int N,
                                                   float* __restrict__ part, int S, int64_t stride, int64_t off) {
  umma::griddep_wait();
  umma::griddep_launch();
  const int lane = threadIdx.x & 31;
  const int n = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (n >= N) return;
  const bf16* row = gT + (int64_t)n * ldt;
  const int nv = n2 >> 3;
  float s = 0.f;
#pragma unroll 4
  for (int j = lane; j < nv; j += 32) {
    const uint4 q = reinterpret_cast<const uint4*>(row)[j];
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 f = __bfloat1622float2(h[e]);
      s += f.x + f.y;
    }
  }
  for (int j = 8 * nv + lane; j < n2; j += 32) s += __bfloat162float(row[j]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane < S) part[(int64_t)lane * stride + off + n] = lane == 0 ? s : 0.f;
}

// grad = sum over splits (fixed order).
__global__ void k_reduce(const float* __restrict__ part, int S, int64_t n, float* __restrict__ grad) {
  umma::griddep_wait();
  umma::griddep_launch();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < S; ++z) s += part[(int64_t)z * n + i];
    grad[i] = s;
  }
}

// Adam (Kingma & Ba 2015) on the float32 master parameters, gradient summed from the
// split partials (S > 0) or read directly (S == 0); refreshes the network's float32 and
// BF16 copies. c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t).
// Store parameter i into the network's copies: float32, BF16 and, for the weights of
// layers 2-4, the transposed BF16 copy W^T [in][out].
__device__ __forceinline__ void store_param(int64_t i, float v, float* pf, bf16* pb, bf16* pbt) {
  pf[i] = v;
  const bf16 b = __float2bfloat16_rn(v);
  pb[i] = b;
  int64_t off, tof;
  int nout;
  if (i >= kOffW2 && i < kOffB2) { off = kOffW2; tof = kOffT2; nout = kHid; }
  else if (i >= kOffW3 && i < kOffB3) { off = kOffW3; tof = kOffT3; nout = kHid; }
  else if (i >= kOffW4 && i < kOffB4) { off = kOffW4; tof = kOffT4; nout = kOut; }
  else return;
  const int64_t r = i - off;              // W[o][ii], o = r / 512, ii = r % 512
  bf16* row = pbt + tof + (r % kHid) * 2 * nout;
  row[r / kHid] = b;
  row[nout + r / kHid] = b;
}

struct AdamArgs {
  const float* part;   // split partials [S][n] (S > 0), else grad
  int S;
  const float* grad;
  float *p, *m, *v;
  float lr, b1, b2, eps, c1, c2;
  float* pf;
  bf16 *pb, *pbt;
};

// Adam update of parameter i: moments, float32 master value and its float32 / BF16 copies;
// returns the BF16 value.
__device__ __forceinline__ bf16 adam_one(const AdamArgs& a, int64_t i) {
  float gi;
  if (a.S > 0) {
    gi = 0.f;
    for (int z = 0; z < a.S; ++z) gi += a.part[(int64_t)z * kNParams + i];
  } else {
    gi = a.grad[i];
  }
  const float mi = a.b1 * a.m[i] + (1.f - a.b1) * gi;
  const float vi = a.b2 * a.v[i] + (1.f - a.b2) * gi * gi;
  a.m[i] = mi;
  a.v[i] = vi;
  const float pi = a.p[i] - a.lr * (mi * a.c1) / (sqrtf(vi * a.c2) + a.eps);
  a.p[i] = pi;
  a.pf[i] = pi;
  const bf16 b = __float2bfloat16_rn(pi);
  a.pb[i] = b;
  return b;
}

// Blocks [0, kAdamTiles): 32 x 32 tiles of W2, W3, W4 (rows o, columns i), updated along i and
// written transposed through shared memory into [W^T | W^T]; the remaining blocks: W1 and the
// biases, one parameter per thread.
constexpr int kAdamTiles = 2 * (kHid / 32) * (kHid / 32) + ((kOut + 31) / 32) * (kHid / 32);
constexpr int64_t kAdamFlat = kOffW2 + 2 * kHid + kOut;   // W1, b1 | b2, b3, b4
__global__ void __launch_bounds__(256) k_adam(const AdamArgs a) {
  umma::griddep_wait();
  umma::griddep_launch();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (blockIdx.x < kAdamTiles) {
    __shared__ bf16 tile[32][34];
    int t = blockIdx.x, nout = kHid;
    int64_t off = kOffW2, tof = kOffT2;
    if (t >= 512) { t -= 512; off = kOffW4; tof = kOffT4; nout = kOut; }
    else if (t >= 256) { t -= 256; off = kOffW3; tof = kOffT3; }
    const int o0 = (t / (kHid / 32)) * 32, i0 = (t % (kHid / 32)) * 32;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int o = o0 + ty + 8 * j;
      if (o < nout) tile[ty + 8 * j][tx] = adam_one(a, off + (int64_t)o * kHid + i0 + tx);
    }
    __syncthreads();
    const int o = o0 + tx;
    if (o < nout)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        bf16* row = a.pbt + tof + (int64_t)(i0 + ty + 8 * j) * 2 * nout;
        const bf16 b = tile[tx][ty + 8 * j];
        row[o] = b;
        row[nout + o] = b;
      }
    return;
  }
  const int64_t j = (int64_t)(blockIdx.x - kAdamTiles) * 256 + threadIdx.x;
  if (j >= kAdamFlat) return;
  int64_t i = j;
  if (j >= kOffW2) {
    const int64_t r = j - kOffW2;
    i = r < kHid ? kOffB2 + r : r < 2 * kHid ? kOffB3 + (r - kHid) : kOffB4 + (r - 2 * kHid);
  }
  adam_one(a, i);
}
constexpr int kAdamBlocks = kAdamTiles + (int)((kAdamFlat + 255) / 256);

__global__ void k_copy_params(const float* __restrict__ p, int64_t n, float* __restrict__ pf, bf16* __restrict__ pb,
                              bf16* __restrict__ pbt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    store_param(i, p[i], pf, pb, pbt);
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

AdamArgs adam_args(gbk_mdn* net, const float* part, int S, const float* grad, float* p, float* m, float* v, float lr,
                   float b1, float b2, float eps, float c1, float c2) {
  AdamArgs a;
  a.part = part; a.S = S; a.grad = grad; a.p = p; a.m = m; a.v = v;
  a.lr = lr; a.b1 = b1; a.b2 = b2; a.eps = eps; a.c1 = c1; a.c2 = c2;
  a.pf = net->pf; a.pb = net->pb; a.pbt = net->pbT;
  return a;
}

int splits_for(int B, int* kps) {
  int S = (B + 511) / 512;
  if (S < 1) S = 1;
  if (S > kMaxSplit) S = kMaxSplit;
  int per = (B + S - 1) / S;
  per = (per + umma::kBK - 1) / umma::kBK * umma::kBK;   // whole 64-wide k tiles per split
  S = (B + per - 1) / per;
  *kps = per;
  return S;
}

// Forward through the four layers; raw outputs to out (float32 [B][272]). With
// transposed = true the hidden activations are also written as [h^T | h^T] [512][ldt].
gbk_status forward(gbk_mdn* net, const bf16* x, int B, float* out, bool transposed, cudaStream_t st) {
  const int64_t offw[4] = {kOffW1, kOffW2, kOffW3, kOffW4}, offb[4] = {kOffB1, kOffB2, kOffB3, kOffB4};
  const bf16* in = x;
  int64_t ldin = kIn;
  gbk_status s;
  for (int l = 0; l < 3; ++l) {
    umma::Args g = margs(net, net->h[l], kHid);
    g.bias = net->pf + offb[l];
    if (transposed) {
      g.CT = net->hT[l];
      g.ldct = net->ldt;
      g.ct_dup = 1;
    }
    if ((s = mm<umma::EPI_BIAS_RELU_BF16>(net, in, ldin, net->pb + offw[l], ldin, B, kHid, (int)ldin, g, 1, st))) return s;
    in = net->h[l];
    ldin = kHid;
  }
  umma::Args g = margs(net, out, kOut);
  g.bias = net->pf + kOffB4;
  return mm<umma::EPI_BIAS_F32>(net, in, kHid, net->pb + kOffW4, kHid, B, kOut, kHid, g, 1, st);
}

// Loss, gradient and backward pass; weight / bias gradient partials to net->part.
// x_t_ready: net->xT already holds [x^T | x^T] (written by the training-row gather).
gbk_status backward(gbk_mdn* net, const bf16* x, const float* u, int B, double* loss, int* S_out, bool x_t_ready,
                    cudaStream_t st) {
  gbk_status s;
  if ((s = forward(net, x, B, net->raw, true, st))) return s;
  if ((s = launch_pdl("mdn loss", k_mdn_loss, dim3((B + kLossRows - 1) / kLossRows), dim3(kLossRows * 32), 0, st,
                       (const float*)net->raw, u, B, 1.0f / (float)B, net->g4, net->g4T, net->ldt, net->nll)))
    return s;
  if (loss && (s = launch_pdl("mdn loss mean", k_mean, dim3(1), dim3(256), 0, st, (const float*)net->nll, B, loss)))
    return s;
  if (!x_t_ready && (s = launch_pdl("mdn input transpose", k_transpose, dim3(kIn / 32, (B + 31) / 32), dim3(32, 8), 0,
                                    st, x, B, kIn, net->xT, net->ldt)))
    return s;
  int kps;
  const int S = splits_for(2 * B, &kps);   // the weight-gradient contraction runs over [hi | lo]: 2 B
  *S_out = S;
  const int64_t offw[4] = {kOffW1, kOffW2, kOffW3, kOffW4}, offb[4] = {kOffB1, kOffB2, kOffB3, kOffB4};
  const int64_t offt[4] = {0, kOffT2, kOffT3, kOffT4};
  const int nout[4] = {kHid, kHid, kHid, kOut}, nin[4] = {kIn, kHid, kHid, kHid};
  const bf16* gcur = net->g4;
  const bf16* gcurT = net->g4T;
  for (int l = 3; l >= 0; --l) {
    const bf16* hinT = l == 0 ? net->xT : net->hT[l - 1];
    // dW_l[o][i] = sum_m g[m][o] hin[m][i] = (g^T) . (hin^T)^T over the batch, split over it
    umma::Args gw = margs(net, net->part + offw[l], nin[l]);
    gw.kps = kps;
    gw.split_stride = kNParams;
    if ((s = mm<umma::EPI_PART_F32>(net, gcurT, net->ldt, hinT, net->ldt, nout[l], nin[l], 2 * B, gw, S, st)))
      return s;
    if ((s = launch_pdl("mdn bias gradient", k_bias_grad, dim3((nout[l] + 7) / 8), dim3(256), 0, st, gcurT, net->ldt,
                        2 * B, nout[l], net->part, S, kNParams, offb[l])))
      return s;
    if (l == 0) break;
    // g_prev[m][i] = sum_o g[m][o] W[o][i] = [hi | lo] . [W^T | W^T]^T (contraction over 2 nout),
    // kept where the forward activation was positive and stored again as a hi / lo pair
    bf16* gn = net->g[l & 1];
    bf16* gnT = net->gT[l & 1];
    umma::Args gx = margs(net, gn, 2 * nin[l]);
    gx.mask = net->h[l - 1];
    gx.ldm = kHid;
    gx.CT = gnT;
    gx.ldct = net->ldt;
    if ((s = mm<umma::EPI_MASK_SPLIT>(net, gcur, 2 * nout[l], net->pbT + offt[l], 2 * nout[l], B, nin[l],
                                       2 * nout[l], gx, 1, st)))
      return s;
    gcur = gn;
    gcurT = gnT;
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
  n->ldt = 2 * ((max_batch + 7) / 8 * 8);   // transposed [hi | lo] / doubled copies: rows 16-byte aligned
  const size_t B = (size_t)max_batch, T = (size_t)n->ldt;
  bool ok = cudaMalloc(&n->pf, kNParams * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->pb, kNParams * sizeof(bf16)) == cudaSuccess &&
            cudaMalloc(&n->pbT, kNT * sizeof(bf16)) == cudaSuccess &&
            cudaMalloc(&n->raw, B * kOut * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->g4, B * 2 * kOut * sizeof(bf16)) == cudaSuccess &&
            cudaMalloc(&n->g4T, T * kOut * sizeof(bf16)) == cudaSuccess &&
            cudaMalloc(&n->xT, T * kIn * sizeof(bf16)) == cudaSuccess &&
            cudaMalloc(&n->nll, B * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->err, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&n->xb, B * kIn * sizeof(bf16)) == cudaSuccess &&
            cudaMalloc(&n->ub, B * kMixDim * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->part, (size_t)kMaxSplit * kNParams * sizeof(float)) == cudaSuccess;
  for (int i = 0; i < 3 && ok; ++i)
    ok = cudaMalloc(&n->h[i], B * kHid * sizeof(bf16)) == cudaSuccess &&
         cudaMalloc(&n->hT[i], T * kHid * sizeof(bf16)) == cudaSuccess;
  for (int i = 0; i < 2 && ok; ++i)
    ok = cudaMalloc(&n->g[i], B * 2 * kHid * sizeof(bf16)) == cudaSuccess &&
         cudaMalloc(&n->gT[i], T * kHid * sizeof(bf16)) == cudaSuccess;
  if (ok) ok = cudaMemset(n->err, 0, sizeof(int)) == cudaSuccess;
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
  cudaFree(n->pf); cudaFree(n->pb); cudaFree(n->pbT); cudaFree(n->raw); cudaFree(n->g4); cudaFree(n->g4T);
  cudaFree(n->xT); cudaFree(n->nll); cudaFree(n->err); cudaFree(n->part); cudaFree(n->xb); cudaFree(n->ub);
  for (int i = 0; i < 3; ++i) { cudaFree(n->h[i]); cudaFree(n->hT[i]); }
  for (int i = 0; i < 2; ++i) { cudaFree(n->g[i]); cudaFree(n->gT[i]); }
  delete n;
  return GBK_OK;
}

extern "C" gbk_status mdn_status(gbk_mdn* net, void* stream) {
  if (!net) return set_error(GBK_EINVAL, "mdn_status: null network");
  int h = 0;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
      cudaMemcpy(&h, net->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(net->err, 0, sizeof(int)) != cudaSuccess) {
    const cudaError_t e = cudaGetLastError();
    return set_error(GBK_ECUDA, "mdn_status: %s", cudaGetErrorString(e));
  }
  if (h & kErrTimeout) return set_error(GBK_ETIMEOUT, "mdn: a tensor-core product gave up waiting (bounded wait)");
  if (h & kErrWalker) return set_error(GBK_ERANGE, "mdn: a training-row index was out of range");
  return GBK_OK;
}

extern "C" gbk_status mdn_set_params(gbk_mdn* net, const float* params, void* stream) {
  if (!net || !params) return set_error(GBK_EINVAL, "mdn_set_params: null argument");
  k_copy_params<<<blocks_for(kNParams), 256, 0, (cudaStream_t)stream>>>(params, kNParams, net->pf, net->pb, net->pbT);
  net->have_params = true;
  return check_launch("mdn_set_params");
}

extern "C" gbk_status mdn_forward(gbk_mdn* net, const uint16_t* x, int32_t batch, float* raw, void* stream) {
  gbk_status s = check_batch(net, batch, "mdn_forward");
  if (s) return s;
  if (!x || !raw) return set_error(GBK_EINVAL, "mdn_forward: null device pointer");
  if (((uintptr_t)x & 15) || ((uintptr_t)raw & 15)) return set_error(GBK_EINVAL, "mdn_forward: misaligned buffer");
  return forward(net, reinterpret_cast<const bf16*>(x), batch, raw, false, (cudaStream_t)stream);
}

extern "C" gbk_status mdn_backward(gbk_mdn* net, const uint16_t* x, const float* u, int32_t batch, float* grad,
                                   double* loss, void* stream) {
  gbk_status s = check_batch(net, batch, "mdn_backward");
  if (s) return s;
  if (!x || !u || !grad) return set_error(GBK_EINVAL, "mdn_backward: null device pointer");
  if ((uintptr_t)x & 15) return set_error(GBK_EINVAL, "mdn_backward: x must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  int S = 0;
  if ((s = backward(net, reinterpret_cast<const bf16*>(x), u, batch, loss, &S, false, st))) return s;
  return launch_pdl("mdn_backward", k_reduce, dim3(blocks_for(kNParams)), dim3(256), 0, st, (const float*)net->part, S,
                    kNParams, grad);
}

extern "C" gbk_status mdn_adam(gbk_mdn* net, float* params, float* m, float* v, const float* grad, int32_t step,
                               float lr, float beta1, float beta2, float eps, void* stream) {
  if (!net || !params || !m || !v || !grad) return set_error(GBK_EINVAL, "mdn_adam: null argument");
  if (step < 1) return set_error(GBK_EINVAL, "mdn_adam: step counts from 1");
  const float c1 = (float)(1.0 / (1.0 - pow((double)beta1, step)));
  const float c2 = (float)(1.0 / (1.0 - pow((double)beta2, step)));
  const gbk_status s = launch_pdl("mdn_adam", k_adam, dim3(kAdamBlocks), dim3(256), 0, (cudaStream_t)stream,
                                  adam_args(net, nullptr, 0, grad, params, m, v, lr, beta1, beta2, eps, c1, c2));
  if (!s) net->have_params = true;
  return s;
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
  if ((s = backward(net, reinterpret_cast<const bf16*>(x), u, batch, loss, &S, false, st))) return s;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 / (1.0 - pow(b1, step))), c2 = (float)(1.0 / (1.0 - pow(b2, step)));
  return launch_pdl("mdn_train_step", k_adam, dim3(kAdamBlocks), dim3(256), 0, st,
                    adam_args(net, net->part, S, nullptr, params, m, v, lr, (float)b1, (float)b2, 1e-8f, c1, c2));
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

extern "C" gbk_status mdn_train_epoch(gbk_mdn* net, float* params, float* m, float* v, const uint16_t* x,
                                      const float* u, int64_t n_rows, const int32_t* order, int32_t batch,
                                      int32_t n_steps, int32_t step0, float lr, double* loss, void* stream) {
  gbk_status s = check_batch(net, batch, "mdn_train_epoch");
  if (s) return s;
  if (!params || !m || !v || !x || !u || !order) return set_error(GBK_EINVAL, "mdn_train_epoch: null device pointer");
  if ((uintptr_t)x & 15) return set_error(GBK_EINVAL, "mdn_train_epoch: x must be 16-byte aligned");
  if (n_steps < 0 || step0 < 0 || n_rows < 1) return set_error(GBK_EINVAL, "mdn_train_epoch: bad counts");
  cudaStream_t st = (cudaStream_t)stream;
  const double b1 = 0.9, b2 = 0.999;
  for (int32_t k = 0; k < n_steps; ++k) {
    if ((s = launch_pdl("mdn_train_epoch(gather)", k_gather_t, dim3(kIn / 64, (batch + 63) / 64), dim3(256), 0, st,
                        reinterpret_cast<const bf16*>(x), u, order + (int64_t)k * batch, batch, n_rows, net->xb, net->ub,
                        net->xT, net->ldt, net->err)))
      return s;
    int S = 0;
    if ((s = backward(net, net->xb, net->ub, batch, k == n_steps - 1 ? loss : nullptr, &S, true, st))) return s;
    const int step = step0 + k + 1;
    const float c1 = (float)(1.0 / (1.0 - pow(b1, step))), c2 = (float)(1.0 / (1.0 - pow(b2, step)));
    if ((s = launch_pdl("mdn_train_epoch(adam)", k_adam, dim3(kAdamBlocks), dim3(256), 0, st,
                        adam_args(net, net->part, S, nullptr, params, m, v, lr, (float)b1, (float)b2, 1e-8f, c1, c2))))
      return s;
  }
  return GBK_OK;
}
