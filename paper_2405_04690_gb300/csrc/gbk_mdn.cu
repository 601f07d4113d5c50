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
  umma::k_umma<kBN, EPI><<<grid, umma::kThreads, SM::bytes, st>>>(ma, mb, g);
  return check_launch("mdn tensor-core product");
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

// Transposes through 32 x 32 shared-memory tiles. split = 0: x [B][cols] -> xt[c][r] and the
// copy xt[c][B + r]; split = 1: x [B][2 cols] = [hi | lo] -> xt[c][r] = hi, xt[c][B + r] = lo.
__global__ void k_transpose(const bf16* __restrict__ x, int B, int cols, int split, bf16* __restrict__ xt,
                            int64_t ldt) {
  __shared__ bf16 t[2][32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int64_t ldx = split ? 2 * (int64_t)cols : cols;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < B && c < cols) {
      t[0][i][threadIdx.x] = x[(int64_t)r * ldx + c];
      t[1][i][threadIdx.x] = split ? x[(int64_t)r * ldx + cols + c] : t[0][i][threadIdx.x];
    }
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < B && c < cols) {
      xt[(int64_t)c * ldt + r] = t[0][threadIdx.x][i];
      xt[(int64_t)c * ldt + B + r] = t[1][threadIdx.x][i];
    }
  }
}

// Training rows of one minibatch: x[order[i]] -> xb[i] (16-byte chunks), u[order[i]] -> ub[i].
__global__ void k_gather(const bf16* __restrict__ x, const float* __restrict__ u, const int32_t* __restrict__ order,
                         int B, int64_t n_rows, bf16* __restrict__ xb, float* __restrict__ ub, int* err) {
  const int64_t total = (int64_t)B * (kIn / 8);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / (kIn / 8)), c = (int)(i % (kIn / 8));
    const int32_t src = order[r];
    if (src < 0 || src >= n_rows) {   // bad index: zero row, error bit, nothing read
      if (c == 0) atomicOr(err, 4);
      reinterpret_cast<uint4*>(xb + (int64_t)r * kIn)[c] = make_uint4(0, 0, 0, 0);
      if (c < kMixDim) ub[(int64_t)r * kMixDim + c] = 0.5f;
      continue;
    }
    reinterpret_cast<uint4*>(xb + (int64_t)r * kIn)[c] = reinterpret_cast<const uint4*>(x + (int64_t)src * kIn)[c];
    if (c < kMixDim) ub[(int64_t)r * kMixDim + c] = u[(int64_t)src * kMixDim + c];
  }
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
  bf16* gr = graw + (int64_t)m * 2 * kOut + k * 17;   // [hi | lo] pairs, row of 2 x 272
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

// Bias gradients: column sums of g = hi + lo ([B][2N]: [hi | lo]) over split z's rows, into
// part + z stride + off.
// Block (32 columns) x (8 row phases); the 8 phase sums are added in a fixed order.
__global__ void k_colsum(const bf16* __restrict__ g, int B, int N, int kps, float* __restrict__ part,
                         int64_t stride, int64_t off) {
  __shared__ float red[8][33];
  const int n = blockIdx.x * 32 + threadIdx.x;
  const int z = blockIdx.y;
  const int r1 = min(B, (z + 1) * kps);
  float s = 0.f;
  if (n < N)
    for (int r = z * kps + threadIdx.y; r < r1; r += 8)
      s += __bfloat162float(g[(int64_t)r * 2 * N + n]) + __bfloat162float(g[(int64_t)r * 2 * N + N + n]);
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && n < N) {
    float t = 0.f;
    for (int i = 0; i < 8; ++i) t += red[i][threadIdx.x];
    part[(int64_t)z * stride + off + n] = t;
  }
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

__global__ void k_adam(const float* __restrict__ part, int S, const float* __restrict__ grad, int64_t n,
                       float* __restrict__ p, float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                       float b2, float eps, float c1, float c2, float* __restrict__ pf, bf16* __restrict__ pb,
                       bf16* __restrict__ pbt) {
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
    store_param(i, pi, pf, pb, pbt);
  }
}

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
gbk_status backward(gbk_mdn* net, const bf16* x, const float* u, int B, double* loss, int* S_out, cudaStream_t st) {
  gbk_status s;
  if ((s = forward(net, x, B, net->raw, true, st))) return s;
  k_mdn_loss<<<(B + 7) / 8, 256, 0, st>>>(net->raw, u, B, 1.0f / (float)B, net->g4, net->nll);
  if ((s = check_launch("mdn loss"))) return s;
  k_transpose<<<dim3((kOut + 31) / 32, (B + 31) / 32), dim3(32, 8), 0, st>>>(net->g4, B, kOut, 1, net->g4T, net->ldt);
  if (loss) {
    k_mean<<<1, 256, 0, st>>>(net->nll, B, loss);
    if ((s = check_launch("mdn loss mean"))) return s;
  }
  k_transpose<<<dim3(kIn / 32, (B + 31) / 32), dim3(32, 8), 0, st>>>(x, B, kIn, 0, net->xT, net->ldt);
  if ((s = check_launch("mdn input transpose"))) return s;
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
    k_colsum<<<dim3((nout[l] + 31) / 32, S), dim3(32, 8), 0, st>>>(gcur, B, nout[l], kps, net->part, kNParams,
                                                                    offb[l]);
    if ((s = check_launch("mdn bias gradient"))) return s;
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
                                                                  beta2, eps, c1, c2, net->pf, net->pb, net->pbT);
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
                                              1e-8f, c1, c2, net->pf, net->pb, net->pbT);
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
  const int gblocks = blocks_for((int64_t)batch * (kIn / 8));
  for (int32_t k = 0; k < n_steps; ++k) {
    k_gather<<<gblocks, 256, 0, st>>>(reinterpret_cast<const bf16*>(x), u, order + (int64_t)k * batch, batch, n_rows,
                                      net->xb, net->ub, net->err);
    if ((s = check_launch("mdn_train_epoch(gather)"))) return s;
    int S = 0;
    if ((s = backward(net, net->xb, net->ub, batch, k == n_steps - 1 ? loss : nullptr, &S, st))) return s;
    const int step = step0 + k + 1;
    const float c1 = (float)(1.0 / (1.0 - pow(b1, step))), c2 = (float)(1.0 / (1.0 - pow(b2, step)));
    k_adam<<<blocks_for(kNParams), 256, 0, st>>>(net->part, S, nullptr, kNParams, params, m, v, lr, (float)b1,
                                                (float)b2, 1e-8f, c1, c2, net->pf, net->pb, net->pbT);
    if ((s = check_launch("mdn_train_epoch(adam)"))) return s;
  }
  return GBK_OK;
}
