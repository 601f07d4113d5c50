// BF16 matrix product on the 5th-generation tensor cores: C[M][N] = sum_k A[m][k] B[n][k]
// (both operands K-contiguous), float32 accumulation in tensor memory.
//
// One CTA of 4 warps per 128 x BN tile of C:
//   warp 0, one lane   TMA producer: 128 x 64 tiles of A and BN x 64 tiles of B, 128-byte
//                      swizzle, into a 4-stage shared-memory ring (mbarrier per stage);
//   warp 1, one lane   MMA issuer: tcgen05.mma kind::f16 (M = 128, N = BN, K = 16) x 4 per
//                      stage, accumulator in TMEM; tcgen05.commit frees each stage;
//   all 4 warps        epilogue: tcgen05.ld of their 32 TMEM lanes (= rows), fused bias /
//                      ReLU / mask, stores (optionally also the transposed BF16 copy the
//                      backward products read as a K-contiguous operand).
// Out-of-range rows and k are zero-filled by TMA. Split-K: blockIdx.z takes the k range
// [z kps, (z + 1) kps), kps a multiple of 64, and writes its own partial slot.
// Every wait is bounded (2 s by %globaltimer); a wait that gives up sets the abort flag,
// the kernel drains what it issued (bounded), frees its TMEM and records kErrTimeout.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace gbk {
namespace umma {

constexpr int kBM = 128, kBK = 64, kStages = 4, kThreads = 128;
constexpr uint64_t kWaitNs = 2000000000ull;

// EPI_BIAS_RELU_BF16: relu(acc + bias) -> BF16 C (and CT; with ct_dup also CT[n ldct + M + m]);
// EPI_BIAS_F32: acc + bias -> float32 C; EPI_PART_F32: acc -> float32 partial slot z;
// EPI_MASK_SPLIT: v = acc where mask > 0, else 0, stored as the BF16 pair hi = bf16(v),
// lo = bf16(v - hi): C[m ldc + n] = hi, C[m ldc + N + n] = lo, CT[n ldct + m] = hi,
// CT[n ldct + M + m] = lo (about 16 significant bits for the back-propagated signal).
enum { EPI_BIAS_RELU_BF16 = 0, EPI_BIAS_F32 = 1, EPI_MASK_SPLIT = 2, EPI_PART_F32 = 3 };

struct Args {
  int M, N, K, kps;                    // kps: k range per split (multiple of 64)
  const float* bias;                   // [N]
  const __nv_bfloat16* mask;           // EPI_MASK: keep (m, n) where mask[m ldm + n] > 0
  int64_t ldm;
  void* C;                             // C(m, n) = C[m ldc + n] (+ z split_stride for EPI_PART)
  int64_t ldc, split_stride;
  __nv_bfloat16* CT;                   // optional transposed BF16 copy: CT[n ldct + m]
  int64_t ldct;
  int ct_dup;                          // EPI_BIAS_RELU_BF16: also CT[n ldct + M + m] (a second copy)
  int* err;                            // device error word
};

template <int BN>
struct Smem {
  static constexpr int a_bytes = kBM * kBK * 2;
  static constexpr int b_bytes = BN * kBK * 2;
  static constexpr int stage_bytes = a_bytes + b_bytes;
  static constexpr size_t bytes = (size_t)kStages * stage_bytes + 1024 /* alignment */ + 256 /* barriers */;
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of the given parity to complete; false on abort or after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (gtimer() - t0 > kWaitNs) {
      *abort_flag = 1;
      return false;
    }
  }
}
// Drain wait (failure path): ignores the abort flag, still bounded.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = gtimer();
  while (!mbar_try(bar, parity) && gtimer() - t0 < kWaitNs) {
  }
}
__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(saddr(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(const void* p) {
  return (uint64_t)((saddr(p) & 0x3FFFF) >> 4) | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}
// Instruction descriptor of kind::f16: BF16 A and B, float32 D, both K-major, M = 128.
template <int BN>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive float32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BN, int EPI>
__global__ void __launch_bounds__(kThreads, 1)
k_umma(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, const Args g) {
  static_assert(BN == 64 || BN == 128 || BN == 256, "tile width");
  typedef Smem<BN> SM;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t base = saddr(smem_raw);
  unsigned char* tiles = smem_raw + (((base + 1023u) & ~1023u) - base);   // 1024-byte aligned (swizzle atom)
  uint64_t* full = reinterpret_cast<uint64_t*>(tiles + kStages * SM::stage_bytes);
  uint64_t* empty = full + kStages;
  uint64_t* accum = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * g.kps;
  const int kend = min(g.K, kbeg + g.kps);
  const int nk = kend > kbeg ? (kend - kbeg + kBK - 1) / kBK : 0;

  if (nk == 0) {   // an empty split writes zeros to its partial slot
    if (EPI == EPI_PART_F32) {
      float* C = reinterpret_cast<float*>(g.C) + (int64_t)blockIdx.z * g.split_stride;
      for (int i = threadIdx.x; i < kBM * BN; i += kThreads) {
        const int m = m0 + i / BN, n = n0 + i % BN;
        if (m < g.M && n < g.N) C[(int64_t)m * g.ldc + n] = 0.f;
      }
    }
    return;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {   // TMEM: BN float32 columns x 128 lanes
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    int loads = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages, n = kb / kStages;
      if (!mbar_wait(&empty[s], (uint32_t)((n & 1) ^ 1), abort_flag)) break;
      unsigned char* sa = tiles + s * SM::stage_bytes;
      mbar_expect_tx(&full[s], (uint32_t)SM::stage_bytes);
      tma_load(sa, &mapA, kbeg + kb * kBK, m0, &full[s]);
      tma_load(sa + SM::a_bytes, &mapB, kbeg + kb * kBK, n0, &full[s]);
      ++loads;
    }
    // the last stages' copies must have landed before the CTA can leave (immediate unless aborted)
    for (int kb = loads > kStages ? loads - kStages : 0; kb < loads; ++kb)
      mbar_drain(&full[kb % kStages], (uint32_t)((kb / kStages) & 1));
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t id = idesc<BN>();
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages, n = kb / kStages;
      if (!mbar_wait(&full[s], (uint32_t)(n & 1), abort_flag)) break;
      fence_after();
      const unsigned char* sa = tiles + s * SM::stage_bytes;
      const uint64_t da = sdesc(sa), db = sdesc(sa + SM::a_bytes);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk)   // K = 16 per MMA: advance 32 bytes inside the swizzled row
        mma(tmem, da + 2 * kk, db + 2 * kk, id, (kb | kk) != 0 ? 1u : 0u);
      commit(&empty[s]);
    }
    commit(accum);   // arrives when every MMA issued above has completed
  }
  __syncwarp();
  bool ok = mbar_wait(accum, 0, abort_flag);
  if (!ok) mbar_drain(accum, 0);   // MMAs already issued finish before TMEM is freed
  fence_after();
  if (ok && !*abort_flag) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float v[32];
      tmem_ld32(trow + (uint32_t)c0, v);
      if (row >= g.M || n0 + c0 >= g.N) continue;
      const int nv = min(32, g.N - (n0 + c0));   // N is a multiple of 8
      const int nb = n0 + c0;
      if (EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_MASK_SPLIT) {
        __nv_bfloat16* C = reinterpret_cast<__nv_bfloat16*>(g.C) + (int64_t)row * g.ldc + nb;
        const __nv_bfloat16* mk = EPI == EPI_MASK_SPLIT ? g.mask + (int64_t)row * g.ldm + nb : nullptr;
#pragma unroll
        for (int q = 0; q < 32; q += 8) {
          if (q >= nv) break;
          __align__(16) __nv_bfloat16 o[8];
          __align__(16) __nv_bfloat16 lo[8];
          uint4 mv;
          if (EPI == EPI_MASK_SPLIT) mv = *reinterpret_cast<const uint4*>(mk + q);
          const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&mv);
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            float x = v[q + e];
            if (EPI == EPI_BIAS_RELU_BF16) x = fmaxf(x + g.bias[nb + q + e], 0.f);
            else if (!(__bfloat162float(mb[e]) > 0.f)) x = 0.f;
            o[e] = __float2bfloat16_rn(x);
            if (EPI == EPI_MASK_SPLIT) lo[e] = __float2bfloat16_rn(x - __bfloat162float(o[e]));
          }
          *reinterpret_cast<uint4*>(C + q) = *reinterpret_cast<const uint4*>(o);
          if (EPI == EPI_MASK_SPLIT) *reinterpret_cast<uint4*>(C + g.N + q) = *reinterpret_cast<const uint4*>(lo);
          if (g.CT) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              __nv_bfloat16* ct = g.CT + (int64_t)(nb + q + e) * g.ldct + row;
              ct[0] = o[e];
              if (EPI == EPI_MASK_SPLIT) ct[g.M] = lo[e];
              else if (g.ct_dup) ct[g.M] = o[e];
            }
          }
        }
      } else {
        float* C = reinterpret_cast<float*>(g.C) + (EPI == EPI_PART_F32 ? (int64_t)blockIdx.z * g.split_stride : 0) +
                   (int64_t)row * g.ldc + nb;
#pragma unroll
        for (int q = 0; q < 32; q += 4) {
          if (q >= nv) break;
          float4 o;
          o.x = v[q]; o.y = v[q + 1]; o.z = v[q + 2]; o.w = v[q + 3];
          if (EPI == EPI_BIAS_F32) {
            o.x += g.bias[nb + q]; o.y += g.bias[nb + q + 1]; o.z += g.bias[nb + q + 2]; o.w += g.bias[nb + q + 3];
          }
          *reinterpret_cast<float4*>(C + q) = o;
        }
      }
    }
  } else if (threadIdx.x == 0 && g.err) {
    atomicOr(g.err, 8);   // kErrTimeout
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
  }
}

}  // namespace umma
}  // namespace gbk
