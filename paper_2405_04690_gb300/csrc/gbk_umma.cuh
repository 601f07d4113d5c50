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
// Launched as a programmatic dependent launch: barrier set-up and the TMEM allocation overlap the
// previous kernel, the operands are read only after griddep_wait().
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
  // tiles, barriers (256 bytes), the tile's bias values (BN floats)
  static constexpr size_t bytes = (size_t)kStages * stage_bytes + 1024 /* alignment */ + 256 + BN * 4;
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// Programmatic dependent launch: a kernel launched with programmatic stream serialization may
// start while the previous kernel of the stream still runs; griddep_wait() returns once that
// kernel has completed and its writes are visible, and no global memory is touched before it.
// griddep_launch() lets the next such kernel start (once every CTA of this grid has called it
// or exited).
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
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
  volatile int* first_issued = reinterpret_cast<volatile int*>(tmem_slot + 2);
  float* sbias = reinterpret_cast<float*>(tiles + kStages * SM::stage_bytes + 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * g.kps;
  const int kend = min(g.K, kbeg + g.kps);
  const int nk = kend > kbeg ? (kend - kbeg + kBK - 1) / kBK : 0;

  if (nk == 0) {   // an empty split writes zeros to its partial slot
    griddep_wait();
    griddep_launch();
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
    *first_issued = 0;
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
  griddep_wait();   // set-up above overlaps the previous kernel; operands are read below
  // Operands of the epilogue, fetched while the products run (global loads placed among the
  // epilogue's stores would wait one after another): the tile's bias values into shared memory
  // by warps 2-3, this thread's row of the mask into registers.
  if ((EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_BIAS_F32) && warp >= 2)
    for (int i = threadIdx.x - 64; i < BN; i += kThreads - 64) sbias[i] = n0 + i < g.N ? g.bias[n0 + i] : 0.f;
  uint4 mrow[EPI == EPI_MASK_SPLIT ? BN / 8 : 1];
  auto load_mask = [&]() {
    if (EPI == EPI_MASK_SPLIT) {
      const int row = m0 + threadIdx.x;
#pragma unroll
      for (int j = 0; j < BN / 8; ++j)
        mrow[j] = row < g.M && n0 + 8 * j < g.N
                      ? *reinterpret_cast<const uint4*>(g.mask + (int64_t)row * g.ldm + n0 + 8 * j)
                      : make_uint4(0, 0, 0, 0);
    }
  };

  if (warp == 0 && lane == 0) {
    int loads = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages, n = kb / kStages;
      if (!mbar_wait(&empty[s], (uint32_t)((n & 1) ^ 1), abort_flag)) break;
      unsigned char* sa = tiles + s * SM::stage_bytes;
      mbar_expect_tx(&full[s], (uint32_t)SM::stage_bytes);
      tma_load(sa, &mapA, kbeg + kb * kBK, m0, &full[s]);
      tma_load(sa + SM::a_bytes, &mapB, kbeg + kb * kBK, n0, &full[s]);
      if (kb == 0) *first_issued = 1;
      ++loads;
    }
    // the last stages' copies must have landed before the CTA can leave (immediate unless aborted)
    for (int kb = loads > kStages ? loads - kStages : 0; kb < loads; ++kb)
      mbar_drain(&full[kb % kStages], (uint32_t)((kb / kStages) & 1));
    load_mask();
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
    load_mask();
  } else if (EPI == EPI_MASK_SPLIT) {
    // the row's mask is read once the first operand tiles are requested (issued earlier, its
    // loads would queue ahead of them); the wait is a hint, bounded at 100 us
    const uint64_t t0 = gtimer();
    while (!*first_issued && !*abort_flag && gtimer() - t0 < 100000ull) {
    }
    load_mask();
  }
  __syncwarp();
  const bool ok = mbar_wait(accum, 0, abort_flag);
  if (!ok) mbar_drain(accum, 0);   // MMAs already issued finish before TMEM is freed
  griddep_launch();                // the next kernel's set-up may overlap this epilogue
  __syncthreads();                 // bias values in shared memory; the abort flag is final
  fence_after();
  if (!*abort_flag) {              // the same for every thread of the CTA
    const int lr = warp * 32 + lane;   // this thread's TMEM lane = row of the tile
    const int row = m0 + lr;
    const int mrows = min(kBM, g.M - m0), ncols = min(BN, g.N - n0);
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    // Staging in the operand ring (free once every product has completed), so that the
    // transposed BF16 copy and the float32 results leave as whole rows of 16-byte stores:
    // sT [2][BN][kTP] BF16 (column n of the tile as a row of kBM values), sF [kBM][kFP] float32.
    constexpr int kTP = kBM + 8, kFP = BN + 4;
    static_assert(2 * BN * kTP * 2 <= kStages * SM::stage_bytes && kBM * kFP * 4 <= kStages * SM::stage_bytes,
                  "staging area");
    __nv_bfloat16* sT = reinterpret_cast<__nv_bfloat16*>(tiles);
    float* sF = reinterpret_cast<float*>(tiles);
    const bool stage_t = (EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_MASK_SPLIT) && g.CT != nullptr;
#pragma unroll
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float v[32];
      tmem_ld32(trow + (uint32_t)c0, v);
      if (row >= g.M || c0 >= ncols) continue;
      const int nv = min(32, ncols - c0);   // N is a multiple of 8
      if (EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_MASK_SPLIT) {
        __nv_bfloat16* C = reinterpret_cast<__nv_bfloat16*>(g.C) + (int64_t)row * g.ldc + n0 + c0;
#pragma unroll
        for (int q = 0; q < 32; q += 8) {
          if (q >= nv) break;
          __align__(16) __nv_bfloat16 o[8];
          __align__(16) __nv_bfloat16 lo[8];
          const uint4 mv = mrow[EPI == EPI_MASK_SPLIT ? (c0 + q) / 8 : 0];
          const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&mv);
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            float x = v[q + e];
            if (EPI == EPI_BIAS_RELU_BF16) x = fmaxf(x + sbias[c0 + q + e], 0.f);
            else if (!(__bfloat162float(mb[e]) > 0.f)) x = 0.f;
            o[e] = __float2bfloat16_rn(x);
            if (EPI == EPI_MASK_SPLIT) lo[e] = __float2bfloat16_rn(x - __bfloat162float(o[e]));
          }
          *reinterpret_cast<uint4*>(C + q) = *reinterpret_cast<const uint4*>(o);
          if (EPI == EPI_MASK_SPLIT) *reinterpret_cast<uint4*>(C + g.N + q) = *reinterpret_cast<const uint4*>(lo);
          if (stage_t) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              sT[(c0 + q + e) * kTP + lr] = o[e];
              if (EPI == EPI_MASK_SPLIT) sT[(BN + c0 + q + e) * kTP + lr] = lo[e];
            }
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < 32; q += 4) {
          if (q >= nv) break;
          float4 o;
          o.x = v[q]; o.y = v[q + 1]; o.z = v[q + 2]; o.w = v[q + 3];
          if (EPI == EPI_BIAS_F32) {
            o.x += sbias[c0 + q]; o.y += sbias[c0 + q + 1]; o.z += sbias[c0 + q + 2]; o.w += sbias[c0 + q + 3];
          }
          *reinterpret_cast<float4*>(sF + lr * kFP + c0 + q) = o;
        }
      }
    }
    __syncthreads();
    if (stage_t) {
      // plane p of CT (columns p M ..): EPI_MASK_SPLIT hi, lo; EPI_BIAS_RELU_BF16 the values, twice with ct_dup
      const int planes = (EPI == EPI_MASK_SPLIT || g.ct_dup) ? 2 : 1;
      const bool vec = mrows == kBM && (g.ldct & 7) == 0 && (g.M & 7) == 0 && ((uintptr_t)g.CT & 15) == 0;
      if (vec) {
        for (int i = threadIdx.x; i < planes * ncols * (kBM / 8); i += kThreads) {
          const int p = i / (ncols * (kBM / 8)), rem = i % (ncols * (kBM / 8));
          const int c = rem / (kBM / 8), j = rem % (kBM / 8);
          const int sp = EPI == EPI_MASK_SPLIT ? p : 0;
          *reinterpret_cast<uint4*>(g.CT + (int64_t)(n0 + c) * g.ldct + (int64_t)p * g.M + m0 + 8 * j) =
              *reinterpret_cast<const uint4*>(sT + (sp * BN + c) * kTP + 8 * j);
        }
      } else {
        for (int i = threadIdx.x; i < planes * ncols * mrows; i += kThreads) {
          const int p = i / (ncols * mrows), rem = i % (ncols * mrows);
          const int c = rem / mrows, r = rem % mrows;
          const int sp = EPI == EPI_MASK_SPLIT ? p : 0;
          g.CT[(int64_t)(n0 + c) * g.ldct + (int64_t)p * g.M + m0 + r] = sT[(sp * BN + c) * kTP + r];
        }
      }
    }
    if (EPI == EPI_BIAS_F32 || EPI == EPI_PART_F32) {   // one warp per row
      float* C = reinterpret_cast<float*>(g.C) + (EPI == EPI_PART_F32 ? (int64_t)blockIdx.z * g.split_stride : 0) +
                 (int64_t)m0 * g.ldc + n0;
      const bool vec = (g.ldc & 3) == 0 && ((uintptr_t)C & 15) == 0 && (ncols & 3) == 0;
      for (int r = warp; r < mrows; r += kThreads / 32) {
        if (vec)
          for (int c = 4 * lane; c < ncols; c += 128)
            *reinterpret_cast<float4*>(C + (int64_t)r * g.ldc + c) = *reinterpret_cast<const float4*>(sF + r * kFP + c);
        else
          for (int c = lane; c < ncols; c += 32) C[(int64_t)r * g.ldc + c] = sF[r * kFP + c];
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
