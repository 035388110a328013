// packgemm.cu -- a GEMM that consumes the packing routine directly (the
// level-3 BLAS use of TTC's sub-tensor transpositions, section 2.1, Figs.
// 2-3): C = alpha * P * Bm, where P is the BF16 panel that the permute plan
// (perm, sizes, outer sizes of A; FP32 -> BF16, round to nearest even) would
// write, viewed as an M x K column-major matrix, and Bm is a BF16 K x N
// column-major matrix.  Instead of writing P to memory and reading it back
// into a GEMM, every CTA gathers its 128 x 64 slices of P straight from A
// (per-row and per-column offset tables: the permutation splits into an
// M part and a K part), rounds it to BF16 into shared memory in the tensor
// cores' K-major layout, and issues tcgen05.mma (M 128, N 256, K 16) into a
// TMEM accumulator; the epilogue reads TMEM with tcgen05.ld and writes C.
//
// Every wait is bounded: a wait that gives up sets the plan's error word,
// which ttc_packed_gemm_check reports, and the CTA still frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ttc.h"
#include "../../include/ttc_debug.h"
#include "kernels.cuh"
#include "plan_impl.h"

using namespace ttc;

namespace ttc {
extern std::atomic<int64_t> g_launches;
}

namespace {

constexpr int kBM = 128, kBN = 256, kBK = 64;     // CTA tile; one MMA is 128 x 256 x 16
constexpr int kPgThreads = 256;
constexpr uint32_t kTmemCols = 256;               // FP32 accumulator: 128 lanes x 256 columns
// shared-memory operand layout: K-major with the 128-byte swizzle.  A row of
// a tile is its kBK = 64 BF16 (128 bytes) along K; 8 rows form a 1024-byte
// atom (the stride byte offset between 8-row groups), and inside an atom the
// 16-byte chunk c of row r sits at chunk c ^ r, so that 8 lanes storing
// either 8 chunks of one row or one chunk of 8 rows hit 32 distinct banks.
// One MMA (K = 16) reads 32 bytes of every row: its descriptor starts 32
// bytes further per K step, and the hardware applies the same XOR.
constexpr int kSBO = 8 * kBK * 2;
constexpr uint64_t kSwizzle128B = 2;               // descriptor layout type
constexpr int kTileA = kBM * kBK * 2;              // 16 KiB: the slice of P
constexpr int kTileB = kBN * kBK * 2;              // 32 KiB: the slice of Bm
constexpr int kStage = kTileA + kTileB;
// dynamic shared memory per CTA: two buffers of two tiles, two barriers and
// the TMEM address, padded so that at most two CTAs are resident on an SM
// (two 256-column accumulators fill the SM's 512 TMEM columns: no
// allocation waits)
constexpr int kPgSmem = 100 * 1024;
constexpr uint32_t kWaitLimit = 1u << 22;          // polls of one barrier phase before giving up
constexpr uint32_t kTestWaitLimit = 1u << 12;      // the same under the testing hook that skips the MMAs

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// shared-memory matrix descriptor of a K-major tile with the 128-byte
// swizzle (atoms 1024-byte aligned: base offset 0; the leading byte offset
// is unused when one MMA's K lies inside a row, and is set to 16 bytes)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = uint64_t((saddr >> 4) & 0x3fffu);
  d |= uint64_t(1) << 16;
  d |= uint64_t((kSBO >> 4) & 0x3fff) << 32;
  d |= uint64_t(1) << 46;                          // descriptor version of this architecture
  d |= kSwizzle128B << 61;
  return d;
}

// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M x N
constexpr uint32_t mma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// byte offset of element (row, k) of a tile (k a multiple of 8: the start of
// a 16-byte chunk)
__device__ __forceinline__ int tile_off(int row, int k) {
  return (row >> 3) * kSBO + (row & 7) * (kBK * 2) + ((((k >> 3) ^ row) & 7) << 4);
}

__device__ __forceinline__ bool barrier_wait(uint32_t bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  return uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(lo))) |
         (uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(hi))) << 16);
}

// One stage's operand slices, staged in registers between the global loads
// and the shared-memory stores, so that the next stage's loads are in flight
// while the tensor cores work on the current one.
struct StageRegs {
  float a[4][8];   // four (row, 8 k) items of P
  uint4 b[8];      // eight (column, 8 k) items of Bm
};

// KVEC: A's stride-1 index lies among the K indices (each group of 8 k is 8
// consecutive, 16-byte aligned floats of A): lanes run along k with two
// 16-byte loads per item; else lanes run along the rows with 8 scalar loads.
template <bool KVEC>
__device__ __forceinline__ void load_stage(StageRegs& R, int t, int m0, int n0, int k0, const float* __restrict__ A,
                                           const int32_t* __restrict__ rowoff, const int32_t* __restrict__ coloff,
                                           const uint16_t* __restrict__ Bm, int M, int N, int K) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int i = t + kPgThreads * j;
    const int r = KVEC ? i / (kBK / 8) : i % kBM, kg = KVEC ? i % (kBK / 8) : i / kBM;
    const int m = m0 + r, kb = k0 + kg * 8;
    if (KVEC) {
      float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
      if (m < M && kb < K) {
        const float4* p = reinterpret_cast<const float4*>(A + (int64_t(rowoff[m]) + coloff[kb]));
        lo = __ldg(p);
        hi = __ldg(p + 1);
      }
      R.a[j][0] = lo.x; R.a[j][1] = lo.y; R.a[j][2] = lo.z; R.a[j][3] = lo.w;
      R.a[j][4] = hi.x; R.a[j][5] = hi.y; R.a[j][6] = hi.z; R.a[j][7] = hi.w;
    } else {
      const int32_t ro = m < M ? rowoff[m] : 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = kb + e;
        R.a[j][e] = (m < M && k < K) ? __ldg(A + (int64_t(ro) + coloff[k])) : 0.f;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < (kBN * kBK / 8) / kPgThreads; ++j) {
    const int i = t + kPgThreads * j;
    const int kg = i % (kBK / 8), r = i / (kBK / 8);
    const int n = n0 + r, kb = k0 + kg * 8;
    R.b[j] = (n < N && kb < K) ? __ldg(reinterpret_cast<const uint4*>(Bm + (int64_t(n) * K + kb)))
                               : make_uint4(0u, 0u, 0u, 0u);
  }
}

template <bool KVEC>
__device__ __forceinline__ void store_stage(const StageRegs& R, int t, uint8_t* sA, uint8_t* sB) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int i = t + kPgThreads * j;
    const int r = KVEC ? i / (kBK / 8) : i % kBM, kg = KVEC ? i % (kBK / 8) : i / kBM;
    *reinterpret_cast<uint4*>(sA + tile_off(r, kg * 8)) =
        make_uint4(pack_bf16x2(R.a[j][0], R.a[j][1]), pack_bf16x2(R.a[j][2], R.a[j][3]),
                   pack_bf16x2(R.a[j][4], R.a[j][5]), pack_bf16x2(R.a[j][6], R.a[j][7]));
  }
#pragma unroll
  for (int j = 0; j < (kBN * kBK / 8) / kPgThreads; ++j) {
    const int i = t + kPgThreads * j;
    *reinterpret_cast<uint4*>(sB + tile_off(i / (kBK / 8), (i % (kBK / 8)) * 8)) = R.b[j];
  }
}

template <bool KVEC>
__global__ void __launch_bounds__(kPgThreads, 2)
    packgemm_kernel(const float* __restrict__ A, const int32_t* __restrict__ rowoff,
                    const int32_t* __restrict__ coloff, const uint16_t* __restrict__ Bm, float* __restrict__ C,
                    int M, int N, int K, float alpha, int* err, int skip_mma) {
  extern __shared__ __align__(1024) uint8_t smem[];
  // skip_mma (testing hook): no MMA is issued or committed, so every wait
  // runs out and takes the error path
  const uint32_t wait_limit = skip_mma ? kTestWaitLimit : kWaitLimit;
  // two buffers of (A slice, B slice), one barrier each
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * kStage);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 2 * kStage + 16);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
  const uint32_t bar0 = smem_addr(bars);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int nk = (K + kBK - 1) / kBK;
  bool ok = true;
  int issued = -1;   // last stage whose MMAs were committed
  StageRegs R;
  load_stage<KVEC>(R, t, m0, n0, 0, A, rowoff, coloff, Bm, M, N, K);
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    uint8_t* sA = smem + buf * kStage;
    uint8_t* sB = sA + kTileA;
    // this buffer was last read by the MMAs of stage kt - 2 (the j-th use of
    // a buffer completes its barrier's phase j)
    if (kt >= 2) {
      const bool mine = barrier_wait(bar0 + 8 * buf, uint32_t((kt - 2) >> 1) & 1u, wait_limit);
      ok = __syncthreads_and(ok && mine) != 0;
      if (!ok) break;
    }
    store_stage<KVEC>(R, t, sA, sB);
    // the slices were written by the generic proxy; the tensor cores read
    // them through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0 && !skip_mma) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
#pragma unroll
      for (int s = 0; s < kBK / 16; ++s) {
        const uint64_t da = smem_desc(a0 + s * 32), db = smem_desc(b0 + s * 32);
        const uint32_t accumulate = (kt > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(mma_idesc(kBM, kBN)), "r"(accumulate)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar0 + 8 * buf)
                   : "memory");
    }
    if (!skip_mma) issued = kt;
    if (kt + 1 < nk) load_stage<KVEC>(R, t, m0, n0, (kt + 1) * kBK, A, rowoff, coloff, Bm, M, N, K);
  }
  // the last commit completes when every MMA before it has completed
  if (ok) {
    const bool mine = issued >= 0 && barrier_wait(bar0 + 8 * (issued & 1), uint32_t(issued >> 1) & 1u, wait_limit);
    ok = __syncthreads_and(mine) != 0;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // accumulator row m0 + 32 * (warp % 4) + lane; warps 0-3 take the first
    // half of the columns, warps 4-7 the second
    const int q = warp & 3, h = warp >> 2;
    const int m = m0 + 32 * q + lane;
#pragma unroll 1
    for (int c = 0; c < kBN / 64; ++c) {
      const int col = (kBN / 2) * h + 32 * c;
      uint32_t r[32];
      const uint32_t taddr = tmem + (uint32_t(32 * q) << 16) + uint32_t(col);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < M) {
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const int n = n0 + col + e;
          if (n < N) C[int64_t(n) * M + m] = __fmul_rn(alpha, __uint_as_float(r[e]));
        }
      }
    }
  } else if (t == 0) {
    atomicExch(err, 1);
    // give the MMAs in flight a last bounded chance to finish before the
    // accumulator is released; if they still have not, the tensor memory is
    // released under them, and the error word says so for good (2)
    if (issued >= 0 && !barrier_wait(bar0 + 8 * (issued & 1), uint32_t(issued >> 1) & 1u, wait_limit))
      atomicExch(err, 2);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ---------------------------------------------------------------------------
// Warp-specialised form (K a multiple of 8, so that Bm's rows have a 16-byte
// pitch): a persistent CTA per SM walks 128 x 256 tiles of C (groups of 16
// row blocks, so that the A slices in flight share L2) with four roles over
// a ring of kWsStages (P slice, Bm slice) buffers:
//   warp 0      -- one thread copies each stage's 256 x 64 slice of Bm with
//                  TMA (a tensor map over this GPU's memory, 128-byte
//                  swizzle) and arms the stage's "full" barrier with its bytes;
//   warps 10-17 -- the pack: they gather the stage's 128 x 64 slice of P from
//                  A through the offset tables, round it to BF16 into the
//                  same swizzled layout, make it visible to the tensor cores
//                  (fence.proxy.async) and arrive on "full" (one arrival a
//                  warp);
//   warp 1      -- one thread issues the MMAs (M 128, N 256, K 16) of each
//                  full stage into one of two TMEM accumulators and commits
//                  the stage to its "empty" barrier, the tile to its
//                  accumulator's barrier;
//   warps 2-9   -- the epilogue of the other accumulator: tcgen05.ld, alpha,
//                  C written one column of 32 rows per instruction.
// The pack then runs ahead of the tensor cores by up to kWsStages stages
// instead of one, no thread holds a prefetch in registers, and the dense Bm
// takes no gather at all.
constexpr int kWsStages = 4;
constexpr int kWsGatherWarps = 8;
constexpr int kWsThreads = 64 + 32 * 8 + 32 * kWsGatherWarps;   // 576
constexpr int kWsGroupM = 16;
constexpr int kWsSmem = 1024 + kWsStages * kStage + 256;

__device__ __forceinline__ void ws_tile_of(int t, int ntm, int ntn, int* mb, int* nb) {
  const int per = kWsGroupM * ntn;
  const int grp = t / per, in = t - grp * per;
  const int first = grp * kWsGroupM;
  const int gsz = ntm - first < kWsGroupM ? ntm - first : kWsGroupM;
  *mb = first + in % gsz;
  *nb = in / gsz;
}

// one stage's 128 x 128 slice of P as E4M3 codes of alpha * a / scale (the
// codes of the FP8 permute), as 4 items of (row, 16 k) per thread
template <bool KVEC>
__device__ __forceinline__ void ws_pack_stage_fp8(int gt, int m0, int k0, const float* __restrict__ A,
                                                  const int32_t* __restrict__ rowoff,
                                                  const int32_t* __restrict__ coloff, int M, int K, float alpha,
                                                  float scale, float rcp, uint8_t* sA) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int i = gt + 32 * kWsGatherWarps * j;
    const int r = KVEC ? i / 8 : i % kBM, kg = KVEC ? i % 8 : i / kBM;
    const int m = m0 + r, kb = k0 + kg * 16;
    float v[16];
    if (KVEC) {
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m < M && kb < K) q = __ldg(reinterpret_cast<const float4*>(A + (int64_t(rowoff[m]) + coloff[kb])) + h);
        v[4 * h] = q.x; v[4 * h + 1] = q.y; v[4 * h + 2] = q.z; v[4 * h + 3] = q.w;
      }
    } else {
      const int32_t ro = m < M ? __ldg(rowoff + m) : 0;
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int k = kb + e;
        v[e] = (m < M && k < K) ? __ldg(A + (int64_t(ro) + __ldg(coloff + k))) : 0.f;
      }
    }
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      w[q] = 0;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        w[q] |= uint32_t(e4m3_of_quotient(__fmul_rn(alpha, v[4 * q + e]), scale, rcp)) << (8 * e);
    }
    // chunk kg of row r: 16 codes (the same 16-byte chunk layout as 8 BF16)
    *reinterpret_cast<uint4*>(sA + tile_off(r, kg * 8)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// one stage's 128 x 64 slice of P, as 4 items of (row, 8 k) per thread
template <bool KVEC>
__device__ __forceinline__ void ws_pack_stage(int gt, int m0, int k0, const float* __restrict__ A,
                                              const int32_t* __restrict__ rowoff,
                                              const int32_t* __restrict__ coloff, int M, int K, uint8_t* sA) {
  float v[4][8];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int i = gt + 32 * kWsGatherWarps * j;
    const int r = KVEC ? i / (kBK / 8) : i % kBM, kg = KVEC ? i % (kBK / 8) : i / kBM;
    const int m = m0 + r, kb = k0 + kg * 8;
    if (KVEC) {
      float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
      if (m < M && kb < K) {
        const float4* p = reinterpret_cast<const float4*>(A + (int64_t(rowoff[m]) + coloff[kb]));
        lo = __ldg(p);
        hi = __ldg(p + 1);
      }
      v[j][0] = lo.x; v[j][1] = lo.y; v[j][2] = lo.z; v[j][3] = lo.w;
      v[j][4] = hi.x; v[j][5] = hi.y; v[j][6] = hi.z; v[j][7] = hi.w;
    } else {
      const int32_t ro = m < M ? __ldg(rowoff + m) : 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = kb + e;
        v[j][e] = (m < M && k < K) ? __ldg(A + (int64_t(ro) + __ldg(coloff + k))) : 0.f;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int i = gt + 32 * kWsGatherWarps * j;
    const int r = KVEC ? i / (kBK / 8) : i % kBM, kg = KVEC ? i % (kBK / 8) : i / kBM;
    *reinterpret_cast<uint4*>(sA + tile_off(r, kg * 8)) =
        make_uint4(pack_bf16x2(v[j][0], v[j][1]), pack_bf16x2(v[j][2], v[j][3]), pack_bf16x2(v[j][4], v[j][5]),
                   pack_bf16x2(v[j][6], v[j][7]));
  }
}

// FP8: P packed as E4M3 codes of alpha * a / *scale_p, Bm read as E4M3
// codes, MMAs of kind::f8f6f4 (K 32), C = *scale_p * *scale_b * P Bm;
// 128 k per stage (still 128-byte rows)
template <bool KVEC, bool FP8>
__global__ void __launch_bounds__(kWsThreads, 1)
    packgemm_ws_kernel(const __grid_constant__ CUtensorMap mapB, const float* __restrict__ A,
                       const int32_t* __restrict__ rowoff, const int32_t* __restrict__ coloff,
                       float* __restrict__ C, int M, int N, int K, float alpha, const float* __restrict__ scale_p,
                       const float* __restrict__ scale_b, int* err, int skip_mma) {
  constexpr int KB = FP8 ? 128 : kBK;                 // k per stage
  // kind::f8f6f4 with E4M3 A and B (format 0), FP32 accumulator
  constexpr uint32_t kIdesc = FP8 ? ((1u << 4) | (uint32_t(kBN >> 3) << 17) | (uint32_t(kBM >> 4) << 24))
                                  : mma_idesc(kBM, kBN);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t wait_limit = skip_mma ? kTestWaitLimit : kWaitLimit;
  constexpr int S = kWsStages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * kStage);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 4);
  const uint32_t full0 = smem_addr(bars), empty0 = full0 + 8 * S;
  const uint32_t afull0 = full0 + 16 * S, aempty0 = afull0 + 16;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int nk = (K + KB - 1) / KB;
  const int ntm = (M + kBM - 1) / kBM, ntn = (N + kBN - 1) / kBN, total = ntm * ntn;

  if (t == 0) {
    for (int s = 0; s < S; ++s) {
      // full: the TMA thread's arrival (with the bytes) and one per pack warp
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full0 + 8 * s), "n"(1 + kWsGatherWarps) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * s) : "memory");
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(afull0 + 8 * b) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(aempty0 + 8 * b) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(2 * kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (t == 0) {
      bool ok = true;
      int it = 0;
      for (int tile = blockIdx.x; tile < total && ok; tile += gridDim.x) {
        int mb, nb;
        ws_tile_of(tile, ntm, ntn, &mb, &nb);
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const int s = it % S;
          if (it >= S && !barrier_wait(empty0 + 8 * s, uint32_t((it / S - 1) & 1), wait_limit)) {
            ok = false;
            break;
          }
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full0 + 8 * s), "r"(kTileB)
                       : "memory");
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
              "[%4];" ::"r"(smem_addr(smem + s * kStage + kTileA)),
              "l"(reinterpret_cast<uint64_t>(&mapB)), "r"(kt * KB), "r"(nb * kBN), "r"(full0 + 8 * s)
              : "memory");
        }
      }
      if (!ok) {
        atomicExch(err, 1);
        // the copies already issued land in this CTA's ring: wait (bounded)
        // for the stages in flight before the CTA may end
        for (int j = (it > S ? it - S : 0); j < it; ++j)
          barrier_wait(full0 + 8 * (j % S), uint32_t((j / S) & 1), wait_limit);
      }
    }
  } else if (warp >= 10) {
    // the pack warps
    const int gt = t - 320;
    const float sp = FP8 ? *scale_p : 1.f, rp = FP8 ? __frcp_rn(sp) : 1.f;
    bool ok = true;
    int it = 0;
    for (int tile = blockIdx.x; tile < total && ok; tile += gridDim.x) {
      int mb, nb;
      ws_tile_of(tile, ntm, ntn, &mb, &nb);
      for (int kt = 0; kt < nk; ++kt, ++it) {
        const int s = it % S;
        if (it >= S && !__all_sync(0xffffffffu, barrier_wait(empty0 + 8 * s, uint32_t((it / S - 1) & 1), wait_limit))) {
          ok = false;
          break;
        }
        if constexpr (FP8)
          ws_pack_stage_fp8<KVEC>(gt, mb * kBM, kt * KB, A, rowoff, coloff, M, K, alpha, sp, rp, smem + s * kStage);
        else
          ws_pack_stage<KVEC>(gt, mb * kBM, kt * KB, A, rowoff, coloff, M, K, smem + s * kStage);
        // written by the generic proxy, read by the tensor cores
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(full0 + 8 * s) : "memory");
      }
    }
    if (!ok && lane == 0) atomicExch(err, 1);
  } else if (warp == 1) {
    if (t == 32) {
      bool ok = true;
      int it = 0, ti = 0, committed = -1;
      for (int tile = blockIdx.x; tile < total && ok; tile += gridDim.x, ++ti) {
        const int b = ti & 1;
        if (ti >= 2 && !barrier_wait(aempty0 + 8 * b, uint32_t((ti / 2 - 1) & 1), wait_limit)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + uint32_t(kTmemCols * b);
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const int s = it % S;
          if (!barrier_wait(full0 + 8 * s, uint32_t((it / S) & 1), wait_limit)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          if (skip_mma) continue;   // testing hook: nothing issued or committed
          const uint32_t a0 = smem_addr(smem + s * kStage), b0 = a0 + kTileA;
#pragma unroll
          for (int q = 0; q < 4; ++q) {   // 32 bytes of every row per MMA: K 16 (BF16) or 32 (E4M3)
            const uint64_t da = smem_desc(a0 + q * 32), db = smem_desc(b0 + q * 32);
            const uint32_t accumulate = (kt > 0 || q > 0) ? 1u : 0u;
            if constexpr (FP8)
              asm volatile(
                  "{\n\t.reg .pred p;\n\t"
                  "setp.ne.b32 p, %4, 0;\n\t"
                  "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc),
                  "l"(da), "l"(db), "r"(kIdesc), "r"(accumulate)
                  : "memory");
            else
              asm volatile(
                  "{\n\t.reg .pred p;\n\t"
                  "setp.ne.b32 p, %4, 0;\n\t"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc),
                  "l"(da), "l"(db), "r"(kIdesc), "r"(accumulate)
                  : "memory");
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           empty0 + 8 * s)
                       : "memory");
          committed = it;
        }
        if (!ok || skip_mma) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         afull0 + 8 * b)
                     : "memory");
      }
      if (!ok || skip_mma) {
        atomicExch(err, 1);
        if (committed >= 0 &&
            !barrier_wait(empty0 + 8 * (committed % S), uint32_t((committed / S) & 1), wait_limit))
          atomicExch(err, 2);   // MMAs may outlive the CTA's tensor memory: reported for good
      }
    }
  } else {
    // epilogue: warp (q, h) writes rows 32 q + lane and columns h * 128 ..
    const int q = warp & 3, h = (warp - 2) >> 2;
    // FP8: the product of the codes times both scales (alpha is in P's codes)
    const float outscale = FP8 ? __fmul_rn(*scale_p, *scale_b) : alpha;
    int ti = 0;
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x, ++ti) {
      const int b = ti & 1;
      int mb, nb;
      ws_tile_of(tile, ntm, ntn, &mb, &nb);
      if (!__all_sync(0xffffffffu, barrier_wait(afull0 + 8 * b, uint32_t((ti / 2) & 1), wait_limit))) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int m = mb * kBM + 32 * q + lane;
#pragma unroll 1
      for (int c = 0; c < kBN / 64; ++c) {
        const int col = (kBN / 2) * h + 32 * c;
        uint32_t r[32];
        const uint32_t taddr = tmem + uint32_t(kTmemCols * b) + (uint32_t(32 * q) << 16) + uint32_t(col);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
              "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
              "=r"(r[30]), "=r"(r[31])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (m < M) {
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int n = nb * kBN + col + e;
            if (n < N) C[int64_t(n) * M + m] = __fmul_rn(outscale, __uint_as_float(r[e]));
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(aempty0 + 8 * b) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTmemCols) : "memory");
}

using EncodeTiledPg = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledPg pg_encode_fn() {
  static EncodeTiledPg fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledPg>(f);
  });
  return fn;
}

// Bm (N rows of K BF16 elements, pitch K) in boxes of 64 x 256, 128-byte
// swizzle, zero fill past its edges; false if it cannot be described
bool pg_map_b(CUtensorMap* map, const void* Bm, int64_t K, int64_t N, bool fp8) {
  EncodeTiledPg fn = pg_encode_fn();
  const int es = fp8 ? 1 : 2;
  if (!fn || (K * es) % 16 || reinterpret_cast<uintptr_t>(Bm) % 16) return false;
  const cuuint64_t dims[2] = {cuuint64_t(K), cuuint64_t(N)};
  const cuuint64_t strides[1] = {cuuint64_t(K) * cuuint64_t(es)};
  const cuuint32_t box[2] = {cuuint32_t(128 / es), cuuint32_t(kBN)};
  const cuuint32_t el[2] = {1, 1};
  return fn(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(Bm),
            dims, strides, box, el,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct PgDev {
  int32_t* tables = nullptr;   // rowoff[M] | coloff[K] | error word
  int* err = nullptr;
  bool ws_attr = false;        // the warp-specialised kernels' shared-memory limit is set
  bool ws_fp8_attr = false;
};

}  // namespace

struct ttc_packed_gemm_s {
  std::mutex mu;
  int64_t M = 0, N = 0, K = 0, spanA = 0;
  float alpha = 1.f;
  bool kvec = false;   // every group of 8 k is 8 consecutive floats of A, 16-byte aligned relative to A
  int skip_mma = 0;    // testing hook (ttc_debug_packed_gemm_skip_mma)
  bool force_classic = false;   // testing hook (ttc_debug_packed_gemm_classic)
  bool kvec16 = false;          // every group of 16 k is 16 consecutive floats of A, 16-byte aligned relative to A
  const float* scale_p = nullptr;   // FP8 operands (ttc_packed_gemm_set_fp8): device scales of P and Bm
  const float* scale_b = nullptr;
  std::vector<int32_t> rowoff, coloff;
  std::map<int, PgDev> dev;
  ~ttc_packed_gemm_s() {
    int cur = 0;
    const bool have = cudaGetDevice(&cur) == cudaSuccess;
    for (auto& kv : dev) {
      if (have) cudaSetDevice(kv.first);
      if (kv.second.tables) cudaFree(kv.second.tables);
    }
    if (have) cudaSetDevice(cur);
  }
};

extern "C" {

ttc_status ttc_packed_gemm_plan(ttc_packed_gemm_t* out, int ndim, const int* perm, const int64_t* sizes,
                                const int64_t* outer_sizes_A, int rank_m, int64_t n, double alpha) {
  if (!out) return fail(TTC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (ndim < 1 || ndim > kMaxDim || !perm || !sizes) return fail(TTC_ERR_INVALID_PERM, "bad ndim, perm or sizes");
  std::vector<int> seen(size_t(ndim), 0);
  for (int d = 0; d < ndim; ++d) {
    if (perm[d] < 0 || perm[d] >= ndim || seen[size_t(perm[d])]++) return fail(TTC_ERR_INVALID_PERM, "not a permutation");
  }
  if (rank_m < 1 || rank_m >= ndim) return fail(TTC_ERR_INVALID_ARG, "rank_m must split the packed indices");
  if (!std::isfinite(alpha)) return fail(TTC_ERR_INVALID_ARG, "alpha not finite");
  std::vector<int64_t> strideA(static_cast<size_t>(ndim));
  int64_t st = 1, span = 1;
  for (int k = 0; k < ndim; ++k) {
    const int64_t o = outer_sizes_A ? outer_sizes_A[k] : sizes[k];
    if (sizes[k] < 1) return fail(TTC_ERR_INVALID_SIZE, "sizes must be >= 1");
    if (o < sizes[k]) return fail(TTC_ERR_INVALID_OUTER, "outer size below size");
    strideA[size_t(k)] = st;
    span += (sizes[k] - 1) * st;
    st *= o;
  }
  if (span >= (int64_t(1) << 31)) return fail(TTC_ERR_INVALID_SIZE, "A spans 2^31 elements or more");
  std::unique_ptr<ttc_packed_gemm_s> g(new (std::nothrow) ttc_packed_gemm_s());
  if (!g) return fail(TTC_ERR_OOM, "host allocation failed");
  // the packed panel's index d is A's index perm[d]; d < rank_m form the
  // row (M) index, the rest the column (K) index, both column-major
  auto offsets = [&](int d0, int d1, std::vector<int32_t>* out_offs) -> int64_t {
    int64_t cnt = 1;
    for (int d = d0; d < d1; ++d) cnt *= sizes[perm[d]];
    if (cnt >= (int64_t(1) << 31)) return -1;
    out_offs->assign(size_t(cnt), 0);
    for (int64_t i = 0; i < cnt; ++i) {
      int64_t r = i, off = 0;
      for (int d = d0; d < d1; ++d) {
        const int64_t s = sizes[perm[d]];
        off += (r % s) * strideA[size_t(perm[d])];
        r /= s;
      }
      (*out_offs)[size_t(i)] = int32_t(off);
    }
    return cnt;
  };
  g->M = offsets(0, rank_m, &g->rowoff);
  g->K = offsets(rank_m, ndim, &g->coloff);
  if (g->M < 0 || g->K < 0) return fail(TTC_ERR_INVALID_SIZE, "a GEMM extent exceeds 2^31 - 1");
  if (g->K % 8) return fail(TTC_ERR_INVALID_SIZE, "K must be a multiple of 8 (16-byte rows of the BF16 matrix)");
  if (n < 1 || n >= (int64_t(1) << 31) || g->M * n >= (int64_t(1) << 62))
    return fail(TTC_ERR_INVALID_SIZE, "bad n");
  if ((g->M + kBM - 1) / kBM > 2147483647 || (n + kBN - 1) / kBN > 65535)
    return fail(TTC_ERR_INVALID_SIZE, "too many tiles");
  g->N = n;
  g->spanA = span;
  g->alpha = float(alpha);
  g->kvec = true;
  for (int64_t k = 0; k < g->K && g->kvec; k += 8) {
    if (g->coloff[size_t(k)] % 4) g->kvec = false;
    for (int e = 1; e < 8 && g->kvec; ++e)
      if (g->coloff[size_t(k + e)] != g->coloff[size_t(k)] + e) g->kvec = false;
  }
  for (int64_t m = 0; m < g->M && g->kvec; ++m)
    if (g->rowoff[size_t(m)] % 4) g->kvec = false;
  g->kvec16 = g->kvec && g->K % 16 == 0;
  for (int64_t k = 0; k < g->K && g->kvec16; k += 16)
    if (g->coloff[size_t(k + 8)] != g->coloff[size_t(k)] + 8) g->kvec16 = false;
  *out = g.release();
  return TTC_OK;
}

ttc_status ttc_packed_gemm_execute(ttc_packed_gemm_t g, const float* A, const void* B, float* C,
                                   ttc_stream_t stream) {
  if (!g) return fail(TTC_ERR_INVALID_ARG, "plan is NULL");
  if (!A || !B || !C) return fail(TTC_ERR_INVALID_ARG, "A, B or C is NULL");
  if (reinterpret_cast<uintptr_t>(A) % 4 || reinterpret_cast<uintptr_t>(C) % 4 ||
      reinterpret_cast<uintptr_t>(B) % 16)
    return fail(TTC_ERR_ALIGN, "A and C need 4-byte, B 16-byte alignment");
  const uintptr_t a = reinterpret_cast<uintptr_t>(A), c = reinterpret_cast<uintptr_t>(C);
  const uintptr_t b = reinterpret_cast<uintptr_t>(B);
  const size_t bytesC = size_t(g->M) * size_t(g->N) * 4, bytesA = size_t(g->spanA) * 4;
  const bool fp8 = g->scale_p != nullptr;
  const size_t bytesB = size_t(g->K) * size_t(g->N) * (fp8 ? 1 : 2);
  if ((c < a + bytesA && a < c + bytesC) || (c < b + bytesB && b < c + bytesC))
    return fail(TTC_ERR_ALIAS, "C overlaps A or B");
  std::lock_guard<std::mutex> lk(g->mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  PgDev& d = g->dev[dev];
  if (!d.tables) {
    const size_t ints = g->rowoff.size() + g->coloff.size() + 1;
    e = cudaMalloc(&d.tables, ints * sizeof(int32_t));
    if (e != cudaSuccess) {
      d.tables = nullptr;
      return e == cudaErrorMemoryAllocation ? fail(TTC_ERR_OOM, "table allocation failed")
                                            : cuda_fail(e, "cudaMalloc");
    }
    e = cudaMemcpy(d.tables, g->rowoff.data(), g->rowoff.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(d.tables + g->rowoff.size(), g->coloff.data(), g->coloff.size() * sizeof(int32_t),
                     cudaMemcpyHostToDevice);
    d.err = d.tables + g->rowoff.size() + g->coloff.size();
    if (e == cudaSuccess) e = cudaMemset(d.err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "table upload");
    e = cudaFuncSetAttribute(packgemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPgSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(packgemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPgSmem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  }
  const dim3 grid(unsigned((g->M + kBM - 1) / kBM), unsigned((g->N + kBN - 1) / kBN));
  const int32_t* rows = d.tables;
  const int32_t* cols = d.tables + g->rowoff.size();
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CUtensorMap mapB;
  std::memset(&mapB, 0, sizeof(mapB));
  const bool kvec = g->kvec && reinterpret_cast<uintptr_t>(A) % 16 == 0;
  if (fp8) {
    // E4M3 operands: the warp-specialised kernel only (kind::f8f6f4)
    if (!pg_map_b(&mapB, B, g->K, g->N, true)) return fail(TTC_ERR_INVALID_ARG, "cannot describe Bm for TMA");
    if (!d.ws_fp8_attr) {
      e = cudaFuncSetAttribute(packgemm_ws_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWsSmem);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(packgemm_ws_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kWsSmem);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
      d.ws_fp8_attr = true;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    const unsigned pgrid = unsigned(std::min<int64_t>(int64_t(grid.x) * int64_t(grid.y), sms));
    if (g->kvec16 && reinterpret_cast<uintptr_t>(A) % 16 == 0)
      packgemm_ws_kernel<true, true><<<pgrid, kWsThreads, kWsSmem, s>>>(mapB, A, rows, cols, C, int(g->M),
                                                                        int(g->N), int(g->K), g->alpha, g->scale_p,
                                                                        g->scale_b, d.err, g->skip_mma);
    else
      packgemm_ws_kernel<false, true><<<pgrid, kWsThreads, kWsSmem, s>>>(mapB, A, rows, cols, C, int(g->M),
                                                                         int(g->N), int(g->K), g->alpha, g->scale_p,
                                                                         g->scale_b, d.err, g->skip_mma);
    ++g_launches;
    e = cudaGetLastError();
    return e == cudaSuccess ? TTC_OK : cuda_fail(e, "packed GEMM launch");
  }
  if (!g->force_classic && kvec && pg_map_b(&mapB, B, g->K, g->N, false)) {
    // the warp-specialised kernel: Bm by TMA, the pack by its own warps.
    // Only where the pack reads A 16 bytes at a time (k dense in A): with
    // scalar loads its 8 warps keep too few bytes in flight to feed the
    // tensor cores (measured 210 against 336 TFLOP/s for the register-staged
    // kernel on a 4096 x 2048 sub-block; 505 against 447 with 16-byte loads)
    if (!d.ws_attr) {
      e = cudaFuncSetAttribute(packgemm_ws_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWsSmem);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
      d.ws_attr = true;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    const int64_t tiles = int64_t(grid.x) * int64_t(grid.y);
    const unsigned pgrid = unsigned(std::min<int64_t>(tiles, sms));
    packgemm_ws_kernel<true, false><<<pgrid, kWsThreads, kWsSmem, s>>>(mapB, A, rows, cols, C, int(g->M),
                                                                       int(g->N), int(g->K), g->alpha, nullptr,
                                                                       nullptr, d.err, g->skip_mma);
    ++g_launches;
    e = cudaGetLastError();
    return e == cudaSuccess ? TTC_OK : cuda_fail(e, "packed GEMM launch");
  }
  if (g->kvec && reinterpret_cast<uintptr_t>(A) % 16 == 0)
    packgemm_kernel<true><<<grid, kPgThreads, kPgSmem, s>>>(A, rows, cols, static_cast<const uint16_t*>(B), C,
                                                             int(g->M), int(g->N), int(g->K), g->alpha, d.err,
                                                             g->skip_mma);
  else
    packgemm_kernel<false><<<grid, kPgThreads, kPgSmem, s>>>(A, rows, cols, static_cast<const uint16_t*>(B), C,
                                                              int(g->M), int(g->N), int(g->K), g->alpha, d.err,
                                                              g->skip_mma);
  ++g_launches;
  e = cudaGetLastError();
  return e == cudaSuccess ? TTC_OK : cuda_fail(e, "packed GEMM launch");
}

ttc_status ttc_packed_gemm_check(ttc_packed_gemm_t g) {
  if (!g) return fail(TTC_ERR_INVALID_ARG, "plan is NULL");
  std::lock_guard<std::mutex> lk(g->mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  auto it = g->dev.find(dev);
  if (it == g->dev.end() || !it->second.err) return TTC_OK;
  int flag = 0;
  e = cudaMemcpy(&flag, it->second.err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "error word read");
  if (!flag) return TTC_OK;
  if (flag == 2)   // sticky: not reset
    return fail(TTC_ERR_TIMEOUT, "a CTA released its tensor memory with MMAs possibly still in flight: tensor-core "
                                 "results on this device are unreliable from then on");
  e = cudaMemset(it->second.err, 0, sizeof(int));      // reported once
  if (e != cudaSuccess) return cuda_fail(e, "error word reset");
  return fail(TTC_ERR_TIMEOUT, "a tensor-core wait gave up");
}

ttc_status ttc_packed_gemm_info(ttc_packed_gemm_t g, int64_t* m, int64_t* n, int64_t* k) {
  if (!g) return fail(TTC_ERR_INVALID_ARG, "plan is NULL");
  if (m) *m = g->M;
  if (n) *n = g->N;
  if (k) *k = g->K;
  return TTC_OK;
}

ttc_status ttc_packed_gemm_set_fp8(ttc_packed_gemm_t g, const float* scale_p, const float* scale_b) {
  if (!g) return fail(TTC_ERR_INVALID_ARG, "plan is NULL");
  if ((scale_p == nullptr) != (scale_b == nullptr)) return fail(TTC_ERR_INVALID_ARG, "give both scales or neither");
  if (scale_p && g->K % 16) return fail(TTC_ERR_INVALID_SIZE, "E4M3 operands need K a multiple of 16");
  if ((scale_p && reinterpret_cast<uintptr_t>(scale_p) % 4) || (scale_b && reinterpret_cast<uintptr_t>(scale_b) % 4))
    return fail(TTC_ERR_ALIGN, "scales need 4-byte alignment");
  std::lock_guard<std::mutex> lk(g->mu);
  g->scale_p = scale_p;
  g->scale_b = scale_b;
  return TTC_OK;
}

ttc_status ttc_debug_packed_gemm_classic(ttc_packed_gemm_t g, int classic) {
  if (!g) return fail(TTC_ERR_INVALID_ARG, "plan is NULL");
  std::lock_guard<std::mutex> lk(g->mu);
  g->force_classic = classic != 0;
  return TTC_OK;
}

ttc_status ttc_debug_packed_gemm_skip_mma(ttc_packed_gemm_t g, int skip) {
  if (!g) return fail(TTC_ERR_INVALID_ARG, "plan is NULL");
  std::lock_guard<std::mutex> lk(g->mu);
  g->skip_mma = skip ? 1 : 0;
  return TTC_OK;
}

ttc_status ttc_packed_gemm_destroy(ttc_packed_gemm_t g) {
  if (!g) return fail(TTC_ERR_INVALID_ARG, "plan is NULL");
  delete g;
  return TTC_OK;
}

}  // extern "C"
