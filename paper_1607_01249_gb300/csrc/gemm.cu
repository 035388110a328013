// gemm.cu -- the BF16 GEMM of the TTGT contractions (section 1: a tensor
// contraction as transposes around one GEMM), on the tensor cores:
//
//   C[rowoff[m] + coloff[n]] = alpha * sum_k A[m, k] B[n, k] + beta * C[...]
//
// with both operands K-major BF16 matrices as this library's permutes write
// them: A holds, for every m, K consecutive elements (row pitch lda >= K), and
// B the same for every n (pitch ldb).  K-major on both sides lets the tensor
// memory accelerator (TMA) copy each 64-element K slice of 128 rows of A and
// 256 rows of B into shared memory in the tensor cores' 128-byte swizzled
// layout directly, with no thread touching the data.  C is FP32 at any
// offsets rowoff[m] + coloff[n]: a column-major matrix, or a tensor whose
// indices the GEMM's rows and columns split between them (the permutation of
// the product folded into the epilogue's stores).
//
// Persistent: one CTA per SM loops over 128 x 256 output tiles with three
// roles:
//   warp 0  -- one thread issues the TMA copies of each K stage into a ring
//              of kStages buffers (an mbarrier per buffer counts the bytes);
//   warp 1  -- allocates two 256-column FP32 accumulators in tensor memory
//              (TMEM, all 512 columns); one thread issues tcgen05.mma (M 128,
//              N 256, K 16) as each buffer fills, commits each stage to the
//              buffer's "empty" barrier so the producer can refill it, and a
//              finished tile to its accumulator's "full" barrier;
//   warps 2-5 -- the epilogue: tcgen05.ld of one accumulator (each warp its
//              32 TMEM lanes), alpha and beta applied, C written, then the
//              accumulator handed back; meanwhile the MMAs of the next tile
//              run in the other accumulator.
// Every mbarrier wait is bounded; a wait that gives up records an error word
// (reported by the caller as TTC_ERR_TIMEOUT), waits (bounded) for its own
// copies and MMAs in flight and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "gemm.h"

namespace ttc {
extern std::atomic<int64_t> g_launches;

namespace {

constexpr int kGM = 128, kGN = 256, kGK = 64;        // CTA tile; one MMA is 128 x 256 x 16
constexpr int kStages = 4;
constexpr int kGThreads = 192;                        // 6 warps
constexpr uint32_t kGTmemCols = 512;                  // two 256-column accumulators
constexpr int kATile = kGM * kGK * 2;                 // 16 KiB
constexpr int kBTile = kGN * kGK * 2;                 // 32 KiB
constexpr int kSBO = 8 * kGK * 2;                     // 1024-byte atoms of 8 rows of 128 bytes
constexpr uint64_t kSwizzle128B = 2;
constexpr int kGroupM = 16;                           // tiles visited in groups of 16 row blocks
// dynamic shared memory: 1024-byte alignment slack, the ring, the barriers
constexpr int kGSmem = 1024 + kStages * (kATile + kBTile) + 256;
constexpr uint32_t kGWaitLimit = 1u << 24;            // polls of one barrier phase before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle
// (atoms 1024-byte aligned; the leading byte offset is unused when one MMA's
// K lies within a 128-byte row and is set to 16 bytes)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = uint64_t((saddr >> 4) & 0x3fffu);
  d |= uint64_t(1) << 16;
  d |= uint64_t((kSBO >> 4) & 0x3fff) << 32;
  d |= uint64_t(1) << 46;
  d |= kSwizzle128B << 61;
  return d;
}

// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M x N
constexpr uint32_t mma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < kGWaitLimit; ++i) {
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

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// output tile t: row block mb and column block nb, visited in groups of
// kGroupM row blocks (all column blocks of a group before the next), so the
// tiles in flight at one time share their A and B slices in L2
__device__ __forceinline__ void tile_of(int t, int ntm, int ntn, int* mb, int* nb) {
  const int per = kGroupM * ntn;
  const int grp = t / per, in = t - grp * per;
  const int first = grp * kGroupM;
  const int gsz = ntm - first < kGroupM ? ntm - first : kGroupM;
  *mb = first + in % gsz;
  *nb = in / gsz;
}

__global__ void __launch_bounds__(kGThreads, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                     float* __restrict__ C, const int64_t* __restrict__ rowoff, const int64_t* __restrict__ coloff,
                     int M, int N, int K, float alpha, float beta, int* err) {
  extern __shared__ uint8_t smem_raw[];
  // the ring must start on a 1024-byte boundary (the swizzle atoms)
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * kATile;
  // barriers: full[S], empty[S], accumulator full[2], accumulator empty[2]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kStages * kBTile);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 4);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * kStages;
  const uint32_t afull0 = full0 + 16 * kStages, aempty0 = afull0 + 16;
  const int t = threadIdx.x, warp = t >> 5;
  const int nk = (K + kGK - 1) / kGK;
  const int ntm = (M + kGM - 1) / kGM, ntn = (N + kGN - 1) / kGN, total = ntm * ntn;

  if (t == 0) {
    for (int s = 0; s < kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * s) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * s) : "memory");
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(afull0 + 8 * b) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(aempty0 + 8 * b) : "memory");   // 4 epilogue warps
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kGTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (t == 0) {
      // producer: the it-th stage of this CTA (over all its tiles) waits for
      // the MMAs of stage it - kStages to have read its buffer (the j-th use
      // of a buffer completes phase j of its barriers)
      bool ok = true;
      int it = 0;
      for (int tile = blockIdx.x; tile < total && ok; tile += gridDim.x) {
        int mb, nb;
        tile_of(tile, ntm, ntn, &mb, &nb);
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const int s = it % kStages;
          if (it >= kStages && !bar_wait(empty0 + 8 * s, uint32_t((it / kStages - 1) & 1))) {
            ok = false;
            break;
          }
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full0 + 8 * s),
                       "r"(kATile + kBTile)
                       : "memory");
          tma_load_2d(smem_u32(sA + s * kATile), &mapA, kt * kGK, mb * kGM, full0 + 8 * s);
          tma_load_2d(smem_u32(sB + s * kBTile), &mapB, kt * kGK, nb * kGN, full0 + 8 * s);
        }
      }
      if (!ok) {
        atomicExch(err, 1);
        // the copies already issued land in this CTA's buffers: wait for them
        // (bounded) before the CTA may end
        for (int j = (it > kStages ? it - kStages : 0); j < it; ++j)
          bar_wait(full0 + 8 * (j % kStages), uint32_t((j / kStages) & 1));
      }
    }
  } else if (warp == 1) {
    if (t == 32) {
      bool ok = true;
      int it = 0, ti = 0, committed = -1;
      for (int tile = blockIdx.x; tile < total && ok; tile += gridDim.x, ++ti) {
        const int b = ti & 1;
        // the epilogue has read this accumulator's previous tile
        if (ti >= 2 && !bar_wait(aempty0 + 8 * b, uint32_t((ti / 2 - 1) & 1))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc_tmem = tmem + uint32_t(256 * b);
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const int s = it % kStages;
          if (!bar_wait(full0 + 8 * s, uint32_t((it / kStages) & 1))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(sA + s * kATile), b0 = smem_u32(sB + s * kBTile);
#pragma unroll
          for (int q = 0; q < kGK / 16; ++q) {
            const uint64_t da = smem_desc(a0 + q * 32), db = smem_desc(b0 + q * 32);
            const uint32_t accumulate = (kt > 0 || q > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc_tmem),
                "l"(da), "l"(db), "r"(mma_idesc(kGM, kGN)), "r"(accumulate)
                : "memory");
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           empty0 + 8 * s)
                       : "memory");
          committed = it;
        }
        if (!ok) break;
        if (nk == 0)   // K = 0: nothing to multiply; the epilogue writes beta * C
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(afull0 + 8 * b) : "memory");
        else
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           afull0 + 8 * b)
                       : "memory");
      }
      if (!ok) {
        atomicExch(err, 1);
        // the MMAs already issued still read the ring and write TMEM: wait
        // (bounded) for the last commit before the accumulators are released
        if (committed >= 0) bar_wait(empty0 + 8 * (committed % kStages), uint32_t((committed / kStages) & 1));
      }
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (accumulator rows)
    const int q = warp & 3, lane = t & 31;
    int ti = 0;
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x, ++ti) {
      const int b = ti & 1;
      if (!bar_wait(afull0 + 8 * b, uint32_t((ti / 2) & 1))) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int mb, nb;
      tile_of(tile, ntm, ntn, &mb, &nb);
      const int m = mb * kGM + 32 * q + lane;
      const int64_t ro = m < M ? __ldg(rowoff + m) : 0;
#pragma unroll 1
      for (int c = 0; c < kGN / 32; ++c) {
        uint32_t r[32];
        const uint32_t taddr = tmem + uint32_t(256 * b) + (uint32_t(32 * q) << 16) + uint32_t(32 * c);
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
            const int n = nb * kGN + 32 * c + e;
            if (n < N) {
              float* cp = C + (ro + __ldg(coloff + n));
              const float acc = K > 0 ? __fmul_rn(alpha, __uint_as_float(r[e])) : 0.f;
              *cp = beta != 0.f ? __fmaf_rn(beta, *cp, acc) : acc;
            }
          }
        }
      }
      // this warp's TMEM reads are done: hand the accumulator back
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(aempty0 + 8 * b) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGTmemCols) : "memory");
}

// cuTensorMapEncodeTiled through the runtime's driver entry points (no link
// against the driver library)
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(f);
  });
  return fn;
}

// a K-major BF16 matrix of `rows` rows of K elements at pitch `ld`, copied in
// boxes of 64 (K) x box_rows, 128-byte swizzle, zero fill past its edges
bool make_map(CUtensorMap* map, const uint16_t* base, int64_t K, int64_t rows, int64_t ld, int box_rows) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cuuint64_t(K), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(ld) * 2};
  const cuuint32_t box[2] = {cuuint32_t(kGK), cuuint32_t(box_rows)};
  const cuuint32_t elem[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(base), dims, strides, box, elem,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

std::mutex g_attr_mu;
bool g_attr_set[64] = {};

}  // namespace

const char* gemm_bf16_check(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int64_t N, int64_t K) {
  if (M < 1 || N < 1 || K < 0) return "empty GEMM";
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return "a GEMM extent exceeds 2^31 - 1";
  if (((M + kGM - 1) / kGM) * ((N + kGN - 1) / kGN) > INT32_MAX) return "too many tiles";
  if (K == 0) return nullptr;   // the operands are not read
  if (lda < K || ldb < K || lda % 8 || ldb % 8) return "row pitches must be >= K and multiples of 8 elements";
  if (reinterpret_cast<uintptr_t>(A) % 16 || reinterpret_cast<uintptr_t>(B) % 16)
    return "operands must be 16-byte aligned";
  return nullptr;
}

cudaError_t gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, const int64_t* rowoff,
                      const int64_t* coloff, int64_t M, int64_t N, int64_t K, float alpha, float beta, int* err,
                      cudaStream_t s) {
  CUtensorMap ma, mb;
  std::memset(&ma, 0, sizeof(ma));
  std::memset(&mb, 0, sizeof(mb));
  // (K = 0: no copies are issued and the maps stay unused)
  if (K > 0 && (!make_map(&ma, static_cast<const uint16_t*>(A), K, M, lda, kGM) ||
                !make_map(&mb, static_cast<const uint16_t*>(B), K, N, ldb, kGN)))
    return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    if (dev >= 0 && dev < 64 && !g_attr_set[dev]) {
      e = cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmem);
      if (e != cudaSuccess) return e;
      g_attr_set[dev] = true;
    }
  }
  const int64_t tiles = ((M + kGM - 1) / kGM) * ((N + kGN - 1) / kGN);
  const unsigned grid = unsigned(std::min<int64_t>(tiles, sms));
  gemm_bf16_kernel<<<grid, kGThreads, kGSmem, s>>>(ma, mb, C, rowoff, coloff, int(M), int(N), int(K), alpha, beta,
                                                   err);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ttc
