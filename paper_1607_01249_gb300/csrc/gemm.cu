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
//   warps 2-9 -- the epilogue: tcgen05.ld of one accumulator (each warp its
//              32 TMEM lanes and half of the columns), alpha and beta
//              applied, C written, then the accumulator handed back;
//              meanwhile the MMAs of the next tile run in the other
//              accumulator.  A warp stores one column of its 32 rows per
//              instruction (consecutive m, one 128-byte line when rowoff is
//              contiguous); the column offsets of each 32-column chunk are
//              read once, one per lane, and broadcast by shuffles, so that no
//              store waits on a load of its own address.
// Every mbarrier wait is bounded; a wait that gives up records an error word
// (reported by the caller as TTC_ERR_TIMEOUT), waits (bounded) for its own
// copies and MMAs in flight and returns.  If the MMAs in flight do not finish
// within that last wait either, the tensor memory is released under them and
// the error word is set to 2, which the caller never clears.
//
// The pair variant (gemm_bf16_pair_kernel) runs the same roles on a cluster
// of two CTAs on neighbouring SMs that share one 256 x BN output tile
// (tcgen05 with cta_group::2): each CTA copies its 128 rows of A and its
// BN/2 rows of B, one thread of the even CTA issues MMAs of M = 256 that read
// both CTAs' shared memory and write 128 accumulator rows into each CTA's
// tensor memory.  Per output element each SM then streams half the B bytes
// of the single-CTA tile, and the smaller stages make a deeper ring.
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

constexpr int kGM = 128, kGK = 64;                   // rows of A per CTA; K per stage (one MMA takes 16)
constexpr int kGEpiWarps = 8;                        // two per TMEM lane quarter, one per half of the columns
constexpr int kGThreads = 64 + 32 * kGEpiWarps;       // producer warp, MMA warp, epilogue warps
constexpr int kATile = kGM * kGK * 2;                 // 16 KiB
constexpr int kSBO = 8 * kGK * 2;                     // 1024-byte atoms of 8 rows of 128 bytes
constexpr uint64_t kSwizzle128B = 2;
constexpr int kGroupM = 16;                           // tiles visited in groups of 16 row blocks
// (dynamic shared memory: 1024-byte alignment slack, the ring, the barriers)
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

// Epilogue offsets of one tile, read before the accumulator is ready so that
// their latency hides behind the MMAs: warp (q, h) writes rows m_base + 32 q
// + lane and the BN/64 column chunks n_base + h BN/2 + 32 c + [0, 32).
template <int BN>
struct EpiOffsets {
  int64_t ro;
  int64_t co[BN / 64];   // lane's column offset in each chunk
  bool mok;
};

template <int BN>
__device__ __forceinline__ void load_offsets(EpiOffsets<BN>& o, int q, int h, int lane, int m_base, int n_base, int M,
                                             int N, const int64_t* __restrict__ rowoff,
                                             const int64_t* __restrict__ coloff) {
  const int m = m_base + 32 * q + lane;
  o.mok = m < M;
  o.ro = o.mok ? __ldg(rowoff + m) : 0;
#pragma unroll
  for (int c = 0; c < BN / 64; ++c) {
    const int n = n_base + (BN / 2) * h + 32 * c + lane;
    o.co[c] = n < N ? __ldg(coloff + n) : 0;
  }
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

// one 32-column chunk: a store per column, lanes on consecutive rows; with
// BETA false C is never read
template <bool BETA>
__device__ __forceinline__ void store_chunk(const uint32_t (&r)[32], int64_t co, bool mok, int64_t ro, int nleft,
                                            float* __restrict__ C, float alpha, float beta, bool kzero) {
#pragma unroll
  for (int e = 0; e < 32; ++e) {
    const int64_t coe = __shfl_sync(0xffffffffu, co, e);   // every lane takes part
    if (mok && e < nleft) {
      float* cp = C + (ro + coe);
      const float acc = kzero ? 0.f : __fmul_rn(alpha, __uint_as_float(r[e]));
      if (BETA)
        *cp = __fmaf_rn(beta, *cp, acc);
      else
        *cp = acc;
    }
  }
}

// Epilogue of one accumulator (TMEM columns from tacc) with the offsets o:
// the next chunk's tensor-memory load is in flight while a chunk is stored.
// kzero: K = 0, the accumulator was never written and counts as zero.
template <int BN>
__device__ __forceinline__ void store_accumulator(uint32_t tacc, const EpiOffsets<BN>& o, int q, int h,
                                                  int n_base, int N, float* __restrict__ C, float alpha, float beta,
                                                  bool kzero) {
  constexpr int NC = BN / 64;
  uint32_t r[2][32];
  const uint32_t t0 = tacc + (uint32_t(32 * q) << 16) + uint32_t((BN / 2) * h);
  tmem_ld32(t0, r[0]);
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (c + 1 < NC) tmem_ld32(t0 + uint32_t(32 * (c + 1)), r[(c + 1) & 1]);
    const int nleft = N - (n_base + (BN / 2) * h + 32 * c);
    if (beta != 0.f)
      store_chunk<true>(r[c & 1], o.co[c], o.mok, o.ro, nleft, C, alpha, beta, kzero);
    else
      store_chunk<false>(r[c & 1], o.co[c], o.mok, o.ro, nleft, C, alpha, beta, kzero);
    if (c + 1 < NC) asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  }
}

// --- CTA pairs (cluster of two) ------------------------------------------

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// the address of the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// bounded wait with cluster-scope acquire (arrivals from the peer CTA)
__device__ __forceinline__ bool bar_wait_cluster(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < kGWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// a TMA copy into this CTA's shared memory whose completion is counted on a
// barrier of either CTA of the pair (bar: a cluster address)
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// commit of the pair's MMAs issued so far to the barrier at offset `bar` in
// both CTAs
__device__ __forceinline__ void commit_pair(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"(uint16_t(3))
      : "memory");
}

template <int BN>
struct PairCfg {
  static constexpr int kBHalf = BN / 2;                     // rows of B per CTA
  static constexpr int kBTile = kBHalf * kGK * 2;
  static constexpr int kStageBytes = kATile + kBTile;       // per CTA
  static constexpr int kStages = BN == 256 ? 7 : BN == 192 ? 8 : 9;
  static constexpr uint32_t kCols = BN == 128 ? 256 : 512;  // two accumulators (a power of two)
  static constexpr uint32_t kAccStride = kCols / 2;         // accumulator b at column b x this
  static constexpr int kSmem = 1024 + kStages * kStageBytes + 256;
};
static_assert(PairCfg<256>::kSmem <= 232448 && PairCfg<192>::kSmem <= 232448 && PairCfg<128>::kSmem <= 232448,
              "shared memory");

template <int BN>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kGThreads, 1)
    gemm_bf16_pair_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                          float* __restrict__ C, const int64_t* __restrict__ rowoff,
                          const int64_t* __restrict__ coloff, int M, int N, int K, float alpha, float beta,
                          int* err) {
  using P = PairCfg<BN>;
  constexpr int S = P::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + S * kATile;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + S * P::kBTile);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 4);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * S;
  const uint32_t afull0 = full0 + 16 * S, aempty0 = afull0 + 16;
  const int t = threadIdx.x, warp = t >> 5;
  const uint32_t rank = cluster_rank();
  const int pair = int(blockIdx.x >> 1), npairs = int(gridDim.x >> 1);
  const int nk = (K + kGK - 1) / kGK;
  const int ntm = (M + 2 * kGM - 1) / (2 * kGM), ntn = (N + BN - 1) / BN, total = ntm * ntn;

  if (t == 0) {
    for (int s = 0; s < S; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * s) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * s) : "memory");
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(afull0 + 8 * b) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(aempty0 + 8 * b), "n"(2 * kGEpiWarps)
                   : "memory");   // the epilogue warps of both CTAs
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
  }
  if (warp == 1) {
    // the same columns in both CTAs' tensor memory
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(P::kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  // both CTAs' barriers initialised and tensor memory allocated before any
  // copy, MMA or arrival crosses between them
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync_all();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (t == 0) {
      // producer (both CTAs): its own rows of A and B, counted on the even
      // CTA's full barrier, which the even CTA arms with both CTAs' bytes
      const uint32_t full_l = map_to_rank(full0, 0);
      bool ok = true;
      int it = 0;
      for (int tile = pair; tile < total && ok; tile += npairs) {
        int mb, nb;
        tile_of(tile, ntm, ntn, &mb, &nb);
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const int s = it % S;
          if (it >= S && !bar_wait(empty0 + 8 * s, uint32_t((it / S - 1) & 1))) {
            ok = false;
            break;
          }
          if (rank == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full0 + 8 * s),
                         "r"(2 * P::kStageBytes)
                         : "memory");
          tma_load_2d_pair(smem_u32(sA + s * kATile), &mapA, kt * kGK, mb * 2 * kGM + int(rank) * kGM, full_l + 8 * s);
          tma_load_2d_pair(smem_u32(sB + s * P::kBTile), &mapB, kt * kGK, nb * BN + int(rank) * P::kBHalf,
                           full_l + 8 * s);
        }
      }
      if (!ok) {
        atomicExch(err, 1);
        // the copies already issued land in these CTAs' buffers: the even CTA
        // waits (bounded) for the stages in flight before the pair may end
        if (rank == 0)
          for (int j = (it > S ? it - S : 0); j < it; ++j) bar_wait(full0 + 8 * (j % S), uint32_t((j / S) & 1));
      }
    }
  } else if (warp == 1) {
    if (t == 32 && rank == 0) {
      // MMA issuer of the pair
      bool ok = true;
      int it = 0, ti = 0, committed = -1;
      for (int tile = pair; tile < total && ok; tile += npairs, ++ti) {
        const int b = ti & 1;
        if (ti >= 2 && !bar_wait_cluster(aempty0 + 8 * b, uint32_t((ti / 2 - 1) & 1))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc_tmem = tmem + P::kAccStride * uint32_t(b);
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const int s = it % S;
          if (!bar_wait(full0 + 8 * s, uint32_t((it / S) & 1))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(sA + s * kATile), b0 = smem_u32(sB + s * P::kBTile);
#pragma unroll
          for (int q = 0; q < kGK / 16; ++q) {
            const uint64_t da = smem_desc(a0 + q * 32), db = smem_desc(b0 + q * 32);
            const uint32_t accumulate = (kt > 0 || q > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc_tmem),
                "l"(da), "l"(db), "r"(mma_idesc(2 * kGM, BN)), "r"(accumulate)
                : "memory");
          }
          commit_pair(empty0 + 8 * s);
          committed = it;
        }
        if (!ok) break;
        commit_pair(afull0 + 8 * b);
      }
      if (!ok) {
        atomicExch(err, 1);
        if (committed >= 0 && !bar_wait(empty0 + 8 * (committed % S), uint32_t((committed / S) & 1)))
          atomicExch(err, 2);   // MMAs may outlive the pair's tensor memory: reported for good
      }
    }
  } else {
    // epilogue (both CTAs): this CTA's 128 rows of the pair's tile
    const int q = warp & 3, h = (warp - 2) >> 2, lane = t & 31;
    const uint32_t aempty_l = map_to_rank(aempty0, 0);
    int ti = 0;
    for (int tile = pair; tile < total; tile += npairs, ++ti) {
      const int b = ti & 1;
      int mb, nb;
      tile_of(tile, ntm, ntn, &mb, &nb);
      EpiOffsets<BN> o;
      load_offsets<BN>(o, q, h, lane, mb * 2 * kGM + int(rank) * kGM, nb * BN, M, N, rowoff, coloff);
      // (the warp leaves together: the tensor-memory loads below are
      // warp-collective)
      if (!__all_sync(0xffffffffu, bar_wait(afull0 + 8 * b, uint32_t((ti / 2) & 1)))) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      store_accumulator<BN>(tmem + P::kAccStride * uint32_t(b), o, q, h, nb * BN, N, C, alpha, beta, false);
      // this warp's reads of the accumulator are done: tell the issuer
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(aempty_l + 8 * b) : "memory");
    }
  }
  // neither CTA frees its tensor memory or leaves while the pair's MMAs,
  // copies or arrivals may still reach it
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync_all();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P::kCols) : "memory");
}

// single-CTA tiles 128 x BN (BN 256, 192 or 128): the ring takes what
// shared memory allows, the two accumulators 2 BN TMEM columns (allocated
// as the next power of two)
template <int BN>
struct SingleCfg {
  static constexpr int kBTile = BN * kGK * 2;
  static constexpr int kStages = BN == 256 ? 4 : BN == 192 ? 5 : 6;
  static constexpr uint32_t kCols = BN == 128 ? 256 : 512;
  static constexpr uint32_t kAccStride = BN == 128 ? 128 : 256;   // accumulator b at column b x this
  static constexpr int kSmem = 1024 + kStages * (kATile + kBTile) + 256;
};
static_assert(SingleCfg<256>::kSmem <= 232448 && SingleCfg<192>::kSmem <= 232448 &&
                  SingleCfg<128>::kSmem <= 232448, "shared memory");

template <int BN>
__global__ void __launch_bounds__(kGThreads, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                     float* __restrict__ C, const int64_t* __restrict__ rowoff, const int64_t* __restrict__ coloff,
                     int M, int N, int K, float alpha, float beta, int* err) {
  using P = SingleCfg<BN>;
  constexpr int kStages = P::kStages;
  constexpr int kBTile = P::kBTile;
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
  const int ntm = (M + kGM - 1) / kGM, ntn = (N + BN - 1) / BN, total = ntm * ntn;

  if (t == 0) {
    for (int s = 0; s < kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * s) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * s) : "memory");
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(afull0 + 8 * b) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(aempty0 + 8 * b), "n"(kGEpiWarps)
                   : "memory");   // the epilogue warps
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(P::kCols)
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
          tma_load_2d(smem_u32(sB + s * kBTile), &mapB, kt * kGK, nb * BN, full0 + 8 * s);
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
        const uint32_t acc_tmem = tmem + P::kAccStride * uint32_t(b);
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
                "l"(da), "l"(db), "r"(mma_idesc(kGM, BN)), "r"(accumulate)
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
        if (committed >= 0 && !bar_wait(empty0 + 8 * (committed % kStages), uint32_t((committed / kStages) & 1)))
          atomicExch(err, 2);   // MMAs may outlive the CTA's tensor memory: reported for good
      }
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (accumulator rows)
    const int q = warp & 3, h = (warp - 2) >> 2, lane = t & 31;
    int ti = 0;
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x, ++ti) {
      const int b = ti & 1;
      int mb, nb;
      tile_of(tile, ntm, ntn, &mb, &nb);
      EpiOffsets<BN> o;
      load_offsets<BN>(o, q, h, lane, mb * kGM, nb * BN, M, N, rowoff, coloff);
      // (the warp leaves together: the tensor-memory loads below are
      // warp-collective)
      if (!__all_sync(0xffffffffu, bar_wait(afull0 + 8 * b, uint32_t((ti / 2) & 1)))) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      store_accumulator<BN>(tmem + P::kAccStride * uint32_t(b), o, q, h, nb * BN, N, C, alpha, beta, K == 0);
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P::kCols) : "memory");
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
bool g_attr_set[64][7] = {};   // per device and GemmVariant
int g_pairs[64] = {};          // co-resident CTA pairs of the pair kernel (0: not yet known)

template <class F>
cudaError_t set_smem_attr(int dev, int which, F* fn, int bytes) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_attr_set[dev][which]) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    g_attr_set[dev][which] = true;
  }
  return cudaSuccess;
}

// clusters of two of the pair kernel that fit on the device at once
int pairs_on(int dev, int sms) {
  {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    if (dev >= 0 && dev < 64 && g_pairs[dev]) return g_pairs[dev];
  }
  if (set_smem_attr(dev, GEMM_PAIR_256, gemm_bf16_pair_kernel<256>, PairCfg<256>::kSmem) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(2 * (sms / 2)));
  cfg.blockDim = dim3(kGThreads);
  cfg.dynamicSmemBytes = PairCfg<256>::kSmem;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, gemm_bf16_pair_kernel<256>, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    n = 0;
  }
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (dev >= 0 && dev < 64) g_pairs[dev] = n;
  return n;
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

int tile_n_of(int v) {
  return (v == GEMM_SINGLE_192 || v == GEMM_PAIR_192) ? 192 : (v == GEMM_SINGLE_128 || v == GEMM_PAIR_128) ? 128 : 256;
}
bool is_pair(int v) { return v == GEMM_PAIR_256 || v == GEMM_PAIR_192 || v == GEMM_PAIR_128; }

template <int BN>
cudaError_t launch_single(int dev, int which, int sms, const CUtensorMap& ma, const CUtensorMap& mb, float* C,
                          const int64_t* rowoff, const int64_t* coloff, int64_t M, int64_t N, int64_t K,
                          float alpha, float beta, int* err, cudaStream_t s) {
  cudaError_t e = set_smem_attr(dev, which, gemm_bf16_kernel<BN>, SingleCfg<BN>::kSmem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = cdiv(M, kGM) * cdiv(N, BN);
  const unsigned grid = unsigned(std::min<int64_t>(tiles, sms));
  gemm_bf16_kernel<BN><<<grid, kGThreads, SingleCfg<BN>::kSmem, s>>>(ma, mb, C, rowoff, coloff, int(M), int(N),
                                                                     int(K), alpha, beta, err);
  return cudaSuccess;
}

template <int BN>
cudaError_t launch_pair(int dev, int which, int pairs, const CUtensorMap& ma, const CUtensorMap& mb, float* C,
                        const int64_t* rowoff, const int64_t* coloff, int64_t M, int64_t N, int64_t K, float alpha,
                        float beta, int* err, cudaStream_t s) {
  cudaError_t e = set_smem_attr(dev, which, gemm_bf16_pair_kernel<BN>, PairCfg<BN>::kSmem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = cdiv(M, 2 * kGM) * cdiv(N, BN);
  const unsigned grid = unsigned(2 * std::min<int64_t>(tiles, pairs));
  gemm_bf16_pair_kernel<BN><<<grid, kGThreads, PairCfg<BN>::kSmem, s>>>(ma, mb, C, rowoff, coloff, int(M), int(N),
                                                                         int(K), alpha, beta, err);
  return cudaSuccess;
}

}  // namespace

const char* gemm_bf16_check(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int64_t N, int64_t K) {
  if (M < 1 || N < 1 || K < 0) return "empty GEMM";
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return "a GEMM extent exceeds 2^31 - 1";
  if (cdiv(M, kGM) * cdiv(N, 128) > INT32_MAX) return "too many tiles";
  if (K == 0) return nullptr;   // the operands are not read
  if (lda < K || ldb < K || lda % 8 || ldb % 8) return "row pitches must be >= K and multiples of 8 elements";
  if (reinterpret_cast<uintptr_t>(A) % 16 || reinterpret_cast<uintptr_t>(B) % 16)
    return "operands must be 16-byte aligned";
  return nullptr;
}

int gemm_bf16_pick(int64_t M, int64_t N, int64_t K, int sms, int pairs) {
  if (sms < 1) return GEMM_SINGLE;
  // time ~ rounds of tiles x K x the shape's cost of one tile per unit of K,
  // plus the last tile's epilogue, which nothing hides.  Costs relative to
  // the 128 x 256 tile, measured on 2304^3 and 4096^3 GEMMs: 128 x 192 0.87,
  // 128 x 128 0.78 (the tensor cores re-read the A slice for every MMA, so
  // narrower tiles save less than their width), a pair's 256 x 256 0.95 per
  // SM, a pair's 256 x 192 0.90 (the same work per SM as 128 x 192 with a
  // third less B per SM, and no faster: the operand stream from L2 is not
  // what limits these tiles), a pair's 256 x 128 1.3; the epilogue about 500
  // units of K for 256 columns.
  const double kk = double(std::max<int64_t>(K, 1));
  int best = GEMM_SINGLE;
  double best_t = 1e300;
  const int cand[6] = {GEMM_SINGLE, GEMM_SINGLE_192, GEMM_SINGLE_128, GEMM_PAIR_256, GEMM_PAIR_192, GEMM_PAIR_128};
  const double cost[6] = {1.0, 0.87, 0.78, 0.95, 0.90, 1.3};
  for (int i = 0; i < 6; ++i) {
    const int v = cand[i];
    if (is_pair(v) && (K == 0 || pairs < 1)) continue;
    const int bn = tile_n_of(v);
    const int64_t tiles = is_pair(v) ? cdiv(M, 2 * kGM) * cdiv(N, bn) : cdiv(M, kGM) * cdiv(N, bn);
    const int64_t rounds = cdiv(tiles, is_pair(v) ? pairs : sms);
    const double t = double(rounds) * kk * cost[i] + 500.0 * bn / 256.0;
    if (t < best_t * 0.999) {
      best_t = t;
      best = v;
    }
  }
  return best;
}

cudaError_t gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, const int64_t* rowoff,
                      const int64_t* coloff, int64_t M, int64_t N, int64_t K, float alpha, float beta, int* err,
                      int variant, int* used, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int pairs = K > 0 ? pairs_on(dev, sms) : 0;
  int v = variant;
  if (v < GEMM_AUTO || v > GEMM_PAIR_192) return cudaErrorInvalidValue;
  if (v == GEMM_AUTO) v = gemm_bf16_pick(M, N, K, sms, pairs);
  if (is_pair(v) && (K == 0 || pairs < 1)) v = GEMM_SINGLE;
  if (used) *used = v;
  const int bn = tile_n_of(v);
  CUtensorMap ma, mb;
  std::memset(&ma, 0, sizeof(ma));
  std::memset(&mb, 0, sizeof(mb));
  // (K = 0: no copies are issued and the maps stay unused)
  if (K > 0 && (!make_map(&ma, static_cast<const uint16_t*>(A), K, M, lda, kGM) ||
                !make_map(&mb, static_cast<const uint16_t*>(B), K, N, ldb, is_pair(v) ? bn / 2 : bn)))
    return cudaErrorInvalidValue;
  switch (v) {
    case GEMM_SINGLE_192:
      e = launch_single<192>(dev, v, sms, ma, mb, C, rowoff, coloff, M, N, K, alpha, beta, err, s);
      break;
    case GEMM_SINGLE_128:
      e = launch_single<128>(dev, v, sms, ma, mb, C, rowoff, coloff, M, N, K, alpha, beta, err, s);
      break;
    case GEMM_PAIR_256:
      e = launch_pair<256>(dev, v, pairs, ma, mb, C, rowoff, coloff, M, N, K, alpha, beta, err, s);
      break;
    case GEMM_PAIR_192:
      e = launch_pair<192>(dev, v, pairs, ma, mb, C, rowoff, coloff, M, N, K, alpha, beta, err, s);
      break;
    case GEMM_PAIR_128:
      e = launch_pair<128>(dev, v, pairs, ma, mb, C, rowoff, coloff, M, N, K, alpha, beta, err, s);
      break;
    default:
      e = launch_single<256>(dev, v, sms, ma, mb, C, rowoff, coloff, M, N, K, alpha, beta, err, s);
  }
  if (e != cudaSuccess) return e;
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ttc
