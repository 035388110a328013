// kernels_impl.cuh -- the sm_103a kernels of one permute-scale-add (Eq. 1).
//
// Every kernel handles one unit of work per CTA (a tile, or a run chunk per
// warp) and is launched with one CTA per unit: with 256 threads and a few
// dozen registers, eight CTAs are resident per SM, each issuing all of its
// loads before any store, and the hardware scheduler starts a new CTA the
// moment one finishes.  That keeps more bytes in flight than a persistent
// loop with software pipelining does on this part (measured).
//
//  tile_kernel    -- generic tile staged in shared memory (the paper's
//                    macro-tile, section 2.2, Fig. 4): threads walk the tile
//                    in A order to load and in B order to store.
//  tile2_kernel   -- the same tile with a 2D lane layout: lanes run along
//                    A's (load) and B's (store) stride-1 runs, warps along the
//                    rows; row offsets are computed once per row.
//  rowcopy_kernel -- perm keeps index 0 with short runs (section 3.2): blocks
//                    of consecutive runs, contiguous in A, copied directly.
//  copy_kernel    -- perm keeps index 0 with long runs: one warp per run chunk,
//                    128-bit accesses when aligned.
//  amax_kernel    -- FP8 output without a caller scale: max |alpha*a| pre-pass.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>

#include "kernels.cuh"
#include "launch.h"

namespace ttc {

extern std::atomic<int64_t> g_launches;
cudaError_t grid_for(const void* fn, int smem, int64_t work, int* grid);

template <int EK>
__device__ __forceinline__ float cta_fp8_scale(const Epilogue& e) {
  if constexpr (EK == EK_FP8) {
    const float s = fp8_scale_of(e);
    if (blockIdx.x == 0 && threadIdx.x == 0 && e.scale_out) *e.scale_out = s;
    return s;
  } else {
    return 1.f;
  }
}

// The coordinate of this CTA's tile: thread 0 decomposes the tile index (a
// loop over the grid indices with indexed parameter loads) and shares it.
__device__ __forceinline__ TileCoord cta_tile_coord(const TileParams& p) {
  __shared__ TileCoord sc;
  if (threadIdx.x == 0) sc = tile_coord(blockIdx.x, p);
  __syncthreads();
  return sc;
}

// ------------------------------------------------------------- generic tile --

template <int DIN, int DOUT, int EK, bool TA, bool TB>
__device__ __forceinline__ void tile_body(const store_t<DIN>* __restrict__ Ab, store_t<DOUT>* __restrict__ Bb,
                                          const TileParams& p, const TileCoord& c, stage_t<DIN>* tile, float scale) {
  using S = stage_t<DIN>;
  using TO = store_t<DOUT>;
  constexpr int K = tile_k_for(sizeof(S));
  int u0, lb0, lc0, lbw0, la0;
  flat_starts(p, threadIdx.x, u0, lb0, lc0, lbw0, la0);
  S v[K];
  // offset 0 (the tile's first element, which always exists) stands in for holes
  walk_read<K, TA>(c, p, p.tabA, u0, lb0,
                   [&](int k, bool, int32_t off, int) { v[k] = to_stage<DIN>(ldg_elem<DIN>(Ab + off)); });
  walk_read<K, TA>(c, p, p.tabA, u0, lb0, [&](int k, bool ok, int32_t, int pos) {
    if (ok) tile[pos] = v[k];
  });
  __syncthreads();
  TO bo[K] = {};
  if constexpr (EK == EK_AXPBY)
    walk_write<K, TB>(c, p, p.tabB, lc0, lbw0, la0, [&](int k, bool, int32_t off, int) { bo[k] = Bb[off]; });
  walk_write<K, TB>(c, p, p.tabB, lc0, lbw0, la0, [&](int k, bool ok, int32_t off, int pos) {
    if (ok) Bb[off] = epilogue_k<DIN, DOUT, EK>(tile[pos], bo[k], p.epi, scale);
  });
}

template <int DIN, int DOUT, int EK>
__global__ void __launch_bounds__(kThreads, 4) tile_kernel(const store_t<DIN>* __restrict__ A,
                                                           store_t<DOUT>* __restrict__ B,
                                                           const __grid_constant__ TileParams p) {
  using S = stage_t<DIN>;
  extern __shared__ __align__(16) unsigned char smem[];
  S* tile = reinterpret_cast<S*>(smem);
  const float scale = cta_fp8_scale<EK>(p.epi);
  const TileCoord c = cta_tile_coord(p);
  const store_t<DIN>* Ab = A + c.baseA;
  store_t<DOUT>* Bb = B + c.baseB;
  if (p.crossA_tab) {
    if (p.crossB_tab) tile_body<DIN, DOUT, EK, true, true>(Ab, Bb, p, c, tile, scale);
    else tile_body<DIN, DOUT, EK, true, false>(Ab, Bb, p, c, tile, scale);
  } else {
    if (p.crossB_tab) tile_body<DIN, DOUT, EK, false, true>(Ab, Bb, p, c, tile, scale);
    else tile_body<DIN, DOUT, EK, false, false>(Ab, Bb, p, c, tile, scale);
  }
}

// ------------------------------------------------------ slot-table tile --
//
// The same tiles as tile_kernel, driven by the plan's slot tables
// (TileParams::slots): for every (k, thread) slot of the load order and of
// the store order, the element's offset in the tile and its shared-memory
// position, two slots per 16-byte table read; the slots visit the tile's
// elements in increasing A offset (loads) and increasing B offset (stores),
// so both sides coalesce whatever the tile's index structure.  A tile cut
// short by the tensor's edge reads each slot's (la, lb) coordinate from a
// second table and masks the slots outside the tile.  The loops carry no
// index arithmetic; the tables are shared by every CTA through L1.

template <int DIN, int DOUT, int EK, bool FULL>
__device__ __forceinline__ void slots_body(const store_t<DIN>* __restrict__ Ab, store_t<DOUT>* __restrict__ Bb,
                                           const TileParams& p, const TileCoord& c, stage_t<DIN>* tile,
                                           float scale) {
  using S = stage_t<DIN>;
  using TO = store_t<DOUT>;
  constexpr int K = tile_k_for(sizeof(S));
  constexpr int Q = K / 4;                      // groups of four slots per thread
  const int t = threadIdx.x;
  // table regions (TileParams::slots): offsets, tile coordinates, positions
  const int4* __restrict__ offs = p.slots + t;
  const uint4* __restrict__ crd = reinterpret_cast<const uint4*>(p.slots + 2 * Q * kThreads) + t;
  const uint2* __restrict__ poss = reinterpret_cast<const uint2*>(p.slots + 4 * Q * kThreads) + t;
  // slot k of this thread holds an element of this tile iff bit k is set
  auto inside = [&](int phase) -> uint32_t {
    if constexpr (FULL) {
      return 0xffffffffu;
    } else {
      uint32_t m = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const uint4 e = __ldg(crd + (phase * Q + q) * kThreads);
        m |= uint32_t((int(e.x >> 16) < c.remA) & (int(e.x & 0xffffu) < c.remB)) << (4 * q);
        m |= uint32_t((int(e.y >> 16) < c.remA) & (int(e.y & 0xffffu) < c.remB)) << (4 * q + 1);
        m |= uint32_t((int(e.z >> 16) < c.remA) & (int(e.z & 0xffffu) < c.remB)) << (4 * q + 2);
        m |= uint32_t((int(e.w >> 16) < c.remA) & (int(e.w & 0xffffu) < c.remB)) << (4 * q + 3);
      }
      return m;
    }
  };
  // position of slot j (0..3) of a packed group; 0xffff marks an empty slot
  auto slot_pos = [](uint2 pp, int j) -> int {
    const uint32_t w = j < 2 ? pp.x : pp.y;
    return int((w >> (16 * (j & 1))) & 0xffffu);
  };
  // ---- load A in address order, stage in shared memory
  {
    const uint32_t m = inside(0);
    S v[K];
    uint2 pk[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int4 o = __ldg(offs + q * kThreads);
      pk[q] = __ldg(poss + q * kThreads);
      const int32_t oo[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bool in = FULL || ((m >> (4 * q + j)) & 1u);
        v[4 * q + j] = to_stage<DIN>(ldg_elem<DIN>(Ab + (in ? oo[j] : 0)));
      }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int pos = slot_pos(pk[q], j);
        const bool in = FULL || ((m >> (4 * q + j)) & 1u);
        if (in && pos != 0xffff) tile[pos] = v[4 * q + j];
      }
  }
  __syncthreads();
  // ---- store B in address order
  const uint32_t m = inside(1);
  if constexpr (EK == EK_AXPBY) {
    int32_t off[K];
    uint2 pk[Q];
    TO bo[K];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int4 o = __ldg(offs + (Q + q) * kThreads);
      pk[q] = __ldg(poss + (Q + q) * kThreads);
      const int32_t oo[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bool in = FULL || ((m >> (4 * q + j)) & 1u);
        off[4 * q + j] = in ? oo[j] : 0;
        bo[4 * q + j] = Bb[off[4 * q + j]];
      }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int pos = slot_pos(pk[q], j);
        const bool in = FULL || ((m >> (4 * q + j)) & 1u);
        if (in && pos != 0xffff)
          Bb[off[4 * q + j]] = epilogue_k<DIN, DOUT, EK>(tile[pos], bo[4 * q + j], p.epi, scale);
      }
  } else {
    // no loads of B: each group's stores go out as soon as its table entry
    // is in, keeping few registers live
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int4 o = __ldg(offs + (Q + q) * kThreads);
      const uint2 pp = __ldg(poss + (Q + q) * kThreads);
      const int32_t oo[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int pos = slot_pos(pp, j);
        const bool in = FULL || ((m >> (4 * q + j)) & 1u);
        if (in && pos != 0xffff) Bb[oo[j]] = epilogue_k<DIN, DOUT, EK>(tile[pos], TO{}, p.epi, scale);
      }
    }
  }
}

template <int DIN, int DOUT, int EK>
__global__ void __launch_bounds__(kThreads, sizeof(stage_t<DIN>) == 4 ? (EK == EK_AXPBY ? 4 : 5) : (EK == EK_AXPBY ? 5 : 8)) tile_slots_kernel(const store_t<DIN>* __restrict__ A,
                                                                 store_t<DOUT>* __restrict__ B,
                                                                 const __grid_constant__ TileParams p) {
  using S = stage_t<DIN>;
  extern __shared__ __align__(16) unsigned char smem[];
  S* tile = reinterpret_cast<S*>(smem);
  const float scale = cta_fp8_scale<EK>(p.epi);
  const TileCoord c = cta_tile_coord(p);
  const store_t<DIN>* Ab = A + c.baseA;
  store_t<DOUT>* Bb = B + c.baseB;
  if (c.remA == p.LA && c.remB == p.LB) slots_body<DIN, DOUT, EK, true>(Ab, Bb, p, c, tile, scale);
  else slots_body<DIN, DOUT, EK, false>(Ab, Bb, p, c, tile, scale);
}

// --------------------------------------------------------- warp-mapped tile --
//
// Constraints (the planner checks them): U <= 32*JU, LB <= 8*K/JU,
// W <= 32*JW, LA <= 8*K/JW.

template <int DIN, int DOUT, int JU, int JW, int EK, bool FULL, bool TA, bool TB>
__device__ __forceinline__ void tile2_body(const store_t<DIN>* __restrict__ Ab, store_t<DOUT>* __restrict__ Bb,
                                           const TileParams& p, const TileCoord& c, stage_t<DIN>* tile,
                                           float scale) {
  using S = stage_t<DIN>;
  using TO = store_t<DOUT>;
  constexpr int K = tile_k_for(sizeof(S));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // every access is predicated on the walk's ok (no branches); the staged
  // value of a lane with no element is read from position 0 and not stored
  S v[K];
  walk2_read<JU, K, FULL, TA, true>(c, p, p.tabA, lane, warp, [&](int k, bool ok, int32_t off, int) {
    if (ok) v[k] = to_stage<DIN>(ldg_elem<DIN>(Ab + off));
  });
  walk2_read<JU, K, FULL, TA, true>(c, p, p.tabA, lane, warp, [&](int k, bool ok, int32_t, int pos) {
    if (ok) tile[pos] = v[k];
  });
  __syncthreads();
  int spre[JW];
  walk2_lane_consts<JW>(p, lane, spre);
  TO bo[K] = {};
  if constexpr (ek_reads_b(EK))
    walk2_write<JW, K, FULL, TB, true>(c, p, p.tabB, lane, warp, spre, [&](int k, bool ok, int32_t off, int) {
      if (ok) bo[k] = Bb[off];
    });
  walk2_write<JW, K, FULL, TB, true>(c, p, p.tabB, lane, warp, spre, [&](int k, bool ok, int32_t off, int pos) {
    const TO y = epilogue_k<DIN, DOUT, EK>(tile[ok ? pos : 0], bo[k], p.epi, scale);
    if (ok) Bb[off] = y;
  });
}

template <int DIN, int DOUT, int JU, int JW, int EK, bool FULL>
__device__ __forceinline__ void tile2_tabs(const store_t<DIN>* __restrict__ Ab, store_t<DOUT>* __restrict__ Bb,
                                           const TileParams& p, const TileCoord& c, stage_t<DIN>* tile,
                                           float scale) {
  if (p.crossA_tab) {
    if (p.crossB_tab) tile2_body<DIN, DOUT, JU, JW, EK, FULL, true, true>(Ab, Bb, p, c, tile, scale);
    else tile2_body<DIN, DOUT, JU, JW, EK, FULL, true, false>(Ab, Bb, p, c, tile, scale);
  } else {
    if (p.crossB_tab) tile2_body<DIN, DOUT, JU, JW, EK, FULL, false, true>(Ab, Bb, p, c, tile, scale);
    else tile2_body<DIN, DOUT, JU, JW, EK, FULL, false, false>(Ab, Bb, p, c, tile, scale);
  }
}

template <int DIN, int DOUT, int JU, int JW, int EK>
__global__ void __launch_bounds__(kThreads, EK == EK_AXPBY && JW == 4 ? 6 : 8) tile2_kernel(const store_t<DIN>* __restrict__ A,
                                                            store_t<DOUT>* __restrict__ B,
                                                            const __grid_constant__ TileParams p) {
  using S = stage_t<DIN>;
  extern __shared__ __align__(16) unsigned char smem[];
  S* tile = reinterpret_cast<S*>(smem);
  const float scale = cta_fp8_scale<EK>(p.epi);
  const TileCoord c = cta_tile_coord(p);
  const store_t<DIN>* Ab = A + c.baseA;
  store_t<DOUT>* Bb = B + c.baseB;
  if (c.remA == p.LA && c.remB == p.LB) tile2_tabs<DIN, DOUT, JU, JW, EK, true>(Ab, Bb, p, c, tile, scale);
  else tile2_tabs<DIN, DOUT, JU, JW, EK, false>(Ab, Bb, p, c, tile, scale);
}

// --------------------------------------------------------- packed-lane tile --
//
// Tiles without a C index of any extents up to 256 x K elements: the lanes of
// a warp are packed over the rows of each side (walkp_read / walkp_write), so
// runs of any length, and the short runs of the tiles at the tensor's edge,
// keep almost every lane busy, at about the per-element cost of the
// warp-mapped walk.


template <int DIN, int DOUT, int JU, int JW, int EK, bool TA, bool TB, int K = tile_k_for(sizeof(stage_t<DIN>))>
__device__ __forceinline__ void tilep_body(const store_t<DIN>* __restrict__ Ab, store_t<DOUT>* __restrict__ Bb,
                                           const TileParams& p, const TileCoord& c, stage_t<DIN>* tile,
                                           float scale) {
  using S = stage_t<DIN>;
  using TO = store_t<DOUT>;
  const int t = threadIdx.x;
  // accesses predicated on the walk's ok, as in tile2_body
  S v[K];
  walkp_read<0, JU, K, TA, true>(c, p, p.tabA, t, [&](int k, bool ok, int32_t off, int) {
    if (ok) v[k] = to_stage<DIN>(ldg_elem<DIN>(Ab + off));
  });
  walkp_read<0, JU, K, TA, true>(c, p, p.tabA, t, [&](int k, bool ok, int32_t, int pos) {
    if (ok) tile[pos] = v[k];
  });
  __syncthreads();
  TO bo[K] = {};
  if constexpr (ek_reads_b(EK))
    walkp_write<0, JW, K, TB, true>(c, p, p.tabB, t, [&](int k, bool ok, int32_t off, int) {
      if (ok) bo[k] = Bb[off];
    });
  walkp_write<0, JW, K, TB, true>(c, p, p.tabB, t, [&](int k, bool ok, int32_t off, int pos) {
    const TO y = epilogue_k<DIN, DOUT, EK>(tile[ok ? pos : 0], bo[k], p.epi, scale);
    if (ok) Bb[off] = y;
  });
}

// the packed-lane tile with its cross-offset kinds (linear or table) resolved
template <int DIN, int DOUT, int JU, int JW, int EK, int KS = tile_k_for(sizeof(stage_t<DIN>))>
__device__ __forceinline__ void tilep_tile(const store_t<DIN>* __restrict__ Ab, store_t<DOUT>* __restrict__ Bb,
                                           const TileParams& p, const TileCoord& c, stage_t<DIN>* tile,
                                           float scale) {
  if (p.crossA_tab) {
    if (p.crossB_tab) tilep_body<DIN, DOUT, JU, JW, EK, true, true, KS>(Ab, Bb, p, c, tile, scale);
    else tilep_body<DIN, DOUT, JU, JW, EK, true, false, KS>(Ab, Bb, p, c, tile, scale);
  } else {
    if (p.crossB_tab) tilep_body<DIN, DOUT, JU, JW, EK, false, true, KS>(Ab, Bb, p, c, tile, scale);
    else tilep_body<DIN, DOUT, JU, JW, EK, false, false, KS>(Ab, Bb, p, c, tile, scale);
  }
}

template <int DIN, int DOUT, int JU, int JW, int EK>
__global__ void __launch_bounds__(kThreads, EK == EK_AXPBY ? 5 : JU == 1 ? 5 : 8) tilep_kernel(
    const store_t<DIN>* __restrict__ A, store_t<DOUT>* __restrict__ B, const __grid_constant__ TileParams p) {
  using S = stage_t<DIN>;
  extern __shared__ __align__(16) unsigned char smem[];
  S* tile = reinterpret_cast<S*>(smem);
  const float scale = cta_fp8_scale<EK>(p.epi);
  const TileCoord c = cta_tile_coord(p);
  tilep_tile<DIN, DOUT, JU, JW, EK>(A + c.baseA, B + c.baseB, p, c, tile, scale);
}

// ------------------------------------------------------------- packed rows --
//
// Tiles with a C index (perm keeps index 0) whose rows are contiguous on
// both sides: each row goes from A to B directly (walk_rowsp), the lanes of a
// warp packed over the rows, so rows of any length keep almost every lane
// busy and no shared memory is needed.

template <int DIN, int DOUT, int J, int EK, bool TA, bool TB, int K>
__device__ __forceinline__ void rowsp_body(const store_t<DIN>* __restrict__ Ab, store_t<DOUT>* __restrict__ Bb,
                                           const TileParams& p, const TileCoord& c, float scale) {
  using S = stage_t<DIN>;
  using TO = store_t<DOUT>;
  const int t = threadIdx.x;
  S v[K];
  TO bo[K] = {};
  int32_t ob[K];     // B offsets of one walk (-1: no element), kept for the stores
  walk_rowsp<J, K, TA, TB>(c, p, p.tabA, p.tabB, t, [&](int k, bool ok, int32_t offA, int32_t offB) {
    v[k] = to_stage<DIN>(ldg_elem<DIN>(Ab + offA));
    if constexpr (ek_reads_b(EK)) bo[k] = Bb[offB];
    ob[k] = ok ? offB : -1;
  });
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (ob[k] >= 0) Bb[ob[k]] = epilogue_k<DIN, DOUT, EK>(v[k], bo[k], p.epi, scale);
}

// the packed rows of one tile with the cross-offset kinds resolved
template <int DIN, int DOUT, int J, int EK, int K = tile_k_for(sizeof(stage_t<DIN>))>
__device__ __forceinline__ void rowsp_tile(const store_t<DIN>* __restrict__ Ab, store_t<DOUT>* __restrict__ Bb,
                                           const TileParams& p, const TileCoord& c, float scale) {
  if (p.crossA_tab) {
    if (p.crossB_tab) rowsp_body<DIN, DOUT, J, EK, true, true, K>(Ab, Bb, p, c, scale);
    else rowsp_body<DIN, DOUT, J, EK, true, false, K>(Ab, Bb, p, c, scale);
  } else {
    if (p.crossB_tab) rowsp_body<DIN, DOUT, J, EK, false, true, K>(Ab, Bb, p, c, scale);
    else rowsp_body<DIN, DOUT, J, EK, false, false, K>(Ab, Bb, p, c, scale);
  }
}

template <int DIN, int DOUT, int J, int EK>
__global__ void __launch_bounds__(kThreads, sizeof(stage_t<DIN>) == 4 ? (EK == EK_AXPBY ? 3 : 4) : (EK == EK_AXPBY ? 5 : 6)) rowsp_kernel(
    const store_t<DIN>* __restrict__ A, store_t<DOUT>* __restrict__ B, const __grid_constant__ TileParams p) {
  const float scale = cta_fp8_scale<EK>(p.epi);
  const TileCoord c = cta_tile_coord(p);
  rowsp_tile<DIN, DOUT, J, EK>(A + c.baseA, B + c.baseB, p, c, scale);
}

// ------------------------------------------------------------ multi-row copy --
//
// perm keeps index 0 and its runs are short: a tile is LC x LA (LC the shared
// stride-1 index, LA consecutive indices of A's next index, dense in A), so
// the tile is one contiguous block of A; each thread issues its K loads, then
// writes each run of LC elements to its B row directly.
template <int DIN, int DOUT, int EK>
__global__ void __launch_bounds__(kThreads) rowcopy_kernel(const store_t<DIN>* __restrict__ A,
                                                           store_t<DOUT>* __restrict__ B,
                                                           const __grid_constant__ TileParams p) {
  using S = stage_t<DIN>;
  using TO = store_t<DOUT>;
  constexpr int K = tile_k_for(sizeof(S));
  const int t = threadIdx.x;
  const float scale = cta_fp8_scale<EK>(p.epi);
  const TileCoord c = cta_tile_coord(p);
  const store_t<DIN>* Ab = A + c.baseA;
  TO* Bb = B + c.baseB;
  S v[K];
  TO bo[K] = {};
  walk_rows<K>(c, p, t, [&](int k, bool, int32_t offA, int32_t offB) {
    v[k] = to_stage<DIN>(ldg_elem<DIN>(Ab + offA));
    if constexpr (EK == EK_AXPBY) bo[k] = Bb[offB];
  });
  walk_rows<K>(c, p, t, [&](int k, bool ok, int32_t, int32_t offB) {
    if (ok) Bb[offB] = epilogue_k<DIN, DOUT, EK>(v[k], bo[k], p.epi, scale);
  });
}

// ---------------------------------------------------------------- copy ----

constexpr int kCopyUnroll = 8;

// One warp per (run, chunk) work item; 8 items per CTA.
template <int DIN, int DOUT, int VEC, int EK>
__global__ void __launch_bounds__(kThreads) copy_kernel(const store_t<DIN>* __restrict__ A,
                                                        store_t<DOUT>* __restrict__ B,
                                                        const __grid_constant__ RowParams p) {
  using TI = store_t<DIN>;
  using TO = store_t<DOUT>;
  const int lane = threadIdx.x & 31;
  const float scale = cta_fp8_scale<EK>(p.epi);
  const uint32_t item = (blockIdx.x * kThreads + threadIdx.x) >> 5;
  if (item >= p.nitems) return;
  const RowCoord rc = row_coord(item, p);
  if constexpr (VEC == 1) {
    const TI* Ar = A + rc.offA;
    TO* Br = B + rc.offB;
    for (int64_t x0 = rc.start + lane; x0 < rc.end; x0 += 32 * kCopyUnroll) {
      stage_t<DIN> a[kCopyUnroll];
      TO b[kCopyUnroll];
#pragma unroll
      for (int j = 0; j < kCopyUnroll; ++j) {
        const int64_t x = x0 + 32 * j;
        if (x < rc.end) {
          a[j] = to_stage<DIN>(ldg_elem<DIN>(Ar + x * p.sa0));
          if constexpr (EK == EK_AXPBY) b[j] = Br[x * p.sb0];
        }
      }
#pragma unroll
      for (int j = 0; j < kCopyUnroll; ++j) {
        const int64_t x = x0 + 32 * j;
        if (x < rc.end) Br[x * p.sb0] = epilogue_k<DIN, DOUT, EK>(a[j], b[j], p.epi, scale);
      }
    }
  } else {
    // unit strides; run length, chunk and every run offset are multiples of
    // VEC and the bases are aligned (checked by the planner and at launch)
    using VI = VecT<TI, VEC>;
    using VO = VecT<TO, VEC>;
    const VI* Av = reinterpret_cast<const VI*>(A + rc.offA);
    VO* Bv = reinterpret_cast<VO*>(B + rc.offB);
    const int64_t vs = rc.start / VEC, ve = rc.end / VEC;
    for (int64_t x0 = vs + lane; x0 < ve; x0 += 32 * kCopyUnroll) {
      VI a[kCopyUnroll];
      VO b[kCopyUnroll];
#pragma unroll
      for (int j = 0; j < kCopyUnroll; ++j) {
        const int64_t x = x0 + 32 * j;
        if (x < ve) {
          a[j] = Av[x];
          if constexpr (EK == EK_AXPBY) b[j] = Bv[x];
        }
      }
#pragma unroll
      for (int j = 0; j < kCopyUnroll; ++j) {
        const int64_t x = x0 + 32 * j;
        if (x < ve) {
          VO o;
#pragma unroll
          for (int e = 0; e < VEC; ++e)
            o.v[e] = epilogue_k<DIN, DOUT, EK>(to_stage<DIN>(a[j].v[e]), b[j].v[e], p.epi, scale);
          Bv[x] = o;
        }
      }
    }
  }
}

// ---------------------------------------------------------------- amax ----

// A warp takes kAmaxItems groups of consecutive row chunks of A's
// sub-tensor at a time (their coordinates decomposed once per chunk, not per
// element; a group is 32 / L chunks for chunks that L < 32 lanes cover) and
// keeps kAmaxItems x kAmaxUnroll loads per lane in flight, so that short rows
// (a packing panel's 48- or 256-element columns) still stream.  One CTA also
// clears `clear_bits`, the word the next execution of the plan accumulates
// into, so no separate reset is launched (two words alternate per plan).
constexpr int kAmaxItems = 4;
constexpr int kAmaxUnroll = 2;

// lanes of a warp per chunk of `chunk` elements read V at a time: the least
// power of two that covers its loads, at most 32
TTC_HD int amax_lanes_per_item(int64_t chunk, int V) {
  const int64_t loads = (chunk + V - 1) / V;
  int L = 32;
  while (L > 1 && L / 2 >= loads) L >>= 1;
  return L;
}

// V > 1: every chunk starts and ends on a 16-byte boundary (RowParams::vec)
// and a lane loads V consecutive elements at a time.
template <int DIN, int V>
__device__ __forceinline__ void amax_load(const store_t<DIN>* __restrict__ A, int64_t i, float alpha_f, float (&v)[V]) {
  if constexpr (V == 1) {
    v[0] = fabsf(__fmul_rn(alpha_f, float(to_stage<DIN>(ldg_elem<DIN>(A + i)))));
  } else {
    static_assert(V * sizeof(store_t<DIN>) == 16, "16-byte loads");
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(A + i));
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < V; ++k) {
      store_t<DIN> x;
      if constexpr (V == 4)
        x = __uint_as_float(u[k]);
      else
        x = store_t<DIN>(uint16_t(u[k / 2] >> (16 * (k & 1))));
      v[k] = fabsf(__fmul_rn(alpha_f, float(to_stage<DIN>(x))));
    }
  }
}

template <int DIN, int V>
__global__ void __launch_bounds__(kThreads) amax_kernel(const store_t<DIN>* __restrict__ A,
                                                        const __grid_constant__ RowParams p, float alpha_f,
                                                        uint32_t* amax_bits, uint32_t* clear_bits) {
  const int t = threadIdx.x, lane = t & 31;
  if (blockIdx.x == 0 && t == 0 && clear_bits) *clear_bits = 0u;
  const uint32_t warp = (blockIdx.x * kThreads + t) >> 5;
  const uint32_t nwarps = (gridDim.x * kThreads) >> 5;
  // short chunks share a warp: L lanes per chunk (a power of two covering
  // its vectors), 32 / L chunks side by side
  const int L = amax_lanes_per_item(p.chunk, V);
  const int per = 32 / L, sub = lane / L, li = lane % L;
  const uint64_t step = uint64_t(kAmaxItems) * per;
  float m = 0.f;
  for (uint64_t i0 = uint64_t(warp) * step; i0 < p.nitems; i0 += uint64_t(nwarps) * step) {
    RowCoord rc[kAmaxItems];
#pragma unroll
    for (int j = 0; j < kAmaxItems; ++j) {
      const uint64_t it = i0 + uint64_t(j) * per + sub;
      rc[j] = row_coord(uint32_t(it < p.nitems ? it : i0), p);
      if (it >= p.nitems) rc[j].end = rc[j].start;     // no such chunk
    }
    for (int64_t x0 = int64_t(li) * V; x0 < p.chunk; x0 += int64_t(L) * kAmaxUnroll * V) {
      float v[kAmaxItems][kAmaxUnroll][V];
      bool ok[kAmaxItems][kAmaxUnroll];
#pragma unroll
      for (int j = 0; j < kAmaxItems; ++j)
#pragma unroll
        for (int u = 0; u < kAmaxUnroll; ++u) {
          const int64_t x = rc[j].start + x0 + int64_t(L) * V * u;
          ok[j][u] = x < rc[j].end;     // (V > 1: whole vectors only)
          amax_load<DIN, V>(A, ok[j][u] ? rc[j].offA + x * p.sa0 : int64_t(0), alpha_f, v[j][u]);
        }
#pragma unroll
      for (int j = 0; j < kAmaxItems; ++j)
#pragma unroll
        for (int u = 0; u < kAmaxUnroll; ++u)
#pragma unroll
          for (int k = 0; k < V; ++k)
            if (ok[j][u] && v[j][u][k] > m) m = v[j][u][k];     // NaN compares false: ignored
    }
  }
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float red[kThreads / 32];
  if (lane == 0) red[t >> 5] = m;
  __syncthreads();
  if (t == 0) {
    float b = 0.f;
    for (int i = 0; i < kThreads / 32; ++i) b = fmaxf(b, red[i]);
    if (b > 0.f) atomicMax(amax_bits, __float_as_uint(b));
  }
}

// ------------------------------------------------------------ launch templates --

// epilogue kind of a plan: compile-time dispatch of the update of Eq. 1
template <int DIN, int DOUT, template <int> class L, class... Args>
cudaError_t with_ek(int mode, int beta_nz, Args&&... args) {
  if constexpr (DOUT == DT_E4M3) {
    return L<EK_FP8>::run(args...);
  } else {
    if (beta_nz) return L<EK_AXPBY>::run(args...);
    if constexpr (DIN == DOUT)
      if (mode == MODE_BITCOPY) return L<EK_COPY>::run(args...);
    return L<EK_SCALE>::run(args...);
  }
}

template <int DIN, int DOUT>
struct TileL {
  template <int EK>
  struct L {
    static cudaError_t run(const void* A, void* B, const TileParams& p, int smem, cudaStream_t s) {
      if (smem > 48 * 1024) {
        int g = 0;
        cudaError_t err = grid_for(reinterpret_cast<const void*>(&tile_kernel<DIN, DOUT, EK>), smem, 1, &g);
        if (err != cudaSuccess) return err;
      }
      tile_kernel<DIN, DOUT, EK><<<p.ntiles, kThreads, smem, s>>>(static_cast<const store_t<DIN>*>(A),
                                                                  static_cast<store_t<DOUT>*>(B), p);
      ++g_launches;
      return cudaGetLastError();
    }
  };
};

template <int DIN, int DOUT>
struct TileSlotsL {
  template <int EK>
  struct L {
    static cudaError_t run(const void* A, void* B, const TileParams& p, int smem, cudaStream_t s) {
      if (smem > 48 * 1024) {
        int g = 0;
        cudaError_t err = grid_for(reinterpret_cast<const void*>(&tile_slots_kernel<DIN, DOUT, EK>), smem, 1, &g);
        if (err != cudaSuccess) return err;
      }
      tile_slots_kernel<DIN, DOUT, EK><<<p.ntiles, kThreads, smem, s>>>(static_cast<const store_t<DIN>*>(A),
                                                                        static_cast<store_t<DOUT>*>(B), p);
      ++g_launches;
      return cudaGetLastError();
    }
  };
};

template <int DIN, int DOUT, int JU, int JW>
struct Tile2L {
  template <int EK>
  struct L {
    static cudaError_t run(const void* A, void* B, const TileParams& p, int smem, cudaStream_t s) {
      if (smem > 48 * 1024) {
        int g = 0;
        cudaError_t err = grid_for(reinterpret_cast<const void*>(&tile2_kernel<DIN, DOUT, JU, JW, EK>), smem, 1, &g);
        if (err != cudaSuccess) return err;
      }
      tile2_kernel<DIN, DOUT, JU, JW, EK><<<p.ntiles, kThreads, smem, s>>>(static_cast<const store_t<DIN>*>(A),
                                                                           static_cast<store_t<DOUT>*>(B), p);
      ++g_launches;
      return cudaGetLastError();
    }
  };
};

template <int DIN, int DOUT, int JU, int JW>
struct TilepL {
  template <int EK>
  struct L {
    static cudaError_t run(int nt, const void* A, void* B, const TileParams& p, int smem, cudaStream_t s) {
      if (smem > 48 * 1024) {
        int g = 0;
        cudaError_t err = grid_for(reinterpret_cast<const void*>(&tilep_kernel<DIN, DOUT, JU, JW, EK>), smem, 1, &g);
        if (err != cudaSuccess) return err;
      }
      tilep_kernel<DIN, DOUT, JU, JW, EK><<<p.ntiles, nt, smem, s>>>(static_cast<const store_t<DIN>*>(A),
                                                                     static_cast<store_t<DOUT>*>(B), p);
      ++g_launches;
      return cudaGetLastError();
    }
  };
};

template <int DIN, int DOUT, int J>
struct RowspL {
  template <int EK>
  struct L {
    static cudaError_t run(const void* A, void* B, const TileParams& p, cudaStream_t s) {
      rowsp_kernel<DIN, DOUT, J, EK><<<p.ntiles, kThreads, 0, s>>>(static_cast<const store_t<DIN>*>(A),
                                                                   static_cast<store_t<DOUT>*>(B), p);
      ++g_launches;
      return cudaGetLastError();
    }
  };
};

template <int DIN, int DOUT>
struct RowcopyL {
  template <int EK>
  struct L {
    static cudaError_t run(const void* A, void* B, const TileParams& p, cudaStream_t s) {
      rowcopy_kernel<DIN, DOUT, EK><<<p.ntiles, kThreads, 0, s>>>(static_cast<const store_t<DIN>*>(A),
                                                                  static_cast<store_t<DOUT>*>(B), p);
      ++g_launches;
      return cudaGetLastError();
    }
  };
};

template <int DIN, int DOUT, int VEC>
struct CopyL {
  template <int EK>
  struct L {
    static cudaError_t run(const void* A, void* B, const RowParams& p, cudaStream_t s) {
      const int64_t blocks = (int64_t(p.nitems) + kThreads / 32 - 1) / (kThreads / 32);
      copy_kernel<DIN, DOUT, VEC, EK><<<unsigned(blocks), kThreads, 0, s>>>(static_cast<const store_t<DIN>*>(A),
                                                                            static_cast<store_t<DOUT>*>(B), p);
      ++g_launches;
      return cudaGetLastError();
    }
  };
};

template <int DIN, int DOUT>
cudaError_t launch_tile2_pair(int ju, int jw, const void* A, void* B, const TileParams& p, int smem,
                              cudaStream_t s) {
#define J(U_, W_)                                                                                          \
  if (ju == U_ && jw == W_)                                                                                \
    return with_ek<DIN, DOUT, Tile2L<DIN, DOUT, U_, W_>::template L>(p.epi.mode, p.epi.beta_nz, A, B, p, smem, s);
  J(1, 1) J(1, 2) J(1, 4) J(2, 1) J(2, 2) J(2, 4) J(4, 1) J(4, 2) J(4, 4)
#undef J
  return cudaErrorInvalidValue;
}

template <int DIN, int DOUT>
cudaError_t launch_tilep_pair(int nt, int ju, int jw, const void* A, void* B, const TileParams& p, int smem,
                              cudaStream_t s) {
  if (nt != kThreads) return cudaErrorInvalidValue;
#define J(U_, W_)                                                                                           \
  if (ju == U_ && jw == W_)                                                                                 \
    return with_ek<DIN, DOUT, TilepL<DIN, DOUT, U_, W_>::template L>(p.epi.mode, p.epi.beta_nz, nt, A, B, p, smem, s);
  J(1, 1) J(1, 2) J(1, 4) J(2, 1) J(2, 2) J(2, 4) J(4, 1) J(4, 2) J(4, 4)
#undef J
  return cudaErrorInvalidValue;
}

template <int DIN, int DOUT>
cudaError_t launch_rowsp_pair(int j, const void* A, void* B, const TileParams& p, cudaStream_t s) {
  constexpr int K = tile_k_for(sizeof(stage_t<DIN>));
#define J_(J) \
  if constexpr (J <= K)     \
    if (j == J) return with_ek<DIN, DOUT, RowspL<DIN, DOUT, J>::template L>(p.epi.mode, p.epi.beta_nz, A, B, p, s);
  J_(1) J_(2) J_(4) J_(8) J_(16)
#undef J_
  return cudaErrorInvalidValue;
}

template <int DIN, int V>
cudaError_t launch_amax_v(const void* A, const RowParams& p, float alpha_f, uint32_t* amax_bits,
                          uint32_t* clear_bits, cudaStream_t s) {
  const void* fn = reinterpret_cast<const void*>(&amax_kernel<DIN, V>);
  int grid = 0;
  const int64_t step = int64_t(kAmaxItems) * (32 / amax_lanes_per_item(p.chunk, V));
  const int64_t groups = (int64_t(p.nitems) + step - 1) / step;
  cudaError_t err = grid_for(fn, 0, (groups + kThreads / 32 - 1) / (kThreads / 32), &grid);
  if (err != cudaSuccess) return err;
  amax_kernel<DIN, V><<<grid, kThreads, 0, s>>>(static_cast<const store_t<DIN>*>(A), p, alpha_f, amax_bits,
                                                clear_bits);
  ++g_launches;
  return cudaGetLastError();
}

template <int DIN>
cudaError_t launch_amax_t(const void* A, const RowParams& p, float alpha_f, uint32_t* amax_bits,
                          uint32_t* clear_bits, cudaStream_t s) {
  constexpr int V = 16 / int(sizeof(store_t<DIN>));
  if (p.vec == V && reinterpret_cast<uintptr_t>(A) % 16 == 0)
    return launch_amax_v<DIN, V>(A, p, alpha_f, amax_bits, clear_bits, s);
  return launch_amax_v<DIN, 1>(A, p, alpha_f, amax_bits, clear_bits, s);
}

}  // namespace ttc
