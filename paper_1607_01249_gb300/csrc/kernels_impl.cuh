// kernels_impl.cuh -- the sm_103a kernels of one permute-scale-add (Eq. 1).
//
//  tile_kernel  -- the index that is stride-1 in A moves (or both share a short
//                  stride-1 index): a CTA stages a tile in shared memory so that
//                  A is read and B is written along their own stride-1 runs
//                  (the paper's macro-tile of section 2.2, one CTA per tile,
//                  persistent over the flat grid of tiles).
//  copy_kernel  -- perm keeps index 0 (section 3.2: the stride-1 index does not
//                  change): runs of index 0 are streamed directly, one warp per
//                  chunk of a run, 128-bit accesses when aligned.
//  amax_kernel  -- FP8 output without a caller scale: max |alpha*a| pre-pass.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>

#include "kernels.cuh"
#include "launch.h"

namespace ttc {

extern std::atomic<int64_t> g_launches;
cudaError_t grid_for(const void* fn, int smem, int64_t work, int* grid);

// ---------------------------------------------------------------- tile ----

// Read phase, part 1: issue the loads of one tile in A order (lc fastest, then
// la, then lb) into registers.  Element k of this thread is tile element
// t + k*kThreads.
template <int DIN, int K>
__device__ __forceinline__ void tile_load(stage_t<DIN> (&v)[K], const store_t<DIN>* __restrict__ Ab,
                                          const TileCoord& c, const TileParams& p, const int32_t* tabA,
                                          int u0, int lb0) {
  walk_read<K>(c, p, tabA, u0, lb0, [&](int k, int32_t off, int) {
    v[k] = to_stage<DIN>(ldg_elem<DIN>(Ab + off));
  });
}

// Read phase, part 2: put the registers into shared memory (A order, rows
// of pitch P per lb).
template <typename S, int K>
__device__ __forceinline__ void tile_stash(const S (&v)[K], S* tile, const TileCoord& c,
                                           const TileParams& p, int u0, int lb0) {
  walk_read<K>(c, p, static_cast<const int32_t*>(nullptr), u0, lb0, [&](int k, int32_t, int pos) {
    tile[pos] = v[k];
  }, /*need_offset=*/false);
}

// Write phase: gather the tile from shared memory in B order (lc fastest,
// then lb, then la), apply the alpha/beta update and store along B's runs.
template <int DIN, int DOUT, int K>
__device__ __forceinline__ void tile_write(const stage_t<DIN>* tile, store_t<DOUT>* __restrict__ Bb,
                                           const TileCoord& c, const TileParams& p, const int32_t* tabB,
                                           float scale, int lc0, int lb0, int la0) {
  using TO = store_t<DOUT>;
  if (p.epi.beta_nz) {
    TO bo[K];
    walk_write<K>(c, p, tabB, lc0, lb0, la0, [&](int k, int32_t off, int) { bo[k] = Bb[off]; });
    walk_write<K>(c, p, tabB, lc0, lb0, la0, [&](int k, int32_t off, int pos) {
      Bb[off] = epilogue<DIN, DOUT>(tile[pos], bo[k], p.epi, scale);
    });
  } else {
    walk_write<K>(c, p, tabB, lc0, lb0, la0, [&](int, int32_t off, int pos) {
      Bb[off] = epilogue<DIN, DOUT>(tile[pos], TO(0), p.epi, scale);
    });
  }
}

// Persistent over the flat grid of tiles; the loads of the next tile are in
// flight while the current tile is written out (register double buffering).
template <int DIN, int DOUT>
__global__ void __launch_bounds__(kThreads, 2) tile_kernel(const store_t<DIN>* __restrict__ A,
                                                           store_t<DOUT>* __restrict__ B,
                                                           const __grid_constant__ TileParams p) {
  using S = stage_t<DIN>;
  extern __shared__ __align__(16) unsigned char smem[];
  int32_t* tabA = reinterpret_cast<int32_t*>(smem);
  int32_t* tabB = tabA + (p.crossA_tab ? p.LB : 0);
  const int ntab = (p.crossA_tab ? p.LB : 0) + (p.crossB_tab ? p.LA : 0);
  S* tile = reinterpret_cast<S*>(smem + ((ntab * 4 + 15) & ~15));

  const int t = threadIdx.x;
  if (p.crossA_tab)
    for (int i = t; i < p.LB; i += kThreads) tabA[i] = p.tabA[i];
  if (p.crossB_tab)
    for (int i = t; i < p.LA; i += kThreads) tabB[i] = p.tabB[i];
  float scale = 1.f;
  if constexpr (DOUT == DT_E4M3) {
    scale = fp8_scale_of(p.epi);
    if (blockIdx.x == 0 && t == 0 && p.epi.scale_out) *p.epi.scale_out = scale;
  }
  // this thread's first element in read order (u, lb) and write order (lc, lb, la)
  const int r_u0 = t % p.U, r_lb0 = t / p.U;
  const int w_lc0 = t % p.LC, w_lb0 = (t / p.LC) % p.LB, w_la0 = t / p.W;
  __syncthreads();

  constexpr int K = tile_k_for(sizeof(S));
  uint32_t tid = blockIdx.x;
  if (tid >= p.ntiles) return;
  TileCoord cur = tile_coord(tid, p);
  S v[K];
  tile_load<DIN, K>(v, A + cur.baseA, cur, p, tabA, r_u0, r_lb0);
  for (;;) {
    tile_stash<S, K>(v, tile, cur, p, r_u0, r_lb0);
    __syncthreads();
    const uint32_t nxt = tid + gridDim.x;
    TileCoord nc = cur;
    if (nxt < p.ntiles) {
      nc = tile_coord(nxt, p);
      tile_load<DIN, K>(v, A + nc.baseA, nc, p, tabA, r_u0, r_lb0);
    }
    tile_write<DIN, DOUT, K>(tile, B + cur.baseB, cur, p, tabB, scale, w_lc0, w_lb0, w_la0);
    __syncthreads();
    if (nxt >= p.ntiles) break;
    tid = nxt;
    cur = nc;
  }
}

// -------------------------------------------------------- tile, warp-mapped --
//
// Same tile and the same shared-memory layout as tile_kernel, but threads are
// mapped in 2D: in the read phase the 32 lanes of a warp cover 32 consecutive
// positions u of an A run (JU chunks of 32 cover U) and the 8 warps take the
// rows lb in turn; in the write phase the lanes cover 32 consecutive positions
// v of a B run (JW chunks cover W) and the warps take the rows la.  All
// per-element index work is then one add per element (row offsets come once
// per row), which keeps the kernel under the memory roof instead of the issue
// roof.  Constraints (the planner checks them): U <= 32*JU, LB <= 128/JU,
// W <= 32*JW, LA <= 128/JW.

template <int DIN, int JU, int K>
__device__ __forceinline__ void tile2_load(stage_t<DIN> (&v)[K], const store_t<DIN>* __restrict__ A,
                                           const TileCoord& c, const TileParams& p, const int32_t* tabA,
                                           int lane, int warp) {
  const store_t<DIN>* Ab = A + c.baseA;
  walk2_read<JU, K>(c, p, tabA, lane, warp, [&](int k, int32_t off, int) {
    v[k] = to_stage<DIN>(ldg_elem<DIN>(Ab + off));
  });
}

template <typename S, int JU, int K>
__device__ __forceinline__ void tile2_stash(const S (&v)[K], S* tile, const TileCoord& c,
                                            const TileParams& p, const int32_t* tabA, int lane, int warp) {
  walk2_read<JU, K>(c, p, tabA, lane, warp, [&](int k, int32_t, int pos) { tile[pos] = v[k]; });
}

template <int DIN, int DOUT, int JW, int K>
__device__ __forceinline__ void tile2_write(const stage_t<DIN>* tile, store_t<DOUT>* __restrict__ B,
                                            const TileCoord& c, const TileParams& p, const int32_t* tabB,
                                            float scale, int lane, int warp, const int (&spre)[JW],
                                            const int32_t (&voff)[JW]) {
  using TO = store_t<DOUT>;
  TO* Bb = B + c.baseB;
  if (p.epi.beta_nz) {
    TO bo[K];
    walk2_write<JW, K>(c, p, tabB, lane, warp, spre, voff, [&](int k, int32_t off, int) { bo[k] = Bb[off]; });
    walk2_write<JW, K>(c, p, tabB, lane, warp, spre, voff, [&](int k, int32_t off, int pos) {
      Bb[off] = epilogue<DIN, DOUT>(tile[pos], bo[k], p.epi, scale);
    });
  } else {
    walk2_write<JW, K>(c, p, tabB, lane, warp, spre, voff, [&](int, int32_t off, int pos) {
      Bb[off] = epilogue<DIN, DOUT>(tile[pos], TO(0), p.epi, scale);
    });
  }
}

template <int DIN, int DOUT, int JU, int JW>
__global__ void __launch_bounds__(kThreads, (JU == 1 || JW == 1) ? 2 : 3) tile2_kernel(const store_t<DIN>* __restrict__ A,
                                                            store_t<DOUT>* __restrict__ B,
                                                            const __grid_constant__ TileParams p) {
  using S = stage_t<DIN>;
  extern __shared__ __align__(16) unsigned char smem[];
  int32_t* tabA = reinterpret_cast<int32_t*>(smem);
  int32_t* tabB = tabA + (p.crossA_tab ? p.LB : 0);
  const int ntab = (p.crossA_tab ? p.LB : 0) + (p.crossB_tab ? p.LA : 0);
  S* tile = reinterpret_cast<S*>(smem + ((ntab * 4 + 15) & ~15));
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (p.crossA_tab)
    for (int i = t; i < p.LB; i += kThreads) tabA[i] = p.tabA[i];
  if (p.crossB_tab)
    for (int i = t; i < p.LA; i += kThreads) tabB[i] = p.tabB[i];
  float scale = 1.f;
  if constexpr (DOUT == DT_E4M3) {
    scale = fp8_scale_of(p.epi);
    if (blockIdx.x == 0 && t == 0 && p.epi.scale_out) *p.epi.scale_out = scale;
  }
  int spre[JW];
  int32_t voff[JW];
  walk2_lane_consts<JW>(p, lane, spre, voff);
  __syncthreads();

  constexpr int K = tile_k_for(sizeof(S));
  uint32_t tid = blockIdx.x;
  if (tid >= p.ntiles) return;
  TileCoord cur = tile_coord(tid, p);
  S v[K];
  tile2_load<DIN, JU, K>(v, A, cur, p, tabA, lane, warp);
  for (;;) {
    tile2_stash<S, JU, K>(v, tile, cur, p, tabA, lane, warp);
    __syncthreads();
    const uint32_t nxt = tid + gridDim.x;
    TileCoord nc = cur;
    if (nxt < p.ntiles) {
      nc = tile_coord(nxt, p);
      tile2_load<DIN, JU, K>(v, A, nc, p, tabA, lane, warp);
    }
    tile2_write<DIN, DOUT, JW, K>(tile, B, cur, p, tabB, scale, lane, warp, spre, voff);
    __syncthreads();
    if (nxt >= p.ntiles) break;
    tid = nxt;
    cur = nc;
  }
}

// ------------------------------------------- tile, warp-mapped, cp.async ring --
//
// tile2's lane layout, but the read phase copies A straight into shared memory
// with asynchronous copies (cp.async, no registers), into a ring of kStages
// tile buffers: the copies of the next kStages-1 tiles are in flight while the
// current tile is written out, so the SM keeps far more bytes in flight than
// register staging allows.  Only for 4- and 8-byte input elements (the
// smallest cp.async is 4 bytes).

constexpr int kStages = 3;

__device__ __forceinline__ void cp_async_elem(void* smem_dst, const void* gsrc, int bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int DIN, int JU, int K, bool FULL>
__device__ __forceinline__ void tile3_issue(stage_t<DIN>* buf, const store_t<DIN>* __restrict__ A,
                                            const TileCoord& c, const TileParams& p, const int32_t* tabA,
                                            int lane, int warp) {
  const store_t<DIN>* Ab = A + c.baseA;
  walk3_read<JU, K, FULL>(c, p, tabA, lane, warp, [&](int, int32_t off, int pos) {
    cp_async_elem(buf + pos, Ab + off, int(sizeof(store_t<DIN>)));
  });
}

template <int DIN, int DOUT, int JW, int K, int EK, bool FULL>
__device__ __forceinline__ void tile3_write(const stage_t<DIN>* tile, store_t<DOUT>* __restrict__ B,
                                            const TileCoord& c, const TileParams& p, const int32_t* tabB,
                                            float scale, int lane, int warp, const int (&spre)[JW]) {
  using TO = store_t<DOUT>;
  TO* Bb = B + c.baseB;
  if constexpr (EK == EK_AXPBY) {
    TO bo[K];
    walk3_write<JW, K, FULL>(c, p, tabB, lane, warp, spre, [&](int k, int32_t off, int) { bo[k] = Bb[off]; });
    walk3_write<JW, K, FULL>(c, p, tabB, lane, warp, spre, [&](int k, int32_t off, int pos) {
      Bb[off] = epilogue_k<DIN, DOUT, EK>(tile[pos], bo[k], p.epi, scale);
    });
  } else {
    walk3_write<JW, K, FULL>(c, p, tabB, lane, warp, spre, [&](int, int32_t off, int pos) {
      Bb[off] = epilogue_k<DIN, DOUT, EK>(tile[pos], TO(0), p.epi, scale);
    });
  }
}

template <int DIN, int DOUT, int JU, int JW, int EK>
__global__ void __launch_bounds__(kThreads, 3) tile3_kernel(const store_t<DIN>* __restrict__ A,
                                                            store_t<DOUT>* __restrict__ B,
                                                            const __grid_constant__ TileParams p, int stage_elems) {
  using S = stage_t<DIN>;
  static_assert(sizeof(S) == sizeof(store_t<DIN>), "cp.async stages the input type as is");
  constexpr int K = tile_k_for(sizeof(S));
  extern __shared__ __align__(16) unsigned char smem[];
  int32_t* tabA = reinterpret_cast<int32_t*>(smem);
  int32_t* tabB = tabA + (p.crossA_tab ? p.LB : 0);
  const int ntab = (p.crossA_tab ? p.LB : 0) + (p.crossB_tab ? p.LA : 0);
  S* ring = reinterpret_cast<S*>(smem + ((ntab * 4 + 15) & ~15));
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (p.crossA_tab)
    for (int i = t; i < p.LB; i += kThreads) tabA[i] = p.tabA[i];
  if (p.crossB_tab)
    for (int i = t; i < p.LA; i += kThreads) tabB[i] = p.tabB[i];
  float scale = 1.f;
  if constexpr (EK == EK_FP8) {
    scale = fp8_scale_of(p.epi);
    if (blockIdx.x == 0 && t == 0 && p.epi.scale_out) *p.epi.scale_out = scale;
  }
  int spre[JW];
  int32_t voff[JW];
  walk2_lane_consts<JW>(p, lane, spre, voff);
  __syncthreads();

  const uint32_t g = gridDim.x;
  uint32_t tid = blockIdx.x;
  if (tid >= p.ntiles) return;
  auto issue = [&](uint32_t q, int stage) {
    const TileCoord c = tile_coord(q, p);
    S* buf = ring + stage * stage_elems;
    if (c.remA == p.LA && c.remB == p.LB) tile3_issue<DIN, JU, K, true>(buf, A, c, p, tabA, lane, warp);
    else tile3_issue<DIN, JU, K, false>(buf, A, c, p, tabA, lane, warp);
  };
  // prologue: the first kStages-1 tiles of this CTA
#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) {
    const uint32_t q = tid + uint32_t(s) * g;
    if (q < p.ntiles) issue(q, s);
    cp_async_commit();
  }
  for (int it = 0;; ++it) {
    const uint32_t q = tid + uint32_t(kStages - 1) * g;
    if (q < p.ntiles) issue(q, (it + kStages - 1) % kStages);
    cp_async_commit();
    cp_async_wait<kStages - 1>();
    __syncthreads();
    const TileCoord c = tile_coord(tid, p);
    const S* tile = ring + (it % kStages) * stage_elems;
    if (c.remA == p.LA && c.remB == p.LB)
      tile3_write<DIN, DOUT, JW, K, EK, true>(tile, B, c, p, tabB, scale, lane, warp, spre);
    else
      tile3_write<DIN, DOUT, JW, K, EK, false>(tile, B, c, p, tabB, scale, lane, warp, spre);
    __syncthreads();
    tid += g;
    if (tid >= p.ntiles) break;
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------- copy ----

constexpr int kCopyUnroll = 4;

template <int DIN, int DOUT, int VEC>
__global__ void __launch_bounds__(kThreads) copy_kernel(const store_t<DIN>* __restrict__ A,
                                                        store_t<DOUT>* __restrict__ B,
                                                        const __grid_constant__ RowParams p) {
  using TI = store_t<DIN>;
  using TO = store_t<DOUT>;
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * kThreads) >> 5;
  float scale = 1.f;
  if constexpr (DOUT == DT_E4M3) {
    scale = fp8_scale_of(p.epi);
    if (blockIdx.x == 0 && threadIdx.x == 0 && p.epi.scale_out) *p.epi.scale_out = scale;
  }
  for (uint32_t item = warp; item < p.nitems; item += nwarps) {
    const RowCoord rc = row_coord(item, p);
    const int64_t offA = rc.offA, offB = rc.offB, start = rc.start, end = rc.end;
    if constexpr (VEC == 1) {
      const TI* Ar = A + offA;
      TO* Br = B + offB;
      for (int64_t x0 = start + lane; x0 < end; x0 += 32 * kCopyUnroll) {
        stage_t<DIN> a[kCopyUnroll];
        TO b[kCopyUnroll];
#pragma unroll
        for (int j = 0; j < kCopyUnroll; ++j) {
          const int64_t x = x0 + 32 * j;
          if (x < end) {
            a[j] = to_stage<DIN>(ldg_elem<DIN>(Ar + x * p.sa0));
            if (p.epi.beta_nz) b[j] = Br[x * p.sb0];
          }
        }
#pragma unroll
        for (int j = 0; j < kCopyUnroll; ++j) {
          const int64_t x = x0 + 32 * j;
          if (x < end) Br[x * p.sb0] = epilogue<DIN, DOUT>(a[j], b[j], p.epi, scale);
        }
      }
    } else {
      // unit strides, len, chunk and all row offsets multiples of VEC, bases aligned
      using VI = VecT<TI, VEC>;
      using VO = VecT<TO, VEC>;
      const VI* Av = reinterpret_cast<const VI*>(A + offA);
      VO* Bv = reinterpret_cast<VO*>(B + offB);
      const int64_t vs = start / VEC, ve = end / VEC;
      for (int64_t x0 = vs + lane; x0 < ve; x0 += 32 * kCopyUnroll) {
        VI a[kCopyUnroll];
        VO b[kCopyUnroll];
#pragma unroll
        for (int j = 0; j < kCopyUnroll; ++j) {
          const int64_t x = x0 + 32 * j;
          if (x < ve) {
            a[j] = Av[x];
            if (p.epi.beta_nz) b[j] = Bv[x];
          }
        }
#pragma unroll
        for (int j = 0; j < kCopyUnroll; ++j) {
          const int64_t x = x0 + 32 * j;
          if (x < ve) {
            VO o;
#pragma unroll
            for (int e = 0; e < VEC; ++e)
              o.v[e] = epilogue<DIN, DOUT>(to_stage<DIN>(a[j].v[e]), b[j].v[e], p.epi, scale);
            Bv[x] = o;
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------- amax ----

template <int DIN>
__global__ void __launch_bounds__(kThreads) amax_kernel(const store_t<DIN>* __restrict__ A,
                                                        const __grid_constant__ RowParams p,
                                                        float alpha_f, uint32_t* amax_bits) {
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * kThreads) >> 5;
  float m = 0.f;
  for (uint32_t item = warp; item < p.nitems; item += nwarps) {
    const RowCoord rc = row_coord(item, p);
    const int64_t start = rc.start, end = rc.end;
    const store_t<DIN>* Ar = A + rc.offA;
    for (int64_t x = start + lane; x < end; x += 32) {
      const float v = fabsf(__fmul_rn(alpha_f, float(to_stage<DIN>(ldg_elem<DIN>(Ar + x * p.sa0)))));
      if (v > m) m = v;     // NaN compares false: ignored
    }
  }
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float red[kThreads / 32];
  if (lane == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.f;
    for (int i = 0; i < kThreads / 32; ++i) b = fmaxf(b, red[i]);
    if (b > 0.f) atomicMax(amax_bits, __float_as_uint(b));
  }
}


// ------------------------------------------------------------ launch templates --

template <int DIN, int DOUT>
cudaError_t launch_tile_t(const void* A, void* B, const TileParams& p, int smem, cudaStream_t s,
                          int grid_override) {
  const void* fn = reinterpret_cast<const void*>(&tile_kernel<DIN, DOUT>);
  int grid = 0;
  cudaError_t err = grid_for(fn, smem, p.ntiles, &grid);
  if (err != cudaSuccess) return err;
  if (grid_override > 0 && grid_override < grid) grid = grid_override;
  tile_kernel<DIN, DOUT><<<grid, kThreads, smem, s>>>(static_cast<const store_t<DIN>*>(A),
                                                     static_cast<store_t<DOUT>*>(B), p);
  ++g_launches;
  return cudaGetLastError();
}

template <int DIN, int DOUT, int JU, int JW>
cudaError_t launch_tile2_t(const void* A, void* B, const TileParams& p, int smem, cudaStream_t s,
                           int grid_override) {
  const void* fn = reinterpret_cast<const void*>(&tile2_kernel<DIN, DOUT, JU, JW>);
  int grid = 0;
  cudaError_t err = grid_for(fn, smem, p.ntiles, &grid);
  if (err != cudaSuccess) return err;
  if (grid_override > 0 && grid_override < grid) grid = grid_override;
  tile2_kernel<DIN, DOUT, JU, JW><<<grid, kThreads, smem, s>>>(static_cast<const store_t<DIN>*>(A),
                                                               static_cast<store_t<DOUT>*>(B), p);
  ++g_launches;
  return cudaGetLastError();
}

template <int DIN, int DOUT, int JU, int JW, int EK>
cudaError_t launch_tile3_t(const void* A, void* B, const TileParams& p, int smem, cudaStream_t s,
                           int grid_override) {
  const void* fn = reinterpret_cast<const void*>(&tile3_kernel<DIN, DOUT, JU, JW, EK>);
  // smem holds the tables and one tile per stage
  const int tile_bytes = p.P * p.LB * int(sizeof(stage_t<DIN>));
  const int stage_elems = (tile_bytes + 15) / 16 * 16 / int(sizeof(stage_t<DIN>));
  const int ring = smem - tile_bytes + kStages * stage_elems * int(sizeof(stage_t<DIN>));
  int grid = 0;
  cudaError_t err = grid_for(fn, ring, p.ntiles, &grid);
  if (err != cudaSuccess) return err;
  if (grid_override > 0 && grid_override < grid) grid = grid_override;
  tile3_kernel<DIN, DOUT, JU, JW, EK><<<grid, kThreads, ring, s>>>(static_cast<const store_t<DIN>*>(A),
                                                                   static_cast<store_t<DOUT>*>(B), p, stage_elems);
  ++g_launches;
  return cudaGetLastError();
}

template <int DIN, int DOUT, int EK>
cudaError_t launch_tile3_ek(int ju, int jw, const void* A, void* B, const TileParams& p, int smem,
                            cudaStream_t s, int grid_override) {
#define J(U_, W_) \
  if (ju == U_ && jw == W_) return launch_tile3_t<DIN, DOUT, U_, W_, EK>(A, B, p, smem, s, grid_override);
  J(1, 2) J(1, 4) J(2, 1) J(2, 2) J(4, 1) J(4, 2)
#undef J
  return cudaErrorInvalidValue;
}

template <int DIN, int DOUT>
cudaError_t launch_tile3_pair(int ju, int jw, int mode, int beta_nz, const void* A, void* B, const TileParams& p,
                              int smem, cudaStream_t s, int grid_override) {
  if constexpr (DIN == DT_BF16) {
    return cudaErrorInvalidValue;
  } else if constexpr (DOUT == DT_E4M3) {
    return launch_tile3_ek<DIN, DOUT, EK_FP8>(ju, jw, A, B, p, smem, s, grid_override);
  } else {
    if (beta_nz) return launch_tile3_ek<DIN, DOUT, EK_AXPBY>(ju, jw, A, B, p, smem, s, grid_override);
    if constexpr (DIN == DOUT)
      if (mode == MODE_BITCOPY) return launch_tile3_ek<DIN, DOUT, EK_COPY>(ju, jw, A, B, p, smem, s, grid_override);
    return launch_tile3_ek<DIN, DOUT, EK_SCALE>(ju, jw, A, B, p, smem, s, grid_override);
  }
}

template <int DIN, int DOUT>
cudaError_t launch_tile2_pair(int ju, int jw, const void* A, void* B, const TileParams& p, int smem,
                              cudaStream_t s, int grid_override) {
#define J(U_, W_) \
  if (ju == U_ && jw == W_) return launch_tile2_t<DIN, DOUT, U_, W_>(A, B, p, smem, s, grid_override);
  J(1, 1) J(1, 2) J(1, 4) J(2, 1) J(2, 2) J(2, 4) J(4, 1) J(4, 2) J(4, 4)
#undef J
  return cudaErrorInvalidValue;
}

template <int DIN, int DOUT, int VEC>
cudaError_t launch_copy_t(const void* A, void* B, const RowParams& p, cudaStream_t s) {
  const void* fn = reinterpret_cast<const void*>(&copy_kernel<DIN, DOUT, VEC>);
  int grid = 0;
  cudaError_t err = grid_for(fn, 0, (int64_t(p.nitems) + 7) / 8, &grid);
  if (err != cudaSuccess) return err;
  copy_kernel<DIN, DOUT, VEC><<<grid, kThreads, 0, s>>>(static_cast<const store_t<DIN>*>(A),
                                                       static_cast<store_t<DOUT>*>(B), p);
  ++g_launches;
  return cudaGetLastError();
}

template <int DIN>
cudaError_t launch_amax_t(const void* A, const RowParams& p, float alpha_f, uint32_t* amax_bits,
                          cudaStream_t s) {
  const void* fn = reinterpret_cast<const void*>(&amax_kernel<DIN>);
  int grid = 0;
  cudaError_t err = grid_for(fn, 0, (int64_t(p.nitems) + 7) / 8, &grid);
  if (err != cudaSuccess) return err;
  amax_kernel<DIN><<<grid, kThreads, 0, s>>>(static_cast<const store_t<DIN>*>(A), p, alpha_f, amax_bits);
  ++g_launches;
  return cudaGetLastError();
}


}  // namespace ttc
