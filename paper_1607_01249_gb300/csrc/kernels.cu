// kernels.cu -- the sm_103a kernels of one permute-scale-add (Eq. 1).
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
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <mutex>
#include <map>

#include "kernels.cuh"
#include "launch.h"

namespace ttc {

std::atomic<int64_t> g_launches{0};

// ---------------------------------------------------------------- tile ----

// Read phase, part 1: issue the loads of one tile in A order (lc fastest, then
// la, then lb) into registers.  Element k of this thread is tile element
// t + k*kThreads.
template <int DIN>
__device__ __forceinline__ void tile_load(stage_t<DIN> (&v)[kTileK], const store_t<DIN>* __restrict__ Ab,
                                          const TileCoord& c, const TileParams& p, const int32_t* tabA,
                                          int u0, int lb0) {
  walk_read(c, p, tabA, u0, lb0, [&](int k, int32_t off, int) {
    v[k] = to_stage<DIN>(ldg_elem<DIN>(Ab + off));
  });
}

// Read phase, part 2: put the registers into shared memory (A order, rows
// of pitch P per lb).
template <typename S>
__device__ __forceinline__ void tile_stash(const S (&v)[kTileK], S* tile, const TileCoord& c,
                                           const TileParams& p, int u0, int lb0) {
  walk_read(c, p, static_cast<const int32_t*>(nullptr), u0, lb0, [&](int k, int32_t, int pos) {
    tile[pos] = v[k];
  }, /*need_offset=*/false);
}

// Write phase: gather the tile from shared memory in B order (lc fastest,
// then lb, then la), apply the alpha/beta update and store along B's runs.
template <int DIN, int DOUT>
__device__ __forceinline__ void tile_write(const stage_t<DIN>* tile, store_t<DOUT>* __restrict__ Bb,
                                           const TileCoord& c, const TileParams& p, const int32_t* tabB,
                                           float scale, int lc0, int lb0, int la0) {
  using TO = store_t<DOUT>;
  stage_t<DIN> w[kTileK];
  TO bo[kTileK];
  const bool bnz = p.epi.beta_nz;
  walk_write(c, p, tabB, lc0, lb0, la0, [&](int k, int32_t off, int pos) {
    w[k] = tile[pos];
    if (bnz) bo[k] = Bb[off];
  });
  walk_write(c, p, tabB, lc0, lb0, la0, [&](int k, int32_t off, int) {
    Bb[off] = epilogue<DIN, DOUT>(w[k], bo[k], p.epi, scale);
  });
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

  uint32_t tid = blockIdx.x;
  if (tid >= p.ntiles) return;
  TileCoord cur = tile_coord(tid, p);
  S v[kTileK];
  tile_load<DIN>(v, A + cur.baseA, cur, p, tabA, r_u0, r_lb0);
  for (;;) {
    tile_stash<S>(v, tile, cur, p, r_u0, r_lb0);
    __syncthreads();
    const uint32_t nxt = tid + gridDim.x;
    TileCoord nc = cur;
    if (nxt < p.ntiles) {
      nc = tile_coord(nxt, p);
      tile_load<DIN>(v, A + nc.baseA, nc, p, tabA, r_u0, r_lb0);
    }
    tile_write<DIN, DOUT>(tile, B + cur.baseB, cur, p, tabB, scale, w_lc0, w_lb0, w_la0);
    __syncthreads();
    if (nxt >= p.ntiles) break;
    tid = nxt;
    cur = nc;
  }
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

// ------------------------------------------------------------- launchers --

namespace {

struct OccKey {
  const void* fn;
  int smem;
  int dev;
  bool operator<(const OccKey& o) const {
    if (fn != o.fn) return fn < o.fn;
    if (smem != o.smem) return smem < o.smem;
    return dev < o.dev;
  }
};
std::mutex g_occ_mu;
std::map<OccKey, int> g_occ;

cudaError_t grid_for(const void* fn, int smem, int64_t work, int* grid) {
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  int blocks = 0;
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    auto it = g_occ.find({fn, smem, dev});
    if (it != g_occ.end()) blocks = it->second;
  }
  if (blocks == 0) {
    if (smem > 48 * 1024) {
      err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (err != cudaSuccess) return err;
    }
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem);
    if (err != cudaSuccess) return err;
    int sms = 0;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    blocks = (per_sm > 0 ? per_sm : 1) * sms;
    std::lock_guard<std::mutex> lk(g_occ_mu);
    g_occ[{fn, smem, dev}] = blocks;
  }
  int64_t g = work < blocks ? work : blocks;
  *grid = int(g < 1 ? 1 : g);
  return cudaSuccess;
}

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

}  // namespace

// Supported (dtype_in, dtype_out) pairs.
#define TTC_FOR_EACH_PAIR(X) \
  X(DT_F32, DT_F32)          \
  X(DT_F32, DT_F64)          \
  X(DT_F32, DT_BF16)         \
  X(DT_F32, DT_E4M3)         \
  X(DT_F64, DT_F64)          \
  X(DT_F64, DT_F32)          \
  X(DT_BF16, DT_BF16)        \
  X(DT_BF16, DT_F32)         \
  X(DT_BF16, DT_E4M3)

bool pair_supported(int din, int dout) {
#define X(I, O) if (din == I && dout == O) return true;
  TTC_FOR_EACH_PAIR(X)
#undef X
  return false;
}

// Widest vector (elements) the copy kernel uses for a pair: 16 bytes of the
// wider of the two types.
int copy_vec_width(int din, int dout) {
  int w = dtype_size(din) > dtype_size(dout) ? dtype_size(din) : dtype_size(dout);
  return 16 / w;
}

cudaError_t launch_tile(int din, int dout, const void* A, void* B, const TileParams& p, int smem,
                        cudaStream_t s, int grid_override) {
#define X(I, O) if (din == I && dout == O) return launch_tile_t<I, O>(A, B, p, smem, s, grid_override);
  TTC_FOR_EACH_PAIR(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_copy(int din, int dout, int vec, const void* A, void* B, const RowParams& p,
                        cudaStream_t s) {
#define X(I, O)                                                                      \
  if (din == I && dout == O) {                                                       \
    constexpr int W = (dtype_size(I) > dtype_size(O) ? 16 / dtype_size(I) : 16 / dtype_size(O)); \
    if (vec == W) return launch_copy_t<I, O, W>(A, B, p, s);                         \
    return launch_copy_t<I, O, 1>(A, B, p, s);                                       \
  }
  TTC_FOR_EACH_PAIR(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_amax(int din, const void* A, const RowParams& p, float alpha_f, uint32_t* amax_bits,
                        cudaStream_t s) {
  if (din == DT_F32) return launch_amax_t<DT_F32>(A, p, alpha_f, amax_bits, s);
  if (din == DT_BF16) return launch_amax_t<DT_BF16>(A, p, alpha_f, amax_bits, s);
  return cudaErrorInvalidValue;
}

int64_t launch_count() { return g_launches.load(); }

}  // namespace ttc
