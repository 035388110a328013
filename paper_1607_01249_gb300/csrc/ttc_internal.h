// ttc_internal.h -- types shared by the planner (host) and the kernels (device).
//
// Vocabulary (after canonicalisation, section 2.1 stage 1):
//   N canonical indices k = 0..N-1 in A's order, sizes s[k], element strides
//   sa[k] in A and sb[k] in B, perm[d] = A index at B position d.
//
// Tile schedule ("macro-tile" of section 2.2, Fig. 4, re-designed for one
// CTA of a GB300 SM): a tile is a box over three disjoint index groups
//   C  -- the index both tensors share as their stride-1 index (only when
//         perm[0] == 0), taken whole; extent LC (1 when absent);
//   GA -- a dense prefix of A's indices after C, the last one possibly cut
//         into blocks; linear extent LA;
//   GB -- a dense prefix of B's indices after C, disjoint from GA, the last
//         possibly cut into blocks; linear extent LB.
// An element of the tile is (lc, la, lb).  Its A offset is
//   (la*LC + lc) * saU + crossA(lb),  crossA = A offset of GB's coordinates,
// and its B offset is
//   (lb*LC + lc) * sbV + crossB(la),  crossB = B offset of GA's coordinates.
// The CTA reads the tile in A order (lc fastest, then la, then lb), keeps it in
// shared memory, and writes it in B order (lc, lb, la), so both global
// streams are coalesced.  Every other index (and the block index of the cut
// indices) forms the flat grid of tiles.
#pragma once

#include <cstdint>

#include "fpint.h"

struct int4;   // CUDA vector type (vector_types.h); only pointers to it appear here

#if defined(__CUDACC__)
#define TTC_HD __host__ __device__ __forceinline__
#else
#define TTC_HD inline
#endif

namespace ttc {

constexpr int kMaxDim = 16;
constexpr int kThreads = 256;          // threads per CTA of every kernel
constexpr int kTileK = 16;             // elements per thread per phase (tile kernels, 4-byte stage)
constexpr int kTileVmax = kThreads * kTileK;
// elements per thread per phase for a stage type of `stage_bytes` bytes:
// 64 bytes of staged data per thread per phase
constexpr int tile_k_for(int stage_bytes) { return stage_bytes == 16 ? 4 : stage_bytes == 8 ? 8 : 16; }

// DT_C64 / DT_C128: single- and double-complex (the paper's "c" and "z",
// section 2.1), stored as (real, imaginary) pairs of binary32 / binary64
enum DType : int { DT_F32 = 0, DT_F64 = 1, DT_BF16 = 2, DT_E4M3 = 3, DT_C64 = 4, DT_C128 = 5 };
constexpr int kNumDTypes = 6;

constexpr int dtype_size(int dt) {
  return dt == DT_C128 ? 16 : (dt == DT_F64 || dt == DT_C64) ? 8 : dt == DT_F32 ? 4 : dt == DT_BF16 ? 2 : 1;
}
constexpr bool is_complex(int dt) { return dt == DT_C64 || dt == DT_C128; }
// bytes of one element of A staged in shared memory (bf16 is widened to f32)
constexpr int stage_bytes_of(int din) { return din == DT_BF16 ? 4 : dtype_size(din); }

// Epilogue modes (the alpha/beta update of Eq. 1 fused into the store).
enum Mode : int {
  MODE_BITCOPY = 0,   // alpha == 1, beta == 0, same type: move the bits
  MODE_AXPBY = 1,     // r = fma(beta, b, alpha*a) (beta == 0: r = alpha*a), rounded to B's type
  MODE_FP8 = 2        // code = e4m3_satfinite(fl32(alpha*a) / scale)
};

// Unsigned division by an invariant divisor through a multiply-high and a
// shift (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, section 4): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, q = (mulhi(m, n) + n) >> l.  Valid for
// n < 2^31 (so that the sum does not overflow); the planner guarantees it.
struct FastDiv {
  uint32_t d = 1, m = 1, l = 0;
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t l = 0;
  while ((uint64_t(1) << l) < d) ++l;
  f.l = l;
  f.m = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
  return f;
}

TTC_HD uint32_t fast_div(uint32_t n, const FastDiv& f) {
#if defined(__CUDA_ARCH__)
  uint32_t hi = __umulhi(n, f.m);
#else
  uint32_t hi = uint32_t((uint64_t(n) * f.m) >> 32);
#endif
  return (hi + n) >> f.l;
}

// One index of the flat grid of tiles (or of rows).
struct GridDim {
  FastDiv div;         // number of blocks along this index
  int64_t stepA;       // A offset per block
  int64_t stepB;       // B offset per block
  int32_t kind;        // 0 = whole index, 1 = cut index of GA, 2 = cut index of GB
  int32_t t;           // tile extent of a cut index
  int32_t s;           // size of a cut index
  int32_t pad;
};

// Epilogue scalars, shared by all kernels.  Complex dtypes also use the
// imaginary parts alpha_*i, beta_*i (zero for real scalars).
struct Epilogue {
  int mode;
  int beta_nz;         // beta != 0: B is read
  float alpha_f, beta_f;
  double alpha_d, beta_d;
  float alpha_fi, beta_fi;
  double alpha_di, beta_di;
  DMulConst alpha_k;           // alpha_d prepared for the integer product (fpint.h)
  const float* scale_in;       // FP8: caller-supplied scale (device) or null
  const uint32_t* amax_bits;   // FP8: amax as float bits (device scratch) when scale_in is null
  float* scale_out;            // FP8: where block 0 records the scale used
};

// Thread layout of one side of a packed-lane tile (tilep_kernel) for one
// run length n: the CTA's threads form `rows` groups of g consecutive
// threads (g * rows <= the thread count); thread t = tu + g * tr takes run
// positions tu + g * j (j < J, the kernel's chunks per run, g * J >= n) of
// rows tr + rows * i.  g as an invariant divisor.
struct PackWalk {
  int n = 1, g = 1, rows = 1;
  FastDiv div;
};

struct TileParams {
  int ngrid;
  uint32_t ntiles;
  // grouped order (0: off): the first two grid indices are visited in groups
  // of `swz` blocks of the first, all blocks of the second within a group,
  // so that consecutive tiles stay close in both tensors
  uint32_t swz;
  GridDim g[kMaxDim];
  int LC, LA, LB;      // group extents
  int U;               // LC*LA  (A-side run, in elements)
  int W;               // LC*LB  (B-side run)
  int V;               // LC*LA*LB
  int P;               // shared-memory pitch of one lb row, in elements
  int fullA;           // GA: product of the whole extents below its cut index (la units)
  int fullB;           // GB: same for lb units
  // offsets inside one tile are 32-bit (the planner only keeps tile shapes
  // whose largest in-tile offset is below 2^31); tile bases are 64-bit
  int32_t saU, sbV;    // strides of the runs u (in A) and v (in B)
  int32_t crossA_lin;  // crossA(lb) = lb * crossA_lin when GB has one index
  int32_t crossB_lin;  // crossB(la) = la * crossB_lin when GA has one index
  int crossA_tab;      // nonzero: crossA comes from a table of LB entries
  int crossB_tab;      // nonzero: crossB comes from a table of LA entries
  const int32_t* tabA; // device table crossA[LB]
  const int32_t* tabB; // device table crossB[LA]
  // Slot tables of tile_slots_kernel: for every (k, thread) slot of the load
  // and of the store order, four slots per 16-byte group [K/4][kThreads]:
  // the element's offset in the tile (int32; load region, then store
  // region), its tile coordinate (la << 16 | lb, 0xffffffff: no element;
  // load, then store) and its shared-memory position (uint16, 0xffff: no
  // element, four per 8 bytes; load, then store).
  const int4* slots;
  // per-thread step of kThreads in the read order (u, lb) and write order (lc, lb, la)
  int rd_du, rd_dlb;
  int wr_dlc, wr_dlb, wr_dla;
  // invariant divisors of the lane/thread decompositions
  FastDiv divU, divLC, divLB, divW;
  // packed-lane tiles (no C index): walk constants of the load side (runs of
  // u = la, rows lb) and of the store side (runs of v = lb, rows la), [0] for
  // the full extent, [1] for the extent a cut index leaves in the last block
  PackWalk pkA[2], pkB[2];
  // packed rows (rowsp_kernel): the row count of a tile's A side, LA and
  // the short last block's, as invariant divisors of the row index
  FastDiv divRA[2];
  Epilogue epi;
};

struct RowParams {
  int nrd;             // indices of a row (all but the run index)
  uint32_t nitems;     // rows * chunks
  FastDiv chunks;      // chunks per row
  FastDiv div[kMaxDim];
  int64_t stA[kMaxDim], stB[kMaxDim];
  int64_t len;         // run length (elements)
  int64_t chunk;       // chunk length (elements)
  int64_t sa0, sb0;    // run strides
  int vec;             // FP8 amax pre-pass: elements per 16-byte load (1: one element per load)
  Epilogue epi;
};

// Kernel-level entry points implemented in the .cu files.
struct LaunchCfg {
  int grid;
  int smem;
};

}  // namespace ttc
