// tma2d.h -- the TMA-staged tile of a two-index transpose (tma2d.cu): its
// geometry, shared by the kernel, the planner and the host schedule checker.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "planner.h"
#include "ttc_internal.h"

namespace ttc {

// B[c + r ldb] <- Eq. 1 of A[r + c lda] for r < R, c < C: a problem whose
// canonical form has two indices, swapped.  A CTA takes a tile of bx rows
// (A's stride-1 index; bx x element size = 128 bytes) by 32 kTmaBoxes
// columns, copied by the tensor memory accelerator as kTmaBoxes boxes of
// bx x 32 into shared memory in the 128-byte swizzle.
constexpr int kTmaBoxes = 4;
constexpr int kTmaBoxBytes = 4096;   // bx x 32 elements of 128 / bx bytes

struct Tma2dGeom {
  int R, C;          // extents (A's stride-1 index, the other)
  int bx;            // box rows: 128 bytes of A's elements
  int tilesR;        // tiles along R
  int64_t tiles;     // tiles in all
  int64_t lda, ldb;  // A's column stride, B's row stride (elements)
};

TTC_HD int64_t tma2d_cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Whether a canonical problem takes the TMA tile: two indices swapped, A's
// and B's stride-1 indices dense, A's column stride a multiple of 16 bytes (the TMA's
// rule for global strides), a real FP32 or FP64 A, and extents and tile
// counts within the kernel's 32-bit arithmetic.
inline bool tma2d_eligible(const Canon& c, int din) {
  if (c.N != 2 || c.perm[0] != 1 || c.perm[1] != 0) return false;
  if (din != DT_F32 && din != DT_F64) return false;
  const int es = dtype_size(din);
  if (c.sa[0] != 1 || c.sb[1] != 1 || (c.sa[1] * es) % 16 != 0) return false;
  if (c.s[0] >= (int64_t(1) << 31) || c.s[1] >= (int64_t(1) << 31) || c.sa[1] >= (int64_t(1) << 36)) return false;
  const int bx = 128 / es;
  return tma2d_cdiv(c.s[0], bx) * tma2d_cdiv(c.s[1], 32 * kTmaBoxes) < (int64_t(1) << 31);
}

inline Tma2dGeom tma2d_geom(const Canon& c, int din) {
  Tma2dGeom g;
  g.R = int(c.s[0]);
  g.C = int(c.s[1]);
  g.bx = 128 / dtype_size(din);
  g.tilesR = int(tma2d_cdiv(g.R, g.bx));
  g.tiles = int64_t(g.tilesR) * tma2d_cdiv(g.C, 32 * kTmaBoxes);
  g.lda = c.sa[1];
  g.ldb = c.sb[0];
  return g;
}

// Origin of tile t: rows r0.., columns c0.. (tiles along R fastest, so that
// consecutive CTAs read neighbouring 128-byte pieces of the same columns).
TTC_HD void tma2d_origin(const Tma2dGeom& g, int64_t t, int* r0, int* c0) {
  *r0 = int(t % g.tilesR) * g.bx;
  *c0 = int(t / g.tilesR) * (32 * kTmaBoxes);
}

// Element j of lane `lane` in warp w for box k: row x = w + 8 j of the box,
// column y = lane (lanes store 32 consecutive elements of a B row).
// Byte position of element (x, y) of a box in shared memory (128-byte
// swizzle: the 16-byte chunk index XORed with the row's index mod 8).
TTC_HD int tma2d_smem_byte(int x, int y, int es) {
  return y * 128 + ((((x * es) >> 4) ^ (y & 7)) << 4) + ((x * es) & 15);
}

// Enqueue the kernel for the canonical problem of geometry g.  A must be
// 16-byte aligned for the TMA path; otherwise (and should a TMA wait give
// up) the kernel reads A directly.
cudaError_t launch_tma2d(int din, int dout, const void* A, void* B, const Tma2dGeom& g, const Epilogue& epi,
                         cudaStream_t s);

}  // namespace ttc
