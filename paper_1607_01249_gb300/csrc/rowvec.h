// rowvec.h -- the multi-row copy with 16-byte accesses (rowvec.cu): its
// element walk, shared by the kernel and the host schedule checker.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"
#include "ttc_internal.h"

namespace ttc {

// Vectors per thread of the vector multi-row copy.
constexpr int kRowVecK = 8;

// Elements per 16-byte load of A (0: the type takes no vector copy).
constexpr int rowvec_width(int din) {
  return din == DT_F32 ? 4 : din == DT_F64 ? 2 : din == DT_BF16 ? 8 : 0;
}

// The multi-row copy tile (perm keeps index 0; LC x remA elements, one
// contiguous block of A, rows of LC elements in B at the linear cross offset
// crossB_lin) in vectors of V consecutive elements: thread t takes the
// vectors starting at u = V (t + kThreads k), k < kRowVecK.  LC is a
// multiple of V, so a vector never straddles two rows.  f(k, ok, A offset,
// B offset) of the vector's first element.
template <class PT, class F>
TTC_HD void walk_rows_vec(const TileCoord& c, const PT& p, int V, int t, F&& f) {
  const int limU = c.remA * p.LC;
#pragma unroll
  for (int k = 0; k < kRowVecK; ++k) {
    const int u = V * (t + kThreads * k);
    const bool ok = u < limU;
    const int la = ok ? int(fast_div(uint32_t(u), p.divLC)) : 0;
    const int lc = u - la * p.LC;
    f(k, ok, ok ? u : 0, ok ? lc + la * p.crossB_lin : 0);
  }
}

// Enqueue the vector multi-row copy (16-byte accesses where the bases allow,
// element accesses otherwise, the same walk).
cudaError_t launch_rowcopy_vec(int din, int dout, const void* A, void* B, const TileParams& p, cudaStream_t s);

}  // namespace ttc
