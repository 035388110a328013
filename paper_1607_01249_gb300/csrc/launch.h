// launch.h -- host entry points of the kernels (implemented in kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "ttc_internal.h"

namespace ttc {

bool pair_supported(int din, int dout);
int copy_vec_width(int din, int dout);
cudaError_t launch_tile(int din, int dout, const void* A, void* B, const TileParams& p, int smem,
                        cudaStream_t s);
cudaError_t launch_tile_slots(int din, int dout, const void* A, void* B, const TileParams& p, int smem,
                              cudaStream_t s);
cudaError_t launch_tile2(int din, int dout, int ju, int jw, const void* A, void* B, const TileParams& p,
                         int smem, cudaStream_t s);
// packed-lane tile kernel with nt (256 or 512) threads per CTA and ju / jw
// (1, 2, 4) run chunks per thread on the load / store side
cudaError_t launch_tilep(int din, int dout, int nt, int ju, int jw, const void* A, void* B, const TileParams& p,
                         int smem, cudaStream_t s);
// packed rows (C tiles copied row by row without staging), j positions per
// thread in each row (1, 2, 4, 8, 16; at most the kernel's slots per thread)
cudaError_t launch_rowsp(int din, int dout, int j, const void* A, void* B, const TileParams& p, cudaStream_t s);
cudaError_t launch_rowcopy(int din, int dout, const void* A, void* B, const TileParams& p, cudaStream_t s);
cudaError_t launch_copy(int din, int dout, int vec, const void* A, void* B, const RowParams& p,
                        cudaStream_t s);
// FP8 pre-pass: max |alpha a| over A's sub-tensor into *amax_bits (which
// must start at 0); clear_bits (may be null) is set to 0 on the way.
cudaError_t launch_amax(int din, const void* A, const RowParams& p, float alpha_f, uint32_t* amax_bits,
                        uint32_t* clear_bits, cudaStream_t s);
int64_t launch_count();
// a kernel that stays busy for ns nanoseconds (bounded), for watchdog tests
cudaError_t launch_delay(uint64_t ns, cudaStream_t s);

}  // namespace ttc
