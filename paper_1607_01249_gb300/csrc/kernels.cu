// kernels.cu -- launch plumbing of the kernels (grid sizing, launch counter,
// dispatch to the per-dtype-pair instantiations in kern_*.cu).  The kernels
// themselves are in kernels_impl.cuh.
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>

#include "kernels_impl.cuh"
#include "launch.h"

namespace ttc {

std::atomic<int64_t> g_launches{0};

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
// largest dynamic shared memory each kernel has been allowed on each device:
// the attribute is an upper bound, so it is only ever raised
std::map<std::pair<const void*, int>, int> g_smem_attr;

}  // namespace

cudaError_t grid_for(const void* fn, int smem, int64_t work, int* grid) {
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  int blocks = 0;
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    if (smem > 48 * 1024) {
      int& cur = g_smem_attr[{fn, dev}];
      if (smem > cur) {
        err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (err != cudaSuccess) return err;
        cur = smem;
      }
    }
    auto it = g_occ.find({fn, smem, dev});
    if (it != g_occ.end()) blocks = it->second;
  }
  if (blocks == 0) {
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


// The dtype pairs with kernels (one kern_<in>_<out>.cu each): the paper's
// s, d, sd, ds, c, z, cz, zc (section 2.1) plus the BF16 and FP8 downcasts.
#define TTC_PAIRS(X)                                                                                      \
  X(DT_F32, DT_F32, f32_f32) X(DT_F32, DT_F64, f32_f64) X(DT_F32, DT_BF16, f32_bf16)                     \
  X(DT_F32, DT_E4M3, f32_e4m3) X(DT_F64, DT_F64, f64_f64) X(DT_F64, DT_F32, f64_f32)                     \
  X(DT_BF16, DT_BF16, bf16_bf16) X(DT_BF16, DT_F32, bf16_f32) X(DT_BF16, DT_E4M3, bf16_e4m3)             \
  X(DT_C64, DT_C64, c64_c64) X(DT_C128, DT_C128, c128_c128) X(DT_C64, DT_C128, c64_c128)                 \
  X(DT_C128, DT_C64, c128_c64)

#define TTC_DECLARE(I, O, P)                                                                              \
  cudaError_t launch_tile_##P(const void*, void*, const TileParams&, int, cudaStream_t);                  \
  cudaError_t launch_tile_slots_##P(const void*, void*, const TileParams&, int, cudaStream_t);            \
  cudaError_t launch_tile2_##P(int, int, const void*, void*, const TileParams&, int, cudaStream_t);       \
  cudaError_t launch_tilep_##P(int, int, int, const void*, void*, const TileParams&, int, cudaStream_t);  \
  cudaError_t launch_copy_##P(int, const void*, void*, const RowParams&, cudaStream_t);                   \
  cudaError_t launch_rowsp_##P(int, const void*, void*, const TileParams&, cudaStream_t);                  \
  cudaError_t launch_rowcopy_##P(const void*, void*, const TileParams&, cudaStream_t);
TTC_PAIRS(TTC_DECLARE)
#undef TTC_DECLARE

bool pair_supported(int din, int dout) {
#define TTC_IS(I, O, P) \
  if (din == I && dout == O) return true;
  TTC_PAIRS(TTC_IS)
#undef TTC_IS
  return false;
}

// Widest vector (elements) the copy kernel uses for a pair: 16 bytes of the
// wider of the two types.
int copy_vec_width(int din, int dout) {
  int w = dtype_size(din) > dtype_size(dout) ? dtype_size(din) : dtype_size(dout);
  return 16 / w;
}

cudaError_t launch_tile_slots(int din, int dout, const void* A, void* B, const TileParams& p, int smem,
                              cudaStream_t s) {
#define TTC_GO(I, O, P) \
  if (din == I && dout == O) return launch_tile_slots_##P(A, B, p, smem, s);
  TTC_PAIRS(TTC_GO)
#undef TTC_GO
  return cudaErrorInvalidValue;
}

cudaError_t launch_tile(int din, int dout, const void* A, void* B, const TileParams& p, int smem,
                        cudaStream_t s) {
#define TTC_GO(I, O, P) \
  if (din == I && dout == O) return launch_tile_##P(A, B, p, smem, s);
  TTC_PAIRS(TTC_GO)
#undef TTC_GO
  return cudaErrorInvalidValue;
}

cudaError_t launch_tile2(int din, int dout, int ju, int jw, const void* A, void* B, const TileParams& p,
                         int smem, cudaStream_t s) {
#define TTC_GO(I, O, P) \
  if (din == I && dout == O) return launch_tile2_##P(ju, jw, A, B, p, smem, s);
  TTC_PAIRS(TTC_GO)
#undef TTC_GO
  return cudaErrorInvalidValue;
}

cudaError_t launch_tilep(int din, int dout, int nt, int ju, int jw, const void* A, void* B, const TileParams& p,
                         int smem, cudaStream_t s) {
#define TTC_GO(I, O, P) \
  if (din == I && dout == O) return launch_tilep_##P(nt, ju, jw, A, B, p, smem, s);
  TTC_PAIRS(TTC_GO)
#undef TTC_GO
  return cudaErrorInvalidValue;
}

cudaError_t launch_copy(int din, int dout, int vec, const void* A, void* B, const RowParams& p,
                        cudaStream_t s) {
#define TTC_GO(I, O, P) \
  if (din == I && dout == O) return launch_copy_##P(vec, A, B, p, s);
  TTC_PAIRS(TTC_GO)
#undef TTC_GO
  return cudaErrorInvalidValue;
}

cudaError_t launch_rowsp(int din, int dout, int j, const void* A, void* B, const TileParams& p, cudaStream_t s) {
#define TTC_GO(I, O, P) \
  if (din == I && dout == O) return launch_rowsp_##P(j, A, B, p, s);
  TTC_PAIRS(TTC_GO)
#undef TTC_GO
  return cudaErrorInvalidValue;
}

cudaError_t launch_rowcopy(int din, int dout, const void* A, void* B, const TileParams& p, cudaStream_t s) {
#define TTC_GO(I, O, P) \
  if (din == I && dout == O) return launch_rowcopy_##P(A, B, p, s);
  TTC_PAIRS(TTC_GO)
#undef TTC_GO
  return cudaErrorInvalidValue;
}

cudaError_t launch_amax(int din, const void* A, const RowParams& p, float alpha_f, uint32_t* amax_bits,
                        uint32_t* clear_bits, cudaStream_t s) {
  if (din == DT_F32) return launch_amax_t<DT_F32>(A, p, alpha_f, amax_bits, clear_bits, s);
  if (din == DT_BF16) return launch_amax_t<DT_BF16>(A, p, alpha_f, amax_bits, clear_bits, s);
  return cudaErrorInvalidValue;
}

int64_t launch_count() { return g_launches.load(); }

// One thread that stays busy for `ns` nanoseconds of the device's global
// timer and returns: bounded by the timer and by an iteration cap, whichever
// ends first.  Used only to make a server epoch outlast its watchdog in tests.
__global__ void delay_kernel(uint64_t ns) {
  uint64_t t0 = 0, t = 0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  // every iteration takes well over 10 ns (a timer read and a sleep), so
  // ns / 10 iterations cover the requested time even if the sleeps are short
  const uint64_t cap = ns / 10 + 1000;
  for (uint64_t i = 0; i < cap; ++i) {
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 >= ns) break;
    __nanosleep(1000);
  }
}

cudaError_t launch_delay(uint64_t ns, cudaStream_t s) {
  delay_kernel<<<1, 1, 0, s>>>(ns);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ttc
