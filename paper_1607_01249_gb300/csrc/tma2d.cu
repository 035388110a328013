// tma2d.cu -- the TMA-staged tile of a two-index transpose (section 2.2's
// macro-tile with its load side done by the tensor memory accelerator).
//
// One CTA per tile of bx x 128 elements (tma2d.h): one thread issues
// kTmaBoxes `cp.async.bulk.tensor.2d` copies of bx x 32 boxes of A (a tensor
// map over this GPU's memory, 128-byte swizzle, zero fill past the edges)
// against one mbarrier; the 256 threads then read the boxes along B's
// stride-1 index and store 32 consecutive B elements per warp instruction,
// with the epilogue of Eq. 1.  The swizzle spreads a column read of a box
// over 8 banks groups (4-way conflicts at most).  The wait for the copies is
// bounded: should it give up, or should A not be 16-byte aligned, the CTA
// reads its elements of A directly instead (the same results).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "kernels_impl.cuh"
#include "tma2d.h"

namespace ttc {

namespace {

constexpr int kTmaThreads = 256;
constexpr int kTmaSmem = 1024 + kTmaBoxes * kTmaBoxBytes + 64;
constexpr uint32_t kTmaWaitLimit = 1u << 22;

__device__ __forceinline__ bool tma_bar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < kTmaWaitLimit; ++i) {
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

template <int DIN, int DOUT, int EK>
__global__ void __launch_bounds__(kTmaThreads) tma2d_kernel(const __grid_constant__ CUtensorMap mapA,
                                                            const store_t<DIN>* __restrict__ A,
                                                            store_t<DOUT>* __restrict__ B,
                                                            const __grid_constant__ Tma2dGeom g,
                                                            const __grid_constant__ Epilogue epi, int use_tma) {
  using TI = store_t<DIN>;
  using TO = store_t<DOUT>;
  constexpr int es = int(sizeof(TI));
  constexpr int bx = 128 / es;
  extern __shared__ uint8_t raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  const uint32_t bar = uint32_t(__cvta_generic_to_shared(sm + kTmaBoxes * kTmaBoxBytes));
  const float scale = cta_fp8_scale<EK>(epi);
  int r0, c0;
  tma2d_origin(g, blockIdx.x, &r0, &c0);
  int nb = 0;
#pragma unroll
  for (int k = 0; k < kTmaBoxes; ++k) nb += c0 + 32 * k < g.C ? 1 : 0;
  bool staged = false;
  if (use_tma) {
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(nb * kTmaBoxBytes)
                   : "memory");
      for (int k = 0; k < nb; ++k)
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];" ::"r"(uint32_t(__cvta_generic_to_shared(sm + k * kTmaBoxBytes))),
            "l"(reinterpret_cast<uint64_t>(&mapA)), "r"(r0), "r"(c0 + 32 * k), "r"(bar)
            : "memory");
    }
    staged = !__syncthreads_or(!tma_bar_wait(bar, 0));
    if (!staged) {
      // the copies may still land: wait for them (bounded) before the CTA
      // ends, and read A directly meanwhile
      tma_bar_wait(bar, 0);
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < nb; ++k) {
    const int c = c0 + 32 * k + lane;
    const uint8_t* box = sm + k * kTmaBoxBytes;
#pragma unroll
    for (int j = 0; j < bx / 8; ++j) {
      const int x = w + 8 * j;
      const int r = r0 + x;
      if (r >= g.R || c >= g.C) continue;
      const TI a = staged ? *reinterpret_cast<const TI*>(box + tma2d_smem_byte(x, lane, es))
                          : __ldg(A + (int64_t(r) + int64_t(c) * g.lda));
      TO* bp = B + (int64_t(c) + int64_t(r) * g.ldb);
      TO b = TO();
      if constexpr (ek_reads_b(EK)) b = *bp;
      *bp = epilogue_k<DIN, DOUT, EK>(to_stage<DIN>(a), b, epi, scale);
    }
  }
}

template <int DIN, int DOUT>
struct Tma2dL {
  template <int EK>
  struct L {
    static cudaError_t run(const CUtensorMap& m, const void* A, void* B, const Tma2dGeom& g, const Epilogue& e,
                           int use_tma, cudaStream_t s) {
      static_assert(kTmaSmem <= 48 * 1024, "dynamic shared memory within the default limit");
      tma2d_kernel<DIN, DOUT, EK><<<unsigned(g.tiles), kTmaThreads, kTmaSmem, s>>>(
          m, static_cast<const store_t<DIN>*>(A), static_cast<store_t<DOUT>*>(B), g, e, use_tma);
      ++g_launches;
      return cudaGetLastError();
    }
  };
};

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled tma_encode_fn() {
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

}  // namespace

cudaError_t launch_tma2d(int din, int dout, const void* A, void* B, const Tma2dGeom& g, const Epilogue& epi,
                         cudaStream_t s) {
  if (g.tiles <= 0) return cudaSuccess;
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  int use_tma = 0;
  EncodeTiled fn = tma_encode_fn();
  if (fn && reinterpret_cast<uintptr_t>(A) % 16 == 0) {
    const int es = dtype_size(din);
    const cuuint64_t dims[2] = {cuuint64_t(g.R), cuuint64_t(g.C)};
    const cuuint64_t strides[1] = {cuuint64_t(g.lda) * cuuint64_t(es)};
    const cuuint32_t box[2] = {cuuint32_t(g.bx), 32};
    const cuuint32_t el[2] = {1, 1};
    use_tma = fn(&m, din == DT_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                 const_cast<void*>(A), dims, strides, box, el, CU_TENSOR_MAP_INTERLEAVE_NONE,
                 CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS
                  ? 1
                  : 0;
  }
#define TTC_TMA(I, O)                                                                                   \
  if (din == I && dout == O)                                                                            \
    return with_ek<I, O, Tma2dL<I, O>::template L>(epi.mode, epi.beta_nz, m, A, B, g, epi, use_tma, s);
  TTC_TMA(DT_F32, DT_F32)
  TTC_TMA(DT_F32, DT_F64)
  TTC_TMA(DT_F32, DT_BF16)
  TTC_TMA(DT_F32, DT_E4M3)
  TTC_TMA(DT_F64, DT_F64)
  TTC_TMA(DT_F64, DT_F32)
#undef TTC_TMA
  return cudaErrorInvalidValue;
}

}  // namespace ttc
