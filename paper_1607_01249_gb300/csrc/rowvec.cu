// rowvec.cu -- the multi-row copy (perm keeps index 0, runs of LC elements,
// a tile one contiguous block of A) with each thread moving kRowVecK vectors
// of 16 bytes of A: twice the bytes in flight of the element-wise rowcopy
// for a quarter of its instructions, so that problems of a few tens of MB
// (GEMM packing panels) stream in fewer, larger CTAs.
#include <cuda_runtime.h>

#include "kernels_impl.cuh"
#include "rowvec.h"

namespace ttc {

namespace {

// V elements of B's type to memory at p, aligned to V x sizeof(T) (VIO) or
// element by element
template <class T, int V, bool VIO>
__device__ __forceinline__ void store_vec(T* p, const T (&v)[V]) {
  if constexpr (VIO && (V * sizeof(T)) % 16 == 0) {
#pragma unroll
    for (int i = 0; i < int(V * sizeof(T) / 16); ++i)
      reinterpret_cast<uint4*>(p)[i] = reinterpret_cast<const uint4*>(v)[i];
  } else if constexpr (VIO && V * sizeof(T) == 8) {
    *reinterpret_cast<uint2*>(p) = *reinterpret_cast<const uint2*>(v);
  } else if constexpr (VIO && V * sizeof(T) == 4) {
    *reinterpret_cast<uint32_t*>(p) = *reinterpret_cast<const uint32_t*>(v);
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) p[i] = v[i];
  }
}

template <class T, int V, bool VIO>
__device__ __forceinline__ void load_vec(const T* __restrict__ p, T (&v)[V]) {
  if constexpr (VIO && (V * sizeof(T)) % 16 == 0) {
#pragma unroll
    for (int i = 0; i < int(V * sizeof(T) / 16); ++i)
      reinterpret_cast<uint4*>(v)[i] = __ldg(reinterpret_cast<const uint4*>(p) + i);
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) v[i] = p[i];
  }
}

template <int DIN, int DOUT, int EK, bool VIO>
__global__ void __launch_bounds__(kThreads, EK == EK_FP8 ? 4 : 1) rowcopy_vec_kernel(const store_t<DIN>* __restrict__ A,
                                                               store_t<DOUT>* __restrict__ B,
                                                               const __grid_constant__ TileParams p) {
  using TI = store_t<DIN>;
  using TO = store_t<DOUT>;
  constexpr int V = rowvec_width(DIN);
  const int t = threadIdx.x;
  const float scale = cta_fp8_scale<EK>(p.epi);
  const TileCoord c = cta_tile_coord(p);
  const TI* Ab = A + c.baseA;
  TO* Bb = B + c.baseB;
  alignas(16) TI v[kRowVecK][V];
  alignas(16) TO bo[kRowVecK][V];
  walk_rows_vec(c, p, V, t, [&](int k, bool ok, int32_t offA, int32_t offB) {
    if (ok) {
      load_vec<TI, V, VIO>(Ab + offA, v[k]);
      if constexpr (ek_reads_b(EK)) {
#pragma unroll
        for (int i = 0; i < V; ++i) bo[k][i] = Bb[offB + i];
      }
    }
  });
  walk_rows_vec(c, p, V, t, [&](int k, bool ok, int32_t, int32_t offB) {
    if (ok) {
      alignas(16) TO r[V];
#pragma unroll
      for (int i = 0; i < V; ++i) r[i] = epilogue_k<DIN, DOUT, EK>(to_stage<DIN>(v[k][i]), bo[k][i], p.epi, scale);
      store_vec<TO, V, VIO>(Bb + offB, r);
    }
  });
}

template <int DIN, int DOUT>
struct RowVecL {
  template <int EK>
  struct L {
    static cudaError_t run(const void* A, void* B, const TileParams& p, bool vio, cudaStream_t s) {
      if (vio)
        rowcopy_vec_kernel<DIN, DOUT, EK, true><<<p.ntiles, kThreads, 0, s>>>(
            static_cast<const store_t<DIN>*>(A), static_cast<store_t<DOUT>*>(B), p);
      else
        rowcopy_vec_kernel<DIN, DOUT, EK, false><<<p.ntiles, kThreads, 0, s>>>(
            static_cast<const store_t<DIN>*>(A), static_cast<store_t<DOUT>*>(B), p);
      ++g_launches;
      return cudaGetLastError();
    }
  };
};

}  // namespace

cudaError_t launch_rowcopy_vec(int din, int dout, const void* A, void* B, const TileParams& p, cudaStream_t s) {
  const int V = rowvec_width(din);
  if (V == 0) return cudaErrorInvalidValue;
  // 16-byte loads need A's base on a 16-byte boundary and the stores B's on
  // V elements of B's type (the planner made every tile offset a multiple
  // of V)
  const size_t sb = size_t(V) * size_t(dtype_size(dout));
  const bool vio = reinterpret_cast<uintptr_t>(A) % 16 == 0 && reinterpret_cast<uintptr_t>(B) % (sb < 16 ? sb : 16) == 0;
#define TTC_RV(I, O) \
  if (din == I && dout == O) return with_ek<I, O, RowVecL<I, O>::template L>(p.epi.mode, p.epi.beta_nz, A, B, p, vio, s);
  TTC_RV(DT_F32, DT_F32)
  TTC_RV(DT_F32, DT_F64)
  TTC_RV(DT_F32, DT_BF16)
  TTC_RV(DT_F32, DT_E4M3)
  TTC_RV(DT_F64, DT_F64)
  TTC_RV(DT_F64, DT_F32)
  TTC_RV(DT_BF16, DT_BF16)
  TTC_RV(DT_BF16, DT_F32)
  TTC_RV(DT_BF16, DT_E4M3)
#undef TTC_RV
  return cudaErrorInvalidValue;
}

}  // namespace ttc
