// kernels.cuh -- device-side building blocks shared by the single-plan
// kernels and the batched persistent kernel.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "ttc_internal.h"

namespace ttc {

// Storage type of each dtype in memory, and the type a tile is staged in
// shared memory (bf16 is widened exactly to f32 on the way in).
template <int DT> struct Store;
template <> struct Store<DT_F32> { using T = float; };
template <> struct Store<DT_F64> { using T = double; };
template <> struct Store<DT_BF16> { using T = uint16_t; };
template <> struct Store<DT_E4M3> { using T = uint8_t; };

template <int DT> struct Stage { using T = float; };
template <> struct Stage<DT_F64> { using T = double; };

template <int DT> using store_t = typename Store<DT>::T;
template <int DT> using stage_t = typename Stage<DT>::T;

template <int DT>
__device__ __forceinline__ stage_t<DT> to_stage(store_t<DT> x) {
  if constexpr (DT == DT_BF16) return __uint_as_float(uint32_t(x) << 16);
  else return x;
}

template <int DT>
__device__ __forceinline__ store_t<DT> ldg_elem(const store_t<DT>* p) {
  return __ldg(p);
}

// value of a B element as the compute type
template <int DT>
__device__ __forceinline__ float out_as_float(store_t<DT> x) {
  if constexpr (DT == DT_BF16) return __uint_as_float(uint32_t(x) << 16);
  else return float(x);
}

template <int DIN, int DOUT>
struct ComputeIsF64 {
  static constexpr bool value = (DIN == DT_F64 || DOUT == DT_F64);
};

// FP8 scale of one execution: caller-supplied, or fl32(amax/448) with the
// degenerate cases mapped to 1.
__device__ __forceinline__ float fp8_scale_of(const Epilogue& e) {
  if (e.scale_in) return *e.scale_in;
  const float amax = __uint_as_float(*e.amax_bits);
  if (!(amax > 0.f) || isinf(amax)) return 1.f;
  const float s = __fdiv_rn(amax, 448.f);
  return s == 0.f ? 1.f : s;
}

// The alpha/beta update of Eq. 1 for one element, in the compute type, then
// one rounding to B's type.  `b` is only meaningful when e.beta_nz.
template <int DIN, int DOUT>
__device__ __forceinline__ store_t<DOUT> epilogue(stage_t<DIN> a, store_t<DOUT> b, const Epilogue& e,
                                                  float scale) {
  if constexpr (DOUT == DT_E4M3) {
    const float v = __fmul_rn(e.alpha_f, float(a));
    const float q = __fdiv_rn(v, scale);
    return store_t<DOUT>(__nv_cvt_float_to_fp8(q, __NV_SATFINITE, __NV_E4M3));
  } else {
    if (e.mode == MODE_BITCOPY) {
      // same dtype in and out (the planner guarantees it)
      if constexpr (DIN == DT_BF16 && DOUT == DT_BF16) return store_t<DOUT>(__float_as_uint(a) >> 16);
      else if constexpr (DIN == DOUT) return a;
    }
    if constexpr (ComputeIsF64<DIN, DOUT>::value) {
      double r = __dmul_rn(e.alpha_d, double(a));
      if (e.beta_nz) r = __fma_rn(e.beta_d, double(b), r);
      if constexpr (DOUT == DT_F64) return r;
      else return __double2float_rn(r);
    } else {
      float r = __fmul_rn(e.alpha_f, float(a));
      if (e.beta_nz) r = __fmaf_rn(e.beta_f, out_as_float<DOUT>(b), r);
      if constexpr (DOUT == DT_BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(r));
      else return r;
    }
  }
}

// The update of Eq. 1 with the mode fixed at compile time (no per-element
// branches): EK_COPY moves bits (alpha = 1, beta = 0, same type), EK_SCALE
// r = alpha*a, EK_AXPBY r = fma(beta, b, alpha*a), EK_FP8 the scaled E4M3 code.
enum EpiKind : int { EK_COPY = 0, EK_SCALE = 1, EK_AXPBY = 2, EK_FP8 = 3 };

template <int DIN, int DOUT, int EK>
__device__ __forceinline__ store_t<DOUT> epilogue_k(stage_t<DIN> a, store_t<DOUT> b, const Epilogue& e,
                                                    float scale) {
  if constexpr (EK == EK_FP8) {
    const float v = __fmul_rn(e.alpha_f, float(a));
    return store_t<DOUT>(__nv_cvt_float_to_fp8(__fdiv_rn(v, scale), __NV_SATFINITE, __NV_E4M3));
  } else if constexpr (EK == EK_COPY) {
    if constexpr (DIN == DT_BF16 && DOUT == DT_BF16) return store_t<DOUT>(__float_as_uint(a) >> 16);
    else return a;
  } else if constexpr (ComputeIsF64<DIN, DOUT>::value) {
    double r = __dmul_rn(e.alpha_d, double(a));
    if constexpr (EK == EK_AXPBY) r = __fma_rn(e.beta_d, double(b), r);
    if constexpr (DOUT == DT_F64) return r;
    else return __double2float_rn(r);
  } else {
    float r = __fmul_rn(e.alpha_f, float(a));
    if constexpr (EK == EK_AXPBY) r = __fmaf_rn(e.beta_f, out_as_float<DOUT>(b), r);
    if constexpr (DOUT == DT_BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(r));
    else return r;
  }
}

template <typename T, int N>
struct alignas(sizeof(T) * N) VecT {
  T v[N];
};

// ------------------------------------------------------------------------
// Index walks of the tile schedule, shared by the kernels and the host-side
// schedule checker (simulate.cu), so that the checker verifies exactly the
// addresses the kernels use.

struct TileCoord {
  int64_t baseA, baseB;   // element offsets of the tile's first element
  int remA, remB;         // valid extents of la and lb in this tile (cut indices)
};

TTC_HD TileCoord tile_coord(uint32_t tid, const TileParams& p) {
  TileCoord c{0, 0, p.LA, p.LB};
  uint32_t r = tid;
  for (int i = 0; i < p.ngrid; ++i) {
    const uint32_t q = fast_div(r, p.g[i].div);
    const uint32_t d = r - q * p.g[i].div.d;
    r = q;
    c.baseA += int64_t(d) * p.g[i].stepA;
    c.baseB += int64_t(d) * p.g[i].stepB;
    const int rem = p.g[i].s - int(d) * p.g[i].t;
    const int ext = rem < p.g[i].t ? rem : p.g[i].t;
    if (p.g[i].kind == 1) c.remA = p.fullA * ext;
    else if (p.g[i].kind == 2) c.remB = p.fullB * ext;
  }
  return c;
}

// Read order: (u, lb) with u = la*LC + lc.  f(k, A offset in tile, smem position)
template <int K = kTileK, class F>
TTC_HD void walk_read(const TileCoord& c, const TileParams& p, const int32_t* tabA, int u0, int lb0, F&& f,
                      bool need_offset = true) {
  const int limU = c.remA * p.LC;
  int u = u0, lb = lb0;
#if defined(__CUDA_ARCH__)
  // opaque: keeps the compiler from precomputing all kTileK index pairs once
  // per thread and holding them in registers across tiles
  asm volatile("" : "+r"(u), "+r"(lb));
#endif
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (lb < c.remB && u < limU) {
      int32_t off = 0;
      if (need_offset) off = u * p.saU + (p.crossA_tab ? tabA[lb] : lb * p.crossA_lin);
      f(k, off, lb * p.P + u);
    }
    u += p.rd_du;
    lb += p.rd_dlb;
    if (u >= p.U) { u -= p.U; ++lb; }
  }
}

// Write order: (lc, lb, la).  f(k, B offset in tile, smem position)
template <int K = kTileK, class F>
TTC_HD void walk_write(const TileCoord& c, const TileParams& p, const int32_t* tabB, int lc0, int lb0, int la0,
                       F&& f) {
  int lc = lc0, lb = lb0, la = la0;
#if defined(__CUDA_ARCH__)
  asm volatile("" : "+r"(lc), "+r"(lb), "+r"(la));
#endif
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (la < c.remA && lb < c.remB) {
      const int32_t off = (lb * p.LC + lc) * p.sbV + (p.crossB_tab ? tabB[la] : la * p.crossB_lin);
      f(k, off, lb * p.P + la * p.LC + lc);
    }
    lc += p.wr_dlc; lb += p.wr_dlb; la += p.wr_dla;
    if (lc >= p.LC) { lc -= p.LC; ++lb; }
    if (lb >= p.LB) { lb -= p.LB; ++la; }
  }
}

// Warp-mapped walks (tile2_kernel).  Read: lanes along u (JU chunks of 32),
// warps along lb.  Write: lanes along v (JW chunks), warps along la.
template <int JU, int K = kTileK, class F>
TTC_HD void walk2_read(const TileCoord& c, const TileParams& p, const int32_t* tabA, int lane, int warp,
                       F&& f) {
  constexpr int RR = K / JU;
  const int limU = c.remA * p.LC;
#pragma unroll
  for (int i = 0; i < RR; ++i) {
    const int r = warp + 8 * i;
    if (r < c.remB) {
      const int32_t row = p.crossA_tab ? tabA[r] : r * p.crossA_lin;
#pragma unroll
      for (int j = 0; j < JU; ++j) {
        const int u = lane + 32 * j;
        if (u < limU) f(i * JU + j, row + u * p.saU, r * p.P + u);
      }
    }
  }
}

// per-lane constants of the write walk: shared-memory offset and B offset of
// the lane's run positions v = lane + 32 j
template <int JW>
TTC_HD void walk2_lane_consts(const TileParams& p, int lane, int (&spre)[JW], int32_t (&voff)[JW]) {
#pragma unroll
  for (int j = 0; j < JW; ++j) {
    const int vv = lane + 32 * j;
    spre[j] = (vv / p.LC) * p.P + vv % p.LC;
    voff[j] = vv * p.sbV;
  }
}

template <int JW, int K = kTileK, class F>
TTC_HD void walk2_write(const TileCoord& c, const TileParams& p, const int32_t* tabB, int lane, int warp,
                        const int (&spre)[JW], const int32_t (&voff)[JW], F&& f) {
  constexpr int RW = K / JW;
  const int limV = c.remB * p.LC;
#pragma unroll
  for (int i = 0; i < RW; ++i) {
    const int la = warp + 8 * i;
    if (la < c.remA) {
      const int32_t row = p.crossB_tab ? tabB[la] : la * p.crossB_lin;
#pragma unroll
      for (int j = 0; j < JW; ++j)
        if (lane + 32 * j < limV) f(i * JW + j, row + voff[j], spre[j] + la * p.LC);
    }
  }
}

// Unit-stride warp-mapped walks (tile3_kernel: both runs have stride 1).
// FULL: the tile is interior (no cut index is short), so no per-element test.
template <int JU, int K, bool FULL, class F>
TTC_HD void walk3_read(const TileCoord& c, const TileParams& p, const int32_t* tabA, int lane, int warp,
                       F&& f) {
  constexpr int RR = K / JU;
  const int limU = c.remA * p.LC;
#pragma unroll
  for (int i = 0; i < RR; ++i) {
    const int r = warp + 8 * i;
    if (FULL ? (r < p.LB) : (r < c.remB)) {
      const int32_t row = (p.crossA_tab ? tabA[r] : r * p.crossA_lin) + lane;
      const int pos = r * p.P + lane;
#pragma unroll
      for (int j = 0; j < JU; ++j)
        if (FULL ? (32 * j < p.U - lane) : (32 * j < limU - lane)) f(i * JU + j, row + 32 * j, pos + 32 * j);
    }
  }
}

template <int JW, int K, bool FULL, class F>
TTC_HD void walk3_write(const TileCoord& c, const TileParams& p, const int32_t* tabB, int lane, int warp,
                        const int (&spre)[JW], F&& f) {
  constexpr int RW = K / JW;
  const int limV = c.remB * p.LC;
#pragma unroll
  for (int i = 0; i < RW; ++i) {
    const int la = warp + 8 * i;
    if (FULL ? (la < p.LA) : (la < c.remA)) {
      const int32_t row = (p.crossB_tab ? tabB[la] : la * p.crossB_lin) + lane;
      const int spos = la * p.LC;
#pragma unroll
      for (int j = 0; j < JW; ++j)
        if (FULL ? (32 * j < p.W - lane) : (32 * j < limV - lane)) f(i * JW + j, row + 32 * j, spre[j] + spos);
    }
  }
}

// Copy schedule: the row and chunk of a work item, as element offsets.
struct RowCoord {
  int64_t offA, offB, start, end;
};

TTC_HD RowCoord row_coord(uint32_t item, const RowParams& p) {
  const uint32_t row = fast_div(item, p.chunks);
  const uint32_t ch = item - row * p.chunks.d;
  RowCoord rc{0, 0, 0, 0};
  uint32_t r = row;
  for (int i = 0; i < p.nrd; ++i) {
    const uint32_t q = fast_div(r, p.div[i]);
    const uint32_t d = r - q * p.div[i].d;
    r = q;
    rc.offA += int64_t(d) * p.stA[i];
    rc.offB += int64_t(d) * p.stB[i];
  }
  rc.start = int64_t(ch) * p.chunk;
  rc.end = rc.start + p.chunk < p.len ? rc.start + p.chunk : p.len;
  return rc;
}

}  // namespace ttc
