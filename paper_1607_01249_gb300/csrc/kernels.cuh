// kernels.cuh -- device-side building blocks shared by the single-plan
// kernels and the batched persistent kernel.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fpint.h"
#include "ttc_internal.h"

namespace ttc {

// Storage type of each dtype in memory, and the type a tile is staged in
// shared memory (bf16 is widened exactly to f32 on the way in).
template <int DT> struct Store;
template <> struct Store<DT_F32> { using T = float; };
template <> struct Store<DT_F64> { using T = double; };
template <> struct Store<DT_BF16> { using T = uint16_t; };
template <> struct Store<DT_E4M3> { using T = uint8_t; };
template <> struct Store<DT_C64> { using T = float2; };     // (real, imaginary)
template <> struct Store<DT_C128> { using T = double2; };

template <int DT> struct Stage { using T = float; };
template <> struct Stage<DT_F64> { using T = double; };
template <> struct Stage<DT_C64> { using T = float2; };
template <> struct Stage<DT_C128> { using T = double2; };

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

// a binary32 or binary64 value as binary64 (exact)
template <typename T>
__device__ __forceinline__ double as_f64(T x) {
  if constexpr (sizeof(T) == 4) return widen_f32(x);
  else return x;
}

// fl64(alpha * x) with the FP64 pipe kept for the fused multiply-adds that
// follow (the complex update: two products and up to six fused
// multiply-adds per element): the integer product of fpint.h when alpha and
// x are normal and so is the result, else the hardware multiply (out of
// line, so that it is issued only by the lanes that need it).  Measured on
// double-complex data: 2480 -> 3078 GB/s with beta, 3254 -> 4388 without.
static __device__ __noinline__ double dmul_hw(double c, double x) { return __dmul_rn(c, x); }

__device__ __forceinline__ double alpha_mul(const Epilogue& e, double x) {
  double r;
  if (e.alpha_k.ok && dmul_normal(e.alpha_k, x, &r)) return r;
  return dmul_hw(e.alpha_d, x);
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

// The E4M3 code (RNE, satfinite) of fl32(v / s), s > 0 finite, without a
// division per element.  q = fl32(v * fl32(1/s)) differs from fl32(v / s) by
// at most 2.5 binary32 ulps (two roundings of relative size 2^-24 each, and
// the quotient's own half ulp).  Take q moved down and up by 2^-20 of its
// magnitude (at least 4 ulps; both ends keep q's sign): when the two ends
// have the same code, no E4M3 rounding boundary lies between them, and since
// rounding to nearest with saturation is monotonic, every value in the band
// (q and fl32(v / s) among them) has that code.  Otherwise (near a boundary,
// a zero of negative sign, infinities, NaN, a reciprocal that overflows) the
// quotient is formed by an IEEE division.  One paired conversion per element.
__device__ __forceinline__ uint8_t e4m3_of_quotient(float v, float s, float r) {
  const float q = __fmul_rn(v, r);
  const float d = __fmul_rn(fabsf(q), 0x1p-20f);
  const __nv_fp8x2_storage_t lh =
      __nv_cvt_float2_to_fp8x2(make_float2(__fsub_rn(q, d), __fadd_rn(q, d)), __NV_SATFINITE, __NV_E4M3);
  const uint8_t lo = uint8_t(lh & 0xffu);
  if (lo == uint8_t(lh >> 8) && q == q && r < __int_as_float(0x7f800000)) return lo;
  return uint8_t(__nv_cvt_float_to_fp8(__fdiv_rn(v, s), __NV_SATFINITE, __NV_E4M3));
}

// The alpha/beta update of Eq. 1 for one element, in the compute type, then
// one rounding to B's type.  `b` is only meaningful when e.beta_nz.
template <int DIN, int DOUT>
__device__ __forceinline__ store_t<DOUT> epilogue(stage_t<DIN> a, store_t<DOUT> b, const Epilogue& e,
                                                  float scale) {
  if constexpr (DOUT == DT_E4M3) {
    const float v = __fmul_rn(e.alpha_f, float(a));
    return store_t<DOUT>(e4m3_of_quotient(v, scale, __frcp_rn(scale)));
  } else {
    if (e.mode == MODE_BITCOPY) {
      // same dtype in and out (the planner guarantees it)
      if constexpr (DIN == DT_BF16 && DOUT == DT_BF16) return store_t<DOUT>(__float_as_uint(a) >> 16);
      else if constexpr (DIN == DOUT) return a;
    }
    if constexpr (ComputeIsF64<DIN, DOUT>::value) {
      double r = __dmul_rn(e.alpha_d, as_f64(a));
      if (e.beta_nz) r = __fma_rn(e.beta_d, as_f64(b), r);
      if constexpr (DOUT == DT_F64) return r;
      else return narrow_f64_rn(r);
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
// EK_RT / EK_RT_B: the mode is read at run time (the batch body, one kernel
// for every problem), without / with B read.
enum EpiKind : int { EK_COPY = 0, EK_SCALE = 1, EK_AXPBY = 2, EK_FP8 = 3, EK_RT = 4, EK_RT_B = 5 };

// whether an epilogue kind reads B
constexpr bool ek_reads_b(int ek) { return ek == EK_AXPBY || ek == EK_RT_B; }

// Complex update (the paper's c, z, cz, zc types), in double-complex when
// either side is double-complex, else in single-complex, with this fixed
// sequence of roundings (ar, ai = alpha; br, bi = beta; (x, y) = a; (u, v) = b):
//   re = fl(ar*x), im = fl(ar*y); if ai != 0: re = fma(-ai, y, re), im = fma(ai, x, im)
//   EK_AXPBY: re = fma(br, u, re), im = fma(br, v, im);
//             if bi != 0: re = fma(-bi, v, re), im = fma(bi, u, im)
// then one rounding per part to B's type.  With real scalars the cross terms
// are skipped, so each part is updated exactly as a real tensor would be.
template <int DIN, int DOUT, int EK>
__device__ __forceinline__ store_t<DOUT> epilogue_complex(stage_t<DIN> a, store_t<DOUT> b, const Epilogue& e) {
  if constexpr (DIN == DT_C128 || DOUT == DT_C128) {
    const double x = as_f64(a.x), y = as_f64(a.y);      // single-complex widens exactly
    double re = alpha_mul(e, x), im = alpha_mul(e, y);
    if (e.alpha_di != 0.0) {
      re = __fma_rn(-e.alpha_di, y, re);
      im = __fma_rn(e.alpha_di, x, im);
    }
    if constexpr (EK == EK_AXPBY) {
      const double u = as_f64(b.x), v = as_f64(b.y);
      re = __fma_rn(e.beta_d, u, re);
      im = __fma_rn(e.beta_d, v, im);
      if (e.beta_di != 0.0) {
        re = __fma_rn(-e.beta_di, v, re);
        im = __fma_rn(e.beta_di, u, im);
      }
    }
    if constexpr (DOUT == DT_C128) return make_double2(re, im);
    else return make_float2(narrow_f64_rn(re), narrow_f64_rn(im));
  } else {
    float re = __fmul_rn(e.alpha_f, a.x), im = __fmul_rn(e.alpha_f, a.y);
    if (e.alpha_fi != 0.f) {
      re = __fmaf_rn(-e.alpha_fi, a.y, re);
      im = __fmaf_rn(e.alpha_fi, a.x, im);
    }
    if constexpr (EK == EK_AXPBY) {
      re = __fmaf_rn(e.beta_f, b.x, re);
      im = __fmaf_rn(e.beta_f, b.y, im);
      if (e.beta_fi != 0.f) {
        re = __fmaf_rn(-e.beta_fi, b.y, re);
        im = __fmaf_rn(e.beta_fi, b.x, im);
      }
    }
    return make_float2(re, im);
  }
}

template <int DIN, int DOUT, int EK>
__device__ __forceinline__ store_t<DOUT> epilogue_k(stage_t<DIN> a, store_t<DOUT> b, const Epilogue& e,
                                                    float scale) {
  if constexpr (EK == EK_RT || EK == EK_RT_B) {
    return epilogue<DIN, DOUT>(a, b, e, scale);
  } else if constexpr (EK == EK_FP8) {
    const float v = __fmul_rn(e.alpha_f, float(a));
    return store_t<DOUT>(e4m3_of_quotient(v, scale, __frcp_rn(scale)));
  } else if constexpr (EK == EK_COPY) {
    if constexpr (DIN == DT_BF16 && DOUT == DT_BF16) return store_t<DOUT>(__float_as_uint(a) >> 16);
    else return a;
  } else if constexpr (is_complex(DIN)) {
    return epilogue_complex<DIN, DOUT, EK>(a, b, e);
  } else if constexpr (ComputeIsF64<DIN, DOUT>::value) {
    // (the integer product of alpha_mul measured slower here than the FP64
    // pipe's multiply: real data carries half the FP64 work per byte of the
    // complex update)
    double r = __dmul_rn(e.alpha_d, as_f64(a));
    if constexpr (EK == EK_AXPBY) r = __fma_rn(e.beta_d, as_f64(b), r);
    if constexpr (DOUT == DT_F64) return r;
    else return narrow_f64_rn(r);
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
  if (p.swz && p.ngrid >= 2) {
    // grouped order: tile tid is block x0 of the first grid index and x1 of
    // the second, taken in groups of swz values of x0 (the last group may be
    // narrower), x0 fastest inside a group; r is then the plain mixed-radix
    // index of (x0, x1, the rest)
    const uint32_t n0 = p.g[0].div.d, n1 = p.g[1].div.d, plane = n0 * n1;
    const uint32_t rest = r / plane, q = r - rest * plane;
    const uint32_t band = q / (p.swz * n1), in = q - band * p.swz * n1;
    const uint32_t width = n0 - band * p.swz < p.swz ? n0 - band * p.swz : p.swz;
    const uint32_t x1 = in / width, x0 = band * p.swz + (in - x1 * width);
    r = rest * plane + x1 * n0 + x0;
  }
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

// The subset of a tile's parameters the walks and the epilogue read, for
// kernels whose parameters are not kernel arguments (the batch): copied into
// registers once per tile instead of being reloaded inside the element loops.
struct WalkP {
  int LC, LA, LB, U, W, P;
  int32_t saU, sbV, crossA_lin, crossB_lin;
  int rd_du, rd_dlb, wr_dlc, wr_dlb, wr_dla;
  FastDiv divU, divLC, divLB;
  const int32_t* tabA;
  const int32_t* tabB;
  Epilogue epi;
};

TTC_HD WalkP walk_params(const TileParams& t) {
  WalkP w;
  w.LC = t.LC; w.LA = t.LA; w.LB = t.LB; w.U = t.U; w.W = t.W; w.P = t.P;
  w.saU = t.saU; w.sbV = t.sbV; w.crossA_lin = t.crossA_lin; w.crossB_lin = t.crossB_lin;
  w.rd_du = t.rd_du; w.rd_dlb = t.rd_dlb; w.wr_dlc = t.wr_dlc; w.wr_dlb = t.wr_dlb; w.wr_dla = t.wr_dla;
  w.divU = t.divU; w.divLC = t.divLC; w.divLB = t.divLB;
  w.tabA = t.tabA; w.tabB = t.tabB;
  w.epi = t.epi;
  return w;
}

// The flat walks' first positions for thread t: read order (u, lb) and write
// order (lc, lb, la), by multiply-high divisions.
template <class PT>
TTC_HD void flat_starts(const PT& p, int t, int& u0, int& lb0, int& lc0, int& lbw0, int& la0) {
  const uint32_t qu = fast_div(uint32_t(t), p.divU);
  u0 = t - int(qu) * p.U;
  lb0 = int(qu);
  const uint32_t qc = fast_div(uint32_t(t), p.divLC);
  lc0 = t - int(qc) * p.LC;
  const uint32_t qb = fast_div(qc, p.divLB);
  lbw0 = int(qc - qb * uint32_t(p.LB));
  la0 = int(qb);
}

// Flat walks (tile_kernel).  Thread t handles tile elements t + k*kThreads,
// k < K.  f(k, ok, offset in tile, smem position) is called for every k; ok
// tells whether the element exists (a short last block leaves holes), and the
// offset is 0 when it does not, so a caller may load unconditionally.  The
// bodies are branch-free (selects instead of ifs): measured ~2x fewer issued
// instructions than the branchy form.  TAB: the cross offsets come from a
// table instead of one multiply.
//
// Read order: (u, lb) with u = la*LC + lc; offset in A.
template <int K, bool TAB, class PT, class F>
TTC_HD void walk_read(const TileCoord& c, const PT& p, const int32_t* tabA, int u0, int lb0, F&& f) {
  const int limU = c.remA * p.LC;
  int u = u0, lb = lb0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const bool ok = (lb < c.remB) & (u < limU);
    const int32_t cross = TAB ? (ok ? tabA[lb] : 0) : lb * p.crossA_lin;
    f(k, ok, ok ? u * p.saU + cross : 0, lb * p.P + u);
    u += p.rd_du;
    lb += p.rd_dlb;
    const bool w = u >= p.U;
    u -= w ? p.U : 0;
    lb += w;
  }
}

// Write order: (lc, lb, la); offset in B.
template <int K, bool TAB, class PT, class F>
TTC_HD void walk_write(const TileCoord& c, const PT& p, const int32_t* tabB, int lc0, int lb0, int la0,
                       F&& f) {
  int lc = lc0, lb = lb0, la = la0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const bool ok = (la < c.remA) & (lb < c.remB);
    const int32_t cross = TAB ? (ok ? tabB[la] : 0) : la * p.crossB_lin;
    f(k, ok, ok ? (lb * p.LC + lc) * p.sbV + cross : 0, lb * p.P + la * p.LC + lc);
    lc += p.wr_dlc;
    lb += p.wr_dlb;
    la += p.wr_dla;
    const bool w1 = lc >= p.LC;
    lc -= w1 ? p.LC : 0;
    lb += w1;
    const bool w2 = lb >= p.LB;
    lb -= w2 ? p.LB : 0;
    la += w2;
  }
}

// Warp-mapped walks (tile2_kernel).  Read: lanes along u (JU chunks of 32),
// warps along lb.  Write: lanes along v (JW chunks), warps along la.
// FULL: an interior tile (no cut index is short).  f(k, ok, offset, smem
// position): rows past the tile's end are skipped (warp-uniform); lanes past
// a run's end get ok == false, and their offset and position are not
// meaningful (callers predicate every access on ok, which keeps the loads and
// stores branch-free).  UNIT: the runs have unit stride on both sides (the
// planner only gives these kernels such tiles), so a lane's chunks sit at
// constant distances from its row offset.
template <int JU, int K, bool FULL, bool TAB, bool UNIT, class PT, class F>
TTC_HD void walk2_read(const TileCoord& c, const PT& p, const int32_t* tabA, int lane, int warp,
                       F&& f) {
  constexpr int RR = K / JU;
  const int limU = FULL ? p.U : c.remA * p.LC;
  const int remB = FULL ? p.LB : c.remB;
  const int32_t su = UNIT ? 1 : p.saU;
  bool uok[JU];
#pragma unroll
  for (int j = 0; j < JU; ++j) uok[j] = lane + 32 * j < limU;
#pragma unroll
  for (int i = 0; i < RR; ++i) {
    const int r = warp + 8 * i;
    if (r < remB) {
      const int32_t row = (TAB ? tabA[r] : r * p.crossA_lin) + lane * su;
      const int pos = r * p.P + lane;
#pragma unroll
      for (int j = 0; j < JU; ++j) f(i * JU + j, uok[j], row + 32 * j * su, pos + 32 * j);
    }
  }
}

// per-lane constants of the write walk: shared-memory offset of the lane's
// run positions v = lane + 32 j
template <int JW, class PT>
TTC_HD void walk2_lane_consts(const PT& p, int lane, int (&spre)[JW]) {
#pragma unroll
  for (int j = 0; j < JW; ++j) {
    const int vv = lane + 32 * j;
    const int q = int(fast_div(uint32_t(vv), p.divLC));
    spre[j] = q * p.P + (vv - q * p.LC);
  }
}

template <int JW, int K, bool FULL, bool TAB, bool UNIT, class PT, class F>
TTC_HD void walk2_write(const TileCoord& c, const PT& p, const int32_t* tabB, int lane, int warp,
                        const int (&spre)[JW], F&& f) {
  constexpr int RW = K / JW;
  const int limV = FULL ? p.W : c.remB * p.LC;
  const int remA = FULL ? p.LA : c.remA;
  const int32_t sv = UNIT ? 1 : p.sbV;
  bool vok[JW];
#pragma unroll
  for (int j = 0; j < JW; ++j) vok[j] = lane + 32 * j < limV;
#pragma unroll
  for (int i = 0; i < RW; ++i) {
    const int la = warp + 8 * i;
    if (la < remA) {
      const int32_t row = (TAB ? tabB[la] : la * p.crossB_lin) + lane * sv;
      const int spos = la * p.LC;
#pragma unroll
      for (int j = 0; j < JW; ++j) f(i * JW + j, vok[j], row + 32 * j * sv, spre[j] + spos);
    }
  }
}

// Packed-lane walks (tilep_kernel).  The tile has no C index (LC = 1): its
// A-side runs are u = la (remA elements, rows lb < remB) and its B-side runs
// v = lb (remB elements, rows la < remA).  On each side the CTA's threads form
// groups of g consecutive threads, one group per row at a time: thread
// t = tu + g*tr takes the run positions tu + g*j (j < J) of rows
// tr + rows*i (i < K/J).  g = ceil(n/J) is chosen per tile class (whole
// tiles, and the short runs of the tiles a cut index leaves short), so the
// lanes of a warp continue from the end of one row into the next instead of
// idling at a run's end, and each thread's offsets advance by constants (one
// add per element, the row's cross offset once per row).  tile2_kernel is
// the case g = 32 with warps as the groups.  f(k, ok, offset in tile, smem
// position): smem holds the tile as lb rows of pitch P in A order; when ok is
// false the offset and position are not meaningful (callers predicate on
// ok).  UNIT as for the warp-mapped walks.
template <int NT, int J, int K, bool TAB, bool UNIT, class F>
TTC_HD void walkp_read(const TileCoord& c, const TileParams& p, const int32_t* tabA, int t, F&& f) {
  constexpr int R = K / J;
  // (the two layouts are selected field by field: indexing the parameter
  // array with a run-time index would copy it to local memory)
  const bool whole = c.remA == p.LA;
  const int g = whole ? p.pkA[0].g : p.pkA[1].g, rows = whole ? p.pkA[0].rows : p.pkA[1].rows;
  const int tr = int(fast_div(uint32_t(t), whole ? p.pkA[0].div : p.pkA[1].div));
  const int tu = t - tr * g;
  const bool active = tr < rows;
  const int32_t su = UNIT ? 1 : p.saU;
  int32_t uoff[J];
  bool uok[J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int u = tu + g * j;
    uok[j] = active && u < c.remA;
    uoff[j] = u * su;
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int lb = tr + rows * i;
    const bool rok = lb < c.remB;
    const int32_t cross = TAB ? (rok && active ? tabA[lb] : 0) : lb * p.crossA_lin;
    const int pos = lb * p.P + tu;
#pragma unroll
    for (int j = 0; j < J; ++j) f(i * J + j, rok && uok[j], uoff[j] + cross, pos + g * j);
  }
}

template <int NT, int J, int K, bool TAB, bool UNIT, class F>
TTC_HD void walkp_write(const TileCoord& c, const TileParams& p, const int32_t* tabB, int t, F&& f) {
  constexpr int R = K / J;
  const bool whole = c.remB == p.LB;
  const int g = whole ? p.pkB[0].g : p.pkB[1].g, rows = whole ? p.pkB[0].rows : p.pkB[1].rows;
  const int tr = int(fast_div(uint32_t(t), whole ? p.pkB[0].div : p.pkB[1].div));
  const int tv = t - tr * g;
  const bool active = tr < rows;
  const int32_t sv = UNIT ? 1 : p.sbV;
  int32_t voff[J];
  bool vok[J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int v = tv + g * j;
    vok[j] = active && v < c.remB;
    voff[j] = v * sv;
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int la = tr + rows * i;
    const bool rok = la < c.remA;
    const int32_t cross = TAB ? (rok && active ? tabB[la] : 0) : la * p.crossB_lin;
    const int pos = tv * p.P + la;
#pragma unroll
    for (int j = 0; j < J; ++j) f(i * J + j, rok && vok[j], voff[j] + cross, pos + g * j * p.P);
  }
}

// Packed rows (rowsp_kernel): a tile with a C index (perm keeps index 0)
// is remA x remB rows (la, lb) of LC elements, each row contiguous in A (at
// la*LC*saU + crossA(lb)) and in B (at lb*LC*sbV + crossB(la)), so rows are
// copied directly, without staging.  Thread t = tu + g*tr takes positions
// tu + g*j (j < J) of rows r = tr + rows*i (i < K/J), r = la + remA*lb; g
// and rows come from the host's layout (pkA[0]).  f(k, ok, A offset, B
// offset).
template <int J, int K, bool TA, bool TB, class F>
TTC_HD void walk_rowsp(const TileCoord& c, const TileParams& p, const int32_t* tabA, const int32_t* tabB, int t,
                       F&& f) {
  constexpr int R = K / J;
  const int g = p.pkA[0].g, rows = p.pkA[0].rows;
  const int tr = int(fast_div(uint32_t(t), p.pkA[0].div));
  const int tu = t - tr * g;
  const bool active = tr < rows;
  const bool whole = c.remA == p.LA;
  const int nrow = c.remA * c.remB;
  const int32_t rowA = p.LC * p.saU, rowB = p.LC * p.sbV;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int r = tr + rows * i;
    const bool rok = active && r < nrow;
    const int lb = int(fast_div(uint32_t(r), whole ? p.divRA[0] : p.divRA[1]));
    const int la = r - lb * c.remA;
    const int32_t baseA = la * rowA + (TA ? (rok ? tabA[lb] : 0) : lb * p.crossA_lin) + tu * p.saU;
    const int32_t baseB = lb * rowB + (TB ? (rok ? tabB[la] : 0) : la * p.crossB_lin) + tu * p.sbV;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      // (positions recomputed per element: arrays of J offsets would not fit
      // in registers next to the staged values)
      const bool ok = rok && tu + g * j < p.LC;
      f(i * J + j, ok, ok ? baseA + g * j * p.saU : 0, ok ? baseB + g * j * p.sbV : 0);
    }
  }
}

// Multi-row copy (perm keeps index 0, short runs): a tile is LC x LA elements,
// LC = the shared stride-1 index, LA consecutive indices of the next A index,
// contiguous in A; thread t takes the flat positions u = t + kThreads*k.
// f(k, A offset in tile, B offset in tile).
template <int K, class PT, class F>
TTC_HD void walk_rows(const TileCoord& c, const PT& p, int t, F&& f) {
  const int limU = c.remA * p.LC;
  const int q = int(fast_div(uint32_t(t), p.divLC));
  int u = t, la = q, lc = t - q * p.LC;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const bool ok = u < limU;
    f(k, ok, ok ? u : 0, ok ? lc + la * p.crossB_lin : 0);
    u += kThreads;
    lc += p.wr_dlc;
    la += p.wr_dla;
    const bool w = lc >= p.LC;
    lc -= w ? p.LC : 0;
    la += w;
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
