// planner.cu -- validation, canonicalisation (index merging) and candidate
// schedules of one permute-scale-add.  Host code only.
//
// Canonicalisation follows section 2.1 stage 1: neighbouring indices are
// merged into a "super index" whose size is the product of their sizes
// (footnote 5: only when ld(i_m) = size(i_m)).  Reading taken here: two
// indices i_m, i_m+1 of A merge when they are also neighbours, in the same
// order, in B, and both memory layouts are dense across them (the stride of
// i_m+1 is the stride of i_m times its size, in A and in B).  Indices of size 1
// are dropped first; neither step changes which element goes where.
//
// Candidate schedules replace TTC's candidate list (section 2.1 stages 2-3,
// section 2.2: blockings b_A, b_B and loop orders; section 2.3 heuristics).
// Here a candidate is a tile shape (which indices form the A-side and B-side
// runs of the tile and how the last of each is cut into blocks) plus the
// order of the flat grid of tiles; a cost model in the spirit of section 2.3
// ranks them (long contiguous runs on both sides = sector efficiency, little
// remainder, enough work per tile), and the autotuner times the best few.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <set>
#include <sstream>

#include "../../include/ttc.h"
#include "kernels.cuh"
#include "launch.h"
#include "planner.h"
#include "rowvec.h"
#include "tma2d.h"

namespace ttc {

namespace {

bool mul_overflows(int64_t a, int64_t b) {
  if (a == 0 || b == 0) return false;
  return a > INT64_MAX / b;
}

// Cost-model constants of one GB300 (only ratios matter for ranking).
constexpr double kHbmBytesPerS = 6.8e12;
constexpr double kLaneInstrPerS = 152.0 * 4 * 32 * 1.9e9;

}  // namespace

double run_efficiency(double bytes, bool write, bool flat) {
  // Measured on GB300 (2D and 3D transposes of aligned and misaligned
  // sizes): a run costs as if it were `bytes + c` long.  For the single-plan
  // kernels c ~ 48 bytes for reads and ~16 bytes for writes: loads are what
  // they wait on, so long A runs pay off, while partial sectors at the ends of
  // B runs are mostly completed in L2 by the neighbouring tile before they are
  // written back.  The batch body's flat walks (half-size tiles, every CTA on
  // a different problem) fit c ~ 16 for reads and ~64 for writes instead.
  if (bytes <= 0) return 1.0;
  if (flat) return bytes / (bytes + (write ? 64.0 : 16.0));
  return bytes / (bytes + (write ? 16.0 : 48.0));
}

std::string Candidate::describe() const {
  std::ostringstream o;
  if (variant == VAR_EMPTY) return "empty";
  if (variant == VAR_COPY) {
    o << "copy chunk=" << chunk << " vec=" << vec;
  } else if (variant == VAR_TMA) {
    o << "tma2d box=" << ta << "x32x" << kTmaBoxes;
  } else {
    o << "tile c=" << has_c << " ga=[";
    for (size_t i = 0; i < ga.size(); ++i) o << (i ? "," : "") << ga[i];
    o << "]/" << ta << " gb=[";
    for (size_t i = 0; i < gb.size(); ++i) o << (i ? "," : "") << gb[i];
    o << "]/" << tb << " j=" << ju << "," << jw << (rows ? " rows" : "") << (rows && vec > 1 ? " vec=" : "");
    if (rows && vec > 1) o << vec;
    o << (slots ? " slots" : "");
    if (pk) o << " pk=" << pk;
    if (swz) o << " swz=" << swz;
    if (rj) o << " rj=" << rj;
    o << " order=[";
    for (size_t i = 0; i < order.size(); ++i) o << (i ? "," : "") << order[i];
    o << "]";
  }
  o << " est_us=" << est_s * 1e6 << " segA=" << seg_a << " segB=" << seg_b;
  return o.str();
}

int canonicalize(int ndim, const int* perm, const int64_t* sizes, const int64_t* outerA,
                 const int64_t* outerB, Canon* c, std::string* err) {
  *c = Canon();
  if (!perm || !sizes) {
    *err = "perm and sizes must not be NULL";
    return TTC_ERR_INVALID_ARG;
  }
  if (ndim < 1 || ndim > kMaxDim) {
    *err = "ndim must be in 1..16";
    return TTC_ERR_INVALID_PERM;
  }
  bool seen[kMaxDim] = {};
  for (int d = 0; d < ndim; ++d) {
    if (perm[d] < 0 || perm[d] >= ndim || seen[perm[d]]) {
      *err = "perm is not a permutation of 0..ndim-1";
      return TTC_ERR_INVALID_PERM;
    }
    seen[perm[d]] = true;
  }
  int64_t oA[kMaxDim], oB[kMaxDim];
  for (int k = 0; k < ndim; ++k) {
    if (sizes[k] < 0) {
      *err = "negative size";
      return TTC_ERR_INVALID_SIZE;
    }
    oA[k] = outerA ? outerA[k] : sizes[k];
    if (oA[k] < sizes[k]) {
      *err = "outer size of A smaller than the size";
      return TTC_ERR_INVALID_OUTER;
    }
  }
  for (int d = 0; d < ndim; ++d) {
    oB[d] = outerB ? outerB[d] : sizes[perm[d]];
    if (oB[d] < sizes[perm[d]]) {
      *err = "outer size of B smaller than the size";
      return TTC_ERR_INVALID_OUTER;
    }
  }
  // strides (column-major, footnote 2) and element count
  int64_t stA[kMaxDim], stB[kMaxDim];
  int64_t acc = 1;
  for (int k = 0; k < ndim; ++k) {
    stA[k] = acc;
    if (mul_overflows(acc, std::max<int64_t>(oA[k], 1))) {
      *err = "A is too large";
      return TTC_ERR_INVALID_SIZE;
    }
    acc *= std::max<int64_t>(oA[k], 1);
  }
  acc = 1;
  for (int d = 0; d < ndim; ++d) {
    stB[d] = acc;
    if (mul_overflows(acc, std::max<int64_t>(oB[d], 1))) {
      *err = "B is too large";
      return TTC_ERR_INVALID_SIZE;
    }
    acc *= std::max<int64_t>(oB[d], 1);
  }
  int64_t n = 1;
  for (int k = 0; k < ndim; ++k) {
    if (mul_overflows(n, sizes[k])) {
      *err = "too many elements";
      return TTC_ERR_INVALID_SIZE;
    }
    n *= sizes[k];
  }
  c->n = n;
  if (n == 0) return TTC_OK;
  int posB[kMaxDim];
  for (int d = 0; d < ndim; ++d) posB[perm[d]] = d;

  struct Ix {
    int64_t s, sa, sb;
    int bpos;
  };
  std::vector<Ix> L;
  for (int k = 0; k < ndim; ++k)
    if (sizes[k] > 1) L.push_back({sizes[k], stA[k], stB[posB[k]], posB[k]});
  if (L.empty()) L.push_back({1, 1, 1, 0});

  // merge neighbours (A order) that are neighbours in the same order in B and
  // dense across the pair in both tensors
  for (bool merged = true; merged && L.size() > 1;) {
    merged = false;
    std::vector<int> rank(L.size());
    std::vector<int> byb(L.size());
    std::iota(byb.begin(), byb.end(), 0);
    std::sort(byb.begin(), byb.end(), [&](int x, int y) { return L[x].bpos < L[y].bpos; });
    for (size_t r = 0; r < byb.size(); ++r) rank[byb[r]] = int(r);
    for (size_t i = 0; i + 1 < L.size(); ++i) {
      if (rank[i + 1] == rank[i] + 1 && L[i + 1].sa == L[i].sa * L[i].s &&
          L[i + 1].sb == L[i].sb * L[i].s) {
        L[i].s *= L[i + 1].s;
        L.erase(L.begin() + i + 1);
        merged = true;
        break;
      }
    }
  }
  c->N = int(L.size());
  std::vector<int> byb(L.size());
  std::iota(byb.begin(), byb.end(), 0);
  std::sort(byb.begin(), byb.end(), [&](int x, int y) { return L[x].bpos < L[y].bpos; });
  c->spanA = 1;
  c->spanB = 1;
  for (int k = 0; k < c->N; ++k) {
    c->s[k] = L[k].s;
    c->sa[k] = L[k].sa;
    c->sb[k] = L[k].sb;
    c->perm[k] = byb[k];
    c->spanA += (L[k].s - 1) * L[k].sa;
    c->spanB += (L[k].s - 1) * L[k].sb;
  }
  return TTC_OK;
}

namespace {

// Block extents considered for a cut index of size s (section 2.2 uses
// b in {w, 2w, 3w, 4w}; here: powers of two, balanced splits, and the
// divisors of s, which leave no remainder -- section 2.3's blocking heuristic).
std::vector<int> cut_options(int64_t s, int64_t cap) {
  std::set<int64_t> o;
  if (s <= cap) o.insert(s);
  for (int64_t p = 2; p < s && p <= cap; p *= 2) o.insert(p);
  for (int64_t j = 2; j <= 16; ++j) {
    int64_t t = (s + j - 1) / j;
    if (t >= 2 && t < s && t <= cap) o.insert(t);
  }
  for (int64_t d = 2; d * d <= s && d <= 4096; ++d) {
    if (s % d == 0) {
      if (d <= cap) o.insert(d);
      if (s / d <= cap && s / d < s) o.insert(s / d);
    }
  }
  return std::vector<int>(o.begin(), o.end());
}

int stage_bytes(int din) { return stage_bytes_of(din); }

// shared-memory pitch (elements) of one lb row; see ttc_internal.h
int pick_pitch(int U, int LC, int LB, int din, int smem_cap) {
  const int banks = 128 / stage_bytes(din);      // 4-byte banks, counted in elements
  int P;
  if (LC <= 1) P = U | 1;
  else P = U + (((LC - U) % banks) + banks) % banks;
  if (int64_t(P) * LB * stage_bytes(din) > smem_cap) P = (LC <= 1) ? (U | 1) : U;
  if (int64_t(P) * LB * stage_bytes(din) > smem_cap) P = U;
  return P;
}

struct TileShape {
  int has_c;
  std::vector<int> ga, gb;
  int ta, tb;
};

// extents of every canonical index inside the tile (1 if not in it)
void tile_extents(const Canon& c, const TileShape& t, int64_t* ext) {
  for (int k = 0; k < c.N; ++k) ext[k] = 1;
  if (t.has_c) ext[0] = c.s[0];
  for (size_t i = 0; i < t.ga.size(); ++i) ext[t.ga[i]] = (i + 1 == t.ga.size()) ? t.ta : c.s[t.ga[i]];
  for (size_t i = 0; i < t.gb.size(); ++i) ext[t.gb[i]] = (i + 1 == t.gb.size()) ? t.tb : c.s[t.gb[i]];
}

// contiguous run (elements) of the tile in memory order of one tensor
double run_length(const Canon& c, const int64_t* ext, const int* order, const int64_t* st) {
  double seg = 1;
  if (st[order[0]] != 1) return 1;
  for (int i = 0; i < c.N; ++i) {
    const int k = order[i];
    if (ext[k] == 1) break;
    seg *= double(ext[k]);
    if (ext[k] < c.s[k]) break;
    if (i + 1 < c.N && st[order[i + 1]] != st[k] * c.s[k]) break;
  }
  return seg;
}

std::vector<int> grid_order(const Canon& c, const int64_t* ext, int mode) {
  std::vector<int> g;
  for (int k = 0; k < c.N; ++k)
    if (ext[k] < c.s[k]) g.push_back(k);
  auto key = [&](int k) -> double {
    const double a = double(ext[k]) * double(c.sa[k]), b = double(ext[k]) * double(c.sb[k]);
    if (mode == 1) return a;
    if (mode == 2) return b;
    // both-local: indices with small steps in both tensors first, so that
    // consecutive tiles touch neighbouring memory on both sides
    if (mode == 3) return std::max(a, b) + 1e-9 * std::min(a, b);
    return std::min(a, b) + 1e-9 * std::max(a, b);
  };
  std::stable_sort(g.begin(), g.end(), [&](int x, int y) { return key(x) < key(y); });
  return g;
}

// Lane-group layout of one side of a packed-lane tile (PackWalk): runs of n
// elements in R rows on nt threads of k slots each, with j run chunks per
// thread: groups of g = ceil(n / j) threads, nt / g groups, each taking every
// (nt / g)-th row.  False if the rows are not covered.
bool pack_layout(int n, int R, int nt, int k, int j, PackWalk* w) {
  if (n < 1 || R < 1) return false;
  const int g = (n + j - 1) / j;
  const int rows = nt / g;
  if (rows < 1 || int64_t(rows) * (k / j) < R) return false;
  if (w) {
    w->n = n;
    w->g = g;
    w->rows = rows;
    w->div = make_fastdiv(uint32_t(g));
  }
  return true;
}

// Chunks per thread of one side (the fewest of 1, 2, 4 whose layout covers
// the whole tile; the short tiles then fit too), or 0 if none does.
int pack_chunks(int n, int R, int nt, int k) {
  for (int j : {1, 2, 4})
    if (pack_layout(n, R, nt, k, j, nullptr)) return j;
  return 0;
}

// Memory time of a tile schedule: the runs of every class of tiles (the
// cut index of GA, and of GB, in a whole block or in the short last block)
// weighted by the class's share of the elements, each run charged the
// per-run overhead of run_efficiency.  A schedule whose tiles are mostly of
// the full size gets the full tile's runs; one whose cut leaves a short last
// block pays for the short runs of those tiles.  `walks`: the index walks'
// coalescing (see the caller); false for slot tables.
double tile_mem_time(const Canon& c, const TileShape& sh, const int64_t* ext, int esA, int esB, bool bnz,
                     bool flat, bool walks) {
  int orderA[kMaxDim], orderB[kMaxDim];
  for (int k = 0; k < c.N; ++k) {
    orderA[k] = k;
    orderB[k] = c.perm[k];
  }
  const int cut[2] = {sh.ga.empty() ? -1 : sh.ga.back(), sh.gb.empty() ? -1 : sh.gb.back()};
  double per_el = 0;
  for (int ea = 0; ea < 2; ++ea)
    for (int eb = 0; eb < 2; ++eb) {
      int64_t e2[kMaxDim];
      for (int k = 0; k < c.N; ++k) e2[k] = ext[k];
      double w = 1;
      bool skip = false;
      const int side[2] = {ea, eb};
      for (int g = 0; g < 2 && !skip; ++g) {
        const int m = cut[g];
        const bool short_side = side[g] != 0;
        if (m < 0 || ext[m] >= c.s[m]) {
          skip = short_side;
          continue;
        }
        const int64_t whole = c.s[m] / ext[m] * ext[m], rest = c.s[m] - whole;
        if (short_side) {
          if (rest == 0) skip = true;
          w *= double(rest) / double(c.s[m]);
          e2[m] = rest;
        } else {
          w *= double(whole) / double(c.s[m]);
        }
      }
      if (skip || w <= 0) continue;
      double ra = run_length(c, e2, orderA, c.sa), rb = run_length(c, e2, orderB, c.sb);
      if (walks) {
        double U = sh.has_c ? double(c.s[0]) : 1, W = U, V = U;
        for (int m : sh.ga) U *= double(e2[m]);
        for (int m : sh.gb) W *= double(e2[m]);
        V = U * W / V;
        if (U == 1) ra = ra >= V ? 8.0 : 1.0;
        if (W == 1) rb = rb >= V ? 8.0 : 1.0;
      }
      per_el += w * (esA / run_efficiency(ra * esA, false, flat) + esB / run_efficiency(rb * esB, true, flat) +
                     (bnz ? esB / run_efficiency(rb * esB, false, flat) : 0.0));
    }
  return double(c.n) * per_el / kHbmBytesPerS;
}

}  // namespace

std::vector<Candidate> make_candidates(const Canon& c, int din, int dout, double beta, int max_keep, int vmax) {
  std::vector<Candidate> out;
  const bool flat = vmax > 0;   // the batch body
  if (c.N == 0) {
    out.push_back(Candidate());
    return out;
  }
  const int esA = dtype_size(din), esB = dtype_size(dout);
  const bool bnz = beta != 0.0;
  const double n = double(c.n);
  int orderA[kMaxDim], orderB[kMaxDim];
  for (int k = 0; k < c.N; ++k) {
    orderA[k] = k;
    orderB[k] = c.perm[k];
  }

  // ---- streaming copy (perm keeps index 0)
  if (c.perm[0] == 0) {
    Candidate k;
    k.variant = VAR_COPY;
    const int64_t len = c.s[0];
    k.chunk = len <= 16384 ? len : 8192;
    const int w = 16 / std::max(esA, esB);
    bool vec_ok = c.sa[0] == 1 && c.sb[0] == 1 && len % w == 0;
    for (int i = 1; i < c.N; ++i) vec_ok = vec_ok && c.sa[i] % w == 0 && c.sb[i] % w == 0;
    k.vec = vec_ok ? w : 1;
    const double nitems = double(c.n / len) * double((len + k.chunk - 1) / k.chunk);
    if (nitems >= 2147483647.0) k.variant = VAR_EMPTY;   // marked unusable below
    const double ra = c.sa[0] == 1 ? double(len) : 1.0, rb = c.sb[0] == 1 ? double(len) : 1.0;
    k.seg_a = ra;
    k.seg_b = rb;
    const double mem = (n * esA / run_efficiency(ra * esA, false, flat) +
                        n * esB / run_efficiency(rb * esB, true, flat) +
                        (bnz ? n * esB / run_efficiency(rb * esB, false, flat) : 0.0)) / kHbmBytesPerS;
    const double rows = n / double(len);
    const double lanes_per_row = std::ceil(double(len) / (32.0 * k.vec)) * 32.0;
    const double issue = (rows * lanes_per_row * 10.0 + rows * 32.0 * (8.0 * c.N)) / kLaneInstrPerS;
    // one warp per row chunk: short rows leave few loads in flight per warp,
    // and scalar rows sustain less than the tile kernels (measured ~0.6x of
    // the multi-row copy for runs of a few hundred elements)
    const double mlp = std::min(1.0, double(len) / (32.0 * 8 * k.vec));
    const double scalar_penalty = (k.vec > 1 || len > 4096) ? 1.0 : 1.6;
    k.est_s = std::max(mem / std::max(mlp, 0.1), issue) * scalar_penalty + 0.2 * std::min(mem, issue) + 2e-6;
    if (k.variant == VAR_COPY) out.push_back(k);
  }

  // ---- multi-row copy: perm keeps index 0 with short runs; G consecutive
  // indices of A's next index make one contiguous block of A per tile
  if (!flat && c.perm[0] == 0 && c.N >= 2 && c.sa[0] == 1 && c.sb[0] == 1 && c.sa[1] == c.s[0]) {
    const int Kt = tile_k_for(stage_bytes(din));
    const int64_t vcap = vmax > 0 ? std::min<int64_t>(vmax, int64_t(kThreads) * Kt) : int64_t(kThreads) * Kt;
    const int64_t cap = vcap / c.s[0];
    if (cap >= 2) {
      for (int G : cut_options(c.s[1], cap)) {
        Candidate k;
        k.variant = VAR_TILE;
        k.rows = 1;
        k.has_c = 1;
        k.ga = {1};
        k.ta = G;
        int64_t ext[kMaxDim];
        TileShape sh{1, k.ga, {}, G, 1};
        tile_extents(c, sh, ext);
        double ntiles = 1;
        for (int q = 0; q < c.N; ++q) ntiles *= std::ceil(double(c.s[q]) / double(ext[q]));
        if (ntiles >= 2147483647.0) continue;
        k.order = grid_order(c, ext, 0);
        const double ra = run_length(c, ext, orderA, c.sa), rb = run_length(c, ext, orderB, c.sb);
        k.seg_a = ra;
        k.seg_b = rb;
        const double mem = (n * esA / run_efficiency(ra * esA, false, flat) +
                            n * esB / run_efficiency(rb * esB, true, flat) +
                        (bnz ? n * esB / run_efficiency(rb * esB, false, flat) : 0.0)) / kHbmBytesPerS;
        const double issue = ntiles * kThreads * Kt * (10.0 + (bnz ? 3 : 0)) / kLaneInstrPerS;
        const double over = ntiles * kThreads * (40.0 + 10.0 * c.N) / kLaneInstrPerS;
        const double fill = double(c.s[0]) * G / double(vcap);   // share of the unrolled slots in use
        // with beta != 0 the multi-row copy reads B in as many separate runs
        // as it writes: measured 1.4-1.7x slower than a staged tile whose B
        // footprint is fewer, longer runs (3D (370,377,481) perm (0,2,1):
        // 3369 against 5405 GB/s), which the per-run overhead does not show
        const double rows_beta = bnz ? 1.5 : 1.0;
        k.est_s = (std::max(mem, issue / std::max(fill, 0.05)) + 0.1 * std::min(mem, issue)) * rows_beta + over + 3e-6;
        out.push_back(k);
      }
    }
  }

  // ---- multi-row copy with 16-byte accesses (rowvec.cu): rows a multiple
  // of the vector, every A and B stride too, so that each thread's vectors
  // are aligned relative to both bases; twice the bytes per thread and a
  // quarter of the instructions of the element-wise copy
  const int V = rowvec_width(din);
  bool vec_rows = !flat && V > 1 && c.perm[0] == 0 && c.N >= 2 && c.sa[0] == 1 && c.sb[0] == 1 &&
                  c.sa[1] == c.s[0] && c.s[0] % V == 0;
  for (int i = 1; vec_rows && i < c.N; ++i) vec_rows = c.sa[i] % V == 0 && c.sb[i] % V == 0;
  if (vec_rows) {
    const int64_t vcap = int64_t(kThreads) * kRowVecK * V;
    const int64_t cap = vcap / c.s[0];
    if (cap >= 2) {
      for (int G : cut_options(c.s[1], cap)) {
        Candidate k;
        k.variant = VAR_TILE;
        k.rows = 1;
        k.vec = V;
        k.has_c = 1;
        k.ga = {1};
        k.ta = G;
        int64_t ext[kMaxDim];
        TileShape sh{1, k.ga, {}, G, 1};
        tile_extents(c, sh, ext);
        double ntiles = 1;
        for (int q = 0; q < c.N; ++q) ntiles *= std::ceil(double(c.s[q]) / double(ext[q]));
        if (ntiles >= 2147483647.0) continue;
        k.order = grid_order(c, ext, 0);
        const double ra = run_length(c, ext, orderA, c.sa), rb = run_length(c, ext, orderB, c.sb);
        k.seg_a = ra;
        k.seg_b = rb;
        const double mem = (n * esA / run_efficiency(ra * esA, false, flat) +
                            n * esB / run_efficiency(rb * esB, true, flat) +
                            (bnz ? n * esB / run_efficiency(rb * esB, false, flat) : 0.0)) / kHbmBytesPerS;
        const double issue = ntiles * kThreads * kRowVecK * (12.0 + (bnz ? 3 * V : 0)) / kLaneInstrPerS;
        const double over = ntiles * kThreads * (40.0 + 10.0 * c.N) / kLaneInstrPerS;
        const double fill = double(c.s[0]) * G / double(vcap);
        const double rows_beta = bnz ? 1.5 : 1.0;
        k.est_s = (std::max(mem, issue / std::max(fill, 0.05)) + 0.1 * std::min(mem, issue)) * rows_beta + over + 3e-6;
        out.push_back(k);
      }
    }
  }

  // ---- staged tile
  const bool hc = c.perm[0] == 0;
  const int c0 = hc ? 1 : 0;
  const int64_t LC = hc ? c.s[0] : 1;
  const int Kt = tile_k_for(stage_bytes(din));
  // elements of one 256-thread tile (packed-lane tiles of twice that volume
  // on 512 threads measured slower than 256-thread ones on every sweep case:
  // fewer, larger CTAs hide the latency between their load and store phases
  // less well)
  const int V1 = vmax > 0 ? std::min(vmax, kThreads * Kt) : kThreads * Kt;
  // the packed-lane kernel needs unit-stride runs on both sides
  const bool pk_ok = !hc && c.sa[0] == 1 && c.sb[c.perm[0]] == 1;
  const int Vmax = V1;
  const int Kp = flat ? vmax / kThreads : Kt;   // slots per thread of the packed kernels
  std::vector<Candidate> tiles;
  if (!(hc && c.N == 1) && LC * 2 <= Vmax) {
    // A-group index list: A order from c0, dense, never B's first index after C
    std::vector<int> ka;
    for (int k = c0; k < c.N; ++k) {
      if (k == c.perm[c0]) break;
      if (k > 0 && c.sa[k] != c.sa[k - 1] * c.s[k - 1]) break;
      ka.push_back(k);
    }
    for (size_t nA = 0; nA <= ka.size(); ++nA) {
      int64_t fullA = 1;
      bool too_big = false;
      for (size_t i = 0; i + 1 < nA; ++i) {
        fullA *= c.s[ka[i]];
        if (LC * fullA * 2 > Vmax) too_big = true;
      }
      if (too_big) break;
      std::vector<int> topts = nA ? cut_options(c.s[ka[nA - 1]], Vmax / (2 * LC * fullA)) : std::vector<int>{1};
      for (int ta : topts) {
        const int64_t LA = fullA * ta;
        if (LC * LA * 2 > Vmax) continue;
        std::vector<int> ga(ka.begin(), ka.begin() + nA);
        std::set<int> inA(ga.begin(), ga.end());
        std::vector<int> kb;
        for (int d = c0; d < c.N; ++d) {
          const int m = c.perm[d];
          if (inA.count(m)) break;
          if (d > 0 && c.sb[m] != c.sb[c.perm[d - 1]] * c.s[c.perm[d - 1]]) break;
          kb.push_back(m);
        }
        for (size_t nB = 0; nB <= kb.size(); ++nB) {
          int64_t fullB = 1;
          bool big = false;
          for (size_t i = 0; i + 1 < nB; ++i) {
            fullB *= c.s[kb[i]];
            if (LC * LA * fullB > Vmax) big = true;
          }
          if (big) break;
          std::vector<int> tbopts = nB ? cut_options(c.s[kb[nB - 1]], Vmax / (LC * LA * fullB)) : std::vector<int>{1};
          for (int tb : tbopts) {
            const int64_t LB = fullB * tb;
            const int64_t V = LC * LA * LB;
            if (V > Vmax || (LA == 1 && LB == 1)) continue;
            TileShape sh{hc ? 1 : 0, ga, std::vector<int>(kb.begin(), kb.begin() + nB), int(ta), int(tb)};
            if (sh.ga.empty()) sh.ta = 1;
            if (sh.gb.empty()) sh.tb = 1;
            int64_t ext[kMaxDim];
            tile_extents(c, sh, ext);
            double ntiles = 1;
            for (int k = 0; k < c.N; ++k) ntiles *= std::ceil(double(c.s[k]) / double(ext[k]));
            if (ntiles >= 2147483647.0) continue;
            {
              // in-tile offsets must fit in 32 bits
              double maxA = double(LC * LA - 1) * double(c.sa[0]), maxB = double(LC * LB - 1) * double(c.sb[c.perm[0]]);
              for (int m : sh.gb) maxA += double(ext[m] - 1) * double(c.sa[m]);
              for (int m : sh.ga) maxB += double(ext[m] - 1) * double(c.sb[m]);
              for (int m : sh.gb) maxA = std::max(maxA, double(c.sa[m]));
              for (int m : sh.ga) maxB = std::max(maxB, double(c.sb[m]));
              if (maxA >= 2147483647.0 || maxB >= 2147483647.0) continue;
            }
            if ((!sh.ga.empty() && c.s[sh.ga.back()] >= (int64_t(1) << 30)) ||
                (!sh.gb.empty() && c.s[sh.gb.back()] >= (int64_t(1) << 30)))
              continue;
            // Slot tables visit a tile's elements in address order on each
            // side, so their runs are the tile footprint's contiguous runs.
            // The index walks (tile2, packed lanes, the batch) load a tile
            // without a C or GA index (U = 1) in GB's order, which steps
            // through A by large strides: a warp's loads do not coalesce.  When
            // the whole tile is one contiguous block of A, L1 still catches
            // most of the reuse (measured as if the runs were 8 elements long);
            // otherwise nothing does.  Likewise for W = 1.
            const double mem = tile_mem_time(c, sh, ext, esA, esB, bnz, flat, true);
            const double mem_s = tile_mem_time(c, sh, ext, esA, esB, bnz, flat, false);
            const double over = ntiles * kThreads * (60.0 + 10.0 * c.N) / kLaneInstrPerS;
            Candidate k;
            k.variant = VAR_TILE;
            k.has_c = sh.has_c;
            k.ga = sh.ga;
            k.ta = sh.ta;
            k.gb = sh.gb;
            k.tb = sh.tb;
            k.order = grid_order(c, ext, 0);
            k.seg_a = run_length(c, ext, orderA, c.sa);
            k.seg_b = run_length(c, ext, orderB, c.sb);
            if (!flat) {
              const double per_slot = 26.0 + (sh.ga.size() > 1 ? 3 : 0) + (sh.gb.size() > 1 ? 3 : 0) + (bnz ? 6 : 0);
              const double issue = ntiles * kTileK * kThreads * per_slot / kLaneInstrPerS;
              k.est_s = std::max(mem, issue) + 0.25 * std::min(mem, issue) + over + 3e-6;
              if (vmax == 0) {
                // single-plan tiles read their whole tiles from slot tables: two
                // slots per 16-byte table read and no index arithmetic.  The
                // table reads cost L1 bandwidth and one more dependent load per
                // phase: measured ~9 % below the warp-mapped kernel on shapes
                // both fit, 30-40 % above the index walk on every shape tried.
                const double per_slot3 = 14.0 + (bnz ? 4 : 0);
                const double issue3 = ntiles * kTileK * kThreads * per_slot3 / kLaneInstrPerS;
                k.slots = 1;
                k.est_s = std::max(1.08 * mem_s, issue3) + 0.25 * std::min(mem_s, issue3) + over + 3e-6;
              }
              tiles.push_back(k);
              // the warp-mapped kernel (single-plan only), when the shape fits
              // one of its lane layouts
              const int64_t U = LC * LA, W = LC * LB;
              // (unit-stride runs on both sides: the warp-mapped walks step
              // their lanes' chunks by constants)
              const bool unit = c.sa[0] == 1 && c.sb[c.perm[0]] == 1;
              int ju = 0, jw = 0;
              for (int j : {1, 2, 4})
                if (!ju && vmax == 0 && U <= 32 * j && LB <= 8 * Kt / j) ju = j;
              for (int j : {1, 2, 4})
                if (!jw && vmax == 0 && W <= 32 * j && LA <= 8 * Kt / j) jw = j;
              // a run shorter than half a warp leaves most lanes idle: every
              // warp access then carries a few elements only (measured slower
              // than the flat walk in the batch body)
              if (U < 16 || W < 16 || !unit) ju = jw = 0;
              if (ju && jw) {
                // lanes past a run's end idle, also in the short tiles at the
                // tensor's edge: every tile costs the full tile's instructions
                const double rows_r = std::ceil(double(LB) / 8.0), rows_w = std::ceil(double(LA) / 8.0);
                const double wi = 8.0 * (rows_r * (ju * 4.0 + 4.0 + (sh.gb.size() > 1 ? 2 : 0)) +
                                         rows_w * (jw * (5.0 + (bnz ? 3.0 : 0.0)) + 4.0 + (sh.ga.size() > 1 ? 2 : 0)));
                const double issue2 = ntiles * 32.0 * wi / kLaneInstrPerS;
                Candidate k2 = k;
                k2.slots = 0;
                k2.ju = ju;
                k2.jw = jw;
                k2.est_s = std::max(mem, issue2) + 0.25 * std::min(mem, issue2) + over + 3e-6;
                tiles.push_back(k2);
              }
            }
            if (hc && (flat || V >= 64)) {
              // packed rows: the C run is contiguous on both sides, so rows
              // are copied directly (no staging); the fewest idle threads
              // whose layout covers the tile's rows (the batch body has the
              // layouts with 1 and Kp positions per row)
              const int nrows = int(LA * LB);
              int best_j = 0, best_active = 0;
              for (int j : {1, 2, 4, 8, 16}) {
                if (j > Kp) break;
                if (flat && j != 1 && j != Kp) continue;
                PackWalk w;
                if (!pack_layout(int(LC), nrows, kThreads, Kp, j, &w)) continue;
                if (w.g * w.rows > best_active) {
                  best_active = w.g * w.rows;
                  best_j = j;
                }
              }
              if (best_j) {
                const double rows_per_thread = double(Kp / best_j);
                const double wi = rows_per_thread * (16.0 + best_j * (4.0 + (bnz ? 3.0 : 0.0))) + 20.0;
                const double issuer = ntiles * kThreads * wi / kLaneInstrPerS;
                Candidate kr = k;
                kr.slots = 0;
                kr.rj = best_j;
                kr.kt = flat ? Kp : 0;
                kr.est_s = std::max(mem, issuer) + 0.25 * std::min(mem, issuer) + over + 3e-6;
                tiles.push_back(kr);
              }
            }
            if (pk_ok && (flat || V >= 64)) {
              // the packed-lane kernel: lane groups of any width, so ragged
              // runs (and the short runs of the edge tiles) idle few lanes
              // (the batch body has the layouts with 1 or 2 chunks on both
              // sides)
              const int nt = kThreads;
              int ju = pack_chunks(int(LA), int(LB), nt, Kp), jw = pack_chunks(int(LB), int(LA), nt, Kp);
              if (flat) {
                const int j = std::max(ju, jw);
                ju = jw = (j == 1 || j == 2) && pack_layout(int(LA), int(LB), nt, Kp, j, nullptr) &&
                                  pack_layout(int(LB), int(LA), nt, Kp, j, nullptr)
                             ? j
                             : 0;
              }
              if (ju && jw) {
                const double wi = (Kp / ju) * (ju * 3.0 + 6.0 + (sh.gb.size() > 1 ? 2 : 0)) +
                                  (Kp / jw) * (jw * (4.0 + (bnz ? 3.0 : 0.0)) + 6.0 + (sh.ga.size() > 1 ? 2 : 0)) + 30.0;
                const double issuep = ntiles * nt * wi / kLaneInstrPerS;
                const double overp = ntiles * nt * (60.0 + 10.0 * c.N) / kLaneInstrPerS;
                Candidate kp = k;
                kp.slots = 0;
                kp.ju = ju;
                kp.jw = jw;
                kp.pk = nt;
                kp.kt = flat ? Kp : 0;
                kp.est_s = std::max(mem, issuep) + 0.25 * std::min(mem, issuep) + overp + 3e-6;
                tiles.push_back(kp);
              }
            }
          }
        }
      }
    }
  }
  std::stable_sort(tiles.begin(), tiles.end(),
                   [](const Candidate& a, const Candidate& b) { return a.est_s < b.est_s; });
  // Keep the best few of every kernel kind (the cost model ranks kinds less
  // reliably than shapes of one kind), then give the best shapes the A-major,
  // B-major and both-local grid orders and the grouped order (measured: the
  // order alone moves a tile schedule by up to 20 %); the autotuner sorts
  // them out.
  auto kind = [](const Candidate& q) { return q.rj ? 5 : q.pk ? 2 : q.rows ? 3 : q.slots ? 0 : q.ju ? 1 : 4; };
  auto same = [](const Candidate& q, const Candidate& k) {
    return q.order == k.order && q.ga == k.ga && q.gb == k.gb && q.ta == k.ta && q.tb == k.tb &&
           q.has_c == k.has_c && q.ju == k.ju && q.jw == k.jw && q.slots == k.slots && q.pk == k.pk &&
           q.rows == k.rows && q.swz == k.swz && q.rj == k.rj;
  };
  const int base_keep = std::max(1, max_keep / 2);
  const int per_kind = std::max(1, base_keep / 3);
  std::vector<Candidate> keep;
  int nkind[6] = {};
  for (const auto& t : tiles) {
    if (int(keep.size()) >= base_keep) break;
    if (nkind[kind(t)] >= per_kind) continue;
    ++nkind[kind(t)];
    keep.push_back(t);
  }
  for (const auto& t : tiles) {       // fill up with the next best of any kind
    if (int(keep.size()) >= base_keep) break;
    bool dup = false;
    for (const auto& q : keep) dup = dup || same(q, t);
    if (!dup) keep.push_back(t);
  }
  const size_t nshape = keep.size();
  std::vector<Candidate> vars;
  int vkind[6] = {};
  for (size_t i = 0; i < nshape; ++i) {
    if (vkind[kind(keep[i])]++ >= 2) continue;
    int64_t ext[kMaxDim];
    TileShape sh{keep[i].has_c, keep[i].ga, keep[i].gb, keep[i].ta, keep[i].tb};
    tile_extents(c, sh, ext);
    for (int mode = 1; mode <= 3; ++mode) {
      for (int swz : {0, 8}) {
        Candidate k = keep[i];
        k.order = grid_order(c, ext, mode);
        k.swz = k.order.size() >= 2 ? swz : 0;
        if (swz && !k.swz) continue;
        bool dup = false;
        for (const auto& q : keep) dup = dup || same(q, k);
        for (const auto& q : vars) dup = dup || same(q, k);
        if (!dup) {
          k.est_s *= swz ? 1.02 : 1.01;
          vars.push_back(k);
        }
      }
    }
  }
  std::stable_sort(vars.begin(), vars.end(),
                   [](const Candidate& a, const Candidate& b) { return a.est_s < b.est_s; });
  for (const auto& v : vars) {
    if (int(keep.size()) >= max_keep) break;
    keep.push_back(v);
  }
  // the copy and the best three multi-row copies, then the tiles
  std::stable_sort(out.begin(), out.end(),
                   [](const Candidate& a, const Candidate& b) { return a.est_s < b.est_s; });
  std::vector<Candidate> rows_keep;
  int nrows = 0, nvrows = 0;
  for (const auto& q : out)
    if (!q.rows || (q.vec > 1 ? nvrows++ < 2 : nrows++ < 3)) rows_keep.push_back(q);
  out.swap(rows_keep);
  out.insert(out.end(), keep.begin(), keep.end());
  std::stable_sort(out.begin(), out.end(),
                   [](const Candidate& a, const Candidate& b) { return a.est_s < b.est_s; });
  // the best vector multi-row copy stays among the candidates even when the
  // model ranks it below the cut (the autotuner decides)
  Candidate best_vrow;
  bool have_vrow = false, kept_vrow = false;
  for (size_t i = 0; i < out.size(); ++i)
    if (out[i].rows && out[i].vec > 1) {
      if (!have_vrow) best_vrow = out[i];
      have_vrow = true;
      kept_vrow = kept_vrow || int(i) < max_keep;
    }
  if (int(out.size()) > max_keep) out.resize(max_keep);
  if (have_vrow && !kept_vrow && max_keep > 1) out.back() = best_vrow;
  // the TMA-staged tile of a two-index transpose, where its strides allow a
  // tensor map: always kept among the candidates (the autotuner decides);
  // modelled at 0.96 of the copy bandwidth (measured 1-6 % above tile2 on
  // aligned 2D FP32 transposes)
  if (!flat && tma2d_eligible(c, din) && max_keep > 0) {
    Candidate k;
    k.variant = VAR_TMA;
    k.ta = 128 / esA;
    k.tb = 32 * kTmaBoxes;
    k.seg_a = double(k.ta);
    k.seg_b = 32.0;
    k.est_s = n * double(esA + esB + (bnz ? esB : 0)) / (0.96 * kHbmBytesPerS) + 2e-6;
    if (int(out.size()) >= max_keep) out.pop_back();
    out.push_back(k);
    std::stable_sort(out.begin(), out.end(),
                     [](const Candidate& a, const Candidate& b) { return a.est_s < b.est_s; });
  }
  return out;
}

void build_tile_params(const Canon& c, const Candidate& k, int din, TileParams* p,
                       std::vector<int32_t>* tabA, std::vector<int32_t>* tabB, int* smem_bytes) {
  *p = TileParams();
  int64_t ext[kMaxDim];
  {
    TileShape sh{k.has_c, k.ga, k.gb, k.ta, k.tb};
    tile_extents(c, sh, ext);
  }
  const int LC = k.has_c ? int(c.s[0]) : 1;
  int LA = 1, LB = 1, fullA = 1, fullB = 1;
  for (size_t i = 0; i < k.ga.size(); ++i) {
    LA *= int(ext[k.ga[i]]);
    if (i + 1 < k.ga.size()) fullA *= int(ext[k.ga[i]]);
  }
  for (size_t i = 0; i < k.gb.size(); ++i) {
    LB *= int(ext[k.gb[i]]);
    if (i + 1 < k.gb.size()) fullB *= int(ext[k.gb[i]]);
  }
  p->LC = LC;
  p->LA = LA;
  p->LB = LB;
  p->U = LC * LA;
  p->W = LC * LB;
  p->V = LC * LA * LB;
  p->fullA = fullA;
  p->fullB = fullB;
  p->saU = int32_t(c.sa[0]);
  p->sbV = int32_t(c.sb[c.perm[0]]);
  // cross offsets: A offset of GB's coordinates (lb), B offset of GA's coordinates (la)
  tabA->clear();
  tabB->clear();
  if (k.gb.size() <= 1) {
    p->crossA_lin = k.gb.empty() ? 0 : int32_t(c.sa[k.gb[0]]);
  } else {
    p->crossA_tab = 1;
    tabA->resize(LB);
    for (int lb = 0; lb < LB; ++lb) {
      int64_t r = lb, off = 0;
      for (int m : k.gb) {
        off += (r % ext[m]) * c.sa[m];
        r /= ext[m];
      }
      (*tabA)[lb] = int32_t(off);
    }
  }
  if (k.ga.size() <= 1) {
    p->crossB_lin = k.ga.empty() ? 0 : int32_t(c.sb[k.ga[0]]);
  } else {
    p->crossB_tab = 1;
    tabB->resize(LA);
    for (int la = 0; la < LA; ++la) {
      int64_t r = la, off = 0;
      for (int m : k.ga) {
        off += (r % ext[m]) * c.sb[m];
        r /= ext[m];
      }
      (*tabB)[la] = int32_t(off);
    }
  }
  // grid
  uint64_t ntiles = 1;
  p->ngrid = 0;
  const int cutA = k.ga.empty() ? -1 : k.ga.back();
  const int cutB = k.gb.empty() ? -1 : k.gb.back();
  for (int gk : k.order) {
    GridDim& g = p->g[p->ngrid++];
    const int64_t nb = (c.s[gk] + ext[gk] - 1) / ext[gk];
    g.div = make_fastdiv(uint32_t(nb));
    g.stepA = ext[gk] * c.sa[gk];
    g.stepB = ext[gk] * c.sb[gk];
    g.kind = 0;
    g.t = int(ext[gk]);
    g.s = int(std::min<int64_t>(c.s[gk], INT32_MAX));
    if (gk == cutA && ext[gk] < c.s[gk]) g.kind = 1;
    if (gk == cutB && ext[gk] < c.s[gk]) g.kind = 2;
    ntiles *= uint64_t(nb);
  }
  p->ntiles = uint32_t(ntiles);
  p->swz = p->ngrid >= 2 ? uint32_t(k.swz) : 0u;
  const int smem_cap = 160 * 1024;
  p->P = pick_pitch(p->U, LC, LB, din, smem_cap);
  // thread steps
  p->rd_du = kThreads % p->U;
  p->rd_dlb = kThreads / p->U;
  p->wr_dlc = kThreads % LC;
  p->wr_dlb = (kThreads / LC) % LB;
  p->wr_dla = kThreads / (LC * LB);
  p->divU = make_fastdiv(uint32_t(p->U));
  p->divLC = make_fastdiv(uint32_t(LC));
  p->divLB = make_fastdiv(uint32_t(LB));
  p->divW = make_fastdiv(uint32_t(p->W));
  if (k.pk) {
    // packed-lane layouts of both sides, for a whole tile and for the tile a
    // cut index leaves short (remA = fullA * (s mod t), likewise remB)
    const int Kt = k.kt ? k.kt : tile_k_for(stage_bytes(din));
    int edgeA = LA, edgeB = LB;
    if (cutA >= 0 && ext[cutA] < c.s[cutA] && c.s[cutA] % ext[cutA]) edgeA = fullA * int(c.s[cutA] % ext[cutA]);
    if (cutB >= 0 && ext[cutB] < c.s[cutB] && c.s[cutB] % ext[cutB]) edgeB = fullB * int(c.s[cutB] % ext[cutB]);
    pack_layout(LA, LB, k.pk, Kt, k.ju, &p->pkA[0]);
    pack_layout(edgeA, LB, k.pk, Kt, k.ju, &p->pkA[1]);
    pack_layout(LB, LA, k.pk, Kt, k.jw, &p->pkB[0]);
    pack_layout(edgeB, LA, k.pk, Kt, k.jw, &p->pkB[1]);
  }
  if (k.rj) {
    // packed rows: g threads per row of LC elements, and the row counts of
    // a whole tile's A side and of the short last block's
    const int Kt = k.kt ? k.kt : tile_k_for(stage_bytes(din));
    int edgeA = LA;
    if (cutA >= 0 && ext[cutA] < c.s[cutA] && c.s[cutA] % ext[cutA]) edgeA = fullA * int(c.s[cutA] % ext[cutA]);
    pack_layout(LC, LA * LB, kThreads, Kt, k.rj, &p->pkA[0]);
    p->divRA[0] = make_fastdiv(uint32_t(LA));
    p->divRA[1] = make_fastdiv(uint32_t(edgeA));
  }
  *smem_bytes = int(((tabA->size() + tabB->size()) * sizeof(int32_t) + 15) & ~size_t(15)) +
                p->P * LB * stage_bytes(din);
}

void build_amax_rows(const Canon& c, int elem_bytes, RowParams* p) {
  // the FP8 pre-pass reads A only: neighbouring indices that are dense in A
  // merge whatever B's order (longer rows to stream)
  Canon a = c;
  int n = 0;
  for (int k = 0; k < c.N; ++k) {
    if (n > 0 && c.sa[k] == a.sa[n - 1] * a.s[n - 1]) {
      a.s[n - 1] *= c.s[k];
    } else {
      a.s[n] = c.s[k];
      a.sa[n] = c.sa[k];
      a.sb[n] = c.sb[k];
      ++n;
    }
  }
  a.N = n;
  // chunks of at most 256 elements: a warp streams a few chunks at a time,
  // and long rows still give every SM many warps' work
  build_row_params(a, a.s[0] <= 256 ? a.s[0] : 256, p);
  // 16-byte loads where every chunk starts and ends on a 16-byte boundary
  // (relative to A's base; the launch checks the base itself)
  const int v = elem_bytes > 0 && elem_bytes < 16 ? 16 / elem_bytes : 1;
  bool ok = v > 1 && p->sa0 == 1 && p->len % v == 0 && p->chunk % v == 0;
  for (int i = 0; ok && i < p->nrd; ++i) ok = p->stA[i] % v == 0;
  p->vec = ok ? v : 1;
}

void build_row_params(const Canon& c, int64_t chunk, RowParams* p) {
  *p = RowParams();
  p->len = c.s[0];
  p->sa0 = c.sa[0];
  p->sb0 = c.sb[0];
  p->chunk = chunk > 0 ? chunk : c.s[0];
  const int64_t nch = (p->len + p->chunk - 1) / p->chunk;
  p->chunks = make_fastdiv(uint32_t(nch));
  uint64_t rows = 1;
  p->nrd = 0;
  for (int k = 1; k < c.N; ++k) {
    p->div[p->nrd] = make_fastdiv(uint32_t(c.s[k]));
    p->stA[p->nrd] = c.sa[k];
    p->stB[p->nrd] = c.sb[k];
    ++p->nrd;
    rows *= uint64_t(c.s[k]);
  }
  p->nitems = uint32_t(rows * uint64_t(nch));
  p->vec = 1;
}

namespace {

// One whole tile (no cut index short) run through the kernel's own index
// walks on the host collects every element's A offset, B offset and
// shared-memory position.  The slots then take the elements in increasing A
// offset (loads) and increasing B offset (stores): consecutive threads touch
// consecutive addresses on both sides whatever the tile's index structure, so
// a tile whose footprint is contiguous in A and in B (e.g. two small indices
// swapped) is read and written as two dense blocks.
struct SlotElem {
  int32_t off;
  int32_t pos;
};

template <int K>
void slot_tables_k(const TileParams& p, int stage_words, const std::vector<int32_t>& tabA,
                   const std::vector<int32_t>& tabB, std::vector<int32_t>* out, int* smem_elems) {
  const TileCoord c{0, 0, p.LA, p.LB};
  std::vector<SlotElem> rd, wr;
  rd.reserve(size_t(p.V));
  wr.reserve(size_t(p.V));
  for (int t = 0; t < kThreads; ++t) {
    int u0, lb0, lc0, lbw0, la0;
    flat_starts(p, t, u0, lb0, lc0, lbw0, la0);
    auto on_rd = [&](int, bool ok, int32_t off, int pos) {
      if (ok) rd.push_back({off, pos});
    };
    auto on_wr = [&](int, bool ok, int32_t off, int pos) {
      if (ok) wr.push_back({off, pos});
    };
    if (p.crossA_tab) walk_read<K, true>(c, p, tabA.data(), u0, lb0, on_rd);
    else walk_read<K, false>(c, p, tabA.data(), u0, lb0, on_rd);
    if (p.crossB_tab) walk_write<K, true>(c, p, tabB.data(), lc0, lbw0, la0, on_wr);
    else walk_write<K, false>(c, p, tabB.data(), lc0, lbw0, la0, on_wr);
  }
  auto by_off = [](const SlotElem& a, const SlotElem& b) { return a.off < b.off || (a.off == b.off && a.pos < b.pos); };
  std::sort(rd.begin(), rd.end(), by_off);
  std::sort(wr.begin(), wr.end(), by_off);
  // Shared-memory layout of the slot kernel: the element of load rank f sits
  // at q = f + (f / g) * s, and then, with x != 0, at q with its low five
  // bits XORed by x times its 32-element block number (a permutation inside
  // each block of 32).  The loads' stores then hit 32 distinct banks per
  // warp (for g >= 32), and the stores' loads, which step through the load
  // ranks by the tile's strides, are spread over the banks by the padding or
  // the swizzle.  (g, s, x) is chosen here by counting the shared-memory
  // wavefronts of both phases, warp by warp, for a few candidates (4-byte
  // banks; an 8-byte element is two words).  The walk's own position
  // (lb*P + la*LC + lc) still gives the tile coordinate.
  std::vector<int32_t> rank(size_t(p.P) * size_t(p.LB), -1);
  for (size_t f = 0; f < rd.size(); ++f) rank[size_t(rd[f].pos)] = int32_t(f);
  const int words = stage_words;
  auto layout = [](int64_t f, int g, int sp, int x) {
    const int64_t q = g ? f + (f / g) * sp : f;
    return x ? (q & ~int64_t(31)) | ((q ^ ((q >> 5) * x)) & 31) : q;
  };
  auto wavefronts = [&](int g, int sp, int x) {
    auto lay = [&](int64_t f) { return layout(f, g, sp, x); };
    int64_t total = 0;
    int cnt[32];
    for (int phase = 0; phase < 2; ++phase) {
      const std::vector<SlotElem>& v = phase ? wr : rd;
      for (size_t w0 = 0; w0 < v.size(); w0 += 32) {
        // one warp access: 32 consecutive slots of one k (kThreads % 32 == 0)
        std::fill(cnt, cnt + 32, 0);
        int worst = 0;
        for (size_t j = w0; j < std::min(v.size(), w0 + 32); ++j) {
          const int64_t f = phase ? rank[size_t(v[j].pos)] : int64_t(j);
          const int64_t word = lay(f) * words;
          for (int x = 0; x < words; ++x) worst = std::max(worst, ++cnt[(word + x) & 31]);
        }
        total += worst;
      }
    }
    return total;
  };
  static const int kLayouts[][3] = {{32, 1, 0}, {0, 0, 0}, {0, 0, 1}, {0, 0, 3}, {0, 0, 5}, {0, 0, 7},
                                    {64, 1, 0}, {128, 1, 0}, {32, 3, 0}, {32, 5, 0}, {32, 2, 0}, {32, 1, 1}};
  int bg = 32, bs = 1, bx = 0;
  int64_t best = -1;
  for (const auto& l : kLayouts) {
    const int64_t w = wavefronts(l[0], l[1], l[2]);
    if (best < 0 || w < best) {
      best = w;
      bg = l[0];
      bs = l[1];
      bx = l[2];
    }
  }
  std::vector<int32_t> remap(rank.size(), -1);
  int32_t top = 0;
  for (size_t f = 0; f < rd.size(); ++f) {
    const int32_t at = int32_t(layout(int64_t(f), bg, bs, bx));
    remap[size_t(rd[f].pos)] = at;
    top = std::max(top, at + 1);
  }
  *smem_elems = top;
  // layout (int32 units): read pairs, write pairs (K*kThreads*2 each), then
  // read and write tile coordinates (K*kThreads each)
  // layout (int32 units, R = K * kThreads): offsets [load R | store R],
  // tile coordinates [load R | store R], then 16-bit shared-memory positions
  // [load R/2 | store R/2]; slot k of thread t is entry ((k/4)*kThreads + t)*4
  // + k%4 of its region (16-bit entries for the positions)
  int32_t* q = out->data();
  const size_t R = size_t(K) * kThreads;
  uint16_t* posq = reinterpret_cast<uint16_t*>(q + 4 * R);
  auto put = [&](int phase, size_t f, const SlotElem* e) {
    const size_t k = f / kThreads, t = f % kThreads;
    const size_t at = ((k / 4) * kThreads + t) * 4 + (k & 3);
    q[size_t(phase) * R + at] = e ? e->off : 0;
    posq[size_t(phase) * R + at] = uint16_t(e ? remap[size_t(e->pos)] : 0xffff);
    // the element's (la, lb) in the tile, from its shared-memory position
    // (lb * P + la * LC + lc); 0xffffffff marks an empty slot
    uint32_t lalb = 0xffffffffu;
    if (e) {
      const int lb = e->pos / p.P, la = (e->pos - lb * p.P) / p.LC;
      lalb = (uint32_t(la) << 16) | uint32_t(lb);
    }
    q[2 * R + size_t(phase) * R + at] = int32_t(lalb);
  };
  for (size_t f = 0; f < size_t(K) * kThreads; ++f) {
    put(0, f, f < rd.size() ? &rd[f] : nullptr);
    put(1, f, f < wr.size() ? &wr[f] : nullptr);
  }
}

}  // namespace

size_t slot_table_ints(int din) { return size_t(tile_k_for(stage_bytes(din))) * kThreads * 5; }

int build_slot_tables(const TileParams& p, int din, const std::vector<int32_t>& tabA,
                      const std::vector<int32_t>& tabB, std::vector<int32_t>* out) {
  out->assign(slot_table_ints(din), 0);
  int elems = 0;
  const int K = tile_k_for(stage_bytes(din));
  if (K == 16) slot_tables_k<16>(p, stage_bytes(din) / 4, tabA, tabB, out, &elems);
  else if (K == 8) slot_tables_k<8>(p, stage_bytes(din) / 4, tabA, tabB, out, &elems);
  else slot_tables_k<4>(p, stage_bytes(din) / 4, tabA, tabB, out, &elems);
  return elems * stage_bytes(din);
}

}  // namespace ttc
