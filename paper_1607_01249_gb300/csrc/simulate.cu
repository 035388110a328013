// simulate.cu -- host-side schedule checker (include/ttc_debug.h).
//
// Runs the kernels' own index walks (kernels.cuh, compiled for the host) for
// every tile / row chunk and every thread, and checks bounds, coverage and
// the element mapping of Eq. 1 against the problem as given to ttc_plan.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ttc.h"
#include "../../include/ttc_debug.h"
#include "kernels.cuh"
#include "plan_impl.h"
#include "batch_impl.h"
#include "planner.h"
#include "rowvec.h"
#include "tma2d.h"

using namespace ttc;

namespace {

template <int JU, int K, bool FULL, class F>
void read2j(const TileCoord& c, const TileParams& tp, const int32_t* tab, int ln, int wp, F&& f) {
  if (tp.crossA_tab) walk2_read<JU, K, FULL, true, true>(c, tp, tab, ln, wp, f);
  else walk2_read<JU, K, FULL, false, true>(c, tp, tab, ln, wp, f);
}

template <int K, bool FULL, class F>
bool read2(int ju, const TileCoord& c, const TileParams& tp, const int32_t* tab, int ln, int wp, F&& f) {
  if (ju == 1) read2j<1, K, FULL>(c, tp, tab, ln, wp, f);
  else if (ju == 2) read2j<2, K, FULL>(c, tp, tab, ln, wp, f);
  else if (ju == 4) read2j<4, K, FULL>(c, tp, tab, ln, wp, f);
  else return false;
  return true;
}

template <int JW, int K, bool FULL, class F>
void write2j(const TileCoord& c, const TileParams& tp, const int32_t* tab, int ln, int wp, F&& f) {
  int sp[JW];
  walk2_lane_consts<JW>(tp, ln, sp);
  if (tp.crossB_tab) walk2_write<JW, K, FULL, true, true>(c, tp, tab, ln, wp, sp, f);
  else walk2_write<JW, K, FULL, false, true>(c, tp, tab, ln, wp, sp, f);
}

template <int K, bool FULL, class F>
bool write2(int jw, const TileCoord& c, const TileParams& tp, const int32_t* tab, int ln, int wp, F&& f) {
  if (jw == 1) write2j<1, K, FULL>(c, tp, tab, ln, wp, f);
  else if (jw == 2) write2j<2, K, FULL>(c, tp, tab, ln, wp, f);
  else if (jw == 4) write2j<4, K, FULL>(c, tp, tab, ln, wp, f);
  else return false;
  return true;
}

struct Checker {
  const ttc_plan_s* p;
  int64_t stA[kMaxDim], stB[kMaxDim];
  int64_t spanA, spanB;
  std::vector<uint8_t> wrote;   // per B element of the span
  int64_t writes = 0;
  std::string err;

  explicit Checker(const ttc_plan_s* plan) : p(plan) {
    int64_t a = 1, b = 1;
    for (int k = 0; k < p->ndim; ++k) {
      stA[k] = a;
      a *= p->outerA0[k];
    }
    for (int d = 0; d < p->ndim; ++d) {
      stB[d] = b;
      b *= p->outerB0[d];
    }
    spanA = p->canon.spanA;
    spanB = p->canon.spanB;
    wrote.assign(size_t(spanB), 0);
  }

  bool fail(const char* what, int64_t x, int64_t y) {
    if (err.empty()) {
      char buf[256];
      std::snprintf(buf, sizeof(buf), "%s (%lld, %lld)", what, (long long)x, (long long)y);
      err = buf;
    }
    return false;
  }

  // Eq. 1: the B offset of the A element at offset offA (outer sizes as given)
  bool expected_b(int64_t offA, int64_t* offB) {
    int64_t idx[kMaxDim];
    int64_t r = offA;
    for (int k = p->ndim - 1; k >= 0; --k) {
      idx[k] = r / stA[k];
      r -= idx[k] * stA[k];
    }
    for (int k = 0; k < p->ndim; ++k)
      if (idx[k] < 0 || idx[k] >= p->sizes0[k]) return fail("A offset outside the sub-tensor", offA, k);
    int64_t b = 0;
    for (int d = 0; d < p->ndim; ++d) b += idx[p->perm0[d]] * stB[d];
    *offB = b;
    return true;
  }

  bool pair(int64_t offA, int64_t offB) {
    if (offA < 0 || offA >= spanA) return fail("A access out of range", offA, spanA);
    if (offB < 0 || offB >= spanB) return fail("B access out of range", offB, spanB);
    int64_t want = 0;
    if (!expected_b(offA, &want)) return false;
    if (want != offB) return fail("element lands at the wrong B offset", offB, want);
    if (wrote[size_t(offB)]) return fail("B element written twice", offB, offA);
    wrote[size_t(offB)] = 1;
    ++writes;
    return true;
  }

  bool tile(const Candidate& k) {
    const int K = tile_k_for(stage_bytes_of(p->din));
    if (K == 4) return tile_k<4>(k);
    if (K == 8) return tile_k<8>(k);
    return tile_k<16>(k);
  }

  // the batch body's tiles (half the slots per thread)
  bool tile_batch(const Candidate& k) {
    if (p->din == DT_F64) return tile_k<batch_k_for(8)>(k);
    return tile_k<batch_k_for(4)>(k);
  }

  template <int K>
  bool tile_k(const Candidate& k) {
    TileParams tp;
    std::vector<int32_t> ta, tb;
    int smem = 0;
    build_tile_params(p->canon, k, p->din, &tp, &ta, &tb, &smem);
    if (smem > 200 * 1024) return fail("shared memory over budget", smem, 0);
    const int nthreads = k.pk ? k.pk : kThreads;
    if ((k.pk || k.ju) && (tp.saU != 1 || tp.sbV != 1))
      return fail("warp-mapped or packed-lane tile without unit-stride runs", tp.saU, tp.sbV);
    const int cover = (k.rows && k.vec > 1) ? kThreads * kRowVecK * k.vec : nthreads * K;
    if (tp.V > cover) return fail("tile larger than the threads cover", tp.V, cover);
    std::vector<int32_t> slots;
    int sbytes = 0;
    if (k.slots) sbytes = build_slot_tables(tp, p->din, ta, tb, &slots);
    const int ncap = k.slots ? sbytes / stage_bytes_of(p->din) : tp.P * tp.LB;
    if (k.slots && sbytes > 200 * 1024) return fail("shared memory over budget", sbytes, 0);
    std::vector<int64_t> posA(static_cast<size_t>(ncap));
    std::vector<uint8_t> used(static_cast<size_t>(ncap));
    for (uint32_t tid = 0; tid < tp.ntiles; ++tid) {
      const TileCoord c = tile_coord(tid, tp);
      std::fill(posA.begin(), posA.end(), -1);
      std::fill(used.begin(), used.end(), 0);
      bool ok = true;
      auto on_read = [&](int, bool valid, int32_t off, int pos) {
        if (!ok || !valid) return;
        if (pos < 0 || pos >= ncap) { ok = fail("shared-memory position out of range (read)", pos, ncap); return; }
        if (posA[size_t(pos)] != -1) { ok = fail("shared-memory position written twice", pos, tid); return; }
        posA[size_t(pos)] = c.baseA + off;
      };
      auto on_write = [&](int, bool valid, int32_t off, int pos) {
        if (!ok || !valid) return;
        if (pos < 0 || pos >= ncap) { ok = fail("shared-memory position out of range (write)", pos, ncap); return; }
        if (posA[size_t(pos)] < 0) { ok = fail("shared-memory position read but never written", pos, tid); return; }
        if (used[size_t(pos)]) { ok = fail("shared-memory position read twice", pos, tid); return; }
        used[size_t(pos)] = 1;
        ok = pair(posA[size_t(pos)], c.baseB + off);
      };
      const bool full = c.remA == tp.LA && c.remB == tp.LB;
      if (k.rj) {
        // packed rows: no staging either
        for (int t = 0; t < kThreads && ok; ++t) {
          auto on_pair = [&](int, bool valid, int32_t offA, int32_t offB) {
            if (ok && valid) ok = pair(c.baseA + offA, c.baseB + offB);
          };
          if (!rowsp_walk<K>(k.rj, c, tp, ta, tb, t, on_pair)) ok = fail("unknown packed-row layout", k.rj, 0);
        }
        if (!ok) return false;
        continue;
      }
      if (k.rows && k.vec > 1) {
        // the vector multi-row copy (rowvec.cu): vectors of V elements, each
        // inside one row, 16-byte aligned relative to A's base and V-aligned
        // relative to B's
        const int V = k.vec;
        if (tp.LC % V) return fail("vector row copy: row length not a multiple of the vector", tp.LC, V);
        for (int t = 0; t < kThreads && ok; ++t)
          walk_rows_vec(c, tp, V, t, [&](int, bool valid, int32_t offA, int32_t offB) {
            if (!ok || !valid) return;
            if ((c.baseA + offA) % V || (c.baseB + offB) % V) {
              ok = fail("vector row copy: unaligned vector", c.baseA + offA, c.baseB + offB);
              return;
            }
            for (int i = 0; i < V && ok; ++i) ok = pair(c.baseA + offA + i, c.baseB + offB + i);
          });
        if (!ok) return false;
        continue;
      }
      if (k.rows) {
        // no staging: each element goes straight from A to B
        for (int t = 0; t < kThreads && ok; ++t)
          walk_rows<K>(c, tp, t, [&](int, bool valid, int32_t offA, int32_t offB) {
            if (ok && valid) ok = pair(c.baseA + offA, c.baseB + offB);
          });
        if (!ok) return false;
        continue;
      }
      if (k.slots) {
        // tile_slots_kernel: slot kk of thread t of phase f is entry
        // ((kk/4)*kThreads + t)*4 + kk%4 of the phase's offset, coordinate
        // and 16-bit position regions (position 0xffff: empty); a tile cut
        // short keeps the slots whose coordinate (la << 16 | lb) lies inside
        const size_t R = size_t(K) * kThreads;
        const uint16_t* posq = reinterpret_cast<const uint16_t*>(slots.data() + 4 * R);
        for (int f = 0; f < 2 && ok; ++f)
          for (int t = 0; t < kThreads && ok; ++t)
            for (int kk = 0; kk < K && ok; ++kk) {
              const size_t at = (size_t(kk / 4) * kThreads + size_t(t)) * 4 + (kk & 3);
              const int32_t off = slots[size_t(f) * R + at];
              const uint32_t lalb = uint32_t(slots[2 * R + size_t(f) * R + at]);
              const int pos = posq[size_t(f) * R + at];
              const bool in = full || (int(lalb >> 16) < c.remA && int(lalb & 0xffffu) < c.remB);
              const bool valid = in && pos != 0xffff;
              if (off < 0) ok = fail("slot table: negative offset", off, pos);
              else if (f == 0) on_read(kk, valid, off, pos);
              else on_write(kk, valid, off, pos);
            }
      } else if (k.pk) {
        if (tp.LC != 1) return fail("packed-lane tile with a C index", tp.LC, 0);
        if (k.pk != 256 && k.pk != 512) ok = fail("unknown packed-lane thread count", k.pk, 0);
        else ok = packed<K>(k.pk, k.ju, k.jw, c, tp, ta, tb, on_read, on_write);
      } else if (k.ju == 0) {
        for (int t = 0; t < kThreads && ok; ++t) {
          int u0, lb0, lc0, lbw0, la0;
          flat_starts(tp, t, u0, lb0, lc0, lbw0, la0);
          if (tp.crossA_tab) walk_read<K, true>(c, tp, ta.data(), u0, lb0, on_read);
          else walk_read<K, false>(c, tp, ta.data(), u0, lb0, on_read);
        }
        for (int t = 0; t < kThreads && ok; ++t) {
          int u0, lb0, lc0, lbw0, la0;
          flat_starts(tp, t, u0, lb0, lc0, lbw0, la0);
          if (tp.crossB_tab) walk_write<K, true>(c, tp, tb.data(), lc0, lbw0, la0, on_write);
          else walk_write<K, false>(c, tp, tb.data(), lc0, lbw0, la0, on_write);
        }
      } else {
        bool known = true;
        for (int t = 0; t < kThreads && ok; ++t) {
          const int ln = t & 31, wp = t >> 5;
          if (full) known = read2<K, true>(k.ju, c, tp, ta.data(), ln, wp, on_read);
          else known = read2<K, false>(k.ju, c, tp, ta.data(), ln, wp, on_read);
          if (!known) ok = fail("unknown lane layout", k.ju, 0);
        }
        for (int t = 0; t < kThreads && ok; ++t) {
          const int ln = t & 31, wp = t >> 5;
          if (full) known = write2<K, true>(k.jw, c, tp, tb.data(), ln, wp, on_write);
          else known = write2<K, false>(k.jw, c, tp, tb.data(), ln, wp, on_write);
          if (!known) ok = fail("unknown lane layout", k.jw, 0);
        }
      }
      for (int q = 0; q < ncap && ok; ++q)
        if (posA[size_t(q)] >= 0 && !used[size_t(q)]) ok = fail("staged element never written out", q, tid);
      if (!ok) return false;
    }
    return true;
  }

  template <int J, int K, class F>
  void rowsp_j(const TileCoord& c, const TileParams& tp, const std::vector<int32_t>& ta,
               const std::vector<int32_t>& tb, int t, F& f) {
    if (tp.crossA_tab) {
      if (tp.crossB_tab) walk_rowsp<J, K, true, true>(c, tp, ta.data(), tb.data(), t, f);
      else walk_rowsp<J, K, true, false>(c, tp, ta.data(), tb.data(), t, f);
    } else {
      if (tp.crossB_tab) walk_rowsp<J, K, false, true>(c, tp, ta.data(), tb.data(), t, f);
      else walk_rowsp<J, K, false, false>(c, tp, ta.data(), tb.data(), t, f);
    }
  }
  template <int K, class F>
  bool rowsp_walk(int j, const TileCoord& c, const TileParams& tp, const std::vector<int32_t>& ta,
                  const std::vector<int32_t>& tb, int t, F& f) {
    if (j == 1) rowsp_j<1, K>(c, tp, ta, tb, t, f);
    else if (j == 2) rowsp_j<2, K>(c, tp, ta, tb, t, f);
    else if (j == 4 && K >= 4) rowsp_j<(K >= 4 ? 4 : 1), K>(c, tp, ta, tb, t, f);
    else if (j == 8 && K >= 8) rowsp_j<(K >= 8 ? 8 : 1), K>(c, tp, ta, tb, t, f);
    else if (j == 16 && K >= 16) rowsp_j<(K >= 16 ? 16 : 1), K>(c, tp, ta, tb, t, f);
    else return false;
    return true;
  }

  // tilep_kernel: every thread's load walk, then every thread's store walk
  template <int J, int K, class F>
  void packed_read(const TileCoord& c, const TileParams& tp, const std::vector<int32_t>& ta, int t, F& f) {
    if (tp.crossA_tab) walkp_read<0, J, K, true, true>(c, tp, ta.data(), t, f);
    else walkp_read<0, J, K, false, true>(c, tp, ta.data(), t, f);
  }
  template <int J, int K, class F>
  void packed_write(const TileCoord& c, const TileParams& tp, const std::vector<int32_t>& tb, int t, F& f) {
    if (tp.crossB_tab) walkp_write<0, J, K, true, true>(c, tp, tb.data(), t, f);
    else walkp_write<0, J, K, false, true>(c, tp, tb.data(), t, f);
  }
  template <int K, class FR, class FW>
  bool packed(int nt, int ju, int jw, const TileCoord& c, const TileParams& tp, const std::vector<int32_t>& ta,
              const std::vector<int32_t>& tb, FR& on_read, FW& on_write) {
    for (int t = 0; t < nt && err.empty(); ++t) {
      if (ju == 1) packed_read<1, K>(c, tp, ta, t, on_read);
      else if (ju == 2) packed_read<2, K>(c, tp, ta, t, on_read);
      else if (ju == 4) packed_read<4, K>(c, tp, ta, t, on_read);
      else return fail("unknown packed-lane chunk count", ju, 0);
    }
    for (int t = 0; t < nt && err.empty(); ++t) {
      if (jw == 1) packed_write<1, K>(c, tp, tb, t, on_write);
      else if (jw == 2) packed_write<2, K>(c, tp, tb, t, on_write);
      else if (jw == 4) packed_write<4, K>(c, tp, tb, t, on_write);
      else return fail("unknown packed-lane chunk count", jw, 0);
    }
    return err.empty();
  }

  bool copy(const Candidate& k) {
    RowParams rp;
    build_row_params(p->canon, k.chunk, &rp);
    for (uint32_t item = 0; item < rp.nitems; ++item) {
      const RowCoord rc = row_coord(item, rp);
      if (k.vec > 1 && (rc.offA % k.vec || rc.offB % k.vec || rc.start % k.vec || rc.end % k.vec))
        return fail("vector access not aligned", item, k.vec);
      for (int64_t x = rc.start; x < rc.end; ++x)
        if (!pair(rc.offA + x * rp.sa0, rc.offB + x * rp.sb0)) return false;
    }
    return true;
  }

  // the TMA tile (tma2d.cu): every tile, box, warp, lane and row of the box
  // as the kernel maps them
  bool tma(const Candidate&) {
    if (!tma2d_eligible(p->canon, p->din)) return fail("TMA tile on a problem it does not fit", 0, 0);
    const Tma2dGeom g = tma2d_geom(p->canon, p->din);
    const int es = dtype_size(p->din);
    for (int64_t t = 0; t < g.tiles && err.empty(); ++t) {
      int r0, c0;
      tma2d_origin(g, t, &r0, &c0);
      if (r0 % g.bx || r0 >= g.R || c0 >= g.C) return fail("TMA tile origin", r0, c0);
      for (int k = 0; k < kTmaBoxes && c0 + 32 * k < g.C; ++k)
        for (int w = 0; w < 8; ++w)
          for (int lane = 0; lane < 32; ++lane)
            for (int j = 0; j < g.bx / 8; ++j) {
              const int x = w + 8 * j, r = r0 + x, col = c0 + 32 * k + lane;
              const int sb = tma2d_smem_byte(x, lane, es);
              if (sb < 0 || sb + es > kTmaBoxBytes || sb % es) return fail("TMA box position", sb, x);
              if (r >= g.R || col >= g.C) continue;
              if (!pair(int64_t(r) + int64_t(col) * g.lda, int64_t(col) + int64_t(r) * g.ldb)) return false;
            }
    }
    return err.empty();
  }

  bool amax() {
    const RowParams& rp = p->amax_rows;
    std::vector<uint8_t> seen(size_t(spanA), 0);
    int64_t visits = 0;
    for (uint32_t item = 0; item < rp.nitems; ++item) {
      const RowCoord rc = row_coord(item, rp);
      if (rp.vec > 1 && (rp.sa0 != 1 || rc.offA % rp.vec || rc.start % rp.vec || rc.end % rp.vec))
        return fail("amax: 16-byte load not aligned", item, rp.vec);
      for (int64_t x = rc.start; x < rc.end; ++x) {
        const int64_t a = rc.offA + x * rp.sa0;
        if (a < 0 || a >= spanA) return fail("amax: A access out of range", a, spanA);
        if (seen[size_t(a)]) return fail("amax: element visited twice", a, item);
        seen[size_t(a)] = 1;
        int64_t b = 0;
        if (!expected_b(a, &b)) return false;
        ++visits;
      }
    }
    if (visits != p->canon.n) return fail("amax: wrong number of elements", visits, p->canon.n);
    return true;
  }
};

}  // namespace

extern "C" ttc_status ttc_debug_verify_schedule(ttc_plan_t plan, int candidate, char* msg, int msglen) {
  auto say = [&](const std::string& s) {
    if (msg && msglen > 0) {
      std::snprintf(msg, size_t(msglen), "%s", s.c_str());
    }
  };
  if (!plan || candidate >= int(plan->cands.size())) {
    say("bad plan or candidate");
    return TTC_ERR_INVALID_ARG;
  }
  say("");
  if (plan->canon.n == 0) return TTC_OK;
  Checker ck(plan);
  Candidate k;
  bool batch = candidate < 0;
  if (batch) {
    // batch-body schedule j = -1 - candidate (ttc_batch_*, the server): 0 is
    // the cost model's choice, the others those ttc_batch_autotune times
    if (plan->dout == DT_E4M3 || is_complex(plan->din)) return TTC_OK;    // never batched
    const int j = -1 - candidate;
    const std::vector<Candidate> bc = make_candidates(plan->canon, plan->din, plan->dout, plan->beta,
                                                      std::max(4, j + 1),
                                                      kThreads * batch_k_for(plan->din == DT_F64 ? 8 : 4));
    if (bc.empty()) return TTC_OK;    // not batchable: the batch runs it as a single-plan kernel
    if (j >= int(bc.size())) {
      say("no such batch candidate");
      return TTC_ERR_INVALID_ARG;
    }
    k = bc[size_t(j)];
    if (k.variant == VAR_COPY) k.chunk = kBatchCopyChunk / (plan->din == DT_F64 ? 2 : 1);
  } else {
    k = plan->cands[candidate];
  }
  bool ok = true;
  if (k.variant == VAR_TILE) ok = batch ? ck.tile_batch(k) : ck.tile(k);
  else if (k.variant == VAR_COPY) ok = ck.copy(k);
  else if (k.variant == VAR_TMA) ok = ck.tma(k);
  if (ok && ck.writes != plan->canon.n) ok = ck.fail("wrong number of B elements written", ck.writes, plan->canon.n);
  if (ok && plan->dout == DT_E4M3 && !batch) ok = ck.amax();
  if (!ok) {
    say(k.describe() + ": " + ck.err);
    return TTC_ERR_INVALID_ARG;
  }
  return TTC_OK;
}

extern "C" ttc_status ttc_debug_describe_candidate(ttc_plan_t plan, int candidate, char* buf, int buflen) {
  if (!plan || !buf || buflen <= 0 || candidate < 0 || candidate >= int(plan->cands.size()))
    return TTC_ERR_INVALID_ARG;
  std::snprintf(buf, size_t(buflen), "%s", plan->cands[size_t(candidate)].describe().c_str());
  return TTC_OK;
}

extern "C" ttc_status ttc_debug_slot_tables(ttc_plan_t plan, int candidate, int32_t* out, int64_t count,
                                            int64_t* needed) {
  if (!plan || !needed || candidate < 0 || candidate >= int(plan->cands.size())) return TTC_ERR_INVALID_ARG;
  const Candidate& k = plan->cands[size_t(candidate)];
  if (k.variant != VAR_TILE || !k.slots) return TTC_ERR_INVALID_ARG;
  TileParams tp;
  std::vector<int32_t> ta, tb, st;
  int smem = 0;
  build_tile_params(plan->canon, k, plan->din, &tp, &ta, &tb, &smem);
  (void)build_slot_tables(tp, plan->din, ta, tb, &st);
  *needed = int64_t(st.size());
  if (!out || count < int64_t(st.size())) return TTC_ERR_INVALID_ARG;
  std::memcpy(out, st.data(), st.size() * sizeof(int32_t));
  return TTC_OK;
}
