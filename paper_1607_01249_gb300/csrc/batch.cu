// batch.cu -- many permute-scale-adds in one persistent kernel launch
// (include/ttc.h, ttc_batch_*).
//
// Every problem of a batch is cut into tiles by its own plan.  A tile is
// processed by one CTA with one of three bodies:
//   BP_TILE -- the generic staged tile (flat walks, offset tables for both
//              cross offsets), for problems whose perm moves index 0 (the
//              warp-mapped walks of tile2_kernel measured slower here: the
//              batch's small problems leave most of their lanes idle);
//   BP_ROWS -- the multi-row copy (perm keeps index 0, short runs);
//   BP_COPY -- one chunk of one long run (perm keeps index 0, long runs).
// Resident CTAs claim tiles from one atomic counter (uneven problems balance
// themselves); a per-tile map names the problem, whose descriptor (pointers,
// tile parameters, epilogue) sits in one device arena owned by the batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ttc.h"
#include "batch_impl.h"
#include "kernels.cuh"
#include "launch.h"
#include "plan_impl.h"
#include "planner.h"

namespace ttc {

extern std::atomic<int64_t> g_launches;
cudaError_t grid_for(const void* fn, int smem, int64_t work, int* grid);

// --------------------------------------------------------------- device --

template <int DIN, int DOUT, bool BNZ, bool TAB>
__device__ __forceinline__ void batch_tile(const BatchDesc& d, const TileCoord& c, unsigned char* smem) {
  using S = stage_t<DIN>;
  using TO = store_t<DOUT>;
  constexpr int K = batch_k_for(sizeof(S));
  const WalkP p = walk_params(d.tp);      // registers, not shared-memory loads per element
  const int t = threadIdx.x;
  const store_t<DIN>* Ab = static_cast<const store_t<DIN>*>(d.A) + c.baseA;
  TO* Bb = static_cast<TO*>(d.B) + c.baseB;
  S v[K];
  TO bo[K] = {};
  if (d.path == BP_ROWS) {
    walk_rows<K>(c, p, t, [&](int k, bool, int32_t offA, int32_t offB) {
      v[k] = to_stage<DIN>(ldg_elem<DIN>(Ab + offA));
      if constexpr (BNZ) bo[k] = Bb[offB];
    });
    walk_rows<K>(c, p, t, [&](int k, bool ok, int32_t, int32_t offB) {
      if (ok) Bb[offB] = epilogue<DIN, DOUT>(v[k], bo[k], p.epi, 1.f);
    });
    return;
  }
  S* tile = reinterpret_cast<S*>(smem);
  int u0, lb0, lc0, lbw0, la0;
  flat_starts(p, t, u0, lb0, lc0, lbw0, la0);
  walk_read<K, TAB>(c, p, p.tabA, u0, lb0,
                    [&](int k, bool, int32_t off, int) { v[k] = to_stage<DIN>(ldg_elem<DIN>(Ab + off)); });
  walk_read<K, TAB>(c, p, p.tabA, u0, lb0, [&](int k, bool ok, int32_t, int pos) {
    if (ok) tile[pos] = v[k];
  });
  __syncthreads();
  if constexpr (BNZ)
    walk_write<K, TAB>(c, p, p.tabB, lc0, lbw0, la0, [&](int k, bool, int32_t off, int) { bo[k] = Bb[off]; });
  walk_write<K, TAB>(c, p, p.tabB, lc0, lbw0, la0, [&](int k, bool ok, int32_t off, int pos) {
    if (ok) Bb[off] = epilogue<DIN, DOUT>(tile[pos], bo[k], p.epi, 1.f);
  });
}

template <int DIN, int DOUT, bool BNZ>
__device__ __forceinline__ void batch_copy(const BatchDesc& d, const RowCoord& rc) {
  using S = stage_t<DIN>;
  using TO = store_t<DOUT>;
  constexpr int K = kBatchCopyChunk / kThreads / (sizeof(S) == 8 ? 2 : 1);
  const int64_t sa0 = d.rp.sa0, sb0 = d.rp.sb0;
  const Epilogue epi = d.rp.epi;
  const int t = threadIdx.x;
  const store_t<DIN>* Ar = static_cast<const store_t<DIN>*>(d.A) + rc.offA;
  TO* Br = static_cast<TO*>(d.B) + rc.offB;
  S v[K];
  TO bo[K] = {};
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t x = rc.start + t + int64_t(k) * kThreads;
    const int64_t xs = x < rc.end ? x : rc.start;
    v[k] = to_stage<DIN>(ldg_elem<DIN>(Ar + xs * sa0));
    if constexpr (BNZ) bo[k] = Br[xs * sb0];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t x = rc.start + t + int64_t(k) * kThreads;
    if (x < rc.end) Br[x * sb0] = epilogue<DIN, DOUT>(v[k], bo[k], epi, 1.f);
  }
}

// one claimed tile of one problem
template <int DIN, int DOUT>
__device__ __noinline__ void batch_unit(const BatchDesc& d, const TileRec& r, unsigned char* smem) {
  if (d.path == BP_COPY) {
    const RowCoord rc{r.baseA, r.baseB, int64_t(r.remA), int64_t(r.remA) + r.remB};
    if (d.rp.epi.beta_nz) batch_copy<DIN, DOUT, true>(d, rc);
    else batch_copy<DIN, DOUT, false>(d, rc);
  } else {
    const TileCoord c{r.baseA, r.baseB, r.remA, r.remB};
    // both cross offsets linear, or both from tables
    if (d.tp.crossA_tab) {
      if (d.tp.epi.beta_nz) batch_tile<DIN, DOUT, true, true>(d, c, smem);
      else batch_tile<DIN, DOUT, false, true>(d, c, smem);
    } else {
      if (d.tp.epi.beta_nz) batch_tile<DIN, DOUT, true, false>(d, c, smem);
      else batch_tile<DIN, DOUT, false, false>(d, c, smem);
    }
  }
}

__device__ __forceinline__ void batch_dispatch(const BatchDesc& d, const TileRec& r, unsigned char* smem) {
  switch (d.din * 4 + d.dout) {
    case DT_F32 * 4 + DT_F32: batch_unit<DT_F32, DT_F32>(d, r, smem); break;
    case DT_F32 * 4 + DT_F64: batch_unit<DT_F32, DT_F64>(d, r, smem); break;
    case DT_F32 * 4 + DT_BF16: batch_unit<DT_F32, DT_BF16>(d, r, smem); break;
    case DT_F64 * 4 + DT_F64: batch_unit<DT_F64, DT_F64>(d, r, smem); break;
    case DT_F64 * 4 + DT_F32: batch_unit<DT_F64, DT_F32>(d, r, smem); break;
    case DT_BF16 * 4 + DT_BF16: batch_unit<DT_BF16, DT_BF16>(d, r, smem); break;
    case DT_BF16 * 4 + DT_F32: batch_unit<DT_BF16, DT_F32>(d, r, smem); break;
    default: break;
  }
}

// The record of tile q of a problem, computed on the device (thread 0) when
// the launch has no precomputed records.
__device__ __forceinline__ TileRec device_rec(const BatchDesc& d, uint32_t prob, uint32_t q) {
  TileRec r;
  r.prob = prob;
  r.pad = 0;
  if (d.path == BP_COPY) {
    const RowCoord rc = row_coord(q, d.rp);
    r.baseA = rc.offA;
    r.baseB = rc.offB;
    r.remA = int32_t(rc.start);
    r.remB = int32_t(rc.end - rc.start);
  } else {
    const TileCoord c = tile_coord(q, d.tp);
    r.baseA = c.baseA;
    r.baseB = c.baseB;
    r.remA = c.remA;
    r.remB = c.remB;
  }
  return r;
}

// problem of global tile g: the last p with tile0[p] <= g (tile0 ascending,
// tile0[0] = 0, nprob entries)
__device__ __forceinline__ uint32_t find_problem(const uint32_t* __restrict__ tile0, uint32_t nprob, uint32_t g) {
  uint32_t lo = 0, hi = nprob;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(tile0 + mid) <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Persistent: resident CTAs claim tiles from one counter (uneven problems
// balance themselves).  The claim of the next tile is issued while the
// current one is processed; the current problem's descriptor is kept in
// shared memory and reloaded only when the problem changes.  A tile's record
// comes either from the precomputed array `recs` (ttc_batch_*, built once and
// replayed) or, when recs is null, from the problem's tile prefix `tile0`
// and its tile parameters on the device (the server, whose epochs are built
// per launch and should cost the host nothing per tile).
__global__ void __launch_bounds__(kThreads, 4) batch_kernel(const BatchDesc* __restrict__ descs,
                                                            const TileRec* __restrict__ recs,
                                                            const uint32_t* __restrict__ tile0, uint32_t nprob,
                                                            uint32_t total, uint32_t* counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  // the claimed tile, double-buffered: thread 0 records the next claim in the
  // other buffer before the end-of-tile barrier, which then also publishes it
  __shared__ uint32_t s_g[2], s_p[2];
  __shared__ TileRec s_rec[2];
  // raw storage: BatchDesc has member initializers, which a __shared__
  // variable cannot run
  __shared__ __align__(16) unsigned char s_desc_raw[sizeof(BatchDesc)];
  BatchDesc& s_desc = *reinterpret_cast<BatchDesc*>(s_desc_raw);
  constexpr int kWords = int(sizeof(BatchDesc) / sizeof(int4));
  static_assert(sizeof(BatchDesc) % sizeof(int4) == 0, "descriptor copied as 16-byte words");
  const int t = threadIdx.x;
  uint32_t have = 0xffffffffu;
  auto claim = [&](int b, uint32_t g) {   // thread 0: remember tile g and its problem in buffer b
    s_g[b] = g;
    if (g < total) {
      if (recs) {
        s_rec[b] = recs[g];
        s_p[b] = s_rec[b].prob;
      } else {
        s_p[b] = find_problem(tile0, nprob, g);
      }
    }
  };
  if (t == 0) claim(0, atomicAdd(counter, 1u));
  __syncthreads();
  for (int b = 0;; b ^= 1) {
    const uint32_t g = s_g[b];
    if (g >= total) break;
    const uint32_t prob = s_p[b];
    uint32_t gn = 0;
    if (t == 0) gn = atomicAdd(counter, 1u);
    if (prob != have) {
      const int4* src = reinterpret_cast<const int4*>(descs + prob);
      int4* dst = reinterpret_cast<int4*>(&s_desc);
      for (int i = t; i < kWords; i += kThreads) dst[i] = src[i];
      have = prob;
      __syncthreads();
    }
    if (!recs) {
      if (t == 0) s_rec[b] = device_rec(s_desc, prob, g - __ldg(tile0 + prob));
      __syncthreads();
    }
    const TileRec r = s_rec[b];
    batch_dispatch(s_desc, r, smem);
    // buffer b^1 was last read at the start of the previous tile, before the
    // previous end-of-tile barrier, so thread 0 may overwrite it now
    if (t == 0) claim(b ^ 1, gn);
    __syncthreads();   // the tile buffer, the descriptor and buffer b^1
  }
}

}  // namespace ttc

// ------------------------------------------------------------------ host --

namespace ttc {

namespace {

std::shared_ptr<const BatchTemplate> make_template(const ttc_plan_s* p) {
  auto t = std::make_shared<BatchTemplate>();
  if (p->canon.n == 0 || p->dout == DT_E4M3 || is_complex(p->din)) return t;
  BatchDesc* d = &t->d;
  std::memset(d, 0, sizeof(*d));
  d->din = p->din;
  d->dout = p->dout;
  // tiles for the batch body: the best schedule with at most its tile volume
  const std::vector<Candidate> bc =
      make_candidates(p->canon, p->din, p->dout, p->beta, 4, kThreads * batch_k_for(p->din == DT_F64 ? 8 : 4));
  const Candidate& k = bc.front();
  if (k.variant == VAR_TILE) {
    std::vector<int32_t> ta, tb;
    int sm = 0;
    build_tile_params(p->canon, k, p->din, &d->tp, &ta, &tb, &sm);
    d->path = k.rows ? BP_ROWS : BP_TILE;
    if (d->path == BP_TILE && (d->tp.crossA_tab || d->tp.crossB_tab)) {
      // the batch body has two walks: both cross offsets linear, or both
      // from tables (a linear one is then written out as a table)
      if (!d->tp.crossA_tab) {
        ta.resize(d->tp.LB);
        for (int i = 0; i < d->tp.LB; ++i) ta[i] = i * d->tp.crossA_lin;
        d->tp.crossA_tab = 1;
      }
      if (!d->tp.crossB_tab) {
        tb.resize(d->tp.LA);
        for (int i = 0; i < d->tp.LA; ++i) tb[i] = i * d->tp.crossB_lin;
        d->tp.crossB_tab = 1;
      }
      t->tabA_count = ta.size();
      t->tabs.insert(t->tabs.end(), ta.begin(), ta.end());
      t->tabs.insert(t->tabs.end(), tb.begin(), tb.end());
    }
    if (d->path == BP_TILE) t->smem = d->tp.P * d->tp.LB * (p->din == DT_F64 ? 8 : 4);
    d->ntiles = d->tp.ntiles;
    d->tp.epi = make_epilogue(p, nullptr);
  } else {
    build_row_params(p->canon, kBatchCopyChunk / (p->din == DT_F64 ? 2 : 1), &d->rp);
    d->path = BP_COPY;
    d->ntiles = d->rp.nitems;
    d->rp.epi = make_epilogue(p, nullptr);
  }
  t->ok = true;
  return t;
}

}  // namespace

namespace {

std::shared_ptr<const BatchTemplate> plan_template(ttc_plan_s* p) {
  std::lock_guard<std::mutex> lk(p->batch_mu);
  if (!p->batch_tmpl) p->batch_tmpl = make_template(p);
  return p->batch_tmpl;
}

}  // namespace

int64_t batch_tiles(ttc_plan_s* p) {
  const std::shared_ptr<const BatchTemplate> t = plan_template(p);
  return t->ok ? int64_t(t->d.ntiles) : -1;
}

bool batch_describe(ttc_plan_s* p, const void* A, void* B, BatchDesc* d, std::vector<int32_t>* tabs,
                    size_t* tabA_count, int* smem) {
  const std::shared_ptr<const BatchTemplate> t = plan_template(p);
  if (!t->ok) return false;
  *d = t->d;
  d->A = A;
  d->B = B;
  *tabA_count = t->tabA_count;
  tabs->insert(tabs->end(), t->tabs.begin(), t->tabs.end());
  *smem = std::max(*smem, t->smem);
  return true;
}

void batch_records(const BatchDesc& d, uint32_t prob, std::vector<TileRec>* recs) {
  for (uint32_t q = 0; q < d.ntiles; ++q) {
    TileRec r;
    r.prob = prob;
    r.pad = 0;
    if (d.path == BP_COPY) {
      const RowCoord rc = row_coord(q, d.rp);
      r.baseA = rc.offA;
      r.baseB = rc.offB;
      r.remA = int32_t(rc.start);
      r.remB = int32_t(rc.end - rc.start);
    } else {
      const TileCoord c = tile_coord(q, d.tp);
      r.baseA = c.baseA;
      r.baseB = c.baseB;
      r.remA = c.remA;
      r.remB = c.remB;
    }
    recs->push_back(r);
  }
}

cudaError_t batch_launch(const BatchDesc* d_descs, const TileRec* d_recs, const uint32_t* d_tile0, uint32_t nprob,
                         uint32_t total, uint32_t* d_counter, int smem, cudaStream_t s) {
  if (total == 0) return cudaSuccess;
  int grid = 0;
  cudaError_t e = grid_for(reinterpret_cast<const void*>(&batch_kernel), smem, int64_t(total), &grid);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(d_counter, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  batch_kernel<<<grid, kThreads, smem, s>>>(d_descs, d_recs, d_tile0, nprob, total, d_counter);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ttc

using namespace ttc;

struct ttc_batch_s {
  struct Item {
    ttc_plan_t plan;
    const void* A;
    void* B;
  };
  std::mutex mu;
  std::vector<Item> items;
  bool dirty = true;
  int dev = -1;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  BatchDesc* d_descs = nullptr;
  TileRec* d_recs = nullptr;
  uint32_t* d_counter = nullptr;
  uint32_t total = 0;
  int smem = 0;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  // problems of at least direct_min elements run as their own single-plan
  // kernels on a side stream, beside the persistent kernel
  int64_t direct_min = int64_t(1) << 21;
  std::vector<Item> direct;
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  ~ttc_batch_s() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (arena) cudaFree(arena);
    if (side) {
      cudaStreamSynchronize(side);
      cudaStreamDestroy(side);
    }
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
  }
};

namespace {

// the batch body's runtime epilogue covers the real non-FP8 pairs only
bool batch_pair_supported(int din, int dout) {
  return pair_supported(din, dout) && dout != DT_E4M3 && !is_complex(din);
}

// Build the descriptors of every problem and upload them (synchronous).
ttc_status batch_build(ttc_batch_s* b) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::vector<BatchDesc> descs;
  std::vector<int32_t> tabs;
  std::vector<size_t> tab_at, tab_na;
  descs.reserve(b->items.size());
  uint64_t total = 0;
  int smem = 0;
  b->direct.clear();
  for (auto& it : b->items) {
    if (b->direct_min > 0 && it.plan->canon.n >= b->direct_min) {
      // set the plan's device resources up now: nothing may allocate or copy
      // synchronously while the launch is captured into a graph
      DevRes* r = nullptr;
      const ttc_status st = ensure_device(it.plan, dev, &r);
      if (st != TTC_OK) return st;
      b->direct.push_back(it);
      continue;
    }
    BatchDesc d;
    size_t na = 0;
    const size_t at = tabs.size();
    if (!batch_describe(it.plan, it.A, it.B, &d, &tabs, &na, &smem)) continue;
    d.tile0 = uint32_t(total);
    total += d.ntiles;
    if (total >= 0x7fffffffull) return fail(TTC_ERR_INVALID_SIZE, "batch has too many tiles");
    descs.push_back(d);
    tab_at.push_back(at);
    tab_na.push_back(na);
  }
  // arena: descriptors | tables | tile records | counter
  const size_t off_tab = (descs.size() * sizeof(BatchDesc) + 255) & ~size_t(255);
  const size_t off_rec = (off_tab + tabs.size() * 4 + 255) & ~size_t(255);
  const size_t off_cnt = (off_rec + total * sizeof(TileRec) + 255) & ~size_t(255);
  const size_t bytes = off_cnt + 256;
  if (b->arena) {
    cudaFree(b->arena);
    b->arena = nullptr;
  }
  e = cudaMalloc(&b->arena, bytes);
  if (e != cudaSuccess) {
    b->arena = nullptr;
    return fail(TTC_ERR_OOM, "batch arena allocation failed");
  }
  char* base = static_cast<char*>(b->arena);
  int32_t* d_tab = reinterpret_cast<int32_t*>(base + off_tab);
  std::vector<TileRec> recs;
  recs.reserve(total);
  for (size_t i = 0; i < descs.size(); ++i) {
    BatchDesc& d = descs[i];
    if (d.path == BP_TILE) {
      d.tp.tabA = d_tab + tab_at[i];
      d.tp.tabB = d_tab + tab_at[i] + tab_na[i];
    }
    batch_records(d, uint32_t(i), &recs);
  }
  e = cudaMemcpy(base, descs.data(), descs.size() * sizeof(BatchDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !tabs.empty()) e = cudaMemcpy(d_tab, tabs.data(), tabs.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && total)
    e = cudaMemcpy(base + off_rec, recs.data(), total * sizeof(TileRec), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "batch upload");
  b->arena_bytes = bytes;
  b->d_descs = reinterpret_cast<BatchDesc*>(base);
  b->d_recs = reinterpret_cast<TileRec*>(base + off_rec);
  b->d_counter = reinterpret_cast<uint32_t*>(base + off_cnt);
  b->total = uint32_t(total);
  b->smem = smem;
  b->dev = dev;
  if (!b->direct.empty() && !b->side) {
    e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "batch side stream");
  }
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  b->dirty = false;
  return TTC_OK;
}

// The persistent kernel on s; the direct problems one after another on the
// side stream, forked from and joined back into s (so that a capture of s
// records both branches).
ttc_status batch_enqueue(ttc_batch_s* b, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  ttc_status st = TTC_OK;
  if (!b->direct.empty()) {
    e = cudaEventRecord(b->fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->fork, 0);
    if (e != cudaSuccess) return cuda_fail(e, "batch fork");
    for (auto& it : b->direct) {
      st = run_plan(it.plan, it.A, it.B, b->side);
      if (st != TTC_OK) break;
    }
    e = cudaEventRecord(b->join, b->side);
    if (e != cudaSuccess && st == TTC_OK) st = cuda_fail(e, "batch join");
  }
  if (b->total && st == TTC_OK) {
    e = batch_launch(b->d_descs, b->d_recs, nullptr, 0, b->total, b->d_counter, b->smem, s);
    if (e != cudaSuccess) st = cuda_fail(e, "batch kernel launch");
  }
  if (!b->direct.empty()) {
    e = cudaStreamWaitEvent(s, b->join, 0);      // always join, so a capture can end
    if (e != cudaSuccess && st == TTC_OK) st = cuda_fail(e, "batch join");
  }
  return st;
}

}  // namespace

extern "C" {

ttc_status ttc_batch_create(ttc_batch_t* out) {
  if (!out) return fail(TTC_ERR_INVALID_ARG, "out is NULL");
  *out = new (std::nothrow) ttc_batch_s();
  return *out ? TTC_OK : fail(TTC_ERR_OOM, "host allocation failed");
}

ttc_status ttc_batch_add(ttc_batch_t b, ttc_plan_t plan, const void* A, void* B) {
  if (!b || !plan) return fail(TTC_ERR_INVALID_ARG, "NULL batch or plan");
  if (!batch_pair_supported(plan->din, plan->dout))
    return fail(TTC_ERR_UNSUPPORTED_DTYPE, "FP8 output and complex types are not supported in a batch");
  if (plan->canon.n > 0) {
    if (!A || !B) return fail(TTC_ERR_INVALID_ARG, "A or B is NULL");
    const uintptr_t a = reinterpret_cast<uintptr_t>(A), bb = reinterpret_cast<uintptr_t>(B);
    if (a % dtype_size(plan->din) || bb % dtype_size(plan->dout))
      return fail(TTC_ERR_ALIGN, "A or B not aligned to its element size");
    const uintptr_t ea = a + uintptr_t(plan->canon.spanA) * dtype_size(plan->din);
    const uintptr_t eb = bb + uintptr_t(plan->canon.spanB) * dtype_size(plan->dout);
    if (a < eb && bb < ea) return fail(TTC_ERR_ALIAS, "the byte ranges of A and B overlap");
  }
  std::lock_guard<std::mutex> lk(b->mu);
  b->items.push_back({plan, A, B});
  b->dirty = true;
  return TTC_OK;
}

ttc_status ttc_batch_execute(ttc_batch_t b, ttc_stream_t stream) {
  if (!b) return fail(TTC_ERR_INVALID_ARG, "batch is NULL");
  std::lock_guard<std::mutex> lk(b->mu);
  if (b->dirty) {
    ttc_status st = batch_build(b);
    if (st != TTC_OK) return st;
  }
  return batch_enqueue(b, reinterpret_cast<cudaStream_t>(stream));
}

ttc_status ttc_batch_graph_launch(ttc_batch_t b, ttc_stream_t stream) {
  if (!b) return fail(TTC_ERR_INVALID_ARG, "batch is NULL");
  std::lock_guard<std::mutex> lk(b->mu);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (b->dirty) {
    ttc_status st = batch_build(b);
    if (st != TTC_OK) return st;
  }
  if (!b->gexec) {
    // capture on a private stream so that the caller's stream may be any stream
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cs);
      return cuda_fail(e, "cudaStreamBeginCapture");
    }
    const int64_t before = g_launches.load();
    ttc_status st = batch_enqueue(b, cs);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    g_launches -= g_launches.load() - before;    // captured, not launched
    if (st != TTC_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      b->gexec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    b->graph = g;
  }
  cudaError_t e = cudaGraphLaunch(b->gexec, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  g_launches += (b->total ? 1 : 0) + int64_t(b->direct.size());
  return TTC_OK;
}

ttc_status ttc_batch_set_direct_threshold(ttc_batch_t b, int64_t min_elements) {
  if (!b) return fail(TTC_ERR_INVALID_ARG, "batch is NULL");
  std::lock_guard<std::mutex> lk(b->mu);
  b->direct_min = min_elements;
  b->dirty = true;
  return TTC_OK;
}

ttc_status ttc_batch_destroy(ttc_batch_t b) {
  if (!b) return fail(TTC_ERR_INVALID_ARG, "batch is NULL");
  delete b;
  return TTC_OK;
}

ttc_status ttc_batch_info(ttc_batch_t b, int64_t* problems, int64_t* tiles) {
  if (!b) return fail(TTC_ERR_INVALID_ARG, "batch is NULL");
  std::lock_guard<std::mutex> lk(b->mu);
  if (problems) *problems = int64_t(b->items.size());
  if (tiles) {
    int64_t t = 0;
    for (auto& it : b->items) {
      BatchDesc d;
      std::vector<int32_t> tabs;
      size_t na = 0;
      int sm = 0;
      if (batch_describe(it.plan, it.A, it.B, &d, &tabs, &na, &sm)) t += d.ntiles;
    }
    *tiles = t;
  }
  return TTC_OK;
}

}  // extern "C"
