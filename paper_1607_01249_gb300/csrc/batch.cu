// batch.cu -- many permute-scale-adds in one kernel launch (include/ttc.h,
// ttc_batch_*).
//
// Every problem of a batch is cut into tiles by its own plan (the batch
// body's schedules: tiles of at most half the single-plan kernels' volume).
// A tile is processed by one CTA with one of three bodies:
//   BP_TILE -- the packed-lane tile (problems whose perm moves index 0): lane
//              groups of any width over the tile's rows, so the many small
//              problems of a batch, whose runs are short and ragged, keep
//              their lanes busy;
//   BP_ROWS -- packed rows (perm keeps index 0, tiles of whole rows copied
//              directly);
//   BP_COPY -- one chunk of one long run (perm keeps index 0, long runs).
// The launch has one CTA per tile of the whole batch; a per-tile record names
// the problem, whose descriptor (pointers, tile parameters, epilogue) sits in
// one device arena owned by the batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "../../include/ttc.h"
#include "batch_impl.h"
#include "kernels_impl.cuh"
#include "launch.h"
#include "plan_impl.h"
#include "planner.h"

namespace ttc {

// --------------------------------------------------------------- device --

template <int DIN, int DOUT, int EK>
__device__ __forceinline__ void batch_copy(const BatchDesc& d, const RowCoord& rc) {
  using S = stage_t<DIN>;
  using TO = store_t<DOUT>;
  constexpr int K = kBatchCopyChunk / kThreads / (sizeof(S) == 8 ? 2 : 1);
  const int64_t sa0 = d.rp.sa0, sb0 = d.rp.sb0;
  const Epilogue& epi = d.rp.epi;
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
    if constexpr (ek_reads_b(EK)) bo[k] = Br[xs * sb0];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t x = rc.start + t + int64_t(k) * kThreads;
    if (x < rc.end) Br[x * sb0] = epilogue_k<DIN, DOUT, EK>(v[k], bo[k], epi, 1.f);
  }
}

// One tile of one problem with the class's body: the packed-lane tile
// (BP_TILE, J run chunks per thread), packed rows (BP_ROWS, J positions per
// row) or a run chunk (BP_COPY); the epilogue's mode is read at run time, B is
// read only for beta != 0 (EK_RT_B).
template <int DIN, int DOUT, int EK, int PATH, int J>
__device__ __forceinline__ void batch_unit_ek(const BatchDesc& d, const TileRec& r, unsigned char* smem) {
  constexpr int K = batch_k_for(sizeof(stage_t<DIN>));
  if constexpr (PATH == BP_COPY) {
    const RowCoord rc{r.baseA, r.baseB, int64_t(r.remA), int64_t(r.remA) + r.remB};
    batch_copy<DIN, DOUT, EK>(d, rc);
  } else {
    const TileCoord c{r.baseA, r.baseB, r.remA, r.remB};
    const store_t<DIN>* Ab = static_cast<const store_t<DIN>*>(d.A) + c.baseA;
    store_t<DOUT>* Bb = static_cast<store_t<DOUT>*>(d.B) + c.baseB;
    if constexpr (PATH == BP_ROWS) {
      rowsp_tile<DIN, DOUT, (J <= K ? J : K), EK, K>(Ab, Bb, d.tp, c, 1.f);
    } else {
      stage_t<DIN>* tile = reinterpret_cast<stage_t<DIN>*>(smem);
      tilep_tile<DIN, DOUT, J, J, EK, K>(Ab, Bb, d.tp, c, tile, 1.f);
    }
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

// One CTA per tile (the paper's independent macro-tiles, section 2.2,
// scheduled across thread blocks): the hardware block scheduler hands out the
// tiles of all problems of one class (dtype pair, beta zero or not; one
// launch per class, so that each launch has its types and epilogue fixed at
// compile time), refilling an SM the moment one of its CTAs ends, which keeps
// more bytes in flight than CTAs that claim tiles in a loop, and lets the
// batch's side-stream kernels share the GPU.  Global tile g = first +
// blockIdx.x.  A tile's record comes from the precomputed array `recs`
// (ttc_batch_*, built once and replayed) or, when recs is null, from the
// problems' tile prefix `tile0` (ascending over all nprob problems) and the
// problem's tile parameters on the device (the server's epochs, built per
// launch at no per-tile host cost).  The problem's descriptor is read from
// global memory, where it stays cached for the problem's other tiles.
template <int DIN, int DOUT, int EK, int PATH, int J>
__global__ void __launch_bounds__(kThreads, 8) batch_kernel(const BatchDesc* __restrict__ descs,
                                                            const TileRec* __restrict__ recs,
                                                            const uint32_t* __restrict__ tile0, uint32_t nprob,
                                                            uint32_t first) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TileRec s_rec;
  const uint32_t g = first + blockIdx.x;
  if (threadIdx.x == 0) {
    if (recs) {
      s_rec = recs[g];
    } else {
      const uint32_t prob = find_problem(tile0, nprob, g);
      s_rec = device_rec(descs[prob], prob, g - __ldg(tile0 + prob));
    }
  }
  __syncthreads();
  const TileRec r = s_rec;
  batch_unit_ek<DIN, DOUT, EK, PATH, J>(descs[r.prob], r, smem);
}

template <int DIN, int DOUT, int EK, int PATH, int J>
cudaError_t launch_batch_body(const BatchDesc* d_descs, const TileRec* d_recs, const uint32_t* d_tile0,
                              uint32_t nprob, uint32_t first, uint32_t count, int smem, cudaStream_t s) {
  const void* fn = reinterpret_cast<const void*>(&batch_kernel<DIN, DOUT, EK, PATH, J>);
  if (smem > 48 * 1024) {
    int g = 0;
    cudaError_t e = grid_for(fn, smem, 1, &g);
    if (e != cudaSuccess) return e;
  }
  batch_kernel<DIN, DOUT, EK, PATH, J><<<count, kThreads, smem, s>>>(d_descs, d_recs, d_tile0, nprob, first);
  ++g_launches;
  return cudaGetLastError();
}

// the body variants of a class: packed-lane tiles with 1 or 2 chunks, packed
// rows with 1 or K positions per row, run chunks
template <int DIN, int DOUT, int EK>
cudaError_t launch_batch_class(int path, int j, const BatchDesc* d_descs, const TileRec* d_recs,
                               const uint32_t* d_tile0, uint32_t nprob, uint32_t first, uint32_t count, int smem,
                               cudaStream_t s) {
  constexpr int K = batch_k_for(sizeof(stage_t<DIN>));
  if (path == BP_COPY)
    return launch_batch_body<DIN, DOUT, EK, BP_COPY, 1>(d_descs, d_recs, d_tile0, nprob, first, count, smem, s);
  if (path == BP_ROWS)
    return j == 1 ? launch_batch_body<DIN, DOUT, EK, BP_ROWS, 1>(d_descs, d_recs, d_tile0, nprob, first, count, smem, s)
                  : launch_batch_body<DIN, DOUT, EK, BP_ROWS, K>(d_descs, d_recs, d_tile0, nprob, first, count, smem, s);
  return j == 1 ? launch_batch_body<DIN, DOUT, EK, BP_TILE, 1>(d_descs, d_recs, d_tile0, nprob, first, count, smem, s)
                : launch_batch_body<DIN, DOUT, EK, BP_TILE, 2>(d_descs, d_recs, d_tile0, nprob, first, count, smem, s);
}

}  // namespace ttc

// ------------------------------------------------------------------ host --

namespace ttc {

namespace {

// the batch body's candidate schedules of a plan, best first by the cost
// model (tiles of at most the batch body's volume)
std::vector<Candidate> batch_candidates(const ttc_plan_s* p, int keep) {
  return make_candidates(p->canon, p->din, p->dout, p->beta, keep, kThreads * batch_k_for(p->din == DT_F64 ? 8 : 4));
}

// the batch template of a plan with schedule k
std::shared_ptr<const BatchTemplate> make_template_for(const ttc_plan_s* p, const Candidate& k) {
  auto t = std::make_shared<BatchTemplate>();
  if (p->canon.n == 0 || p->dout == DT_E4M3 || is_complex(p->din)) return t;
  BatchDesc* d = &t->d;
  std::memset(d, 0, sizeof(*d));
  d->din = p->din;
  d->dout = p->dout;
  d->beta_nz = p->beta_nonzero() ? 1 : 0;
  if (k.variant == VAR_TILE) {
    std::vector<int32_t> ta, tb;
    int sm = 0;
    build_tile_params(p->canon, k, p->din, &d->tp, &ta, &tb, &sm);
    d->path = k.rj ? BP_ROWS : BP_TILE;
    d->j = k.rj ? k.rj : k.ju;
    if (d->tp.crossA_tab || d->tp.crossB_tab) {
      t->tabA_count = ta.size();
      t->tabs.insert(t->tabs.end(), ta.begin(), ta.end());
      t->tabs.insert(t->tabs.end(), tb.begin(), tb.end());
    }
    if (d->path == BP_TILE) t->smem = d->tp.P * d->tp.LB * stage_bytes_of(p->din);
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

// the cost model's choice (the template a plan starts with)
std::shared_ptr<const BatchTemplate> make_template(const ttc_plan_s* p) {
  if (p->canon.n == 0 || p->dout == DT_E4M3 || is_complex(p->din)) return std::make_shared<BatchTemplate>();
  const std::vector<Candidate> bc = batch_candidates(p, 4);
  if (bc.empty()) return std::make_shared<BatchTemplate>();   // the batch runs it as a single-plan kernel
  return make_template_for(p, bc.front());
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

int batch_class(const BatchDesc& d) {
  const int body = d.path == BP_COPY ? 4 : (d.path == BP_ROWS ? 2 : 0) + (d.j == 1 ? 0 : 1);
  return ((d.din * kNumDTypes + d.dout) * 2 + (d.beta_nz ? 1 : 0)) * 8 + body;
}

void batch_ranges(const std::vector<BatchDesc>& descs, std::vector<BatchRange>* ranges) {
  ranges->clear();
  for (const BatchDesc& d : descs) {
    const int cls = batch_class(d);
    if (ranges->empty() || ranges->back().cls != cls)
      ranges->push_back({cls, d.din, d.dout, d.beta_nz, d.path, d.j, d.tile0, 0});
    ranges->back().count += d.ntiles;
  }
}

cudaError_t batch_launch(const BatchDesc* d_descs, const TileRec* d_recs, const uint32_t* d_tile0, uint32_t nprob,
                         const std::vector<BatchRange>& ranges, int smem, cudaStream_t s) {
  for (const BatchRange& r : ranges) {
    if (r.count == 0) continue;
    cudaError_t e = cudaErrorInvalidValue;
#define TTC_BC(I, O)                                                                                     \
  if (r.din == I && r.dout == O)                                                                          \
    e = r.bnz ? launch_batch_class<I, O, EK_RT_B>(r.path, r.j, d_descs, d_recs, d_tile0, nprob, r.first, r.count, \
                                                  smem, s)                                                        \
              : launch_batch_class<I, O, EK_RT>(r.path, r.j, d_descs, d_recs, d_tile0, nprob, r.first, r.count, smem, s);
    TTC_BC(DT_F32, DT_F32) TTC_BC(DT_F32, DT_F64) TTC_BC(DT_F32, DT_BF16) TTC_BC(DT_F64, DT_F64)
    TTC_BC(DT_F64, DT_F32) TTC_BC(DT_BF16, DT_BF16) TTC_BC(DT_BF16, DT_F32)
#undef TTC_BC
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
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
  uint32_t total = 0;
  int smem = 0;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  // problems of at least direct_min elements (if > 0) run as their own
  // single-plan kernels on a side stream, beside the batch kernels; off by
  // default: with one CTA per tile the batch kernels move even the largest
  // problems of a mixed batch faster than a stream of single-plan launches
  int64_t direct_min = 0;
  std::vector<Item> direct;
  std::vector<BatchRange> ranges;   // the class launches of the batch kernel
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  // every other class launch runs on this stream, forked from and joined
  // back into the caller's, so that one class's last wave overlaps the next
  // class's first
  cudaStream_t lane2 = nullptr;
  cudaEvent_t fork2 = nullptr, join2 = nullptr;
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
    if (lane2) {
      cudaStreamSynchronize(lane2);
      cudaStreamDestroy(lane2);
    }
    if (fork2) cudaEventDestroy(fork2);
    if (join2) cudaEventDestroy(join2);
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
    if (!batch_describe(it.plan, it.A, it.B, &d, &tabs, &na, &smem)) {
      // a problem the batch body cannot take runs as its own kernel
      if (it.plan->canon.n > 0) {
        DevRes* r = nullptr;
        const ttc_status st = ensure_device(it.plan, dev, &r);
        if (st != TTC_OK) return st;
        b->direct.push_back(it);
      }
      continue;
    }
    descs.push_back(d);
    tab_at.push_back(at);
    tab_na.push_back(na);
  }
  // problems ordered by class (one kernel launch per class), each class in
  // the order the problems were added; then every problem's first tile
  {
    std::vector<size_t> idx(descs.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(),
                     [&](size_t x, size_t y) { return batch_class(descs[x]) < batch_class(descs[y]); });
    std::vector<BatchDesc> d2;
    std::vector<size_t> at2, na2;
    for (size_t i : idx) {
      d2.push_back(descs[i]);
      at2.push_back(tab_at[i]);
      na2.push_back(tab_na[i]);
    }
    descs.swap(d2);
    tab_at.swap(at2);
    tab_na.swap(na2);
  }
  for (BatchDesc& d : descs) {
    d.tile0 = uint32_t(total);
    total += d.ntiles;
    if (total >= 0x7fffffffull) return fail(TTC_ERR_INVALID_SIZE, "batch has too many tiles");
  }
  batch_ranges(descs, &b->ranges);
  // arena: descriptors | tables | tile records
  const size_t off_tab = (descs.size() * sizeof(BatchDesc) + 255) & ~size_t(255);
  const size_t off_rec = (off_tab + tabs.size() * 4 + 255) & ~size_t(255);
  const size_t bytes = (off_rec + total * sizeof(TileRec) + 255) & ~size_t(255);
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
    if (d.path != BP_COPY) {
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
  b->total = uint32_t(total);
  b->smem = smem;
  b->dev = dev;
  if (!b->direct.empty() && !b->side) {
    e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "batch side stream");
  }
  if (b->ranges.size() > 1 && !b->lane2) {
    e = cudaStreamCreateWithFlags(&b->lane2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork2, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join2, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "batch second class stream");
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

// The batch kernel on s; the direct problems one after another on the
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
    if (b->ranges.size() > 1 && b->lane2) {
      // classes alternate between s and the batch's second stream
      std::vector<BatchRange> even, odd;
      for (size_t i = 0; i < b->ranges.size(); ++i) (i % 2 ? odd : even).push_back(b->ranges[i]);
      e = cudaEventRecord(b->fork2, s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->lane2, b->fork2, 0);
      if (e != cudaSuccess) return cuda_fail(e, "batch fork");
      cudaError_t e1 = batch_launch(b->d_descs, b->d_recs, nullptr, 0, odd, b->smem, b->lane2);
      e = cudaEventRecord(b->join2, b->lane2);
      if (e == cudaSuccess && e1 == cudaSuccess)
        e1 = batch_launch(b->d_descs, b->d_recs, nullptr, 0, even, b->smem, s);
      const cudaError_t e2 = cudaStreamWaitEvent(s, b->join2, 0);   // always join, so a capture can end
      if (e1 != cudaSuccess) st = cuda_fail(e1, "batch kernel launch");
      else if (e != cudaSuccess || e2 != cudaSuccess) st = cuda_fail(e != cudaSuccess ? e : e2, "batch join");
    } else {
      e = batch_launch(b->d_descs, b->d_recs, nullptr, 0, b->ranges, b->smem, s);
      if (e != cudaSuccess) st = cuda_fail(e, "batch kernel launch");
    }
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
  g_launches += int64_t(b->ranges.size()) + int64_t(b->direct.size());
  return TTC_OK;
}

ttc_status ttc_batch_set_direct_threshold(ttc_batch_t b, int64_t min_elements) {
  if (!b) return fail(TTC_ERR_INVALID_ARG, "batch is NULL");
  std::lock_guard<std::mutex> lk(b->mu);
  b->direct_min = min_elements;
  b->dirty = true;
  return TTC_OK;
}

ttc_status ttc_batch_autotune(ttc_batch_t b, int max_candidates, ttc_stream_t stream, int64_t* retuned) {
  if (!b) return fail(TTC_ERR_INVALID_ARG, "batch is NULL");
  if (max_candidates < 1) return fail(TTC_ERR_INVALID_ARG, "max_candidates must be >= 1");
  std::lock_guard<std::mutex> lk(b->mu);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (retuned) *retuned = 0;
  // the distinct plans that run in the batch body
  std::vector<ttc_plan_s*> plans;
  std::set<ttc_plan_s*> seen;
  size_t maxA = 16, maxB = 16;
  for (auto& it : b->items) {
    ttc_plan_s* p = it.plan;
    if (p->canon.n == 0 || (b->direct_min > 0 && p->canon.n >= b->direct_min)) continue;
    if (!seen.insert(p).second) continue;
    plans.push_back(p);
    maxA = std::max(maxA, size_t(p->canon.spanA) * dtype_size(p->din));
    maxB = std::max(maxB, size_t(p->canon.spanB) * dtype_size(p->dout));
  }
  if (plans.empty()) return TTC_OK;
  // temporary tensors (the caller's are not touched) and one problem's
  // descriptor, tables and records, grown as needed
  void *dA = nullptr, *dB = nullptr, *scratch = nullptr;
  size_t scratch_bytes = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&dA, maxA);
  if (e == cudaSuccess) e = cudaMalloc(&dB, maxB);
  if (e == cudaSuccess) e = cudaMemsetAsync(dA, 0, maxA, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dB, 0, maxB, s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  ttc_status st = e == cudaSuccess ? TTC_OK : fail(TTC_ERR_OOM, "batch autotune buffers");
  constexpr int kReps = 3;
  for (size_t pi = 0; pi < plans.size() && st == TTC_OK; ++pi) {
    ttc_plan_s* p = plans[pi];
    const std::vector<Candidate> bc = batch_candidates(p, std::max(4, max_candidates));
    const int n = std::min<int>(max_candidates, int(bc.size()));
    if (n < 2) continue;   // nothing to choose between
    std::shared_ptr<const BatchTemplate> best;
    float best_ms = 0.f;
    int best_i = -1;
    for (int i = 0; i < n && st == TTC_OK; ++i) {
      std::shared_ptr<const BatchTemplate> t = make_template_for(p, bc[size_t(i)]);
      if (!t->ok || t->d.ntiles == 0) continue;
      BatchDesc d = t->d;
      d.A = dA;
      d.B = dB;
      d.tile0 = 0;
      std::vector<TileRec> recs;
      batch_records(d, 0, &recs);
      const size_t off_tab = (sizeof(BatchDesc) + 255) & ~size_t(255);
      const size_t off_rec = (off_tab + t->tabs.size() * 4 + 255) & ~size_t(255);
      const size_t bytes = off_rec + recs.size() * sizeof(TileRec);
      if (bytes > scratch_bytes) {
        // the previous scratch may still be read by queued launches
        if (scratch) {
          e = cudaStreamSynchronize(s);
          if (e == cudaSuccess) e = cudaFree(scratch);
          scratch = nullptr;
          scratch_bytes = 0;
          if (e != cudaSuccess) {
            st = cuda_fail(e, "batch autotune scratch");
            break;
          }
        }
        if (cudaMalloc(&scratch, bytes) != cudaSuccess) {
          scratch = nullptr;
          st = fail(TTC_ERR_OOM, "batch autotune scratch allocation failed");
          break;
        }
        scratch_bytes = bytes;
      }
      char* base = static_cast<char*>(scratch);
      if (d.path != BP_COPY) {
        d.tp.tabA = reinterpret_cast<int32_t*>(base + off_tab);
        d.tp.tabB = d.tp.tabA + t->tabA_count;
      }
      // (synchronous copies: the previous candidate's launches have ended
      // before this one's descriptor replaces theirs)
      e = cudaStreamSynchronize(s);
      if (e == cudaSuccess) e = cudaMemcpy(base, &d, sizeof(BatchDesc), cudaMemcpyHostToDevice);
      if (e == cudaSuccess && !t->tabs.empty())
        e = cudaMemcpy(base + off_tab, t->tabs.data(), t->tabs.size() * 4, cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(base + off_rec, recs.data(), recs.size() * sizeof(TileRec), cudaMemcpyHostToDevice);
      std::vector<BatchRange> ranges;
      batch_ranges(std::vector<BatchDesc>{d}, &ranges);
      const BatchDesc* dd = reinterpret_cast<const BatchDesc*>(base);
      const TileRec* dr = reinterpret_cast<const TileRec*>(base + off_rec);
      if (e == cudaSuccess) e = batch_launch(dd, dr, nullptr, 0, ranges, t->smem, s);   // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      for (int r = 0; r < kReps && e == cudaSuccess; ++r) e = batch_launch(dd, dr, nullptr, 0, ranges, t->smem, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        st = cuda_fail(e, "batch autotune timing");
        break;
      }
      if (!best || ms < best_ms) {
        best = t;
        best_ms = ms;
        best_i = i;
      }
    }
    if (st == TTC_OK && best) {
      std::lock_guard<std::mutex> pl(p->batch_mu);
      p->batch_tmpl = best;
      if (retuned && best_i != 0) ++*retuned;
    }
  }
  if (dA || dB || scratch) cudaStreamSynchronize(s);
  if (scratch) cudaFree(scratch);
  if (dA) cudaFree(dA);
  if (dB) cudaFree(dB);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  b->dirty = true;   // the next launch takes the chosen templates
  return st;
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
