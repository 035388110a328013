// capi.cu -- the C ABI (include/ttc.h): plans, execution, FP8 scale, autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/ttc.h"
#include "launch.h"
#include "plan_impl.h"
#include "planner.h"
#include "rowvec.h"
#include "tma2d.h"

using namespace ttc;

namespace ttc {

thread_local std::string g_last_error;

ttc_status fail(ttc_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

ttc_status cuda_fail(cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(TTC_ERR_CUDA, m);
}

// ------------------------------------------------------------ tune cache --
namespace {
std::mutex g_tune_mu;
std::map<std::string, std::string> g_tune;   // key -> candidate description
}  // namespace

namespace {
std::mutex g_name_mu;
std::map<int, std::string> g_dev_names;
std::string device_name(int dev) {
  std::lock_guard<std::mutex> lk(g_name_mu);
  auto it = g_dev_names.find(dev);
  if (it != g_dev_names.end()) return it->second;
  char name[256] = "unknown";
  cudaDeviceProp prop;
  if (dev >= 0 && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) std::snprintf(name, sizeof(name), "%s", prop.name);
  for (char* q = name; *q; ++q)
    if (*q == ' ' || *q == ':' || *q == '\t') *q = '_';
  g_dev_names[dev] = name;
  return name;
}
std::string cand_key(const Candidate& c) {
  const std::string d = c.describe();
  return d.substr(0, d.find(" est_us"));
}
}  // namespace

std::string plan_key(const ttc_plan_s* p, int dev) {
  std::ostringstream o;
  o << device_name(dev) << ":" << p->din << ">" << p->dout << ":b" << p->beta_nonzero() << ":N" << p->canon.N;
  for (int k = 0; k < p->canon.N; ++k)
    o << ":" << p->canon.s[k] << "/" << p->canon.sa[k] << "/" << p->canon.sb[k] << "/" << p->canon.perm[k];
  return o.str();
}

// The candidate an earlier autotune chose for this canonical problem on
// this device, or -1 (the caller holds p->mu).
int remembered_choice(const ttc_plan_s* p, int dev) {
  const std::string key = plan_key(p, dev);
  std::lock_guard<std::mutex> tl(g_tune_mu);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return -1;
  for (size_t i = 0; i < p->cands.size(); ++i)
    if (cand_key(p->cands[i]) == it->second) return int(i);
  return -1;
}

// ------------------------------------------------------- device resources --

ttc_status ensure_device(ttc_plan_s* p, int dev, DevRes** out) {
  std::lock_guard<std::mutex> lk(p->mu);
  DevRes& r = p->dev[dev];
  if (r.base == nullptr) {
    // scratch: amax word + scale, room for the largest cross tables, then
    // (16-byte aligned) the slot tables if a candidate uses them
    size_t tab = 0;
    bool slots = false;
    for (auto& c : p->cands) {
      if (c.variant != VAR_TILE) continue;
      TileParams tp;
      std::vector<int32_t> ta, tb;
      int sm = 0;
      build_tile_params(p->canon, c, p->din, &tp, &ta, &tb, &sm);
      tab = std::max(tab, (ta.size() + tb.size()) * sizeof(int32_t));
      slots = slots || c.slots;
    }
    tab = (tab + 255) & ~size_t(255);
    r.bytes = 256 + tab + (slots ? slot_table_ints(p->din) * sizeof(int32_t) : 0);
    cudaError_t e = cudaMalloc(&r.base, r.bytes);
    if (e != cudaSuccess) {
      r.base = nullptr;
      return e == cudaErrorMemoryAllocation ? fail(TTC_ERR_OOM, "device scratch allocation failed")
                                            : cuda_fail(e, "cudaMalloc");
    }
    r.amax = reinterpret_cast<uint32_t*>(r.base);
    r.scale = reinterpret_cast<float*>(static_cast<char*>(r.base) + 16);
    r.amax_phase = 0;
    e = cudaMemset(r.base, 0, 256);     // both amax words start at 0
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
    r.tables = reinterpret_cast<int32_t*>(static_cast<char*>(r.base) + 256);
    r.slots = slots ? reinterpret_cast<int4*>(static_cast<char*>(r.base) + 256 + tab) : nullptr;
    r.sel = -1;
    // a remembered autotune result for this canonical problem on this device
    if (!p->user_selected) {
      const int i = remembered_choice(p, dev);
      if (i >= 0) p->sel = i;
    }
  }
  if (r.sel != p->sel) {
    const Candidate& k = p->cands[p->sel];
    if (k.variant == VAR_TILE) {
      std::vector<int32_t> ta, tb;
      build_tile_params(p->canon, k, p->din, &r.tp, &ta, &tb, &r.smem);
      std::vector<int32_t> all(ta);
      all.insert(all.end(), tb.begin(), tb.end());
      if (!all.empty()) {
        cudaError_t e = cudaMemcpy(r.tables, all.data(), all.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "table upload");
      }
      r.tp.tabA = r.tables;
      r.tp.tabB = r.tables + ta.size();
      r.tp.slots = nullptr;
      if (k.slots && r.slots) {
        std::vector<int32_t> st;
        const int sbytes = build_slot_tables(r.tp, p->din, ta, tb, &st);
        cudaError_t e = cudaMemcpy(r.slots, st.data(), st.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "slot table upload");
        r.tp.slots = r.slots;
        r.smem = sbytes;
      }
    } else if (k.variant == VAR_COPY) {
      build_row_params(p->canon, k.chunk, &r.rp);
    }
    r.sel = p->sel;
  }
  *out = &r;
  return TTC_OK;
}

Epilogue make_epilogue(const ttc_plan_s* p, const DevRes* r) {
  Epilogue e;
  const bool unit = p->alpha == 1.0 && p->alpha_im == 0.0 && !p->beta_nonzero();
  e.mode = (p->dout == DT_E4M3) ? MODE_FP8 : (unit && p->din == p->dout) ? MODE_BITCOPY : MODE_AXPBY;
  e.beta_nz = p->beta_nonzero();
  e.alpha_f = float(p->alpha);
  e.beta_f = float(p->beta);
  e.alpha_d = p->alpha;
  e.beta_d = p->beta;
  e.alpha_fi = float(p->alpha_im);
  e.beta_fi = float(p->beta_im);
  e.alpha_di = p->alpha_im;
  e.beta_di = p->beta_im;
  e.alpha_k = make_dmul_const(p->alpha);
  e.scale_in = p->user_scale;
  e.amax_bits = r ? r->amax : nullptr;
  e.scale_out = r ? r->scale : nullptr;
  return e;
}

// Launch the selected candidate (and the FP8 amax pre-pass when needed).
ttc_status run_plan(ttc_plan_s* p, const void* A, void* B, cudaStream_t s) {
  if (p->canon.n == 0) return TTC_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  DevRes* r = nullptr;
  ttc_status st = ensure_device(p, dev, &r);
  if (st != TTC_OK) return st;
  const Candidate& k = p->cands[r->sel];
  Epilogue epi = make_epilogue(p, r);
  if (p->dout == DT_E4M3 && !p->user_scale) {
    // this execution accumulates into one amax word and clears the other for
    // the next execution (in stream order, after this one's kernels)
    uint32_t* cur = r->amax + r->amax_phase;
    uint32_t* next = r->amax + (1 - r->amax_phase);
    r->amax_phase ^= 1;
    epi.amax_bits = cur;
    e = launch_amax(p->din, A, p->amax_rows, float(p->alpha), cur, next, s);
    if (e != cudaSuccess) {
      r->amax_phase ^= 1;      // `next` was not cleared: this word is still the one to use
      return cuda_fail(e, "amax kernel launch");
    }
  }
  if (k.variant == VAR_TILE) {
    TileParams tp = r->tp;
    tp.epi = epi;
    e = k.rows ? (k.vec > 1 ? launch_rowcopy_vec(p->din, p->dout, A, B, tp, s) : launch_rowcopy(p->din, p->dout, A, B, tp, s))
        : k.rj ? launch_rowsp(p->din, p->dout, k.rj, A, B, tp, s)
        : k.pk ? launch_tilep(p->din, p->dout, k.pk, k.ju, k.jw, A, B, tp, r->smem, s)
        : k.ju ? launch_tile2(p->din, p->dout, k.ju, k.jw, A, B, tp, r->smem, s)
        : tp.slots ? launch_tile_slots(p->din, p->dout, A, B, tp, r->smem, s)
                   : launch_tile(p->din, p->dout, A, B, tp, r->smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "tile kernel launch");
  } else if (k.variant == VAR_COPY) {
    RowParams rp = r->rp;
    rp.epi = epi;
    int vec = k.vec;
    const uintptr_t a = reinterpret_cast<uintptr_t>(A), b = reinterpret_cast<uintptr_t>(B);
    if (vec > 1 && (a % (size_t(vec) * dtype_size(p->din)) || b % (size_t(vec) * dtype_size(p->dout)))) vec = 1;
    if (vec > 1 && rp.chunk % vec) vec = 1;
    e = launch_copy(p->din, p->dout, vec, A, B, rp, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy kernel launch");
  } else if (k.variant == VAR_TMA) {
    e = launch_tma2d(p->din, p->dout, A, B, tma2d_geom(p->canon, p->din), epi, s);
    if (e != cudaSuccess) return cuda_fail(e, "TMA tile kernel launch");
  }
  return TTC_OK;
}

}  // namespace ttc

// ================================================================ C ABI ===

extern "C" {

const char* ttc_status_string(ttc_status s) {
  switch (s) {
    case TTC_OK: return "TTC_OK";
    case TTC_ERR_INVALID_PERM: return "TTC_ERR_INVALID_PERM";
    case TTC_ERR_INVALID_SIZE: return "TTC_ERR_INVALID_SIZE";
    case TTC_ERR_INVALID_OUTER: return "TTC_ERR_INVALID_OUTER";
    case TTC_ERR_UNSUPPORTED_DTYPE: return "TTC_ERR_UNSUPPORTED_DTYPE";
    case TTC_ERR_ALIAS: return "TTC_ERR_ALIAS";
    case TTC_ERR_ALIGN: return "TTC_ERR_ALIGN";
    case TTC_ERR_OOM: return "TTC_ERR_OOM";
    case TTC_ERR_CUDA: return "TTC_ERR_CUDA";
    case TTC_ERR_TIMEOUT: return "TTC_ERR_TIMEOUT";
    case TTC_ERR_BUDGET: return "TTC_ERR_BUDGET";
    case TTC_ERR_INVALID_ARG: return "TTC_ERR_INVALID_ARG";
    case TTC_ERR_NOT_READY: return "TTC_ERR_NOT_READY";
  }
  return "TTC_ERR_UNKNOWN";
}

const char* ttc_last_error(void) { return ttc::g_last_error.c_str(); }

int64_t ttc_launch_count(void) { return ttc::launch_count(); }

}  // extern "C"

namespace {

// candidate schedules a plan keeps (the autotuner times up to this many)
constexpr int kPlanCandidates = 24;

ttc_status plan_create(ttc_plan_t* out, int ndim, const int* perm, const int64_t* sizes,
                       const int64_t* outer_sizes_A, const int64_t* outer_sizes_B, ttc_dtype dtype_in,
                       ttc_dtype dtype_out, double alpha, double alpha_im, double beta, double beta_im) {
  if (!out) return fail(TTC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  const int din = int(dtype_in), dout = int(dtype_out);
  if (din < 0 || din >= kNumDTypes || dout < 0 || dout >= kNumDTypes || !pair_supported(din, dout))
    return fail(TTC_ERR_UNSUPPORTED_DTYPE, "unsupported dtype pair");
  if (dout == DT_E4M3 && beta != 0.0)
    return fail(TTC_ERR_UNSUPPORTED_DTYPE, "FP8 output supports beta == 0 only");
  if (!std::isfinite(alpha) || !std::isfinite(beta) || !std::isfinite(alpha_im) || !std::isfinite(beta_im))
    return fail(TTC_ERR_INVALID_ARG, "alpha/beta not finite");
  if (!is_complex(din) && (alpha_im != 0.0 || beta_im != 0.0))
    return fail(TTC_ERR_UNSUPPORTED_DTYPE, "complex alpha/beta need complex tensors");
  std::unique_ptr<ttc_plan_s> p(new (std::nothrow) ttc_plan_s());
  if (!p) return fail(TTC_ERR_OOM, "host allocation failed");
  std::string err;
  int rc = canonicalize(ndim, perm, sizes, outer_sizes_A, outer_sizes_B, &p->canon, &err);
  if (rc != TTC_OK) return fail(ttc_status(rc), err);
  p->ndim = ndim;
  for (int k = 0; k < ndim; ++k) {
    p->perm0[k] = perm[k];
    p->sizes0[k] = sizes[k];
    p->outerA0[k] = outer_sizes_A ? outer_sizes_A[k] : sizes[k];
  }
  for (int d = 0; d < ndim; ++d) p->outerB0[d] = outer_sizes_B ? outer_sizes_B[d] : sizes[perm[d]];
  p->din = din;
  p->dout = dout;
  p->alpha = alpha;
  p->beta = beta;
  p->alpha_im = alpha_im;
  p->beta_im = beta_im;
  p->cands = make_candidates(p->canon, din, dout, p->beta_nonzero() ? 1.0 : 0.0, kPlanCandidates);
  if (p->cands.empty()) return fail(TTC_ERR_INVALID_SIZE, "no schedule fits this problem");
  if (p->canon.n > 0) {
    build_amax_rows(p->canon, dtype_size(p->din), &p->amax_rows);
    if (dout == DT_E4M3 && double(p->canon.n) / double(p->canon.s[0]) >= 2147483647.0)
      return fail(TTC_ERR_INVALID_SIZE, "too many rows for the FP8 amax pass");
  }
  *out = p.release();
  return TTC_OK;
}

}  // namespace

extern "C" {

ttc_status ttc_plan(ttc_plan_t* out, int ndim, const int* perm, const int64_t* sizes,
                    const int64_t* outer_sizes_A, const int64_t* outer_sizes_B, ttc_dtype dtype_in,
                    ttc_dtype dtype_out, double alpha, double beta) {
  return plan_create(out, ndim, perm, sizes, outer_sizes_A, outer_sizes_B, dtype_in, dtype_out, alpha, 0.0, beta,
                     0.0);
}

ttc_status ttc_plan_complex(ttc_plan_t* out, int ndim, const int* perm, const int64_t* sizes,
                            const int64_t* outer_sizes_A, const int64_t* outer_sizes_B, ttc_dtype dtype_in,
                            ttc_dtype dtype_out, double alpha_re, double alpha_im, double beta_re,
                            double beta_im) {
  return plan_create(out, ndim, perm, sizes, outer_sizes_A, outer_sizes_B, dtype_in, dtype_out, alpha_re,
                     alpha_im, beta_re, beta_im);
}

ttc_status ttc_plan_destroy(ttc_plan_t plan) {
  if (!plan) return fail(TTC_ERR_INVALID_ARG, "plan is NULL");
  int cur = 0;
  bool have = cudaGetDevice(&cur) == cudaSuccess;
  for (auto& kv : plan->dev) {
    if (kv.second.base) {
      if (have) cudaSetDevice(kv.first);
      cudaFree(kv.second.base);
    }
  }
  if (have) cudaSetDevice(cur);
  delete plan;
  return TTC_OK;
}

ttc_status ttc_execute(ttc_plan_t plan, const void* A, void* B, ttc_stream_t stream) {
  if (!plan) return fail(TTC_ERR_INVALID_ARG, "plan is NULL");
  if (plan->canon.n == 0) return TTC_OK;
  if (!A || !B) return fail(TTC_ERR_INVALID_ARG, "A or B is NULL");
  const uintptr_t a = reinterpret_cast<uintptr_t>(A), b = reinterpret_cast<uintptr_t>(B);
  if (a % dtype_size(plan->din) || b % dtype_size(plan->dout))
    return fail(TTC_ERR_ALIGN, "A or B not aligned to its element size");
  const uintptr_t ea = a + uintptr_t(plan->canon.spanA) * dtype_size(plan->din);
  const uintptr_t eb = b + uintptr_t(plan->canon.spanB) * dtype_size(plan->dout);
  if (a < eb && b < ea) return fail(TTC_ERR_ALIAS, "the byte ranges of A and B overlap");
  return run_plan(plan, A, B, reinterpret_cast<cudaStream_t>(stream));
}

ttc_status ttc_plan_set_fp8_scale(ttc_plan_t plan, const float* d_scale) {
  if (!plan) return fail(TTC_ERR_INVALID_ARG, "plan is NULL");
  if (plan->dout != DT_E4M3) return fail(TTC_ERR_INVALID_ARG, "plan does not produce FP8");
  plan->user_scale = d_scale;
  return TTC_OK;
}

ttc_status ttc_plan_get_fp8_scale(ttc_plan_t plan, float* d_scale_out, ttc_stream_t stream) {
  if (!plan || !d_scale_out) return fail(TTC_ERR_INVALID_ARG, "NULL argument");
  if (plan->dout != DT_E4M3) return fail(TTC_ERR_INVALID_ARG, "plan does not produce FP8");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  auto it = plan->dev.find(dev);
  if (it == plan->dev.end() || !it->second.base) return fail(TTC_ERR_INVALID_ARG, "plan not executed on this device");
  e = cudaMemcpyAsync(d_scale_out, it->second.scale, sizeof(float), cudaMemcpyDeviceToDevice,
                      reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
  return TTC_OK;
}

ttc_status ttc_plan_get_info(ttc_plan_t plan, ttc_plan_info* info) {
  if (!plan || !info) return fail(TTC_ERR_INVALID_ARG, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  const Canon& c = plan->canon;
  info->ndim = c.N;
  for (int k = 0; k < c.N; ++k) {
    info->perm[k] = c.perm[k];
    info->sizes[k] = c.s[k];
    info->stride_A[k] = c.sa[k];
    info->stride_B[k] = c.sb[k];
  }
  info->n = c.n;
  const int sa = dtype_size(plan->din), sb = dtype_size(plan->dout);
  info->algorithmic_bytes = c.n * (sa + (plan->beta_nonzero() ? 2 * sb : sb));
  const Candidate& k = plan->cands[plan->sel];
  info->variant = k.rows ? TTC_VARIANT_ROWCOPY : k.variant == VAR_TMA ? TTC_VARIANT_TMA_TILE : k.variant;
  info->candidate = plan->sel;
  info->ncandidates = int(plan->cands.size());
  if (k.variant == VAR_TILE) {
    TileParams tp;
    std::vector<int32_t> ta, tb;
    int sm = 0;
    build_tile_params(c, k, plan->din, &tp, &ta, &tb, &sm);
    info->tile_c = tp.LC;
    info->tile_a = tp.LA;
    info->tile_b = tp.LB;
    info->ntiles = tp.ntiles;
    info->vec_in = info->vec_out = k.rows ? k.vec : 1;
    info->lanes_a = k.pk ? 0 : 32 * k.ju;
    info->lanes_b = k.pk ? 0 : 32 * k.jw;
    info->slot_tables = k.slots;
    info->packed_threads = k.pk;
    info->packed_rows = k.rj;
  } else if (k.variant == VAR_COPY) {
    RowParams rp;
    build_row_params(c, k.chunk, &rp);
    info->tile_c = int(std::min<int64_t>(c.s[0], INT32_MAX));
    info->tile_a = info->tile_b = 1;
    info->ntiles = rp.nitems;
    info->vec_in = info->vec_out = k.vec;
  } else if (k.variant == VAR_TMA) {
    const Tma2dGeom g = tma2d_geom(c, plan->din);
    info->tile_c = 1;
    info->tile_a = g.bx;
    info->tile_b = 32 * kTmaBoxes;
    info->ntiles = g.tiles;
    info->vec_in = info->vec_out = 1;
  }
  return TTC_OK;
}

ttc_status ttc_plan_select_candidate(ttc_plan_t plan, int index) {
  if (!plan) return fail(TTC_ERR_INVALID_ARG, "plan is NULL");
  if (index < 0 || index >= int(plan->cands.size())) return fail(TTC_ERR_INVALID_ARG, "no such candidate");
  std::lock_guard<std::mutex> lk(plan->mu);
  plan->sel = index;
  plan->user_selected = true;
  return TTC_OK;
}

ttc_status ttc_plan_autotune(ttc_plan_t plan, int max_candidates, ttc_stream_t stream, float* best_ms) {
  if (!plan) return fail(TTC_ERR_INVALID_ARG, "plan is NULL");
  if (plan->canon.n == 0) {
    if (best_ms) *best_ms = 0.f;
    return TTC_OK;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int nc = std::min<int>(max_candidates > 0 ? max_candidates : 1, int(plan->cands.size()));
  const size_t bytesA = size_t(plan->canon.spanA) * dtype_size(plan->din);
  const size_t bytesB = size_t(plan->canon.spanB) * dtype_size(plan->dout);
  void *dA = nullptr, *dB = nullptr;
  cudaError_t e = cudaMalloc(&dA, bytesA);
  if (e != cudaSuccess) return fail(TTC_ERR_OOM, "autotune buffer allocation failed");
  e = cudaMalloc(&dB, bytesB);
  if (e != cudaSuccess) {
    cudaFree(dA);
    return fail(TTC_ERR_OOM, "autotune buffer allocation failed");
  }
  cudaMemsetAsync(dA, 0, bytesA, s);
  cudaMemsetAsync(dB, 0, bytesB, s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int saved = plan->sel;
  int best = saved;
  float best_t = 1e30f;
  ttc_status st = TTC_OK;
  // repetitions: enough to cover ~2 ms per candidate, at least 3
  const double bytes = double(plan->canon.n) * (dtype_size(plan->din) + dtype_size(plan->dout));
  const int reps = int(std::min(50.0, std::max(3.0, 2e-3 * 5e12 / std::max(bytes, 1.0))));
  for (int i = 0; i < nc && st == TTC_OK; ++i) {
    plan->sel = i;
    st = run_plan(plan, dA, dB, s);   // warm-up (uploads tables)
    if (st != TTC_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == TTC_OK; ++r) st = run_plan(plan, dA, dB, s);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "autotune timing");
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (ms < best_t) {
      best_t = ms;
      best = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(dA);
  cudaFree(dB);
  plan->sel = (st == TTC_OK) ? best : saved;
  if (st != TTC_OK) return st;
  if (best_ms) *best_ms = best_t;
  int dev = 0;
  cudaGetDevice(&dev);
  const std::string key = plan_key(plan, dev);
  plan->user_selected = true;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = cand_key(plan->cands[best]);
  return TTC_OK;
}

ttc_status ttc_tune_cache_save(const char* path) {
  if (!path) return fail(TTC_ERR_INVALID_ARG, "path is NULL");
  std::ofstream f(path);
  if (!f) return fail(TTC_ERR_INVALID_ARG, "cannot open file");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& kv : g_tune) f << kv.first << "\t" << kv.second << "\n";
  return TTC_OK;
}

ttc_status ttc_tune_cache_load(const char* path) {
  if (!path) return fail(TTC_ERR_INVALID_ARG, "path is NULL");
  std::ifstream f(path);
  if (!f) return fail(TTC_ERR_INVALID_ARG, "cannot open file");
  std::string line;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  while (std::getline(f, line)) {
    const size_t t = line.find('\t');
    if (t == std::string::npos) continue;
    g_tune[line.substr(0, t)] = line.substr(t + 1);
  }
  return TTC_OK;
}

}  // extern "C"
