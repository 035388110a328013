// noalloc.cu -- ttc_execute_noalloc (include/ttc.h): a plan's execution with
// its device scratch (FP8 amax word and scale, tile offset tables) in a
// static device array instead of memory the plan allocates.
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/ttc.h"
#include "launch.h"
#include "plan_impl.h"
#include "planner.h"

using namespace ttc;

namespace {

// Layout of the static array: [0,4) amax bits, [16,20) scale, [256, end)
// offset tables (int32).
constexpr size_t kAmaxOff = 0;
constexpr size_t kScaleOff = 16;
constexpr size_t kTableOff = 256;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[TTC_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// The array's device address on `dev` (looked up once per device, with that
// device current).  In host code the symbol itself is only a host-side
// stand-in, so the kernels always receive this address instead.
ttc_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(TTC_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return TTC_OK;
}

}  // namespace

extern "C" ttc_status ttc_execute_noalloc(ttc_plan_t plan, const void* A, void* B, float* d_scale_out,
                                          ttc_stream_t stream) {
  if (!plan) return fail(TTC_ERR_INVALID_ARG, "plan is NULL");
  const Canon& c = plan->canon;
  if (c.n == 0) return TTC_OK;
  if (!A || !B) return fail(TTC_ERR_INVALID_ARG, "A or B is NULL");
  const uintptr_t a = reinterpret_cast<uintptr_t>(A), b = reinterpret_cast<uintptr_t>(B);
  if (a % dtype_size(plan->din) || b % dtype_size(plan->dout))
    return fail(TTC_ERR_ALIGN, "A or B not aligned to its element size");
  const uintptr_t ea = a + uintptr_t(c.spanA) * dtype_size(plan->din);
  const uintptr_t eb = b + uintptr_t(c.spanB) * dtype_size(plan->dout);
  if (a < eb && b < ea) return fail(TTC_ERR_ALIAS, "the byte ranges of A and B overlap");

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const Candidate& k = plan->cands[plan->sel];
  TileParams tp;
  RowParams rp;
  std::vector<int32_t> ta, tb;
  int smem = 0;
  size_t table_bytes = 0;
  if (k.variant == VAR_TILE) {
    build_tile_params(c, k, plan->din, &tp, &ta, &tb, &smem);
    table_bytes = (ta.size() + tb.size()) * sizeof(int32_t);
  } else if (k.variant == VAR_COPY) {
    build_row_params(c, k.chunk, &rp);
  }
  if (kTableOff + table_bytes > size_t(TTC_NOALLOC_SCRATCH_BYTES))
    return fail(TTC_ERR_INVALID_SIZE, "schedule needs " + std::to_string(kTableOff + table_bytes) +
                                          " bytes of scratch; the static scratch holds " +
                                          std::to_string(TTC_NOALLOC_SCRATCH_BYTES));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  unsigned char* scratch = nullptr;
  ttc_status st = scratch_address(dev, &scratch);
  if (st != TTC_OK) return st;
  uint32_t* amax = reinterpret_cast<uint32_t*>(scratch + kAmaxOff);
  float* scale = reinterpret_cast<float*>(scratch + kScaleOff);
  int32_t* tables = reinterpret_cast<int32_t*>(scratch + kTableOff);

  Epilogue epi = make_epilogue(plan, nullptr);
  epi.amax_bits = amax;
  epi.scale_out = d_scale_out ? d_scale_out : scale;
  if (plan->dout == DT_E4M3 && !plan->user_scale) {
    e = cudaMemsetAsync(amax, 0, sizeof(uint32_t), s);    // the array keeps the last call's amax
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    e = launch_amax(plan->din, A, plan->amax_rows, float(plan->alpha), amax, nullptr, s);
    if (e != cudaSuccess) return cuda_fail(e, "amax kernel launch");
  }
  if (k.variant == VAR_TILE) {
    // pageable sources: the copy has left them once cudaMemcpyAsync returns
    if (!ta.empty()) {
      e = cudaMemcpyAsync(tables, ta.data(), ta.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return cuda_fail(e, "table upload");
    }
    if (!tb.empty()) {
      e = cudaMemcpyAsync(tables + ta.size(), tb.data(), tb.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return cuda_fail(e, "table upload");
    }
    tp.tabA = tables;
    tp.tabB = tables + ta.size();
    tp.epi = epi;
    e = k.rows ? launch_rowcopy(plan->din, plan->dout, A, B, tp, s)
        : k.ju ? launch_tile2(plan->din, plan->dout, k.ju, k.jw, A, B, tp, smem, s)
             : launch_tile(plan->din, plan->dout, A, B, tp, smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "tile kernel launch");
  } else if (k.variant == VAR_COPY) {
    rp.epi = epi;
    int vec = k.vec;
    if (vec > 1 && (a % (size_t(vec) * dtype_size(plan->din)) || b % (size_t(vec) * dtype_size(plan->dout)))) vec = 1;
    if (vec > 1 && rp.chunk % vec) vec = 1;
    e = launch_copy(plan->din, plan->dout, vec, A, B, rp, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy kernel launch");
  }
  return TTC_OK;
}
