// noalloc.cu -- ttc_execute_noalloc (include/ttc.h): a plan's execution with
// its device scratch (FP8 amax word and scale, tile offset tables) in a
// static device array instead of memory the plan allocates.
#include <cuda.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ttc.h"
#include "launch.h"
#include "plan_impl.h"
#include "planner.h"
#include "rowvec.h"
#include "tma2d.h"

using namespace ttc;

namespace {

// Layout of the static array: [0,4) amax bits, [16,20) scale, [256, end)
// offset tables (int32).
constexpr size_t kAmaxOff = 0;
constexpr size_t kScaleOff = 16;
constexpr size_t kTableOff = 256;

__device__ __align__(256) unsigned char g_noalloc_scratch[TTC_NOALLOC_SCRATCH_BYTES];

// The current CUDA context's process-unique id (cuCtxGetId), through the
// driver entry points that the runtime hands out (no link against the driver
// library); 0 when there is no current context or the driver lacks the calls.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

struct ScratchAddr {
  unsigned long long ctx = 0;
  void* ptr = nullptr;
};
std::mutex g_mu;
std::map<int, ScratchAddr> g_addr;

// The array's device address on `dev`, which is current.  In host code the
// symbol itself is only a host-side stand-in, so the kernels always receive
// this address.  It is looked up (cudaGetSymbolAddress) at the first call on
// each device and again whenever the device's context has changed since (a
// device reset, or another context made current), so a stale address is
// never handed to a kernel.
ttc_status scratch_address(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  const unsigned long long ctx = current_context_id();
  ScratchAddr& a = g_addr[dev];
  if (!a.ptr || ctx == 0 || a.ctx != ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      a = ScratchAddr();
      return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
    }
    // the lookup made the device's context current if it was not yet
    a.ctx = ctx ? ctx : current_context_id();
    a.ptr = p;
  }
  *out = static_cast<unsigned char*>(a.ptr);
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
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  // the plan's selected schedule, or the one an autotune remembered for this
  // problem on this device (as ttc_execute's first use on a device takes it)
  int sel = 0;
  {
    std::lock_guard<std::mutex> lk(plan->mu);
    sel = plan->sel;
    if (!plan->user_selected) {
      const int i = remembered_choice(plan, dev);
      if (i >= 0) sel = i;
    }
  }
  const Candidate& k = plan->cands[size_t(sel)];
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
  if (!ta.empty() || !tb.empty()) {
    // the offset tables are copied from host memory this call owns only until
    // it returns, which a captured copy would still refer to
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone)
      return fail(TTC_ERR_INVALID_ARG, "the schedule uploads offset tables, which a stream capture cannot take");
  }
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
    e = k.rows ? (k.vec > 1 ? launch_rowcopy_vec(plan->din, plan->dout, A, B, tp, s)
                            : launch_rowcopy(plan->din, plan->dout, A, B, tp, s))
        : k.rj ? launch_rowsp(plan->din, plan->dout, k.rj, A, B, tp, s)
        : k.pk ? launch_tilep(plan->din, plan->dout, k.pk, k.ju, k.jw, A, B, tp, smem, s)
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
  } else if (k.variant == VAR_TMA) {
    // (the tensor map travels as a kernel parameter: no scratch)
    e = launch_tma2d(plan->din, plan->dout, A, B, tma2d_geom(c, plan->din), epi, s);
    if (e != cudaSuccess) return cuda_fail(e, "TMA tile kernel launch");
  }
  return TTC_OK;
}
