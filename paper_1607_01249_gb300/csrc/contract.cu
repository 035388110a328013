// contract.cu -- tensor contractions by Transpose-Transpose-GEMM-Transpose
// (TTGT), the use of tensor transpositions that motivates the paper
// (section 1): each operand is permuted (and for the BF16 GEMM path
// downcast) by this library's permute-scale-add kernels into a matrix, the
// contraction runs as one GEMM, and the product is permuted into C with
// Eq. 1's beta update.  The BF16 mode permutes both operands into K-major
// BF16 matrices (the contracted indices fastest, the row pitch padded to a
// multiple of 8 elements) and runs this library's tensor-core GEMM
// (gemm.cu); the exact FP32 and FP64 modes run a cuBLAS GEMM in pedantic
// math (SIMT FP32/FP64, no reduced-precision substitution), with an operand
// already laid out as a matrix in either order passed as it is.  A C laid out
// as [free A indices, free B indices] or the reverse takes the GEMM's output
// directly.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ttc.h"
#include "../../include/ttc_debug.h"
#include "gemm.h"
#include "plan_impl.h"

using namespace ttc;

namespace {

// One operand's role in the GEMM: either the tensor itself (op N or T) or a
// workspace matrix that a transpose plan fills.
struct Operand {
  ttc_plan_t plan = nullptr;   // null: the tensor is used in place
  bool trans = false;          // GEMM op: the stored matrix is the transpose of the one needed
  int64_t ld = 1;              // leading dimension of the stored matrix
  size_t ws_bytes = 0;         // workspace bytes when plan is set
};

struct DevState {
  cublasHandle_t handle = nullptr;
  void* ws = nullptr;          // A' | B' | C' workspaces | error word of the tensor-core GEMM
  size_t bytes = 0;
  int* err = nullptr;
  // the two operand permutes run side by side: B's on `side`, forked from
  // and joined back into the caller's stream by the two events
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

}  // namespace

struct ttc_contraction_s {
  std::mutex mu;
  int dtype = 0, gemm_dtype = 0;
  double alpha = 1.0, beta = 0.0;
  int64_t M = 1, N = 1, K = 1;
  bool swap = false;           // C is [free B, free A]: compute C^T = B'^T A'^T
  Operand opA, opB;
  int64_t kpitch = 0;          // BF16 mode: row pitch of the K-major operands (K rounded up to 8)
  std::vector<int64_t> offs;   // BF16 mode: C offsets of the GEMM's rows (M' entries), then columns (N')
  bool use_cublas = false;     // testing hook: the BF16 mode's GEMM on cuBLAS (a timed comparison)
  int gemm_variant = 0;        // testing hook: the tensor-core GEMM's tile shape (GemmVariant; 0 = pick)
  int gemm_used = 0;           // the tile shape of the last execution
  ttc_plan_t planC = nullptr;  // C' -> C with beta, when C is not a GEMM output layout
  size_t wsC = 0;
  int64_t sizeA = 0, sizeB = 0, sizeC = 0;   // elements of each tensor
  // BF16 mode: what the K-major operands are built from, and the other
  // order of the contracted labels (B's, when it differs from A's) that the
  // autotuner may take instead (both operands share the order; the GEMM and
  // C's offsets do not depend on it)
  std::vector<int> mA, mB, freeA, freeB, kalt;
  std::vector<int64_t> sA, sB;
  std::map<int, int64_t> ext;
  std::map<int, DevState> dev;
  ~ttc_contraction_s() {
    if (opA.plan) ttc_plan_destroy(opA.plan);
    if (opB.plan) ttc_plan_destroy(opB.plan);
    if (planC) ttc_plan_destroy(planC);
    int cur = 0;
    const bool have = cudaGetDevice(&cur) == cudaSuccess;
    for (auto& kv : dev) {
      if (have) cudaSetDevice(kv.first);
      if (kv.second.handle) cublasDestroy(kv.second.handle);
      if (kv.second.ws) cudaFree(kv.second.ws);
      if (kv.second.fork) cudaEventDestroy(kv.second.fork);
      if (kv.second.join) cudaEventDestroy(kv.second.join);
      if (kv.second.side) cudaStreamDestroy(kv.second.side);
    }
    if (have) cudaSetDevice(cur);
  }
};

namespace {

bool positions_of(const std::vector<int>& modes, const std::vector<int>& want, std::vector<int>* pos) {
  pos->clear();
  for (int m : want) {
    auto it = std::find(modes.begin(), modes.end(), m);
    if (it == modes.end()) return false;
    pos->push_back(int(it - modes.begin()));
  }
  return true;
}

// the permutation (B position d <- tensor index perm[d]) that lays `modes`
// out in the order `order`
std::vector<int> perm_to(const std::vector<int>& modes, const std::vector<int>& order) {
  std::vector<int> p;
  positions_of(modes, order, &p);
  return p;
}

bool is_concat(const std::vector<int>& modes, const std::vector<int>& a, const std::vector<int>& b) {
  std::vector<int> c(a);
  c.insert(c.end(), b.begin(), b.end());
  return c == modes;
}

// Set up operand X (modes `mx`, sizes `sx`) to appear in the GEMM as the
// matrix [rows..., cols...] (rows stride 1), rows x cols = R x Cc.
ttc_status setup_operand(const std::vector<int>& mx, const std::vector<int64_t>& sx, const std::vector<int>& rows,
                         const std::vector<int>& cols, int64_t R, int64_t Cc, int din, int dgemm, double scale,
                         Operand* op) {
  const bool same_type = din == dgemm;
  // already a matrix in either orientation: used in place, or (BF16 GEMM)
  // downcast in its own layout, a streaming copy
  const bool as_is = is_concat(mx, rows, cols), flipped = !as_is && is_concat(mx, cols, rows);
  if (as_is || flipped) {
    op->trans = flipped;
    op->ld = std::max<int64_t>(flipped ? Cc : R, 1);
    if (same_type) return TTC_OK;
  }
  std::vector<int> order(rows);
  order.insert(order.end(), cols.begin(), cols.end());
  if (flipped) {
    order = cols;
    order.insert(order.end(), rows.begin(), rows.end());
  }
  const std::vector<int> p = perm_to(mx, order);
  ttc_plan_t plan = nullptr;
  const ttc_status st = ttc_plan(&plan, int(mx.size()), p.data(), sx.data(), nullptr, nullptr, ttc_dtype(din),
                                 ttc_dtype(dgemm), scale, 0.0);
  if (st != TTC_OK) return st;
  op->plan = plan;
  if (!flipped) {
    op->trans = false;
    op->ld = std::max<int64_t>(R, 1);
  }
  op->ws_bytes = size_t(R) * size_t(Cc) * size_t(dtype_size(dgemm));
  return TTC_OK;
}

// BF16 mode: operand X (modes `mx`, sizes `sx`) as a K-major BF16 matrix:
// for every free position (`frees`, column-major) the contracted indices
// (`contracted`, column-major) at consecutive addresses, at a row pitch of
// K rounded up to a multiple of 8 elements (the last contracted index's
// outer extent is widened; the padding is never read).  rows = product of
// the free extents.
ttc_status setup_kmajor(const std::vector<int>& mx0, const std::vector<int64_t>& sx0,
                        const std::vector<int>& contracted0, const std::vector<int>& frees,
                        std::map<int, int64_t> ext, int64_t rows, int din, int64_t* kpitch, Operand* op) {
  std::vector<int> mx(mx0), contracted(contracted0);
  std::vector<int64_t> sx(sx0);
  if (contracted.empty()) {
    // an outer product (K = 1): a contracted index of extent 1 stands in,
    // appended to the operand, so that the rows still have a pitch
    int dummy = 0;
    for (const auto& kv : ext) dummy = std::max(dummy, kv.first + 1);
    mx.push_back(dummy);
    sx.push_back(1);
    contracted.push_back(dummy);
    ext[dummy] = 1;
  }
  std::vector<int> order(contracted);
  order.insert(order.end(), frees.begin(), frees.end());
  const std::vector<int> p = perm_to(mx, order);
  std::vector<int64_t> outer;
  int64_t below = 1;   // product of the contracted extents before the last one
  for (size_t i = 0; i < order.size(); ++i) outer.push_back(ext.at(order[i]));
  for (size_t i = 0; i + 1 < contracted.size(); ++i) below *= ext.at(contracted[i]);
  const int64_t last = ext.at(contracted.back());
  int64_t o = last;
  while ((below * o) % 8) ++o;
  outer[contracted.size() - 1] = o;
  ttc_plan_t plan = nullptr;
  const ttc_status st = ttc_plan(&plan, int(mx.size()), p.data(), sx.data(), nullptr, outer.data(), ttc_dtype(din),
                                 TTC_BF16, 1.0, 0.0);
  if (st != TTC_OK) return st;
  op->plan = plan;
  op->trans = false;
  op->ld = below * o;
  op->ws_bytes = size_t(below * o) * size_t(std::max<int64_t>(rows, 1)) * 2;
  *kpitch = below * o;
  return TTC_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

ttc_status cublas_fail(cublasStatus_t s, const char* where) {
  return fail(TTC_ERR_CUDA, std::string(where) + ": cuBLAS status " + std::to_string(int(s)));
}

}  // namespace

extern "C" {

ttc_status ttc_contraction_plan(ttc_contraction_t* out, int nA, const int* modes_A, const int64_t* sizes_A, int nB,
                                const int* modes_B, const int64_t* sizes_B, int nC, const int* modes_C,
                                const int64_t* sizes_C, ttc_dtype dtype, ttc_dtype gemm_dtype, double alpha,
                                double beta) {
  if (!out) return fail(TTC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nA < 0 || nB < 0 || nC < 0 || nA > kMaxDim || nB > kMaxDim || nC > kMaxDim)
    return fail(TTC_ERR_INVALID_PERM, "tensor order out of range");
  if ((nA && (!modes_A || !sizes_A)) || (nB && (!modes_B || !sizes_B)) || (nC && (!modes_C || !sizes_C)))
    return fail(TTC_ERR_INVALID_ARG, "NULL modes or sizes");
  const int dt = int(dtype), dg = int(gemm_dtype);
  const bool ok_types = (dt == DT_F32 && (dg == DT_F32 || dg == DT_BF16)) || (dt == DT_F64 && dg == DT_F64);
  if (!ok_types) return fail(TTC_ERR_UNSUPPORTED_DTYPE, "supported: f32 (f32 or bf16 GEMM), f64 (f64 GEMM)");
  if (!std::isfinite(alpha) || !std::isfinite(beta)) return fail(TTC_ERR_INVALID_ARG, "alpha/beta not finite");
  std::vector<int> mA(modes_A, modes_A + nA), mB(modes_B, modes_B + nB), mC(modes_C, modes_C + nC);
  std::vector<int64_t> sA(sizes_A, sizes_A + nA), sB(sizes_B, sizes_B + nB), sC(sizes_C, sizes_C + nC);
  // every label: its extent (consistent) and the tensors it appears in
  std::map<int, int64_t> ext;
  std::map<int, int> where;   // bit 0: A, 1: B, 2: C
  auto note = [&](const std::vector<int>& m, const std::vector<int64_t>& s, int bit) -> ttc_status {
    for (size_t i = 0; i < m.size(); ++i) {
      if (s[i] < 0) return fail(TTC_ERR_INVALID_SIZE, "negative size");
      if (where[m[i]] & (1 << bit)) return fail(TTC_ERR_INVALID_PERM, "a label repeats within one tensor");
      where[m[i]] |= 1 << bit;
      auto it = ext.find(m[i]);
      if (it != ext.end() && it->second != s[i]) return fail(TTC_ERR_INVALID_SIZE, "a label has two extents");
      ext[m[i]] = s[i];
    }
    return TTC_OK;
  };
  ttc_status st = note(mA, sA, 0);
  if (st == TTC_OK) st = note(mB, sB, 1);
  if (st == TTC_OK) st = note(mC, sC, 2);
  if (st != TTC_OK) return st;
  std::vector<int> contracted, freeA, freeB;   // contracted in A's order, free in C's order
  for (int m : mA)
    if (where[m] == 3) contracted.push_back(m);
  for (int m : mC) {
    if (where[m] == 5) freeA.push_back(m);
    else if (where[m] == 6) freeB.push_back(m);
    else if (where[m] == 7) return fail(TTC_ERR_INVALID_PERM, "a label in A, B and C (batched) is not supported");
    else return fail(TTC_ERR_INVALID_PERM, "a label of C appears in neither A nor B");
  }
  for (auto& kv : where)
    if (kv.second == 1 || kv.second == 2) return fail(TTC_ERR_INVALID_PERM, "a label appears in one operand only");
  std::unique_ptr<ttc_contraction_s> c(new (std::nothrow) ttc_contraction_s());
  if (!c) return fail(TTC_ERR_OOM, "host allocation failed");
  c->dtype = dt;
  c->gemm_dtype = dg;
  c->alpha = alpha;
  c->beta = beta;
  auto prod = [&](const std::vector<int>& ls) {
    int64_t p = 1;
    for (int l : ls) p *= ext[l];
    return p;
  };
  c->M = prod(freeA);
  c->N = prod(freeB);
  c->K = prod(contracted);
  c->sizeA = prod(mA);
  c->sizeB = prod(mB);
  c->sizeC = prod(mC);
  if (c->M > INT32_MAX || c->N > INT32_MAX || c->K > INT32_MAX)
    return fail(TTC_ERR_INVALID_SIZE, "a GEMM extent exceeds 2^31 - 1");
  // C as the GEMM output: [freeA, freeB] directly, [freeB, freeA] by
  // computing the transpose; else through C' and a final transpose with beta
  if (dg == DT_BF16) {
    // Both operands K-major BF16 for the tensor-core GEMM, and C written by
    // the GEMM's epilogue at offset rowoff[m] + coloff[n] in any layout (the
    // transpose of the product folded into the stores): the GEMM's rows are
    // the free labels of the operand that holds C's stride-1 label, so that
    // consecutive rows are consecutive in C; each operand's free labels in
    // C's order.  With an empty extent nothing is permuted.
    const bool b_rows = !mC.empty() && where[mC[0]] == 6;
    c->swap = b_rows;
    c->kpitch = 8;
    if (c->K > 0 && c->M > 0 && c->N > 0) {
      st = setup_kmajor(mA, sA, contracted, freeA, ext, c->M, dt, &c->kpitch, &c->opA);
      if (st == TTC_OK) st = setup_kmajor(mB, sB, contracted, freeB, ext, c->N, dt, &c->kpitch, &c->opB);
      if (st != TTC_OK) return st;
      std::vector<int> kB;
      for (int m : mB)
        if (where[m] == 3) kB.push_back(m);
      if (kB != contracted) {
        c->kalt = kB;
        c->mA = mA;
        c->mB = mB;
        c->sA = sA;
        c->sB = sB;
        c->freeA = freeA;
        c->freeB = freeB;
        c->ext = ext;
      }
    }
    std::map<int, int64_t> strideC;
    int64_t acc = 1;
    for (size_t i = 0; i < mC.size(); ++i) {
      strideC[mC[i]] = acc;
      acc *= sC[i];
    }
    auto offsets = [&](const std::vector<int>& labels) {
      int64_t cnt = 1;
      for (int l : labels) cnt *= ext[l];
      for (int64_t i = 0; i < cnt; ++i) {
        int64_t r = i, off = 0;
        for (int l : labels) {
          off += (r % ext[l]) * strideC[l];
          r /= ext[l];
        }
        c->offs.push_back(off);
      }
    };
    offsets(b_rows ? freeB : freeA);
    offsets(b_rows ? freeA : freeB);
    // the timed comparison on cuBLAS writes the product as a column-major
    // matrix [rows, columns]; a C of another layout then takes it through a
    // permute plan with beta (the unfused route)
    const std::vector<int>& rl = b_rows ? freeB : freeA;
    const std::vector<int>& cl = b_rows ? freeA : freeB;
    std::vector<int> cp(rl);
    cp.insert(cp.end(), cl.begin(), cl.end());
    if (cp != mC && c->M > 0 && c->N > 0) {
      std::vector<int64_t> scp;
      for (int l : cp) scp.push_back(ext[l]);
      const std::vector<int> p = perm_to(cp, mC);
      st = ttc_plan(&c->planC, int(cp.size()), p.data(), scp.data(), nullptr, nullptr, ttc_dtype(dt), ttc_dtype(dt),
                    1.0, beta);
      if (st != TTC_OK) return st;
      c->wsC = size_t(c->M) * size_t(c->N) * size_t(dtype_size(dt));
    }
    *out = c.release();
    return TTC_OK;
  }
  const bool direct = is_concat(mC, freeA, freeB);
  const bool swapped = !direct && is_concat(mC, freeB, freeA);
  std::vector<int> fa(freeA), fb(freeB);
  if (!direct && !swapped) {
    // C is permuted anyway: keep the free indices in their operands' own order
    fa.clear();
    fb.clear();
    for (int m : mA)
      if (where[m] == 5) fa.push_back(m);
    for (int m : mB)
      if (where[m] == 6) fb.push_back(m);
  }
  c->swap = swapped;
  // the A operand as the M x K matrix [fa, contracted]; B as K x N [contracted, fb]
  st = setup_operand(mA, sA, fa, contracted, c->M, c->K, dt, dg, 1.0, &c->opA);
  if (st == TTC_OK) st = setup_operand(mB, sB, contracted, fb, c->K, c->N, dt, dg, 1.0, &c->opB);
  if (st != TTC_OK) return st;
  if (!direct && !swapped) {
    std::vector<int> cp(fa);
    cp.insert(cp.end(), fb.begin(), fb.end());     // C' index order
    std::vector<int64_t> scp;
    for (int l : cp) scp.push_back(ext[l]);
    const std::vector<int> p = perm_to(cp, mC);     // C position d <- C' index p[d]
    st = ttc_plan(&c->planC, int(cp.size()), p.data(), scp.data(), nullptr, nullptr, ttc_dtype(dt), ttc_dtype(dt),
                  1.0, beta);
    if (st != TTC_OK) return st;
    c->wsC = size_t(c->M) * size_t(c->N) * size_t(dtype_size(dt));
  }
  *out = c.release();
  return TTC_OK;
}

ttc_status ttc_contraction_execute(ttc_contraction_t c, const void* A, const void* B, void* C, ttc_stream_t stream) {
  if (!c) return fail(TTC_ERR_INVALID_ARG, "contraction is NULL");
  if (c->sizeC == 0) return TTC_OK;
  if (!C || (c->K > 0 && (!A || !B))) return fail(TTC_ERR_INVALID_ARG, "A, B or C is NULL");
  const uintptr_t pc = reinterpret_cast<uintptr_t>(C);
  const size_t es = size_t(dtype_size(c->dtype));
  for (const void* X : {A, B}) {
    const uintptr_t px = reinterpret_cast<uintptr_t>(X);
    const size_t bx = size_t(X == A ? c->sizeA : c->sizeB) * es;
    if (X && px < pc + size_t(c->sizeC) * es && pc < px + bx)
      return fail(TTC_ERR_ALIAS, "C overlaps an operand");
  }
  if (pc % es || reinterpret_cast<uintptr_t>(A) % es || reinterpret_cast<uintptr_t>(B) % es)
    return fail(TTC_ERR_ALIGN, "a pointer is not aligned to its element size");
  std::lock_guard<std::mutex> lk(c->mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  DevState& ds = c->dev[dev];
  const size_t need = align256(c->opA.ws_bytes) + align256(c->opB.ws_bytes) + align256(c->wsC) +
                      align256(c->offs.size() * sizeof(int64_t)) + 256;
  if (!ds.handle) {
    cublasStatus_t cs = cublasCreate(&ds.handle);
    if (cs != CUBLAS_STATUS_SUCCESS) {
      ds.handle = nullptr;
      return cublas_fail(cs, "cublasCreate");
    }
    // exact FP32/FP64 GEMMs (no reduced-precision tensor-core substitution)
    cublasSetMathMode(ds.handle, c->gemm_dtype == DT_BF16 ? CUBLAS_DEFAULT_MATH : CUBLAS_PEDANTIC_MATH);
  }
  if (need && !ds.ws) {
    e = cudaMalloc(&ds.ws, need);
    if (e != cudaSuccess) {
      ds.ws = nullptr;
      return e == cudaErrorMemoryAllocation ? fail(TTC_ERR_OOM, "workspace allocation failed")
                                            : cuda_fail(e, "cudaMalloc");
    }
    ds.bytes = need;
    ds.err = reinterpret_cast<int*>(static_cast<char*>(ds.ws) + need - 256);
    if (c->opA.plan && c->opB.plan) {
      // (without them both permutes stay on the caller's stream)
      if (cudaStreamCreateWithFlags(&ds.side, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&ds.fork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&ds.join, cudaEventDisableTiming) != cudaSuccess) {
        (void)cudaGetLastError();
        if (ds.side) cudaStreamDestroy(ds.side);
        if (ds.fork) cudaEventDestroy(ds.fork);
        if (ds.join) cudaEventDestroy(ds.join);
        ds.side = nullptr;
        ds.fork = ds.join = nullptr;
      }
    }
    e = cudaMemset(ds.err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
    if (!c->offs.empty()) {
      e = cudaMemcpy(static_cast<char*>(ds.ws) + align256(c->opA.ws_bytes) + align256(c->opB.ws_bytes) +
                         align256(c->wsC),
                     c->offs.data(), c->offs.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_fail(e, "offset table upload");
    }
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ds.ws);
  void* wa = w;
  void* wb = w + align256(c->opA.ws_bytes);
  void* wc = w + align256(c->opA.ws_bytes) + align256(c->opB.ws_bytes);
  // (empty contractions, K = 0, leave alpha * 0 + beta * C: the GEMM below
  // handles k = 0 as a pure beta scaling)
  const void* ga = A;
  const void* gb = B;
  const bool permA = c->opA.plan && c->K > 0 && c->M > 0;
  const bool permB = c->opB.plan && c->K > 0 && c->N > 0;
  // both operands permuted: B's permute on the side stream, so that the two
  // launches fill each other's ramp and tail
  const bool side = permA && permB && ds.side;
  if (side) {
    e = cudaEventRecord(ds.fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ds.side, ds.fork, 0);
    if (e != cudaSuccess) return cuda_fail(e, "fork of the operand permutes");
  }
  if (permA) {
    ttc_status st = run_plan(c->opA.plan, A, wa, s);
    if (st != TTC_OK) return st;
    ga = wa;
  }
  if (permB) {
    ttc_status st = run_plan(c->opB.plan, B, wb, side ? ds.side : s);
    if (st != TTC_OK) return st;
    gb = wb;
  }
  if (side) {
    e = cudaEventRecord(ds.join, ds.side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ds.join, 0);
    if (e != cudaSuccess) return cuda_fail(e, "join of the operand permutes");
  }
  void* gc = c->planC ? wc : C;
  const double beta_g = c->planC ? 0.0 : c->beta;
  if (c->kpitch && !c->use_cublas) {
    // the tensor-core GEMM on the K-major operands, rows from the operand
    // holding C's stride-1 label, C written through the offset tables
    if (c->M == 0 || c->N == 0) return TTC_OK;
    const bool sw = c->swap;
    const void* X = sw ? gb : ga;
    const void* Y = sw ? ga : gb;
    const int64_t m = sw ? c->N : c->M, n = sw ? c->M : c->N;
    const int64_t* rows = reinterpret_cast<const int64_t*>(static_cast<char*>(wc) + align256(c->wsC));
    if (const char* why = gemm_bf16_check(X, c->kpitch, Y, c->kpitch, m, n, c->K)) return fail(TTC_ERR_INVALID_SIZE, why);
    e = gemm_bf16(X, c->kpitch, Y, c->kpitch, static_cast<float*>(C), rows, rows + m, m, n, c->K, float(c->alpha),
                  float(c->beta), ds.err, c->gemm_variant, &c->gemm_used, s);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core GEMM launch");
    return TTC_OK;
  }
  cublasStatus_t cs = cublasSetStream(ds.handle, s);
  if (cs != CUBLAS_STATUS_SUCCESS) return cublas_fail(cs, "cublasSetStream");
  // column-major GEMM: C (M x N) = op(A') (M x K) op(B') (K x N); with swap,
  // C^T (N x M) = op(B')^T op(A')^T
  const bool sw = c->swap;
  const int m = int(sw ? c->N : c->M), n = int(sw ? c->M : c->N), k = int(c->K);
  const void* X = sw ? gb : ga;
  const void* Y = sw ? ga : gb;
  const Operand& ox = sw ? c->opB : c->opA;
  const Operand& oy = sw ? c->opA : c->opB;
  // op of the first factor: A' stored [M x K] is used as is; with swap the
  // first factor is B'^T, i.e. the stored K x N matrix transposed
  const cublasOperation_t tx = (ox.trans != sw) ? CUBLAS_OP_T : CUBLAS_OP_N;
  const cublasOperation_t ty = (oy.trans != sw) ? CUBLAS_OP_T : CUBLAS_OP_N;
  const int ldx = int(std::max<int64_t>(ox.ld, 1)), ldy = int(std::max<int64_t>(oy.ld, 1));
  const int ldc = std::max(m, 1);
  if (m == 0 || n == 0) return TTC_OK;
  if (c->dtype == DT_F64) {
    const double al = c->alpha, be = beta_g;
    cs = cublasDgemm(ds.handle, tx, ty, m, n, k, &al, static_cast<const double*>(X), ldx,
                     static_cast<const double*>(Y), ldy, &be, static_cast<double*>(gc), ldc);
  } else if (c->gemm_dtype == DT_F32) {
    const float al = float(c->alpha), be = float(beta_g);
    cs = cublasSgemm(ds.handle, tx, ty, m, n, k, &al, static_cast<const float*>(X), ldx,
                     static_cast<const float*>(Y), ldy, &be, static_cast<float*>(gc), ldc);
  } else if (c->kpitch) {
    // the timed comparison: the same K-major BF16 operands on cuBLAS, the
    // product [rows, columns] into C or, for another layout, into C' and a
    // permute plan
    const float al = float(c->alpha), be = float(beta_g);
    const int kp = int(c->kpitch);
    cs = cublasGemmEx(ds.handle, CUBLAS_OP_T, CUBLAS_OP_N, m, n, k, &al, X, CUDA_R_16BF, kp, Y, CUDA_R_16BF, kp, &be,
                      gc, CUDA_R_32F, ldc, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
  } else {
    const float al = float(c->alpha), be = float(beta_g);
    cs = cublasGemmEx(ds.handle, tx, ty, m, n, k, &al, X, CUDA_R_16BF, ldx, Y, CUDA_R_16BF, ldy, &be, gc,
                      CUDA_R_32F, ldc, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
  }
  if (cs != CUBLAS_STATUS_SUCCESS) return cublas_fail(cs, "GEMM");
  if (c->planC) return run_plan(c->planC, wc, C, s);
  return TTC_OK;
}

ttc_status ttc_contraction_info(ttc_contraction_t c, int64_t* m, int64_t* n, int64_t* k, int* transposes) {
  if (!c) return fail(TTC_ERR_INVALID_ARG, "contraction is NULL");
  if (m) *m = c->M;
  if (n) *n = c->N;
  if (k) *k = c->K;
  if (transposes) *transposes = (c->opA.plan ? 1 : 0) + (c->opB.plan ? 2 : 0) + (c->planC ? 4 : 0);
  return TTC_OK;
}

ttc_status ttc_contraction_autotune(ttc_contraction_t c, int max_candidates, ttc_stream_t stream) {
  if (!c) return fail(TTC_ERR_INVALID_ARG, "contraction is NULL");
  std::lock_guard<std::mutex> lk(c->mu);
  if (!c->kalt.empty() && c->dev.empty() && c->opA.plan && c->opB.plan) {
    // BF16 mode before its first execution: the contracted labels in A's
    // order or in B's, whichever pair of operand permutes times faster
    float ta = 0.f, tb = 0.f, ta2 = 0.f, tb2 = 0.f;
    ttc_status st = ttc_plan_autotune(c->opA.plan, max_candidates, stream, &ta);
    if (st == TTC_OK) st = ttc_plan_autotune(c->opB.plan, max_candidates, stream, &tb);
    if (st != TTC_OK) return st;
    Operand a2, b2;
    int64_t kp2 = 8;
    st = setup_kmajor(c->mA, c->sA, c->kalt, c->freeA, c->ext, c->M, c->dtype, &kp2, &a2);
    if (st == TTC_OK) st = setup_kmajor(c->mB, c->sB, c->kalt, c->freeB, c->ext, c->N, c->dtype, &kp2, &b2);
    if (st == TTC_OK) st = ttc_plan_autotune(a2.plan, max_candidates, stream, &ta2);
    if (st == TTC_OK) st = ttc_plan_autotune(b2.plan, max_candidates, stream, &tb2);
    if (st == TTC_OK && ta2 + tb2 < 0.98f * (ta + tb)) {
      std::swap(c->opA, a2);
      std::swap(c->opB, b2);
      c->kpitch = kp2;
    }
    if (a2.plan) ttc_plan_destroy(a2.plan);
    if (b2.plan) ttc_plan_destroy(b2.plan);
    if (st != TTC_OK) return st;
    c->kalt.clear();   // decided
    if (c->planC) return ttc_plan_autotune(c->planC, max_candidates, stream, nullptr);
    return TTC_OK;
  }
  for (ttc_plan_t p : {c->opA.plan, c->opB.plan, c->planC}) {
    if (!p) continue;
    const ttc_status st = ttc_plan_autotune(p, max_candidates, stream, nullptr);
    if (st != TTC_OK) return st;
  }
  return TTC_OK;
}

ttc_status ttc_contraction_check(ttc_contraction_t c) {
  if (!c) return fail(TTC_ERR_INVALID_ARG, "contraction is NULL");
  std::lock_guard<std::mutex> lk(c->mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  auto it = c->dev.find(dev);
  if (it == c->dev.end() || !it->second.err) return TTC_OK;
  int flag = 0;
  e = cudaMemcpy(&flag, it->second.err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "error word read");
  if (!flag) return TTC_OK;
  if (flag == 2)   // sticky: not reset
    return fail(TTC_ERR_TIMEOUT, "a CTA released its tensor memory with MMAs possibly still in flight: tensor-core "
                                 "results on this device are unreliable from then on");
  e = cudaMemset(it->second.err, 0, sizeof(int));      // reported once
  if (e != cudaSuccess) return cuda_fail(e, "error word reset");
  return fail(TTC_ERR_TIMEOUT, "a tensor-core wait of the GEMM gave up");
}

ttc_status ttc_debug_contraction_use_cublas(ttc_contraction_t c, int use) {
  if (!c) return fail(TTC_ERR_INVALID_ARG, "contraction is NULL");
  std::lock_guard<std::mutex> lk(c->mu);
  c->use_cublas = use != 0;
  return TTC_OK;
}

ttc_status ttc_debug_contraction_gemm_variant(ttc_contraction_t c, int variant, int* last_used) {
  if (!c) return fail(TTC_ERR_INVALID_ARG, "contraction is NULL");
  if (variant > 6) return fail(TTC_ERR_INVALID_ARG, "variant must be -1..6");
  std::lock_guard<std::mutex> lk(c->mu);
  if (variant >= 0) c->gemm_variant = variant;
  if (last_used) *last_used = c->gemm_used;
  return TTC_OK;
}

ttc_status ttc_contraction_destroy(ttc_contraction_t c) {
  if (!c) return fail(TTC_ERR_INVALID_ARG, "contraction is NULL");
  delete c;
  return TTC_OK;
}

}  // extern "C"
