// plan_impl.h -- the plan object behind the opaque ttc_plan_t handle.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ttc.h"
#include "planner.h"
#include "ttc_internal.h"

namespace ttc {

// Device-side resources of a plan on one device: a small scratch area (FP8
// amax word and scale) and the cross-offset tables of the selected schedule.
struct DevRes {
  void* base = nullptr;
  size_t bytes = 0;
  uint32_t* amax = nullptr;   // two words: executions alternate between them
  int amax_phase = 0;         // the word the next execution accumulates into
  float* scale = nullptr;
  int32_t* tables = nullptr;
  int4* slots = nullptr;     // slot tables of tile_kernel (when a candidate uses them)
  int sel = -1;          // candidate the parameters below were built for
  TileParams tp;
  RowParams rp;
  int smem = 0;
};

struct BatchTemplate;   // the plan's description for the batch body (batch_impl.h)

}  // namespace ttc

struct ttc_plan_s {
  std::mutex mu;
  // the problem as given (for the schedule checker)
  int ndim = 0;
  int perm0[ttc::kMaxDim] = {};
  int64_t sizes0[ttc::kMaxDim] = {}, outerA0[ttc::kMaxDim] = {}, outerB0[ttc::kMaxDim] = {};
  int din = 0, dout = 0;
  double alpha = 1.0, beta = 0.0;
  double alpha_im = 0.0, beta_im = 0.0;   // imaginary parts (complex dtypes only)
  bool beta_nonzero() const { return beta != 0.0 || beta_im != 0.0; }
  ttc::Canon canon;
  std::vector<ttc::Candidate> cands;
  int sel = 0;
  bool user_selected = false;
  const float* user_scale = nullptr;
  ttc::RowParams amax_rows;
  std::map<int, ttc::DevRes> dev;
  // computed on first use by batch_describe, then shared by every batch and
  // server request of this plan
  std::mutex batch_mu;
  std::shared_ptr<const ttc::BatchTemplate> batch_tmpl;
};

namespace ttc {
ttc_status fail(ttc_status s, const std::string& msg);
ttc_status cuda_fail(cudaError_t e, const char* where);
ttc_status run_plan(ttc_plan_s* p, const void* A, void* B, cudaStream_t s);
ttc_status ensure_device(ttc_plan_s* p, int dev, DevRes** out);
int remembered_choice(const ttc_plan_s* p, int dev);
Epilogue make_epilogue(const ttc_plan_s* p, const DevRes* r);
std::string plan_key(const ttc_plan_s* p, int dev);
}  // namespace ttc
