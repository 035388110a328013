// batch_impl.h -- descriptors of the batched launch, shared by the batch API
// (batch.cu) and the server (server.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "plan_impl.h"
#include "ttc_internal.h"

namespace ttc {

// BP_TILE: packed-lane tile (no C index); BP_ROWS: packed rows (C tiles,
// no staging); BP_COPY: chunks of long runs
enum BatchPath : int { BP_TILE = 0, BP_ROWS = 1, BP_COPY = 2 };

struct alignas(16) BatchDesc {
  const void* A;
  void* B;
  int din, dout, path;
  int j;             // BP_TILE: run chunks per thread on both sides (1 or 2); BP_ROWS: positions per row (1 or K)
  int beta_nz;       // B is read
  uint32_t tile0;    // first global tile of this problem
  uint32_t ntiles;
  int pad;
  TileParams tp;     // BP_TILE, BP_ROWS
  RowParams rp;      // BP_COPY
};

constexpr int kBatchCopyChunk = 2048;   // elements of a run per BP_COPY tile

// elements per thread per phase in the batch body: half of the single-plan
// kernels' (tiles of at most 2048 four-byte or 1024 eight-byte elements): the
// body reads its problem's parameters from global memory into registers,
// which full tiles would spill
constexpr int batch_k_for(int stage_bytes) { return tile_k_for(stage_bytes) / 2; }

// Where one tile of the batch lies, precomputed on the host so that a CTA
// needs one load to start on a claimed tile.  For BP_COPY: baseA/baseB are
// the run's offsets, remA the first element of the chunk, remB its length.
struct TileRec {
  uint32_t prob;
  int32_t remA, remB, pad;
  int64_t baseA, baseB;
};


// What batch_describe derives from the plan alone, kept in the plan.
struct BatchTemplate {
  bool ok = false;
  BatchDesc d;
  std::vector<int32_t> tabs;
  size_t tabA_count = 0;
  int smem = 0;
};

// The descriptor of one problem for the batch body (path, tile parameters or
// run chunks, epilogue).  Offset tables are appended to *tabs (crossA then
// crossB); their device address is filled in when the arena is laid out.
// Returns false for problems the batch body cannot take (FP8 output, empty).
bool batch_describe(ttc_plan_s* p, const void* A, void* B, BatchDesc* d, std::vector<int32_t>* tabs,
                    size_t* tabA_count, int* smem);

// Tiles of the plan in the batch body, or -1 if the body cannot take it.
int64_t batch_tiles(ttc_plan_s* p);

// Append the records of every tile of problem `prob` to *recs.
void batch_records(const BatchDesc& d, uint32_t prob, std::vector<TileRec>* recs);

// The problems of one class (dtype pair, beta zero or not, body and its
// chunk count), consecutive in the descriptor array, and their tiles
// [first, first + count).
struct BatchRange {
  int cls, din, dout, bnz, path, j;
  uint32_t first, count;
};

// The class key of a problem, by which a batch orders its problems.
int batch_class(const BatchDesc& d);

// The class ranges of descriptors already ordered by class (tile0 set).
void batch_ranges(const std::vector<BatchDesc>& descs, std::vector<BatchRange>* ranges);

// Enqueue the batch kernels, one launch per class range, one CTA per tile.
// With d_recs null each kernel derives its tiles' records on the device from
// d_tile0 (the first global tile of each of the nprob problems, ascending).
cudaError_t batch_launch(const BatchDesc* d_descs, const TileRec* d_recs, const uint32_t* d_tile0, uint32_t nprob,
                         const std::vector<BatchRange>& ranges, int smem, cudaStream_t s);

}  // namespace ttc
