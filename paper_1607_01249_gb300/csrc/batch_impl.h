// batch_impl.h -- descriptors of the batched launch, shared by the batch API
// (batch.cu) and the server (server.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "plan_impl.h"
#include "ttc_internal.h"

namespace ttc {

enum BatchPath : int { BP_TILE = 0, BP_ROWS = 1, BP_COPY = 2 };

struct alignas(16) BatchDesc {
  const void* A;
  void* B;
  int din, dout, path, pad;
  uint32_t tile0;    // first global tile of this problem
  uint32_t ntiles;
  TileParams tp;     // BP_TILE, BP_ROWS
  RowParams rp;      // BP_COPY
};

constexpr int kBatchCopyChunk = 2048;   // elements of a run per BP_COPY tile

// elements per thread per phase in the batch body: half of the single-plan
// kernels' (tiles of at most 2048 four-byte or 1024 eight-byte elements), so
// that the descriptor fields fit in registers next to the staged data
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

// Enqueue the counter reset and the persistent kernel (grid from occupancy).
// With d_recs null the kernel derives each tile's record on the device from
// d_tile0 (the first global tile of each of the nprob problems, ascending).
cudaError_t batch_launch(const BatchDesc* d_descs, const TileRec* d_recs, const uint32_t* d_tile0, uint32_t nprob,
                         uint32_t total, uint32_t* d_counter, int smem, cudaStream_t s);

}  // namespace ttc
