// planner.h -- host-side planning of one permute-scale-add (Eq. 1).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "ttc_internal.h"

namespace ttc {

// The problem after validation, dropping of size-1 indices and merging of
// neighbouring indices into super-indices (section 2.1 stage 1, footnote 5).
struct Canon {
  int N = 0;                 // 0 when the problem is empty (some size is 0)
  int64_t s[kMaxDim] = {};   // sizes, A order
  int64_t sa[kMaxDim] = {};  // element strides in A
  int64_t sb[kMaxDim] = {};  // element strides in B of the same (A-ordered) index
  int perm[kMaxDim] = {};    // perm[d] = A index at B position d
  int64_t n = 0;             // elements
  int64_t spanA = 0;         // 1 + largest element offset touched in A (0 if empty)
  int64_t spanB = 0;
};

enum Variant : int { VAR_EMPTY = 0, VAR_COPY = 1, VAR_TILE = 2, VAR_TMA = 3 };   // VAR_TMA: tma2d.h

// One schedule the planner considers (a "candidate" in the paper's sense,
// section 2.2: tile extents and the order of the flat grid).
struct Candidate {
  int variant = VAR_EMPTY;
  // tile variant: groups of the tile
  int has_c = 0;               // index 0 is the shared run C
  std::vector<int> ga;         // A indices of GA, in A order (last one may be cut)
  int ta = 1;                  // tile extent of GA's last index
  std::vector<int> gb;         // A indices of GB, in B order (last one may be cut)
  int tb = 1;                  // tile extent of GB's last index
  std::vector<int> order;      // grid indices (A index ids), fastest first
  int ju = 0, jw = 0;          // >0: warp-mapped tile kernel with JU/JW chunks of 32 lanes
  int rows = 0;                // multi-row copy kernel (perm keeps index 0, GB empty, no staging)
  int slots = 0;               // tile_kernel from precomputed slot tables (whole tiles)
  int pk = 0;                  // >0: packed-lane tile kernel with pk (256 or 512) threads per CTA
  int swz = 0;                 // grouped grid order (TileParams::swz), 0: plain
  int rj = 0;                  // >0: packed rows (C tiles copied row by row), rj positions per thread and row
  int kt = 0;                  // packed kernels: slots per thread their layouts assume (0: the single-plan kernels')
  // copy variant
  int64_t chunk = 0;
  int vec = 1;                 // vector width usable when pointers are aligned
  // model
  double est_s = 0;            // estimated seconds per execution
  double seg_a = 0, seg_b = 0; // contiguous run lengths (elements) on each side
  std::string describe() const;
};

// Validation + canonicalisation.  Returns 0 (TTC_OK) or a ttc_status code
// with a message in *err.
int canonicalize(int ndim, const int* perm, const int64_t* sizes, const int64_t* outerA,
                 const int64_t* outerB, Canon* c, std::string* err);

// Candidate schedules, best estimate first (at most max_keep).
// vmax > 0: schedules of the batch body instead (tiles of at most vmax
// elements, vmax / 256 slots per thread: packed-lane tiles, packed rows and
// run chunks only).
std::vector<Candidate> make_candidates(const Canon& c, int din, int dout, double beta, int max_keep, int vmax = 0);

// Kernel parameters of a candidate.  Host tables (crossA, crossB) are
// returned in tabA/tabB; the device pointers are filled in by the caller.
void build_tile_params(const Canon& c, const Candidate& k, int din, TileParams* p,
                       std::vector<int32_t>* tabA, std::vector<int32_t>* tabB, int* smem_bytes);
void build_row_params(const Canon& c, int64_t chunk, RowParams* p);
// Rows of the FP8 amax pre-pass over A's (sub-)tensor: A-dense neighbours
// merged regardless of B (only A offsets are meaningful), with the width
// of its 16-byte loads (elem_bytes: the size of an A element).
void build_amax_rows(const Canon& c, int elem_bytes, RowParams* p);

// Slot tables of a tile for tile_slots_kernel (layout: TileParams::slots);
// `tabA`/`tabB` are the host cross tables of the same parameters.  Returns
// the shared-memory bytes of the tile in the kernel's layout.
int build_slot_tables(const TileParams& p, int din, const std::vector<int32_t>& tabA,
                      const std::vector<int32_t>& tabB, std::vector<int32_t>* out);
size_t slot_table_ints(int din);

// Estimated memory efficiency of reading (write = false) or writing a
// contiguous run of `bytes` bytes that starts at an arbitrary element offset,
// for the single-plan kernels or (flat = true) the batch body.
double run_efficiency(double bytes, bool write, bool flat = false);

}  // namespace ttc
