// kernels_pair.cuh -- instantiates the kernels of one (dtype_in, dtype_out)
// pair; each kern_<in>_<out>.cu defines TTC_DIN, TTC_DOUT and TTC_PAIR and
// includes this file, so that the pairs compile in parallel.
#include "kernels_impl.cuh"

#define TTC_CAT2(a, b) a##b
#define TTC_CAT(a, b) TTC_CAT2(a, b)

namespace ttc {

cudaError_t TTC_CAT(launch_tile_, TTC_PAIR)(const void* A, void* B, const TileParams& p, int smem, cudaStream_t s) {
  return with_ek<TTC_DIN, TTC_DOUT, TileL<TTC_DIN, TTC_DOUT>::template L>(p.epi.mode, p.epi.beta_nz, A, B, p, smem, s);
}

cudaError_t TTC_CAT(launch_tile_slots_, TTC_PAIR)(const void* A, void* B, const TileParams& p, int smem,
                                                  cudaStream_t s) {
  return with_ek<TTC_DIN, TTC_DOUT, TileSlotsL<TTC_DIN, TTC_DOUT>::template L>(p.epi.mode, p.epi.beta_nz, A, B, p, smem,
                                                                              s);
}

cudaError_t TTC_CAT(launch_tile2_, TTC_PAIR)(int ju, int jw, const void* A, void* B, const TileParams& p, int smem,
                                             cudaStream_t s) {
  return launch_tile2_pair<TTC_DIN, TTC_DOUT>(ju, jw, A, B, p, smem, s);
}

cudaError_t TTC_CAT(launch_tilep_, TTC_PAIR)(int nt, int ju, int jw, const void* A, void* B, const TileParams& p,
                                             int smem, cudaStream_t s) {
  return launch_tilep_pair<TTC_DIN, TTC_DOUT>(nt, ju, jw, A, B, p, smem, s);
}

cudaError_t TTC_CAT(launch_rowsp_, TTC_PAIR)(int j, const void* A, void* B, const TileParams& p, cudaStream_t s) {
  return launch_rowsp_pair<TTC_DIN, TTC_DOUT>(j, A, B, p, s);
}

cudaError_t TTC_CAT(launch_rowcopy_, TTC_PAIR)(const void* A, void* B, const TileParams& p, cudaStream_t s) {
  return with_ek<TTC_DIN, TTC_DOUT, RowcopyL<TTC_DIN, TTC_DOUT>::template L>(p.epi.mode, p.epi.beta_nz, A, B, p, s);
}

cudaError_t TTC_CAT(launch_copy_, TTC_PAIR)(int vec, const void* A, void* B, const RowParams& p, cudaStream_t s) {
  constexpr int W = (dtype_size(TTC_DIN) > dtype_size(TTC_DOUT) ? 16 / dtype_size(TTC_DIN) : 16 / dtype_size(TTC_DOUT));
  if (vec == W)
    return with_ek<TTC_DIN, TTC_DOUT, CopyL<TTC_DIN, TTC_DOUT, W>::template L>(p.epi.mode, p.epi.beta_nz, A, B, p, s);
  return with_ek<TTC_DIN, TTC_DOUT, CopyL<TTC_DIN, TTC_DOUT, 1>::template L>(p.epi.mode, p.epi.beta_nz, A, B, p, s);
}

}  // namespace ttc
