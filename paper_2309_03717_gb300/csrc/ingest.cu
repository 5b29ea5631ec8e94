// ingest.cu -- ingest of one shower's contiguous track arrays.
#include "ingest.cuh"

namespace c8r {

size_t tile_bytes(int precision) { return precision == C8R_FP64 ? kTileBytesF64 : kTileBytesMixed; }

cudaError_t launch_ingest(int precision, const TrackPtrs& t, int64_t n, void* tiles, const MedParams& M,
                          unsigned long long* kept, cudaStream_t st, unsigned long long* form) {
  if (n <= 0) return cudaSuccess;
  const int64_t n_pad = (n + kTileT - 1) / kTileT * kTileT;
  return launch_ingest_map(precision, t, ingest_detail::IdentityMap{n}, n_pad, tiles, M, kept, st, form);
}

}  // namespace c8r
