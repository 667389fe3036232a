// Loading a YET in pieces: the launcher that chunks one range of trials, so
// that the trials whose ids have arrived are chunked while the ids of later
// trials are still being copied from the host.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace ara {

// Number of pieces a host-to-device id copy is split into (the last piece's
// chunking is the only part not hidden behind the copy).
constexpr int kLoadPieces = 8;
// Smallest piece worth its own copy and launch: 2^24 ids (64 MB).
constexpr int kLoadPieceShift = 24;

// Chunk trials [t0, t1) of the YET (the layout of launch_pad_ids: off/coff
// are the full raw and chunk offset arrays, ids are read from src[off[t]]);
// last = true also writes the sentinel tail after chunk coff[t1], so it is
// given only with t1 = n_trials.  Out-of-catalog ids add to *bad_count.
cudaError_t launch_pad_ids_range(const int32_t *src, const int64_t *off, const int64_t *coff,
                                 int64_t t0, int64_t t1, bool last, int4 *dst, int32_t catalog,
                                 bool packed, unsigned long long *bad_count, cudaStream_t s);

}  // namespace ara
