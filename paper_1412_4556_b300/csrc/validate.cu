// Device-side ingest of a freshly copied YET: every event id must lie in the
// catalog (Section III: ids are drawn from the catalogue of events), and
// time-stamps, when given, must be finite and ascending within each trial
// (Section III: each trial is ordered by ascending time-stamp).  Violations
// are counted; the host turns a nonzero count into a status code, so a bad
// input never reaches a kernel that would index with it.
#include "ara_internal.cuh"

namespace ara {

// One warp per trial: position i of trial t is checked against i + 1.
__global__ void check_ts_kernel(const int64_t *__restrict__ offsets, int64_t n_trials,
                                const float *__restrict__ ts, unsigned long long *bad) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long local = 0;
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < n_trials;
       t += warps) {
    const int64_t s = offsets[t], e = offsets[t + 1];
    for (int64_t i = s + lane; i < e; i += 32) {
      const float a = ts[i];
      bool ok = isfinite(a);
      if (i + 1 < e) ok = ok && (a <= ts[i + 1]);
      local += ok ? 0ull : 1ull;
    }
  }
  for (int m = 16; m > 0; m >>= 1) local += __shfl_xor_sync(0xFFFFFFFFu, local, m);
  if (lane == 0 && local) atomicAdd(bad, local);
}

// Copy the YET ids into the engine's padded layout: trial t occupies
// dst[poff[t] .. poff[t+1]), a multiple of 4 positions, so every 16-byte
// chunk of dst belongs to exactly one trial; the gap after the trial's
// events and the 16 positions after the last trial hold the sentinel id
// (= catalog size, whose table entry is zero).  Ids outside the catalog are
// counted (and replaced by the sentinel, so no later kernel indexes with
// them).  One warp per trial.
__global__ void pad_ids_kernel(const int32_t *__restrict__ src, const int64_t *__restrict__ off,
                               const int64_t *__restrict__ poff, int64_t n_trials,
                               int32_t *__restrict__ dst, int32_t catalog,
                               unsigned long long *bad) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t w0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  unsigned long long local = 0;
  for (int64_t t = w0; t < n_trials; t += warps) {
    const int64_t s = off[t], n = off[t + 1] - s;
    const int64_t d = poff[t], dn = poff[t + 1] - d;
    for (int64_t i = lane; i < dn; i += 32) {
      int32_t v = catalog;
      if (i < n) {
        v = src[s + i];
        if (v < 0 || v >= catalog) {
          ++local;
          v = catalog;
        }
      }
      dst[d + i] = v;
    }
  }
  if (w0 == 0 && lane < 16) dst[poff[n_trials] + lane] = catalog;
  for (int m = 16; m > 0; m >>= 1) local += __shfl_xor_sync(0xFFFFFFFFu, local, m);
  if (lane == 0 && local) atomicAdd(bad, local);
}

cudaError_t launch_pad_ids(const int32_t *src, const int64_t *off, const int64_t *poff,
                           int64_t n_trials, int32_t *dst, int32_t catalog,
                           unsigned long long *bad_count, cudaStream_t s) {
  int64_t blocks = (n_trials + 7) / 8;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  pad_ids_kernel<<<(int)blocks, 256, 0, s>>>(src, off, poff, n_trials, dst, catalog, bad_count);
  return cudaGetLastError();
}

cudaError_t launch_check_ts(const int64_t *offsets, int64_t n_trials, const float *ts,
                            unsigned long long *bad_count, cudaStream_t s) {
  if (n_trials <= 0) return cudaSuccess;
  int64_t blocks = (n_trials + 7) / 8;
  if (blocks > 148 * 8) blocks = 148 * 8;
  check_ts_kernel<<<(int)blocks, 256, 0, s>>>(offsets, n_trials, ts, bad_count);
  return cudaGetLastError();
}

}  // namespace ara
