// Device-side checks of a freshly copied YET: every event id must lie in the
// catalog (Section III: ids are drawn from the catalogue of events), and
// time-stamps, when given, must be finite and ascending within each trial
// (Section III: each trial is ordered by ascending time-stamp).  Violations
// are counted; the host turns a nonzero count into a status code, so a bad
// input never reaches a kernel that would index with it.
#include "ara_internal.cuh"

namespace ara {

__global__ void check_ids_kernel(const int32_t *__restrict__ ids, int64_t n, int32_t catalog,
                                 unsigned long long *bad) {
  unsigned long long local = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int32_t v = ids[i];
    local += (v < 0 || v >= catalog) ? 1ull : 0ull;
  }
  for (int m = 16; m > 0; m >>= 1) local += __shfl_xor_sync(0xFFFFFFFFu, local, m);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(bad, local);
}

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

cudaError_t launch_check_ids(const int32_t *ids, int64_t n, int32_t catalog,
                             unsigned long long *bad_count, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  check_ids_kernel<<<(int)blocks, 256, 0, s>>>(ids, n, catalog, bad_count);
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
