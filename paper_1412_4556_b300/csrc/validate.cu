// Device-side ingest of a freshly copied YET: every event id must lie in the
// catalog (Section III: a trial's events come from the event catalogue), and
// time-stamps, when given, must be finite and nondecreasing within each
// trial (Section III: a trial lists its events in time order).  Violations
// are counted; the host turns a nonzero count into a status code, so a bad
// input never reaches a kernel that would index with it.
#include "ara_internal.cuh"
#include "yet_load.cuh"

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

// Copy the YET ids into the engine's chunked layout.  Trial t occupies the
// 16-byte chunks [coff[t], coff[t+1]); a chunk holds 4 plain 32-bit ids, or,
// when every id and the sentinel fit in 21 bits, 6 ids packed as
// id0 | id1 << 21 | id2 << 42 in each 64-bit half.  The positions after a
// trial's last event and the kChunkTail chunks after the last trial hold the
// sentinel id (= catalog size, whose table entry is zero), so every chunk
// belongs to exactly one trial.  Ids outside the catalog are counted and
// replaced by the sentinel, so no later kernel indexes with them.  One warp
// per trial, one chunk per lane; one launch covers the trials [t0, t1), and
// the launch of the last range also writes the tail.
__device__ __forceinline__ int32_t ingest_id(const int32_t *src, int64_t i, int64_t n,
                                             int32_t catalog, unsigned long long &bad) {
  if (i >= n) return catalog;
  const int32_t v = src[i];
  if (v < 0 || v >= catalog) {
    ++bad;
    return catalog;
  }
  return v;
}

template <bool PACKED>
__global__ void pad_ids_kernel(const int32_t *__restrict__ src, const int64_t *__restrict__ off,
                               const int64_t *__restrict__ coff, int64_t t0, int64_t t1,
                               bool write_tail, int4 *__restrict__ dst, int32_t catalog,
                               unsigned long long *bad_count) {
  constexpr int IPC = PACKED ? 6 : 4;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t w0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  unsigned long long bad = 0;
  for (int64_t t = t0 + w0; t < t1; t += warps) {
    const int64_t s = off[t], n = off[t + 1] - s;
    const int64_t c0 = coff[t], nc = coff[t + 1] - c0;
    for (int64_t j = lane; j < nc; j += 32) {
      int32_t v[IPC];
#pragma unroll
      for (int k = 0; k < IPC; ++k) v[k] = ingest_id(src + s, j * IPC + k, n, catalog, bad);
      dst[c0 + j] = PACKED ? pack6(v) : make_int4(v[0], v[1], v[2], v[3]);
    }
  }
  if (write_tail && w0 == 0 && lane < kChunkTail) {
    int32_t v[6] = {catalog, catalog, catalog, catalog, catalog, catalog};
    dst[coff[t1] + lane] = PACKED ? pack6(v) : make_int4(catalog, catalog, catalog, catalog);
  }
  for (int m = 16; m > 0; m >>= 1) bad += __shfl_xor_sync(0xFFFFFFFFu, bad, m);
  if (lane == 0 && bad) atomicAdd(bad_count, bad);
}

cudaError_t launch_pad_ids_range(const int32_t *src, const int64_t *off, const int64_t *coff,
                                 int64_t t0, int64_t t1, bool last, int4 *dst, int32_t catalog,
                                 bool packed, unsigned long long *bad_count, cudaStream_t s) {
  int64_t blocks = (t1 - t0 + 7) / 8;
  if (blocks > (int64_t)current_sm_count() * 16) blocks = (int64_t)current_sm_count() * 16;
  if (blocks < 1) blocks = 1;
  if (packed)
    pad_ids_kernel<true><<<(int)blocks, 256, 0, s>>>(src, off, coff, t0, t1, last, dst, catalog, bad_count);
  else
    pad_ids_kernel<false><<<(int)blocks, 256, 0, s>>>(src, off, coff, t0, t1, last, dst, catalog, bad_count);
  return cudaGetLastError();
}

cudaError_t launch_pad_ids(const int32_t *src, const int64_t *off, const int64_t *coff,
                           int64_t n_trials, int4 *dst, int32_t catalog, bool packed,
                           unsigned long long *bad_count, cudaStream_t s) {
  return launch_pad_ids_range(src, off, coff, 0, n_trials, true, dst, catalog, packed, bad_count, s);
}

cudaError_t launch_check_ts(const int64_t *offsets, int64_t n_trials, const float *ts,
                            unsigned long long *bad_count, cudaStream_t s) {
  if (n_trials <= 0) return cudaSuccess;
  int64_t blocks = (n_trials + 7) / 8;
  if (blocks > (int64_t)current_sm_count() * 8) blocks = (int64_t)current_sm_count() * 8;
  check_ts_kernel<<<(int)blocks, 256, 0, s>>>(offsets, n_trials, ts, bad_count);
  return cudaGetLastError();
}

}  // namespace ara
