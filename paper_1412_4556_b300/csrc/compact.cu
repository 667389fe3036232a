// Compact id stream for repeated pricing.
//
// A trial's loss (Algorithm 1, Section III) does not depend on the order of
// its events: the engine sums exactly, so any order gives the same bits.  For
// YLT passes the ids of each trial can therefore be stored sorted and coded as
// differences: a 16-byte chunk then holds 8 ids (a 21-bit base and seven
// 15-bit steps) instead of 6 -- 2.0 bytes per id instead of 2.67 -- and the id
// stream, which every pass reads from HBM, shrinks by a quarter.  Trials that
// do not fit (more than kCompactMaxTrial events, or a step of 2^15 - 1 or more
// between sorted neighbours, as in short trials over a large catalog) keep
// the 6-per-chunk absolute layout; a flag in bit 62 of the trial's chunk
// offset tells the kernel which.  The stored-order layout stays for the Year
// Event Loss Table, whose entries follow the stored (time) order.
//
// Chunk layout (two 64-bit halves lo, hi):
//   lo = base | d1 << 21 | d2 << 36 | (d3 & 0x1FFF) << 51
//   hi = d3 >> 13 | d4 << 2 | d5 << 17 | d6 << 32 | d7 << 47
// id_k = id_{k-1} + d_k; a step of 0x7FFF marks an empty slot (the rest of the
// trial's last chunk).
#include "ara_internal.cuh"

namespace ara {

namespace {

constexpr int kSortThreads = 256;

__device__ __forceinline__ void unpack6(int4 c, uint32_t (&id)[6]) {
  constexpr uint32_t M = 0x1FFFFFu;
  id[0] = (uint32_t)c.x & M;
  id[1] = __funnelshift_r((uint32_t)c.x, (uint32_t)c.y, 21) & M;
  id[2] = ((uint32_t)c.y >> 10) & M;
  id[3] = (uint32_t)c.z & M;
  id[4] = __funnelshift_r((uint32_t)c.z, (uint32_t)c.w, 21) & M;
  id[5] = ((uint32_t)c.w >> 10) & M;
}

// Sort each trial's ids (stored in the 6-per-chunk layout) in shared memory,
// write them to sorted[raw_off[t] ..], and decide the trial's layout:
// count_flag[t] = chunk count | (1 << 62 when the difference layout fits).
__global__ void __launch_bounds__(kSortThreads)
compact_sort_kernel(const int64_t *__restrict__ raw_off, const int64_t *__restrict__ coff,
                    const int4 *__restrict__ chunks, int64_t n_trials, uint32_t *__restrict__ sorted,
                    int64_t *__restrict__ count_flag) {
  __shared__ uint32_t s[kCompactMaxTrial];
  __shared__ int s_ok;
  const int64_t t = blockIdx.x;
  if (t >= n_trials) return;
  const int tid = threadIdx.x;
  const int64_t n = raw_off[t + 1] - raw_off[t];
  const int64_t c0 = coff[t], nc = coff[t + 1] - c0;
  if (n == 0 || n > kCompactMaxTrial) {
    if (tid == 0) count_flag[t] = nc;
    return;
  }
  int P = 2;
  while (P < n) P <<= 1;
  for (int64_t j = tid; j < nc; j += blockDim.x) {
    uint32_t id[6];
    unpack6(chunks[c0 + j], id);
#pragma unroll
    for (int i = 0; i < 6; ++i)
      if (j * 6 + i < n) s[j * 6 + i] = id[i];
  }
  for (int i = (int)n + tid; i < P; i += blockDim.x) s[i] = 0xFFFFFFFFu;
  if (tid == 0) s_ok = 1;
  __syncthreads();
  // bitonic sort, ascending
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < P; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const uint32_t a = s[i], b = s[ixj];
          if ((a > b) == ((i & k) == 0)) {
            s[i] = b;
            s[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  uint32_t *out = sorted + raw_off[t];
  bool ok = true;
  for (int i = tid; i < n; i += blockDim.x) {
    out[i] = s[i];
    if ((i & 7) != 0 && s[i] - s[i - 1] >= 0x7FFFu) ok = false;
  }
  if (!ok) s_ok = 0;
  __syncthreads();
  if (tid == 0) count_flag[t] = s_ok ? (((n + 7) / 8) | ((int64_t)1 << 62)) : nc;
}

// One warp per trial: write the trial's chunks at dcoff[t] (flag stripped).
__global__ void compact_encode_kernel(const int64_t *__restrict__ raw_off, const int64_t *__restrict__ coff,
                                      const int4 *__restrict__ chunks, int64_t n_trials,
                                      const uint32_t *__restrict__ sorted, const int64_t *__restrict__ dcoff,
                                      int4 *__restrict__ dchunks) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < n_trials; t += warps) {
    const int64_t d0 = dcoff[t] & kCompactOffsetMask;
    const int64_t d1 = dcoff[t + 1] & kCompactOffsetMask;
    if ((dcoff[t] >> 62) & 1) {
      const int64_t n = raw_off[t + 1] - raw_off[t];
      const uint32_t *src = sorted + raw_off[t];
      for (int64_t g = lane; g < d1 - d0; g += 32) {
        uint32_t v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = g * 8 + k < n ? src[g * 8 + k] : 0u;
        unsigned long long d[8];
#pragma unroll
        for (int k = 1; k < 8; ++k) d[k] = g * 8 + k < n ? (unsigned long long)(v[k] - v[k - 1]) : 0x7FFFull;
        const unsigned long long lo = (unsigned long long)v[0] | (d[1] << 21) | (d[2] << 36) | ((d[3] & 0x1FFFull) << 51);
        const unsigned long long hi = (d[3] >> 13) | (d[4] << 2) | (d[5] << 17) | (d[6] << 32) | (d[7] << 47);
        dchunks[d0 + g] = make_int4((int)(uint32_t)lo, (int)(uint32_t)(lo >> 32), (int)(uint32_t)hi,
                                    (int)(uint32_t)(hi >> 32));
      }
    } else {
      const int64_t c0 = coff[t];
      for (int64_t j = lane; j < d1 - d0; j += 32) dchunks[d0 + j] = chunks[c0 + j];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < kChunkTail) {
    const int64_t end = dcoff[n_trials] & kCompactOffsetMask;
    dchunks[end + threadIdx.x] = make_int4(0, 0, 0, 0);  // never read as ids (every load is bounded)
  }
}

}  // namespace

int4 delta_sentinel_chunk(int32_t sentinel) {
  const unsigned long long e = 0x7FFFull;
  const unsigned long long lo = (unsigned long long)(uint32_t)sentinel | (e << 21) | (e << 36) | ((e & 0x1FFFull) << 51);
  const unsigned long long hi = (e >> 13) | (e << 2) | (e << 17) | (e << 32) | (e << 47);
  return make_int4((int)(uint32_t)lo, (int)(uint32_t)(lo >> 32), (int)(uint32_t)hi, (int)(uint32_t)(hi >> 32));
}

cudaError_t launch_compact_sort(const int64_t *raw_off, const int64_t *coff, const int4 *chunks, int64_t n_trials,
                                uint32_t *sorted, int64_t *count_flag, cudaStream_t s) {
  if (n_trials <= 0) return cudaSuccess;
  for (int64_t first = 0; first < n_trials; first += (int64_t)1 << 30) {
    const int64_t n = n_trials - first < ((int64_t)1 << 30) ? n_trials - first : ((int64_t)1 << 30);
    compact_sort_kernel<<<(unsigned)n, kSortThreads, 0, s>>>(raw_off + first, coff + first, chunks, n, sorted,
                                                             count_flag + first);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_compact_encode(const int64_t *raw_off, const int64_t *coff, const int4 *chunks, int64_t n_trials,
                                  const uint32_t *sorted, const int64_t *dcoff, int4 *dchunks, cudaStream_t s) {
  compact_encode_kernel<<<148 * 8, 256, 0, s>>>(raw_off, coff, chunks, n_trials, sorted, dcoff, dchunks);
  return cudaGetLastError();
}

}  // namespace ara
