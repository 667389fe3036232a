// Compact id stream for repeated pricing.
//
// A trial's loss (Algorithm 1, Section III) does not depend on the order of
// its events: the engine sums exactly, so any order gives the same bits.  For
// YLT passes the ids of each trial can therefore be reordered so that each
// chunk's ids ascend in small steps, and coded as differences: a 16-byte chunk
// then holds 8 ids (a 21-bit base and seven 15-bit steps) instead of 6 -- 2.0
// bytes per id instead of 2.67 -- and the id stream, which every pass reads
// from HBM, shrinks by a quarter.  Trials that do not fit (a step of 2^15 - 1
// or more, as in short trials over a large catalog) keep the 6-per-chunk
// absolute layout; a flag in bit 62 of the trial's chunk offset tells the
// kernel which.  The stored-order layout stays for the Year
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

constexpr int kBucketShift = 13;                      // buckets of 8192 ids
constexpr int kBuckets = (1 << 21) >> kBucketShift;  // 256: packed ids are below 2^21
constexpr int kSortWarps = 4;
constexpr int kStage = 1536;                // ids of a trial sorted in shared memory
constexpr int kPad = kStage + kStage / 8;  // group buffer, 9 words a group
constexpr int kWarpWords = kStage + kPad + kBuckets;
constexpr int kSortSmem = kSortWarps * kWarpWords * 4;  // 56,320 bytes
constexpr int kScanBlocks = 1024;

__device__ __forceinline__ void unpack6(int4 c, uint32_t (&id)[6]) {
  constexpr uint32_t M = 0x1FFFFFu;
  id[0] = (uint32_t)c.x & M;
  id[1] = __funnelshift_r((uint32_t)c.x, (uint32_t)c.y, 21) & M;
  id[2] = ((uint32_t)c.y >> 10) & M;
  id[3] = (uint32_t)c.z & M;
  id[4] = __funnelshift_r((uint32_t)c.z, (uint32_t)c.w, 21) & M;
  id[5] = ((uint32_t)c.w >> 10) & M;
}

// Compare-exchange: a gets the smaller key, b the larger.
__device__ __forceinline__ void order2(uint32_t &a, uint32_t &b) {
  const uint32_t lo = min(a, b), hi = max(a, b);
  a = lo;
  b = hi;
}

// Sorts 8 keys with a 19-comparator network (checked exhaustively against all
// 0/1 inputs, which by the 0-1 principle covers every input).
__device__ __forceinline__ void sort8(uint32_t (&v)[8]) {
  order2(v[0], v[2]); order2(v[1], v[3]); order2(v[4], v[6]); order2(v[5], v[7]);
  order2(v[0], v[4]); order2(v[1], v[5]); order2(v[2], v[6]); order2(v[3], v[7]);
  order2(v[0], v[1]); order2(v[2], v[3]); order2(v[4], v[5]); order2(v[6], v[7]);
  order2(v[2], v[4]); order2(v[3], v[5]);
  order2(v[1], v[4]); order2(v[3], v[6]);
  order2(v[1], v[2]); order2(v[3], v[4]); order2(v[5], v[6]);
}

// Exclusive offsets of the bucket counts in hist (in place); lane l owns
// buckets [8l, 8l + 8).
__device__ __forceinline__ void scan_buckets(uint32_t *hist, int lane) {
  constexpr int PER = kBuckets / 32;
  uint32_t h[PER], own = 0u;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    h[k] = hist[lane * PER + k];
    own += h[k];
  }
  uint32_t incl = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  uint32_t run = incl - own;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    hist[lane * PER + k] = run;
    run += h[k];
  }
}

// Places id (bucket b, or b = ~0 for an idle lane) at its stable position:
// the bucket's next free slot, ranked by lane among the lanes sharing b.  The
// lowest lane of each bucket claims the slots for all of them; atomics on one
// bucket come from one lane per warp-wide step, in step order.  Returns the
// position (undefined for an idle lane).
__device__ __forceinline__ uint32_t bucket_slot(uint32_t *hist, uint32_t b, bool in, unsigned lt) {
  const unsigned peers = __match_any_sync(0xFFFFFFFFu, b);
  const uint32_t rank = (uint32_t)__popc(peers & lt);
  uint32_t at = 0u;
  if (in && rank == 0u) at = atomicAdd(&hist[b], (uint32_t)__popc(peers));
  at = __shfl_sync(0xFFFFFFFFu, at, __ffs((int)peers) - 1);
  return at + rank;
}

// Sorts each group of 8 of the n ids (group g at a[g * STRIDE + k]) and
// returns whether every step inside this lane's groups is below 0x7FFF.
template <int STRIDE>
__device__ __forceinline__ bool sort_groups(uint32_t *a, int64_t n, int lane) {
  bool fits = true;
  const int64_t ng = (n + 7) / 8;
  for (int64_t g = lane; g < ng; g += 32) {
    uint32_t v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = g * 8 + k < n ? a[g * STRIDE + k] : 0xFFFFFFFFu;
    sort8(v);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (g * 8 + k < n) {
        a[g * STRIDE + k] = v[k];
        if (k > 0 && v[k] - v[k - 1] >= 0x7FFFu) fits = false;
      }
    }
  }
  return fits;
}

// One warp per trial.  The difference code needs each group of 8 ids (the
// ids of one chunk) ascending with small steps, not a sorted trial: the ids
// are bucketed by their high bits (buckets of 8192 ids, a stable counting
// sort), then each group of 8 is sorted by a network.  Inside a group, ids of
// one bucket differ by less than 8192 and ids of adjacent buckets by less than
// 16384, so the steps fit 15 bits unless the trial leaves buckets empty, the
// case in which fully sorted neighbours are far apart too.  The result goes
// to sorted[raw_off[t] ..] and count_flag[t] = chunk count | (1 << 62 when
// every step fits).  Trials of up to kStage ids work in shared memory (the
// group buffer padded to 9 words a group, so the group sort reads without
// bank conflicts); longer ones work in place in sorted.  The bucket ranks
// follow a fixed order of the trial's ids, so the result is the same on
// every run.
__global__ void __launch_bounds__(kSortWarps * 32)
compact_sort_kernel(const int64_t *__restrict__ raw_off, const int64_t *__restrict__ coff,
                    const int4 *__restrict__ chunks, int64_t n_trials, uint32_t *sorted,
                    int64_t *__restrict__ count_flag) {
  extern __shared__ uint32_t s_sort[];
  const int lane = threadIdx.x & 31;
  uint32_t *stage = s_sort + (threadIdx.x >> 5) * kWarpWords;
  uint32_t *grp = stage + kStage;
  uint32_t *hist = grp + kPad;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t n_warps = (int64_t)gridDim.x * kSortWarps;
  for (int64_t t = (int64_t)blockIdx.x * kSortWarps + (threadIdx.x >> 5); t < n_trials; t += n_warps) {
    const int64_t r0 = raw_off[t], n = raw_off[t + 1] - r0;
    const int64_t c0 = coff[t], nc = coff[t + 1] - c0;
    if (n == 0) {
      if (lane == 0) count_flag[t] = nc;
      continue;
    }
    const bool staged = n <= kStage;
    for (int b = lane; b < kBuckets; b += 32) hist[b] = 0u;
    __syncwarp();
    for (int64_t j = lane; j < nc; j += 32) {
      uint32_t id[6];
      unpack6(chunks[c0 + j], id);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const int64_t p = j * 6 + i;
        if (p < n) {
          if (staged) stage[p] = id[i];
          atomicAdd(&hist[id[i] >> kBucketShift], 1u);
        }
      }
    }
    __syncwarp();
    scan_buckets(hist, lane);
    __syncwarp();
    uint32_t *out = sorted + r0;
    bool fits;
    if (staged) {
      for (int p0 = 0; p0 < (int)n; p0 += 32) {  // stable order: the stored order
        const int p = p0 + lane;
        const bool in = p < (int)n;
        const uint32_t id = in ? stage[p] : 0u;
        const uint32_t q = bucket_slot(hist, in ? id >> kBucketShift : 0xFFFFFFFFu, in, lt);
        if (in) grp[q + (q >> 3)] = id;
      }
      __syncwarp();
      fits = sort_groups<9>(grp, n, lane);
      __syncwarp();
      for (int p = lane; p < (int)n; p += 32) out[p] = grp[p + (p >> 3)];
    } else {
      for (int64_t jb = 0; jb < nc; jb += 32) {  // stable order: (32 chunks, slot, lane)
        const int64_t j = jb + lane;
        uint32_t id[6] = {0u, 0u, 0u, 0u, 0u, 0u};
        if (j < nc) unpack6(chunks[c0 + j], id);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          const bool in = j < nc && j * 6 + i < n;
          const uint32_t q = bucket_slot(hist, in ? id[i] >> kBucketShift : 0xFFFFFFFFu, in, lt);
          if (in) out[q] = id[i];
        }
      }
      __threadfence_block();
      __syncwarp();
      fits = sort_groups<8>(out, n, lane);
    }
    fits = __all_sync(0xFFFFFFFFu, fits);
    if (lane == 0) count_flag[t] = fits ? (((n + 7) / 8) | ((int64_t)1 << 62)) : nc;
    __syncwarp();  // the buffers are reused for the next trial only after every lane is done
  }
}

// Block b of the scan covers trials [b * per, (b + 1) * per).
__global__ void __launch_bounds__(1024) scan_block_sums_kernel(const int64_t *__restrict__ count_flag, int64_t n,
                                                               int64_t per, int64_t *__restrict__ bsum) {
  __shared__ int64_t s_warp[32];
  const int64_t a = (int64_t)blockIdx.x * per, e = min(a + per, n);
  int64_t own = 0;
  for (int64_t i = a + threadIdx.x; i < e; i += blockDim.x) own += count_flag[i] & kCompactOffsetMask;
  for (int o = 16; o > 0; o >>= 1) own += __shfl_xor_sync(0xFFFFFFFFu, own, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = own;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t sum = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += s_warp[w];
    bsum[blockIdx.x] = sum;
  }
}

// Exclusive scan of nb <= 1024 block sums in place, by one CTA; bsum[nb]
// gets the total.
__global__ void __launch_bounds__(1024) scan_block_offsets_kernel(int64_t *bsum, int nb) {
  __shared__ int64_t s_warp[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t own = tid < nb ? bsum[tid] : 0;
  int64_t incl = own;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  int64_t run = incl - own;
  for (int w = 0; w < wid; ++w) run += s_warp[w];
  __syncthreads();
  if (tid < nb) bsum[tid] = run;
  if (tid == 1023) bsum[nb] = run + own;
}

// Block b scans its trials from offset bsum[b]: dcoff[t] = offset | flag and,
// in place, count_plain[t] = offset; the last block also writes entry n.
__global__ void __launch_bounds__(1024) scan_apply_kernel(int64_t *count_plain, int64_t n, int64_t per,
                                                          const int64_t *__restrict__ bsum, int nb,
                                                          int64_t *__restrict__ dcoff) {
  constexpr int64_t FLAG = (int64_t)1 << 62;
  __shared__ int64_t s_warp[32];
  __shared__ int64_t s_carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t a = (int64_t)blockIdx.x * per, e = min(a + per, n);
  if (tid == 0) s_carry = bsum[blockIdx.x];
  __syncthreads();
  for (int64_t base = a; base < e; base += 1024) {
    const int64_t i = base + tid;
    const int64_t raw = i < e ? count_plain[i] : 0;
    const int64_t v = raw & kCompactOffsetMask;
    int64_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    int64_t run = s_carry + incl - v;
    for (int w = 0; w < wid; ++w) run += s_warp[w];
    if (i < e) {
      dcoff[i] = run | (raw & FLAG);
      count_plain[i] = run;
    }
    __syncthreads();  // every thread has read s_carry and s_warp
    if (tid == 1023) s_carry = run + v;
    __syncthreads();
  }
  if (blockIdx.x == nb - 1 && tid == 0) {
    dcoff[n] = bsum[nb];
    count_plain[n] = bsum[nb];
  }
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
  cudaError_t e = cudaFuncSetAttribute(compact_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortSmem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, compact_sort_kernel, kSortWarps * 32,
                                                         kSortSmem)) != cudaSuccess)
    return e;
  const int64_t want = (n_trials + kSortWarps - 1) / kSortWarps;
  const int64_t resident = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  const int blocks = (int)(want < resident ? want : resident);
  compact_sort_kernel<<<blocks, kSortWarps * 32, kSortSmem, s>>>(raw_off, coff, chunks, n_trials, sorted,
                                                                 count_flag);
  return cudaGetLastError();
}

cudaError_t launch_compact_scan(int64_t *count_plain, int64_t n_trials, int64_t *dcoff, int64_t *bsum,
                                cudaStream_t s) {
  const int64_t per = n_trials > 0 ? (n_trials + kScanBlocks - 1) / kScanBlocks : 1;
  const int nb = n_trials > 0 ? (int)((n_trials + per - 1) / per) : 1;
  scan_block_sums_kernel<<<nb, 1024, 0, s>>>(count_plain, n_trials, per, bsum);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  scan_block_offsets_kernel<<<1, 1024, 0, s>>>(bsum, nb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  scan_apply_kernel<<<nb, 1024, 0, s>>>(count_plain, n_trials, per, bsum, nb, dcoff);
  return cudaGetLastError();
}

cudaError_t launch_compact_encode(const int64_t *raw_off, const int64_t *coff, const int4 *chunks, int64_t n_trials,
                                  const uint32_t *sorted, const int64_t *dcoff, int4 *dchunks, cudaStream_t s) {
  compact_encode_kernel<<<current_sm_count() * 8, 256, 0, s>>>(raw_off, coff, chunks, n_trials, sorted, dcoff, dchunks);
  return cudaGetLastError();
}

}  // namespace ara
