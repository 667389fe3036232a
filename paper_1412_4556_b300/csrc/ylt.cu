// The Year Loss Table kernel: Algorithm 1 (Section III), steps 1-4, for every
// trial of the YET, with steps 1-3 already folded into the per-event table.
//
// For trial t with occurrences k = offsets[t] .. offsets[t+1]-1:
//     S_t   = sum_k o(id_k)                  (occurrence-net losses, step 3)
//     YLT_t = min(max(S_t - AggR, 0), AggL)  (aggregate terms, step 4)
// The aggregate clamp applied to the running sum after every event ends at
// the clamp of the final sum (the per-event increments telescope), so one
// clamp per trial gives the trial loss.
//
// B300 design:
//  * One warp per trial; each warp owns a contiguous run of trials, so the
//    YET id stream is read once, in 16-byte coalesced loads, U loads in flight
//    per lane, with an evict-first L2 policy.
//  * The layer's zero-skip bitmap sits in shared memory.  Only occurrences
//    whose bit is set fetch their table entry (a random 16-byte gather served
//    by L2, evict-last); the rest add an exact zero and are skipped.
//  * Table entries are 128-bit fixed-point integers; each lane sums them with
//    add/add-with-carry, and the warp combines lanes with shuffles.  The
//    integer sum is exact, so the result does not depend on the order of
//    the additions or on the launch shape, and B300's low FP64 add rate is
//    kept off the per-occurrence path.  One correctly rounded conversion to
//    binary64 per trial precedes the FP64 aggregate clamp.
#include <cstdlib>

#include "ara_internal.cuh"

namespace ara {

__device__ __forceinline__ unsigned long long policy_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ unsigned long long policy_evict_last() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ int4 ld_ids(const int4 *p, unsigned long long pol) {
  int4 v;
  asm volatile(
      "ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p), "l"(pol));
  return v;
}

__device__ __forceinline__ ulonglong2 ld_entry(const ulonglong2 *p, unsigned long long pol) {
  ulonglong2 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
               : "=l"(v.x), "=l"(v.y)
               : "l"(p), "l"(pol));
  return v;
}

template <int U>
__global__ void __launch_bounds__(kYltThreads, 1)
ylt_fp64_kernel(const int64_t *__restrict__ offsets, const int32_t *__restrict__ ids,
                int64_t n_trials, const ulonglong2 *__restrict__ table,
                const uint4 *__restrict__ bitmap4, int bm_words4, uint32_t bm_add, int bm_shift,
                int q, double agg_ret, double agg_lim, double *__restrict__ ylt) {
  extern __shared__ uint4 s_bm4[];
  for (int i = threadIdx.x; i < bm_words4; i += blockDim.x) s_bm4[i] = bitmap4[i];
  __syncthreads();
  const uint32_t *s_bm = reinterpret_cast<const uint32_t *>(s_bm4);

  const unsigned long long pol_ids = policy_evict_first();
  const unsigned long long pol_tab = policy_evict_last();
  const int lane = threadIdx.x & 31;
  const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t t_begin = n_trials * w / n_warps;
  const int64_t t_end = n_trials * (w + 1) / n_warps;
  const int4 *ids4 = reinterpret_cast<const int4 *>(ids);

  for (int64_t t = t_begin; t < t_end; ++t) {
    const int64_t s = offsets[t];
    const int64_t e = offsets[t + 1];
    const int64_t base = s & ~3ll;              // 16-byte aligned start
    const int32_t lo_r = (int32_t)(s - base);   // first valid position (0..3)
    const int32_t hi_r = (int32_t)(e - base);   // one past the last valid position
    U128 acc{0ull, 0ull};
    for (int32_t c = 4 * lane; c < hi_r; c += 128 * U) {
      int4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int32_t r = c + 128 * u;
        v[u] = (r < hi_r) ? ld_ids(ids4 + ((base + r) >> 2), pol_ids) : make_int4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int32_t r = c + 128 * u;
        const int32_t idv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t id = (uint32_t)idv[i];
          const uint32_t pos = bitmap_pos(id, bm_add, bm_shift);
          const uint32_t word = s_bm[pos >> 5];
          const bool in_trial = (r + i >= lo_r) && (r + i < hi_r);
          if (in_trial && ((word >> (pos & 31)) & 1u)) {
            const ulonglong2 x = ld_entry(table + id, pol_tab);
            add128(acc, x.x, x.y);
          }
        }
      }
    }
    acc = warp_sum_u128(acc);
    if (lane == 0) {
      const double S = from_fixed(acc, q);
      ylt[t] = fmin(fmax(__dsub_rn(S, agg_ret), 0.0), agg_lim);
    }
  }
}

template <int U>
static cudaError_t launch_u(const int64_t *offsets, const int32_t *ids, int64_t n_trials,
                            const ulonglong2 *table, const uint32_t *bitmap, BitmapLayout bm,
                            int q, double agg_ret, double agg_lim, double *ylt,
                            const YltLaunch &cfg, cudaStream_t s) {
  cudaError_t err = cudaFuncSetAttribute(ylt_fp64_kernel<U>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cfg.smem);
  if (err != cudaSuccess) return err;
  ylt_fp64_kernel<U><<<cfg.blocks, cfg.threads, cfg.smem, s>>>(
      offsets, ids, n_trials, table, reinterpret_cast<const uint4 *>(bitmap), bm.words / 4,
      bm.add, bm.shift, q, agg_ret, agg_lim, ylt);
  return cudaGetLastError();
}

cudaError_t launch_ylt_fp64(const int64_t *offsets, const int32_t *ids, int64_t n_trials,
                            const ulonglong2 *table, const uint32_t *bitmap, BitmapLayout bm,
                            int q, double agg_ret, double agg_lim, double *ylt,
                            const YltLaunch &cfg, cudaStream_t s) {
  if (n_trials <= 0) return cudaSuccess;
  switch (cfg.unroll) {
    case 1: return launch_u<1>(offsets, ids, n_trials, table, bitmap, bm, q, agg_ret, agg_lim, ylt, cfg, s);
    case 2: return launch_u<2>(offsets, ids, n_trials, table, bitmap, bm, q, agg_ret, agg_lim, ylt, cfg, s);
    case 4: return launch_u<4>(offsets, ids, n_trials, table, bitmap, bm, q, agg_ret, agg_lim, ylt, cfg, s);
    default: return launch_u<8>(offsets, ids, n_trials, table, bitmap, bm, q, agg_ret, agg_lim, ylt, cfg, s);
  }
}

cudaError_t plan_ylt(int device, const BitmapLayout &bm, double mean_trial_len, YltLaunch *out) {
  int sms = 0;
  cudaError_t err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (err != cudaSuccess) return err;
  int unroll = mean_trial_len >= 768.0 ? 8 : mean_trial_len >= 384.0 ? 4 : mean_trial_len >= 160.0 ? 2 : 1;
  if (const char *env = std::getenv("ARA_YLT_UNROLL")) {
    int u = std::atoi(env);
    if (u == 1 || u == 2 || u == 4 || u == 8) unroll = u;
  }
  out->threads = kYltThreads;
  out->smem = (size_t)bm.words * 4u;
  out->unroll = unroll;
  const void *fn = unroll == 1 ? (const void *)ylt_fp64_kernel<1>
                 : unroll == 2 ? (const void *)ylt_fp64_kernel<2>
                 : unroll == 4 ? (const void *)ylt_fp64_kernel<4>
                               : (const void *)ylt_fp64_kernel<8>;
  err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out->smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kYltThreads, out->smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  out->blocks = sms * per_sm;
  return cudaSuccess;
}

}  // namespace ara
