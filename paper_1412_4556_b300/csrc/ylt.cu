// The Year Loss Table kernel: Algorithm 1 (Section III), steps 1-4, for every
// trial of the YET, with steps 1-3 already folded into the per-event table.
//
// For trial t with occurrences id_k (the trial's events in stored order):
//     S_t   = sum_k o(id_k)                  (occurrence-net losses, step 3)
//     YLT_t = min(max(S_t - AggR, 0), AggL)  (aggregate terms, step 4)
// The aggregate clamp applied to the running sum after every event ends at
// the clamp of the final sum (the per-event increments telescope), so one
// clamp per trial gives the trial loss.
//
// B300 design:
//  * One warp per trial; each warp owns a contiguous run of trials, so the
//    YET id stream is read once, in 16-byte coalesced loads, U loads in flight
//    per lane, with an evict-first L2 policy; one lane bulk-prefetches the
//    next trial into L2.  The engine stores every trial as whole 16-byte
//    chunks (4 plain ids, or 6 ids of 21 bits when the catalog allows, which
//    cuts the id stream by a third), padded with a sentinel event whose table
//    entry is zero, so each chunk belongs to one trial and no per-event
//    bounds test is needed.
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
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p), "l"(pol));
  return v;
}

__device__ __forceinline__ ulonglong2 ld_entry(const ulonglong2 *p, unsigned long long pol) {
  ulonglong2 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
               : "=l"(v.x), "=l"(v.y)
               : "l"(p), "l"(pol));
  return v;
}

// Table entry of `id` if `hit`, else zero: a predicated 16-byte gather, so
// occurrences whose bitmap bit is clear cost no memory request.
__device__ __forceinline__ ulonglong2 gather_if(const ulonglong2 *p, uint32_t hit,
                                                unsigned long long pol) {
  ulonglong2 v = make_ulonglong2(0ull, 0ull);
  asm("{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %2, 0;\n\t"
      "@p ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u64 {%0, %1}, [%3], %4;\n\t}"
      : "+l"(v.x), "+l"(v.y)
      : "r"(hit), "l"(p), "l"(pol));
  return v;
}

// One bulk copy-engine request pulls a whole trial's ids (a contiguous,
// 16-byte aligned run) into L2, so the warp's own loads of that trial hit L2.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The ids of one 16-byte chunk: four plain 32-bit ids, or six 21-bit ids
// packed three to a 64-bit half (see pack6).
template <bool PACKED>
__device__ __forceinline__ void chunk_ids(int4 c, uint32_t (&id)[PACKED ? 6 : 4]) {
  if constexpr (PACKED) {
    constexpr uint32_t M = 0x1FFFFFu;
    id[0] = (uint32_t)c.x & M;
    id[1] = __funnelshift_r((uint32_t)c.x, (uint32_t)c.y, 21) & M;
    id[2] = ((uint32_t)c.y >> 10) & M;
    id[3] = (uint32_t)c.z & M;
    id[4] = __funnelshift_r((uint32_t)c.z, (uint32_t)c.w, 21) & M;
    id[5] = ((uint32_t)c.w >> 10) & M;
  } else {
    id[0] = (uint32_t)c.x;
    id[1] = (uint32_t)c.y;
    id[2] = (uint32_t)c.z;
    id[3] = (uint32_t)c.w;
  }
}

// Table entries of `id` for G layers (16 bytes each, interleaved) if `hit`,
// else zeros; G = 2 is one 32-byte load, i.e. one L2 sector for two layers.
template <int G>
__device__ __forceinline__ void gather_group(const ulonglong2 *table, uint32_t id, uint32_t hit,
                                             unsigned long long pol, ulonglong2 (&x)[G]) {
  if constexpr (G == 1) {
    x[0] = gather_if(table + id, hit, pol);
  } else {
    unsigned long long a = 0ull, b = 0ull, c = 0ull, d = 0ull;
    asm("{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "@p ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u64 {%0, %1, %2, %3}, [%5], %6;\n\t}"
        : "+l"(a), "+l"(b), "+l"(c), "+l"(d)
        : "r"(hit), "l"(table + 2 * (size_t)id), "l"(pol));
    x[0] = make_ulonglong2(a, b);
    x[1] = make_ulonglong2(c, d);
  }
}

template <int G>
struct GroupOut {
  LayerOut l[G];
};

// G layers share one pass over the YET: one zero-skip bitmap (the union of
// the layers' bitmaps), one gather per occurrence that any layer needs, and
// one 128-bit accumulator per layer.
template <int U, bool PACKED, int G>
__global__ void __launch_bounds__(kYltThreads, 1)
ylt_fp64_kernel(const int64_t *__restrict__ coff, const int4 *__restrict__ chunks,
                int64_t n_trials, const ulonglong2 *__restrict__ table,
                const uint4 *__restrict__ bitmap4, int bm_words4, uint32_t bm_mul,
                int4 sent4, GroupOut<G> out) {
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

  int64_t p_next = t_begin < t_end ? coff[t_begin] : 0;
  if (lane == 0 && t_begin < t_end) {
    const int64_t b = coff[t_begin + 1];
    if (b > p_next) prefetch_l2(chunks + p_next, (uint32_t)((b - p_next) * 16));
  }
  for (int64_t t = t_begin; t < t_end; ++t) {
    const int64_t p0 = p_next;
    p_next = coff[t + 1];
    // While this trial is summed, its successor's ids travel to L2.
    if (lane == 0 && t + 1 < t_end) {
      const int64_t b = coff[t + 2];
      if (b > p_next) prefetch_l2(chunks + p_next, (uint32_t)((b - p_next) * 16));
    }
    const int4 *tp = chunks + p0;
    const int nk = (int)(p_next - p0);  // 16-byte chunks of this trial
    U128 acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = U128{0ull, 0ull};
    for (int base = 0; base < nk; base += 32 * U) {
      int4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        v[u] = sent4;
        const int j = base + 32 * u + lane;
        if (base + 32 * u < nk && j < nk) v[u] = ld_ids(tp + j, pol_ids);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (base + 32 * u >= nk) break;  // warp-uniform: the rest of this step is empty
        uint32_t idv[PACKED ? 6 : 4];
        chunk_ids<PACKED>(v[u], idv);
#pragma unroll
        for (int i = 0; i < (PACKED ? 6 : 4); ++i) {
          const uint32_t id = idv[i];
          const uint32_t word = s_bm[bitmap_word(id, bm_mul)];
          const uint32_t hit = __funnelshift_r(word, word, id) & 1u;  // bit id & 31
          ulonglong2 x[G];
          gather_group<G>(table, id, hit, pol_tab, x);
#pragma unroll
          for (int g = 0; g < G; ++g) add128(acc[g], x[g].x, x[g].y);
        }
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const U128 sum = warp_sum_u128(acc[g]);
      const LayerOut &L = out.l[g];
      if (lane == 0) L.ylt[t] = trial_loss(sum, L.q, L.af, L.agg_ret, L.agg_lim);
    }
  }
}

template <int U, bool PACKED, int G>
static cudaError_t launch_u(const int64_t *coff, const int4 *chunks, int64_t n_trials,
                            const ulonglong2 *table, const uint32_t *bitmap, BitmapLayout bm,
                            int32_t sentinel, const LayerOut *outs, const YltLaunch &cfg,
                            cudaStream_t s) {
  cudaError_t err = cudaFuncSetAttribute(ylt_fp64_kernel<U, PACKED, G>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cfg.smem);
  if (err != cudaSuccess) return err;
  int32_t sv[6] = {sentinel, sentinel, sentinel, sentinel, sentinel, sentinel};
  const int4 sent4 = PACKED ? pack6(sv) : make_int4(sentinel, sentinel, sentinel, sentinel);
  GroupOut<G> go;
  for (int g = 0; g < G; ++g) go.l[g] = outs[g];
  ylt_fp64_kernel<U, PACKED, G><<<cfg.blocks, cfg.threads, cfg.smem, s>>>(
      coff, chunks, n_trials, table, reinterpret_cast<const uint4 *>(bitmap), bm.words / 4, bm.mul,
      sent4, go);
  return cudaGetLastError();
}

template <bool PACKED, int G>
static cudaError_t launch_pg(const int64_t *coff, const int4 *chunks, int64_t n_trials,
                             const ulonglong2 *table, const uint32_t *bitmap, BitmapLayout bm,
                             int32_t sentinel, const LayerOut *outs, const YltLaunch &cfg,
                             cudaStream_t s) {
  switch (cfg.unroll) {
    case 1: return launch_u<1, PACKED, G>(coff, chunks, n_trials, table, bitmap, bm, sentinel, outs, cfg, s);
    case 2: return launch_u<2, PACKED, G>(coff, chunks, n_trials, table, bitmap, bm, sentinel, outs, cfg, s);
    default: return launch_u<4, PACKED, G>(coff, chunks, n_trials, table, bitmap, bm, sentinel, outs, cfg, s);
  }
}

cudaError_t launch_ylt_group(const int64_t *coff, const int4 *chunks, bool packed, int64_t n_trials,
                             const ulonglong2 *table, const uint32_t *bitmap, BitmapLayout bm,
                             int32_t sentinel, int G, const LayerOut *outs, const YltLaunch &cfg,
                             cudaStream_t s) {
  if (n_trials <= 0) return cudaSuccess;
  if (G == 2)
    return packed ? launch_pg<true, 2>(coff, chunks, n_trials, table, bitmap, bm, sentinel, outs, cfg, s)
                  : launch_pg<false, 2>(coff, chunks, n_trials, table, bitmap, bm, sentinel, outs, cfg, s);
  return packed ? launch_pg<true, 1>(coff, chunks, n_trials, table, bitmap, bm, sentinel, outs, cfg, s)
                : launch_pg<false, 1>(coff, chunks, n_trials, table, bitmap, bm, sentinel, outs, cfg, s);
}

template <bool PACKED, int G>
static const void *kernel_ptr(int unroll) {
  return unroll == 1 ? (const void *)ylt_fp64_kernel<1, PACKED, G>
       : unroll == 2 ? (const void *)ylt_fp64_kernel<2, PACKED, G>
                     : (const void *)ylt_fp64_kernel<4, PACKED, G>;
}

cudaError_t plan_ylt(int device, const BitmapLayout &bm, double mean_chunks, bool packed, int G,
                     int unroll_hint, YltLaunch *out) {
  int sms = 0;
  cudaError_t err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (err != cudaSuccess) return err;
  // Chunks per lane of a typical trial.  Measured on B300 with ~8 chunks per
  // lane (1000-event trials): U = 2 beats 4 and 8 (fewer wasted slots in the
  // last step of a trial, more warps' worth of registers free).
  const double per_lane = mean_chunks / 32.0;
  int unroll = per_lane > 1.5 ? 2 : 1;
  if (unroll_hint == 1 || unroll_hint == 2 || unroll_hint == 4) unroll = unroll_hint;
  if (const char *env = std::getenv("ARA_YLT_UNROLL")) {
    int u = std::atoi(env);
    if (u == 1 || u == 2 || u == 4) unroll = u;
  }
  out->threads = kYltThreads;
  out->smem = (size_t)bm.words * 4u;
  out->unroll = unroll;
  const void *fn = G == 2 ? (packed ? kernel_ptr<true, 2>(unroll) : kernel_ptr<false, 2>(unroll))
                          : (packed ? kernel_ptr<true, 1>(unroll) : kernel_ptr<false, 1>(unroll));
  err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out->smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kYltThreads, out->smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  out->blocks = sms * per_sm;
  return cudaSuccess;
}

// Interleave two layers' tables (entry e of layer a then of layer b, 32 bytes
// per event) and OR their zero-skip bitmaps, for a two-layer pass.
__global__ void interleave_kernel(const ulonglong2 *__restrict__ ta, const ulonglong2 *__restrict__ tb,
                                  int64_t entries, ulonglong2 *__restrict__ out,
                                  const uint32_t *__restrict__ ba, const uint32_t *__restrict__ bb,
                                  int32_t words, uint32_t *__restrict__ bout) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < entries; e += stride) {
    out[2 * e] = ta[e];
    out[2 * e + 1] = tb[e];
  }
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += stride)
    bout[w] = ba[w] | bb[w];
}

cudaError_t launch_interleave(const ulonglong2 *ta, const ulonglong2 *tb, int64_t entries,
                              ulonglong2 *out, const uint32_t *ba, const uint32_t *bb,
                              int32_t words, uint32_t *bout, cudaStream_t s) {
  interleave_kernel<<<148 * 8, 256, 0, s>>>(ta, tb, entries, out, ba, bb, words, bout);
  return cudaGetLastError();
}

}  // namespace ara
