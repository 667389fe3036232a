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
//    next trials into L2 (when the table leaves L2 room for it).  The engine stores every trial as whole 16-byte
//    chunks (4 plain ids, or 6 ids of 21 bits when the catalog allows, which
//    cuts the id stream by a third), padded with a sentinel event whose table
//    entry is zero, so each chunk belongs to one trial and no per-event
//    bounds test is needed.
//  * The layer's zero-skip bitmap sits in shared memory.  Only occurrences
//    whose bit is set fetch their table entry (a random 16-byte gather served
//    by L2, evict-last); the rest add an exact zero and are skipped.
//  * FP64 layers' table entries are 128-bit fixed-point integers; each lane
//    sums them with add/add-with-carry, and the warp combines lanes with
//    shuffles.  FP32-table layers use 64-bit entries on a grid chosen so that
//    no trial sum reaches 2^64: half the table bytes, so one 32-byte sector
//    holds an event's entries for four layers.  The
//    integer sum is exact, so the result does not depend on the order of
//    the additions or on the launch shape, and B300's low FP64 add rate is
//    kept off the per-occurrence path.  One correctly rounded conversion to
//    binary64 per trial precedes the FP64 aggregate clamp.
#include <cstdlib>
#include <type_traits>

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

// One bulk copy-engine request pulls a whole trial's ids (a contiguous,
// 16-byte aligned run) into L2, so the warp's own loads of that trial hit L2.
// The prefetched lines carry the id stream's evict-first policy, so the
// stream does not push the layer tables out of L2.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes, unsigned long long pol) {
  asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(p), "r"(bytes), "l"(pol)
               : "memory");
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

// The 8 ids of a difference-coded chunk (see compact.cu): a 21-bit base and
// seven 15-bit steps; a step of 0x7FFF marks an empty slot, read as the
// sentinel id (table entry zero).
template <bool FULL>
__device__ __forceinline__ void delta_ids(int4 c, uint32_t zero_id, uint32_t (&id)[8]) {
  const uint32_t x = (uint32_t)c.x, y = (uint32_t)c.y, z = (uint32_t)c.z, w = (uint32_t)c.w;
  uint32_t d[8];
  d[1] = __funnelshift_r(x, y, 21) & 0x7FFFu;
  d[2] = (y >> 4) & 0x7FFFu;
  d[3] = ((y >> 19) & 0x1FFFu) | ((z & 3u) << 13);
  d[4] = (z >> 2) & 0x7FFFu;
  d[5] = (z >> 17) & 0x7FFFu;
  d[6] = w & 0x7FFFu;
  d[7] = (w >> 15) & 0x7FFFu;
  uint32_t cur = x & 0x1FFFFFu;
  id[0] = cur;
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    cur += d[k];
    id[k] = FULL || d[k] != 0x7FFFu ? cur : zero_id;  // FULL: a chunk that is not a trial's last
  }
}

// Accumulators of G layers: 128-bit for 16-byte entries, 64-bit for 8-byte.
template <int EB, int G>
struct Acc {
  U128 v[G];
};
template <int G>
struct Acc<8, G> {
  unsigned long long v[G];
};

// Adds the table entries of `id` for G layers (EB bytes each, interleaved,
// EB * G <= 32: one L2 sector) to the accumulators when `hit` is set.  The
// gather is predicated, so occurrences whose bitmap bit is clear cost no
// memory request.
template <int EB, int G>
__device__ __forceinline__ void gather_add(Acc<EB, G> &acc, const void *table, uint32_t id, uint32_t hit,
                                           unsigned long long pol) {
  if constexpr (EB == 16 && G == 1) {
    unsigned long long a = 0ull, b = 0ull;
    asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t"
        "@p ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u64 {%0, %1}, [%3], %4;\n\t}"
        : "+l"(a), "+l"(b)
        : "r"(hit), "l"(static_cast<const ulonglong2 *>(table) + id), "l"(pol));
    add128(acc.v[0], a, b);
  } else if constexpr (EB == 16 && G == 2) {
    unsigned long long a = 0ull, b = 0ull, c = 0ull, d = 0ull;
    asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "@p ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u64 {%0, %1, %2, %3}, [%5], %6;\n\t}"
        : "+l"(a), "+l"(b), "+l"(c), "+l"(d)
        : "r"(hit), "l"(static_cast<const ulonglong2 *>(table) + 2 * (size_t)id), "l"(pol));
    add128(acc.v[0], a, b);
    add128(acc.v[1], c, d);
  } else if constexpr (EB == 8 && G == 1) {
    unsigned long long a = 0ull;
    asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "@p ld.global.nc.L1::no_allocate.L2::cache_hint.u64 %0, [%2], %3;\n\t}"
        : "+l"(a)
        : "r"(hit), "l"(static_cast<const unsigned long long *>(table) + id), "l"(pol));
    acc.v[0] += a;
  } else if constexpr (EB == 8 && G == 2) {
    unsigned long long a = 0ull, b = 0ull;
    asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t"
        "@p ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u64 {%0, %1}, [%3], %4;\n\t}"
        : "+l"(a), "+l"(b)
        : "r"(hit), "l"(static_cast<const unsigned long long *>(table) + 2 * (size_t)id), "l"(pol));
    acc.v[0] += a;
    acc.v[1] += b;
  } else {
    static_assert(EB == 8 && G == 4, "entry width x group must fill at most one 32-byte sector");
    unsigned long long a = 0ull, b = 0ull, c = 0ull, d = 0ull;
    asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "@p ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u64 {%0, %1, %2, %3}, [%5], %6;\n\t}"
        : "+l"(a), "+l"(b), "+l"(c), "+l"(d)
        : "r"(hit), "l"(static_cast<const unsigned long long *>(table) + 4 * (size_t)id), "l"(pol));
    acc.v[0] += a;
    acc.v[1] += b;
    acc.v[2] += c;
    acc.v[3] += d;
  }
}

// Sum over the LPT consecutive lanes of a group (LPT a power of two <= 32).
template <int LPT>
__device__ __forceinline__ U128 group_sum_u128(U128 v) {
#pragma unroll
  for (int m = LPT / 2; m > 0; m >>= 1) {
    U128 o = shfl_xor_u128(v, m);
    add128(v, o.lo, o.hi);
  }
  return v;
}

template <int LPT>
__device__ __forceinline__ unsigned long long group_sum_u64(unsigned long long v) {
#pragma unroll
  for (int m = LPT / 2; m > 0; m >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, m);
  return v;
}

template <int G>
struct GroupOut {
  LayerOut l[G];
};

// G layers share one pass over the YET: one zero-skip bitmap (the union of
// the layers' bitmaps), one gather per occurrence that any layer needs, and
// one 128-bit accumulator per layer.  A warp sums 32 / LPT consecutive trials
// side by side, LPT lanes per trial: fewer lanes idle in the last step of a
// trial, and one group reduction and one epilogue serve 32 / LPT trials.
template <int U, int LAYOUT, int EB, int G, int LPT, int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
ylt_fp64_kernel(const int64_t *__restrict__ coff, const int4 *__restrict__ chunks,
                int64_t n_trials, const void *__restrict__ table,
                const uint4 *__restrict__ bitmap4, int bm_words4, uint32_t bm_mul,
                int4 sent4, int4 sentd, uint32_t zero_id, GroupOut<G> out, int do_prefetch) {
  // LAYOUT 0: 4 plain ids per chunk; 1: 6 packed ids; 2: per trial either 6
  // packed ids or 8 difference-coded ids (flag in bit 62 of its offset).
  constexpr bool PACKED = LAYOUT >= 1;
  constexpr int IDS = LAYOUT == 2 ? 8 : (PACKED ? 6 : 4);
  constexpr int64_t OFF = LAYOUT == 2 ? kCompactOffsetMask : ~(int64_t)0;
  constexpr int TPW = 32 / LPT;  // trials per warp step
  extern __shared__ uint4 s_bm4[];
  for (int i = threadIdx.x; i < bm_words4; i += blockDim.x) s_bm4[i] = bitmap4[i];
  __syncthreads();
  const uint32_t *s_bm = reinterpret_cast<const uint32_t *>(s_bm4);

  const unsigned long long pol_ids = policy_evict_first();
  const unsigned long long pol_tab = policy_evict_last();
  const int lane = threadIdx.x & 31;
  const int grp = lane / LPT;
  const int gl = lane % LPT;
  const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t t_begin = n_trials * w / n_warps;
  const int64_t t_end = n_trials * (w + 1) / n_warps;

  // Offsets of the next warp step's trials and the L2 prefetch range of the
  // step after it are loaded one step ahead, so no step waits on them.
  int64_t pa = 0, pe = 0;  // chunk range of this lane's trial in the next step (flag kept in pa)
  if (t_begin + grp < t_end) {
    pa = coff[t_begin + grp];
    pe = coff[t_begin + grp + 1] & OFF;
  }
  int64_t fa = 0, fb = 0;  // lane 0: chunk range prefetched at the top of the next step
  if (lane == 0 && t_begin < t_end) {
    const int64_t a = coff[t_begin] & OFF, b = coff[min(t_begin + TPW, t_end)] & OFF;
    if (b > a && do_prefetch) prefetch_l2(chunks + a, (uint32_t)((b - a) * 16), pol_ids);
    fa = b;
    fb = coff[min(t_begin + 2 * TPW, t_end)] & OFF;
  }
  for (int64_t t0 = t_begin; t0 < t_end; t0 += TPW) {
    const int64_t t = t0 + grp;
    const bool valid = t < t_end;
    const bool dfl = LAYOUT == 2 && ((pa >> 62) & 1);  // difference-coded trial
    const int64_t p0 = pa & OFF;
    const int nk = (int)(pe - p0);  // 16-byte chunks of trial t (0 if not valid)
    pa = pe = 0;
    if (t + TPW < t_end) {
      pa = coff[t + TPW];
      pe = coff[t + TPW + 1] & OFF;
    }
    // While these trials are summed, the next ones' ids travel to L2.
    if (lane == 0) {
      if (fb > fa && do_prefetch) prefetch_l2(chunks + fa, (uint32_t)((fb - fa) * 16), pol_ids);
      fa = fb;
      fb = coff[min(t0 + 3 * TPW, t_end)] & OFF;
    }
    const int4 sentv = dfl ? sentd : sent4;
    int nk_max = nk, nk_min = nk;
    if constexpr (TPW > 1) {
      nk_max = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)nk);
      if constexpr (LAYOUT == 2) nk_min = (int)__reduce_min_sync(0xFFFFFFFFu, (unsigned)nk);
    }
    const int4 *tp = chunks + p0;
    Acc<EB, G> acc;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if constexpr (EB == 16)
        acc.v[g] = U128{0ull, 0ull};
      else
        acc.v[g] = 0ull;
    }
    // Software-pipelined: the ids of step base + LPT*U are in flight while
    // the current step's bitmap tests and gathers run.
    int4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      v[u] = sentv;
      const int j = LPT * u + gl;
      if (j < nk) v[u] = ld_ids(tp + j, pol_ids);
    }
    for (int base = 0; base < nk_max; base += LPT * U) {
      int4 vn[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        vn[u] = sentv;
        const int j = base + LPT * (U + u) + gl;
        if (j < nk) vn[u] = ld_ids(tp + j, pol_ids);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (base + LPT * u >= nk_max) break;  // warp-uniform: the rest of this step is empty
        uint32_t idv[IDS];
        if constexpr (LAYOUT == 2) {
          if (dfl) {
            // warp-uniform: no lane holds the last chunk of its trial, so no slot is empty
            if (base + LPT * (u + 1) < nk_min)
              delta_ids<true>(v[u], zero_id, idv);
            else
              delta_ids<false>(v[u], zero_id, idv);
          } else {
            uint32_t id6[6];
            chunk_ids<true>(v[u], id6);
#pragma unroll
            for (int i = 0; i < 6; ++i) idv[i] = id6[i];
            idv[6] = idv[7] = zero_id;
          }
        } else {
          chunk_ids<PACKED>(v[u], idv);
        }
#pragma unroll
        for (int i = 0; i < IDS; ++i) {
          const uint32_t id = idv[i];
          const uint32_t word = s_bm[bitmap_word(id, bm_mul)];
          const uint32_t hit = __funnelshift_r(word, word, id) & 1u;  // bit id & 31
          gather_add<EB, G>(acc, table, id, hit, pol_tab);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = vn[u];
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      U128 sum;
      if constexpr (EB == 16)
        sum = group_sum_u128<LPT>(acc.v[g]);
      else
        sum = U128{group_sum_u64<LPT>(acc.v[g]), 0ull};
      const LayerOut &L = out.l[g];
      const double y = trial_loss(sum, L.q, L.af, L.agg_ret, L.agg_lim);
      if (gl == 0 && valid) L.ylt[t] = y;
    }
  }
}

template <int U, int LAYOUT, int EB, int G, int LPT, int THREADS>
static cudaError_t launch_u(const int64_t *coff, const int4 *chunks, int64_t n_trials, const void *table,
                            const uint32_t *bitmap, BitmapLayout bm, int32_t sentinel, const LayerOut *outs,
                            const YltLaunch &cfg, cudaStream_t s) {
  cudaError_t err = cudaFuncSetAttribute(ylt_fp64_kernel<U, LAYOUT, EB, G, LPT, THREADS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
  if (err != cudaSuccess) return err;
  int32_t sv[6] = {sentinel, sentinel, sentinel, sentinel, sentinel, sentinel};
  const int4 sent4 = LAYOUT >= 1 ? pack6(sv) : make_int4(sentinel, sentinel, sentinel, sentinel);
  const int4 sentd = delta_sentinel_chunk(sentinel);
  GroupOut<G> go;
  for (int g = 0; g < G; ++g) go.l[g] = outs[g];
  ylt_fp64_kernel<U, LAYOUT, EB, G, LPT, THREADS><<<cfg.blocks, THREADS, cfg.smem, s>>>(
      coff, chunks, n_trials, table, reinterpret_cast<const uint4 *>(bitmap), bm.words / 4, bm.mul, sent4, sentd,
      (uint32_t)sentinel, go, cfg.prefetch);
  return cudaGetLastError();
}

// The kernel for (unroll, lanes per trial, threads per CTA) as a function
// pointer and as a launch, for one (LAYOUT, EB, G).
template <int LAYOUT, int EB, int G>
struct YltVariants {
  template <int THREADS>
  static const void *fn_t(int unroll, int lpt) {
    if (lpt == 16)
      return unroll == 1 ? (const void *)ylt_fp64_kernel<1, LAYOUT, EB, G, 16, THREADS>
                         : (const void *)ylt_fp64_kernel<2, LAYOUT, EB, G, 16, THREADS>;
    return unroll == 1 ? (const void *)ylt_fp64_kernel<1, LAYOUT, EB, G, 32, THREADS>
                       : (const void *)ylt_fp64_kernel<2, LAYOUT, EB, G, 32, THREADS>;
  }
  static const void *fn(int unroll, int lpt, int threads) {
    return threads == 768 ? fn_t<768>(unroll, lpt) : fn_t<1024>(unroll, lpt);
  }
  template <int THREADS>
  static cudaError_t launch_t(const int64_t *coff, const int4 *chunks, int64_t n_trials, const void *table,
                              const uint32_t *bitmap, BitmapLayout bm, int32_t sentinel, const LayerOut *outs,
                              const YltLaunch &cfg, cudaStream_t s) {
    if (cfg.lanes_per_trial == 16)
      return cfg.unroll == 1
                 ? launch_u<1, LAYOUT, EB, G, 16, THREADS>(coff, chunks, n_trials, table, bitmap, bm, sentinel, outs,
                                                           cfg, s)
                 : launch_u<2, LAYOUT, EB, G, 16, THREADS>(coff, chunks, n_trials, table, bitmap, bm, sentinel, outs,
                                                           cfg, s);
    return cfg.unroll == 1
               ? launch_u<1, LAYOUT, EB, G, 32, THREADS>(coff, chunks, n_trials, table, bitmap, bm, sentinel, outs,
                                                         cfg, s)
               : launch_u<2, LAYOUT, EB, G, 32, THREADS>(coff, chunks, n_trials, table, bitmap, bm, sentinel, outs,
                                                         cfg, s);
  }
  static cudaError_t launch(const int64_t *coff, const int4 *chunks, int64_t n_trials, const void *table,
                            const uint32_t *bitmap, BitmapLayout bm, int32_t sentinel, const LayerOut *outs,
                            const YltLaunch &cfg, cudaStream_t s) {
    if (cfg.threads == 768)
      return launch_t<768>(coff, chunks, n_trials, table, bitmap, bm, sentinel, outs, cfg, s);
    return launch_t<1024>(coff, chunks, n_trials, table, bitmap, bm, sentinel, outs, cfg, s);
  }
};

// Dispatch on (id layout, entry bytes, group size) -> F<LAYOUT, EB, G>.
template <template <int, int, int> class F, int EB, int G, typename... A>
static auto dispatch_layout(int layout, A... a) {
  if (layout == 2) return F<2, EB, G>::call(a...);
  if (layout == 1) return F<1, EB, G>::call(a...);
  return F<0, EB, G>::call(a...);
}

template <template <int, int, int> class F, typename... A>
static auto dispatch(int layout, int eb, int G, A... a) {
  if (eb == 16) {
    if (G == 2) return dispatch_layout<F, 16, 2>(layout, a...);
    return dispatch_layout<F, 16, 1>(layout, a...);
  }
  if (G == 4) return dispatch_layout<F, 8, 4>(layout, a...);
  if (G == 2) return dispatch_layout<F, 8, 2>(layout, a...);
  return dispatch_layout<F, 8, 1>(layout, a...);
}

template <int LAYOUT, int EB, int G>
struct LaunchF {
  static cudaError_t call(const int64_t *coff, const int4 *chunks, int64_t n_trials, const void *table,
                          const uint32_t *bitmap, BitmapLayout bm, int32_t sentinel, const LayerOut *outs,
                          const YltLaunch *cfg, cudaStream_t s) {
    return YltVariants<LAYOUT, EB, G>::launch(coff, chunks, n_trials, table, bitmap, bm, sentinel, outs, *cfg, s);
  }
};

template <int LAYOUT, int EB, int G>
struct FnF {
  static const void *call(int unroll, int lpt, int threads) {
    return YltVariants<LAYOUT, EB, G>::fn(unroll, lpt, threads);
  }
};

cudaError_t launch_ylt_group(const int64_t *coff, const int4 *chunks, int layout, int64_t n_trials,
                             const void *table, int entry_bytes, const uint32_t *bitmap, BitmapLayout bm,
                             int32_t sentinel, int G, const LayerOut *outs, const YltLaunch &cfg,
                             cudaStream_t s) {
  if (n_trials <= 0) return cudaSuccess;
  if (!(entry_bytes == 16 && (G == 1 || G == 2)) && !(entry_bytes == 8 && (G == 1 || G == 2 || G == 4)))
    return cudaErrorInvalidValue;
  if (layout < 0 || layout > 2) return cudaErrorInvalidValue;
  return dispatch<LaunchF>(layout, entry_bytes, G, coff, chunks, n_trials, table, bitmap, bm, sentinel, outs,
                           &cfg, s);
}

cudaError_t plan_ylt(int device, const BitmapLayout &bm, double mean_chunks, int layout, int entry_bytes,
                     int G, size_t table_bytes, YltShape hint, YltLaunch *out) {
  if (!(entry_bytes == 16 && (G == 1 || G == 2)) && !(entry_bytes == 8 && (G == 1 || G == 2 || G == 4)))
    return cudaErrorInvalidValue;
  int sms = 0;
  cudaError_t err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (err != cudaSuccess) return err;
  // Lanes per trial: a group of LPT lanes wastes on average LPT/2 chunk
  // slots in the last step of each trial, and one group reduction plus one
  // epilogue per warp step serve 32 / LPT trials.  Measured on B300 with
  // 167-chunk trials (Poisson(1000) events, 6 ids a chunk): 16 lanes per
  // trial beat 32 by 8% and 8 by 23%.
  int lpt = mean_chunks >= 24.0 ? 16 : 32;
  // Unroll: U chunk loads per lane per step; the loop already keeps the
  // next step's loads in flight, and U = 1 measured as fast as U = 2 with 16
  // lanes per trial (1.06 ms against 1.09 ms for 1e9 occurrences).
  int unroll = 1;
  // L2 bulk prefetch of the next trials' ids: measured on B300 it takes the
  // one-layer kernel from 1.30 to 1.06 ms (32 MB table), but with a 64 MB
  // interleaved table (two FP64 or four FP32-table layers) the prefetched ids
  // push table lines out of L2 and turning it off saves 10-14%.
  int prefetch = table_bytes <= (size_t)40 << 20 ? 1 : 0;
  if (hint.prefetch == 0 || hint.prefetch == 1) prefetch = hint.prefetch;
  if (hint.unroll == 1 || hint.unroll == 2) unroll = hint.unroll;
  if (hint.lanes_per_trial == 16 || hint.lanes_per_trial == 32) lpt = hint.lanes_per_trial;
  if (const char *env = std::getenv("ARA_YLT_UNROLL")) {
    int u = std::atoi(env);
    if (u == 1 || u == 2) unroll = u;
  }
  if (const char *env = std::getenv("ARA_YLT_LPT")) {
    int l = std::atoi(env);
    if (l == 16 || l == 32) lpt = l;
  }
  int threads = kYltThreads;
  if (hint.threads == 768 || hint.threads == 1024) threads = hint.threads;
  if (const char *env = std::getenv("ARA_YLT_THREADS")) {
    int t = std::atoi(env);
    if (t == 768 || t == 1024) threads = t;
  }
  out->threads = threads;
  out->smem = (size_t)bm.words * 4u;
  out->unroll = unroll;
  out->lanes_per_trial = lpt;
  out->prefetch = prefetch;
  if (layout < 0 || layout > 2) return cudaErrorInvalidValue;
  const void *fn = dispatch<FnF>(layout, entry_bytes, G, unroll, lpt, threads);
  err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out->smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, out->smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  out->blocks = sms * per_sm;
  return cudaSuccess;
}

// Interleave G layers' tables (entry e of layer 0, then of layer 1, ...:
// EB * G bytes per event, one 32-byte sector for G = 32 / EB) and OR their
// zero-skip bitmaps, for a G-layer pass.
template <int EB, int G>
__global__ void interleave_kernel(Tables4 in, int64_t entries, void *__restrict__ out, Bitmaps4 bin,
                                  int32_t words, uint32_t *__restrict__ bout) {
  using E = typename std::conditional<EB == 16, ulonglong2, unsigned long long>::type;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  E *o = static_cast<E *>(out);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < entries; e += stride) {
#pragma unroll
    for (int g = 0; g < G; ++g) o[G * e + g] = static_cast<const E *>(in.t[g])[e];
  }
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += stride) {
    uint32_t v = 0u;
#pragma unroll
    for (int g = 0; g < G; ++g) v |= bin.b[g][w];
    bout[w] = v;
  }
}

cudaError_t launch_interleave(const Tables4 &in, int entry_bytes, int G, int64_t entries, void *out,
                              const Bitmaps4 &bin, int32_t words, uint32_t *bout, cudaStream_t s) {
  const dim3 grid(current_sm_count() * 8), block(256);
  if (entry_bytes == 16 && G == 2)
    interleave_kernel<16, 2><<<grid, block, 0, s>>>(in, entries, out, bin, words, bout);
  else if (entry_bytes == 8 && G == 2)
    interleave_kernel<8, 2><<<grid, block, 0, s>>>(in, entries, out, bin, words, bout);
  else if (entry_bytes == 8 && G == 4)
    interleave_kernel<8, 4><<<grid, block, 0, s>>>(in, entries, out, bin, words, bout);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace ara
