// Year Event Loss Table: the per-occurrence increments of Algorithm 1's
// aggregate step (Section III, step 4 applied after every event of a trial),
// and each trial's largest increment for occurrence exceedance (OEP) reports.
//
// For trial t with occurrence-net losses o_1..o_n (stored order):
//     P_k   = o_1 + ... + o_k                      (running sum)
//     a_k   = min(max(P_k - AggR, 0), AggL)        (aggregate terms)
//     inc_k = a_k - a_{k-1},   a_0 = 0             (YELT entry of occurrence k)
// and the trial loss is a_n (the YLT entry).
//
// B300 design: 16 lanes per trial (8 for the report variant) walk the
// trial's 16-byte id chunks in order, one chunk per lane per step, two (four)
// trials side by side in a warp.  Each lane
// gathers its chunk's table entries (zero-skip bitmap in shared memory, as
// in the YLT kernel), forms their prefix sums, and the trial's lanes turn their
// totals into an exclusive scan with shuffles: a segmented scan whose
// segments are the trials.  The running
// sums are 128-bit fixed-point integers, so every P_k is exact; when the
// aggregate terms lie on the table's grid the clamps and differences are
// exact integers too and each increment is rounded to binary64 once.  With
// per-occurrence output the entries are gathered from a copy of the table
// holding each event's binary64 value beside its entry (one 32-byte sector
// for FP64 layers), so an increment inside the layer is read, not converted,
// and needs no second gather.
#include "ara_internal.cuh"

namespace ara {

namespace {

// L2 policies: the id chunks (read once) and the increments (written once)
// pass through L2 marked evict-first, the table gathers evict-last, so that
// the stream does not push the layer's table out of L2 (measured on the
// paper-scale YET: 4.68 -> 3.94 ms with per-occurrence output).
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ unsigned long long l2_evict_last() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ ulonglong2 gather_or_zero(const ulonglong2 *p, uint32_t hit, unsigned long long pol) {
  unsigned long long a = 0ull, b = 0ull;
  asm("{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %2, 0;\n\t"
      "@p ld.global.nc.L2::cache_hint.v2.u64 {%0, %1}, [%3], %4;\n\t}"
      : "+l"(a), "+l"(b)
      : "r"(hit), "l"(p), "l"(pol));
  return make_ulonglong2(a, b);
}

__device__ __forceinline__ unsigned long long gather_or_zero8(const unsigned long long *p, uint32_t hit,
                                                              unsigned long long pol) {
  unsigned long long a = 0ull;
  asm("{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "@p ld.global.nc.L2::cache_hint.u64 %0, [%2], %3;\n\t}"
      : "+l"(a)
      : "r"(hit), "l"(p), "l"(pol));
  return a;
}

// A table entry as a 128-bit integer (zero without a load when hit is 0).
template <int EB>
__device__ __forceinline__ U128 entry_or_zero(const void *table, uint32_t id, uint32_t hit, unsigned long long pol) {
  if constexpr (EB == 16) {
    const ulonglong2 e = gather_or_zero(static_cast<const ulonglong2 *>(table) + id, hit, pol);
    return U128{e.x, e.y};
  } else {
    return U128{gather_or_zero8(static_cast<const unsigned long long *>(table) + id, hit, pol), 0ull};
  }
}

// An entry and its binary64 value from the interleaved table: one 32-byte
// (16-byte entries) or 16-byte (8-byte entries) load, zero when hit is 0.
template <int EB>
__device__ __forceinline__ void gather_comb(const ulonglong2 *comb, uint32_t id, uint32_t hit, unsigned long long pol,
                                            U128 &e, unsigned long long &f64) {
  unsigned long long a = 0ull, b = 0ull, c = 0ull, d = 0ull;
  if constexpr (EB == 16) {
    asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "@p ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u64 {%0, %1, %2, %3}, [%5], %6;\n\t}"
        : "+l"(a), "+l"(b), "+l"(c), "+l"(d)
        : "r"(hit), "l"(comb + 2 * (size_t)id), "l"(pol));
    e = U128{a, b};
    f64 = c;
  } else {
    asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t"
        "@p ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u64 {%0, %1}, [%3], %4;\n\t}"
        : "+l"(a), "+l"(b)
        : "r"(hit), "l"(comb + id), "l"(pol));
    e = U128{a, 0ull};
    f64 = b;
  }
  (void)d;
}

__device__ __forceinline__ int4 ld_chunk(const int4 *p, unsigned long long pol) {
  int4 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p), "l"(pol));
  return v;
}

__device__ __forceinline__ void st_out2(double *p, double a, double b, unsigned long long pol) {
  asm volatile("st.global.L1::no_allocate.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(a), "d"(b),
               "l"(pol)
               : "memory");
}

// 32 bytes at a 32-byte aligned address (256-bit store, sm_100 and later).
__device__ __forceinline__ void st_out4(double *p, double a, double b, double c, double d, unsigned long long pol) {
  asm volatile("st.global.L1::no_allocate.L2::cache_hint.v4.f64 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "d"(a),
               "d"(b), "d"(c), "d"(d), "l"(pol)
               : "memory");
}

__device__ __forceinline__ void st_out(double *p, double a, unsigned long long pol) {
  asm volatile("st.global.L1::no_allocate.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(a), "l"(pol) : "memory");
}

__device__ __forceinline__ U128 add(U128 a, U128 b) {
  add128(a, b.lo, b.hi);
  return a;
}

// Aggregate clamp of a running sum on the fixed-point grid (exact terms).
__device__ __forceinline__ U128 clamp_fixed(U128 P, const AggFixed &af) {
  U128 d{0ull, 0ull};
  if (ge128(P, af.ret)) d = sub128(P, af.ret);
  if (ge128(d, af.lim)) d = af.lim;
  return d;
}

__device__ __forceinline__ double clamp_fp64(U128 P, int q, double agg_ret, double agg_lim) {
  return fmin(fmax(__dsub_rn(from_fixed(P, q), agg_ret), 0.0), agg_lim);
}

// Shuffles within groups of W consecutive lanes.
template <int W>
__device__ __forceinline__ U128 shfl_up_u128(U128 v, int d) {
  U128 r;
  r.lo = __shfl_up_sync(0xFFFFFFFFu, v.lo, d, W);
  r.hi = __shfl_up_sync(0xFFFFFFFFu, v.hi, d, W);
  return r;
}

template <int W>
__device__ __forceinline__ U128 shfl_u128(U128 v, int src) {
  U128 r;
  r.lo = __shfl_sync(0xFFFFFFFFu, v.lo, src, W);
  r.hi = __shfl_sync(0xFFFFFFFFu, v.hi, src, W);
  return r;
}

template <bool PACKED>
__device__ __forceinline__ void chunk_ids_y(int4 c, uint32_t (&id)[PACKED ? 6 : 4]) {
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

// OUT: the per-occurrence increments are written (else only the trial
// maxima and losses, as for the return period report).  768-thread CTAs:
// one per SM (the bitmap), 80 registers a thread, which leaves room to load
// the next step's chunk a step ahead without spilling (measured on the
// paper-scale YET with output: 3.29 ms against 3.56 ms for 1024 threads
// without the early load, 3.63 ms with it, 3.89 ms at 768 threads without
// it; report pass 2.15 against 2.18 ms).
constexpr int kYeltThreads = 768;

template <bool PACKED, int EB, bool OUT>
__global__ void __launch_bounds__(kYeltThreads, 1)
yelt_kernel(const int64_t *__restrict__ coff, const int4 *__restrict__ chunks,
            const int64_t *__restrict__ raw_off, int64_t n_trials, const void *__restrict__ table,
            const uint4 *__restrict__ bitmap4, int bm_words4, uint32_t bm_mul, int4 sent4, LayerOut L,
            double *__restrict__ yelt, double *__restrict__ occ_max, const ulonglong2 *__restrict__ comb,
            const unsigned int *__restrict__ inexact) {
  constexpr int IDS = PACKED ? 6 : 4;
  // lanes per trial (measured: 16 with per-occurrence output, 8 without)
  constexpr int kLanes = OUT ? 16 : 8;
  constexpr int kTrialsPerWarp = 32 / kLanes;  // trials a warp walks side by side
  extern __shared__ uint4 s_bm4[];
  for (int i = threadIdx.x; i < bm_words4; i += blockDim.x) s_bm4[i] = bitmap4[i];
  __syncthreads();
  const uint32_t *s_bm = reinterpret_cast<const uint32_t *>(s_bm4);
  const int lane = threadIdx.x & 31;
  const int grp = lane / kLanes;  // which of the warp's trials this lane works on
  const int gl = lane % kLanes;   // lane within that trial's group
  const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t t_begin = n_trials * w / n_warps;
  const int64_t t_end = n_trials * (w + 1) / n_warps;
  const bool exact = L.af.exact != 0;
  const unsigned long long pol_stream = l2_evict_first();
  const unsigned long long pol_tab = l2_evict_last();
  // the binary64 values hold exactly the entries' values: read increments from them
  const bool use64 = OUT && *inexact == 0u;
  // AggR + AggL on the grid, saturated (an unreachable limit stays unreachable)
  U128 ret_lim = add(L.af.ret, L.af.lim);
  if (!ge128(ret_lim, L.af.ret)) ret_lim = U128{~0ull, ~0ull};

  for (int64_t t0 = t_begin; t0 < t_end; t0 += kTrialsPerWarp) {
    const int64_t t = t0 + grp;
    const bool valid_t = t < t_end;
    const int64_t p0 = valid_t ? coff[t] : 0;
    const int nk = valid_t ? (int)(coff[t + 1] - p0) : 0;
    const int64_t r0 = valid_t ? raw_off[t] : 0;
    const int64_t nr = valid_t ? raw_off[t + 1] - r0 : 0;  // occurrences of trial t
    int nk_max = nk;
    if constexpr (kTrialsPerWarp > 1) nk_max = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)nk);
    U128 carry{0ull, 0ull};                  // running sum before this step
    unsigned long long best = 0ull;          // largest increment seen by this lane, as bits
                                             // (increments are >= 0: bits order like values)
    U128 best_fx{0ull, 0ull};                // !OUT: largest entry of the steps inside the layer
    // The next step's chunk is loaded a step ahead.
    int4 vnext = gl < nk ? ld_chunk(chunks + p0 + gl, pol_stream) : sent4;
    for (int base = 0; base < nk_max; base += kLanes) {
      const int j = base + gl;
      const int4 v = vnext;
      vnext = j + kLanes < nk ? ld_chunk(chunks + p0 + j + kLanes, pol_stream) : sent4;
      uint32_t id[IDS];
      chunk_ids_y<PACKED>(v, id);
      // Without output the entries stay in registers; with output only their
      // binary64 values do (the per-occurrence path, rare, gathers an entry
      // again: the line is still in L2).
      U128 x[OUT ? 1 : IDS];
      unsigned long long f[OUT ? IDS : 1];
      uint32_t hits = 0u;
      U128 tot{0ull, 0ull};
#pragma unroll
      for (int i = 0; i < IDS; ++i) {
        const uint32_t word = s_bm[bitmap_word(id[i], bm_mul)];
        const uint32_t hit = __funnelshift_r(word, word, id[i]) & 1u;
        if constexpr (OUT) {
          hits |= hit << i;
          U128 e;
          gather_comb<EB>(comb, id[i], hit, pol_tab, e, f[i]);
          tot = add(tot, e);
        } else {
          x[i] = entry_or_zero<EB>(table, id[i], hit, pol_tab);
          tot = add(tot, x[i]);
        }
      }
      // entry i of this lane's chunk (with output: gathered again, from the
      // interleaved table whose line this step has just brought into L2)
      auto entry = [&](int i) -> U128 {
        if constexpr (OUT) {
          // the entry is the first 16 (8) bytes of the event's 32 (16) in the interleaved table
          if constexpr (EB == 16)
            return entry_or_zero<16>(comb, 2 * id[i], (hits >> i) & 1u, pol_tab);
          else
            return entry_or_zero<8>(comb, 2 * id[i], (hits >> i) & 1u, pol_tab);
        } else {
          return x[i];
        }
      };
      // inclusive scan of the lane totals across the trial's lanes
      U128 incl = tot;
#pragma unroll
      for (int d = 1; d < kLanes; d <<= 1) {
        const U128 o = shfl_up_u128<kLanes>(incl, d);
        if (gl >= d) incl = add(incl, o);
      }
      const U128 step_total = shfl_u128<kLanes>(incl, kLanes - 1);
      // running sum before this lane's first id: carry + exclusive prefix
      U128 P = sub128(add(carry, incl), tot);
      const int64_t k0 = (int64_t)j * IDS;  // index of id[0] within the trial
      const int64_t left = nr - k0;          // this lane's ids that are occurrences (may be <= 0)
      const int valid = left < IDS ? (int)(left > 0 ? left : 0) : IDS;
      double *const out = OUT ? yelt + r0 + k0 : nullptr;
      // Fast path (warp-uniform): every lane's chunk lies wholly below the
      // retention (a stays 0), wholly beyond the exhausted limit (a stays
      // AggL), or wholly inside the layer (a_k = P_k - AggR, so each
      // increment is the occurrence's own entry, exactly).
      bool inside = false;
      bool fast = false;
      if (exact) {
        const U128 P1 = add(P, tot);
        inside = ge128(P, L.af.ret) && ge128(ret_lim, P1);
        fast = __all_sync(0xFFFFFFFFu, inside || ge128(L.af.ret, P1) || ge128(P, ret_lim));
      }
      if constexpr (!OUT) {
        if (fast) {
          // Inside the layer an increment is its entry, and the conversion is
          // monotone: keep the largest entry, convert it once per trial.  Slots
          // past the trial's end hold the sentinel (entry 0), which cannot
          // raise a maximum, so only the stores need the slot count.
          if (inside) {
#pragma unroll
            for (int i = 0; i < IDS; ++i)
              if (ge128(x[i], best_fx)) best_fx = x[i];
          }
          carry = add(carry, step_total);
          continue;
        }
      }
      if (fast) {
        double inc[IDS];
#pragma unroll
        for (int i = 0; i < IDS; ++i) {
          if constexpr (OUT) {
            if (use64)
              inc[i] = inside ? __longlong_as_double((long long)f[i]) : 0.0;
            else
              inc[i] = inside ? from_fixed_exact(entry(i), L.q) : 0.0;
          } else {
            inc[i] = inside ? from_fixed_exact(x[i], L.q) : 0.0;
          }
          const unsigned long long b = (unsigned long long)__double_as_longlong(inc[i]);
          best = b > best ? b : best;
        }
        if (OUT) {
          if (valid == IDS) {
            const uintptr_t a = reinterpret_cast<uintptr_t>(out);
            if (IDS == 6 && (a & 15u) == 0u) {
              // 48 bytes a lane: a 32-byte store on the lane's 32-byte aligned
              // part and a 16-byte store on the rest (which part comes first
              // alternates from lane to lane; selects keep the warp converged)
              const bool lo32 = (a & 31u) == 0u;
              double *p4 = lo32 ? out : out + 2;
              double *p2 = lo32 ? out + 4 : out;
              st_out4(p4, lo32 ? inc[0] : inc[2], lo32 ? inc[1] : inc[3], lo32 ? inc[2] : inc[4],
                      lo32 ? inc[3] : inc[5], pol_stream);
              st_out2(p2, lo32 ? inc[4] : inc[0], lo32 ? inc[5] : inc[1], pol_stream);
            } else if ((a & 15u) == 0u) {
              // 16-byte stores where the pair is aligned (the parity of r0 is the
              // same for every lane of a trial), so a warp writes half as many sectors
#pragma unroll
              for (int i = 0; i + 1 < IDS; i += 2) st_out2(out + i, inc[i], inc[i + 1], pol_stream);
            } else {
              st_out(out, inc[0], pol_stream);
#pragma unroll
              for (int i = 1; i + 1 < IDS; i += 2) st_out2(out + i, inc[i], inc[i + 1], pol_stream);
              st_out(out + IDS - 1, inc[IDS - 1], pol_stream);
            }
          } else {
#pragma unroll
            for (int i = 0; i < IDS; ++i)
              if (i < valid) st_out(out + i, inc[i], pol_stream);
          }
        }
        carry = add(carry, step_total);
        continue;
      }
      U128 a_fx = exact ? clamp_fixed(P, L.af) : U128{0ull, 0ull};
      double a_fp = exact ? 0.0 : clamp_fp64(P, L.q, L.agg_ret, L.agg_lim);
#pragma unroll
      for (int i = 0; i < IDS; ++i) {
        const U128 e = entry(i);
        P = add(P, e);
        double inc;
        if (exact) {
          const U128 a = clamp_fixed(P, L.af);
          const U128 d = sub128(a, a_fx);
          a_fx = a;
          if constexpr (!OUT) {
            // Only the largest increment is kept: one equal to its entry
            // (the id lies inside the layer) joins the largest entry,
            // converted once per trial; one of 0 cannot raise it; only a
            // crossing id (d strictly between) is converted here.  Slots past
            // the trial's end hold entry 0 and leave d = 0.
            if (d.lo == e.lo && d.hi == e.hi) {
              if (ge128(d, best_fx)) best_fx = d;
            } else if ((d.lo | d.hi) != 0ull) {
              const unsigned long long b = (unsigned long long)__double_as_longlong(from_fixed_int(d, L.q));
              best = b > best ? b : best;
            }
            continue;
          }
          // with output: an id inside the layer is its own binary64 value,
          // one that changes nothing is 0; only a crossing id is converted
          if ((d.lo | d.hi) == 0ull)
            inc = 0.0;
          else if (use64 && d.lo == e.lo && d.hi == e.hi)
            inc = __longlong_as_double((long long)f[i]);
          else
            inc = from_fixed_int(d, L.q);
        } else {
          const double a = clamp_fp64(P, L.q, L.agg_ret, L.agg_lim);
          inc = __dsub_rn(a, a_fp);
          a_fp = a;
        }
        if (i < valid) {
          const unsigned long long b = (unsigned long long)__double_as_longlong(inc);
          best = b > best ? b : best;
          if (OUT) st_out(out + i, inc, pol_stream);
        }
      }
      carry = add(carry, step_total);
    }
    if (!OUT) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(from_fixed_exact(best_fx, L.q));
      best = b > best ? b : best;
    }
#pragma unroll
    for (int m = kLanes / 2; m > 0; m >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, best, m);
      best = o > best ? o : best;
    }
    if (gl == 0 && valid_t) {
      if (occ_max) occ_max[t] = __longlong_as_double((long long)best);
      if (L.ylt) L.ylt[t] = trial_loss(carry, L.q, L.af, L.agg_ret, L.agg_lim);
    }
  }
}

}  // namespace

template <bool PACKED, int EB, bool OUT>
static cudaError_t launch_yelt_t(const int64_t *coff, const int4 *chunks, const int64_t *raw_off, int64_t n_trials,
                                 const void *table, const uint32_t *bitmap, BitmapLayout bm, int32_t sentinel,
                                 const LayerOut &L, double *yelt, double *occ_max, int sms, cudaStream_t s,
                                 const ulonglong2 *comb, const unsigned int *inexact) {
  const size_t smem = (size_t)bm.words * 4u;
  cudaError_t err = cudaFuncSetAttribute(yelt_kernel<PACKED, EB, OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  int32_t sv[6] = {sentinel, sentinel, sentinel, sentinel, sentinel, sentinel};
  const int4 sent4 = PACKED ? pack6(sv) : make_int4(sentinel, sentinel, sentinel, sentinel);
  yelt_kernel<PACKED, EB, OUT><<<sms, kYeltThreads, smem, s>>>(coff, chunks, raw_off, n_trials, table,
                                                          reinterpret_cast<const uint4 *>(bitmap), bm.words / 4,
                                                          bm.mul, sent4, L, yelt, occ_max, comb, inexact);
  return cudaGetLastError();
}

cudaError_t launch_yelt(const int64_t *coff, const int4 *chunks, const int64_t *raw_off, bool packed,
                        int64_t n_trials, const void *table, int entry_bytes, const uint32_t *bitmap,
                        BitmapLayout bm, int32_t sentinel, const LayerOut &L, double *yelt, double *occ_max,
                        int device, cudaStream_t s, const ulonglong2 *comb, const unsigned int *inexact) {
  if (n_trials <= 0) return cudaSuccess;
  if (yelt != nullptr && (comb == nullptr || inexact == nullptr)) return cudaErrorInvalidValue;
  int sms = 0;
  cudaError_t err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (err != cudaSuccess) return err;
  const bool out = yelt != nullptr;
#define ARA_YELT_LAUNCH(P, E, O)                                                                             \
  launch_yelt_t<P, E, O>(coff, chunks, raw_off, n_trials, table, bitmap, bm, sentinel, L, yelt, occ_max, sms, s, \
                         comb, inexact)
  if (entry_bytes == 16) {
    if (packed) return out ? ARA_YELT_LAUNCH(true, 16, true) : ARA_YELT_LAUNCH(true, 16, false);
    return out ? ARA_YELT_LAUNCH(false, 16, true) : ARA_YELT_LAUNCH(false, 16, false);
  }
  if (packed) return out ? ARA_YELT_LAUNCH(true, 8, true) : ARA_YELT_LAUNCH(true, 8, false);
  return out ? ARA_YELT_LAUNCH(false, 8, true) : ARA_YELT_LAUNCH(false, 8, false);
#undef ARA_YELT_LAUNCH
}

namespace {

__global__ void yelt_comb_kernel(const void *__restrict__ table, int entry_bytes, const double *__restrict__ table64,
                                 int64_t n, ulonglong2 *__restrict__ comb) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long f = (unsigned long long)__double_as_longlong(table64[e]);
    if (entry_bytes == 16) {
      comb[2 * e] = static_cast<const ulonglong2 *>(table)[e];
      comb[2 * e + 1] = make_ulonglong2(f, 0ull);
    } else {
      comb[e] = make_ulonglong2(static_cast<const unsigned long long *>(table)[e], f);
    }
  }
}

}  // namespace

cudaError_t launch_yelt_comb(const void *table, int entry_bytes, const double *table64, int64_t n_events,
                             ulonglong2 *comb, cudaStream_t s) {
  if (n_events <= 0) return cudaSuccess;
  if (entry_bytes != 16 && entry_bytes != 8) return cudaErrorInvalidValue;
  int64_t blocks = (n_events + 255) / 256;
  if (blocks > (int64_t)current_sm_count() * 8) blocks = (int64_t)current_sm_count() * 8;
  yelt_comb_kernel<<<(int)blocks, 256, 0, s>>>(table, entry_bytes, table64, n_events, comb);
  return cudaGetLastError();
}

}  // namespace ara
