// Internal declarations shared by the engine's translation units: device
// helpers for exact fixed-point accumulation, the per-ELT descriptor the fold
// kernel reads, and the launch wrappers each kernel file exports.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ara {

// ---------------------------------------------------------------- tuning
constexpr int kFoldEventsPerCta = 2048;  // catalog events folded by one CTA
constexpr int kFoldThreads = 256;
constexpr int kFoldStage = 2048;         // ELT entries staged in smem per chunk
constexpr int kMaxLayerElts = 1024;      // ELTs one layer may cover
constexpr int kYltThreads = 1024;        // threads per YLT CTA (32 warps)
constexpr int kMaxReturnPeriods = 16;
constexpr int kChunkTail = 4;            // sentinel chunks after the last trial
constexpr int32_t kPackedIdLimit = (1 << 21) - 1;  // catalog sizes whose ids pack in 21 bits

// Six ids of at most 21 bits in one 16-byte chunk (three per 64-bit half).
__host__ __device__ inline int4 pack6(const int32_t *v) {
  const unsigned long long lo = (unsigned long long)(uint32_t)v[0] |
                                ((unsigned long long)(uint32_t)v[1] << 21) |
                                ((unsigned long long)(uint32_t)v[2] << 42);
  const unsigned long long hi = (unsigned long long)(uint32_t)v[3] |
                                ((unsigned long long)(uint32_t)v[4] << 21) |
                                ((unsigned long long)(uint32_t)v[5] << 42);
  return make_int4((int)(uint32_t)lo, (int)(uint32_t)(lo >> 32), (int)(uint32_t)hi,
                   (int)(uint32_t)(hi >> 32));
}
constexpr int kSelectThreads = 512;

// ------------------------------------------------------ ELT descriptor
// One ELT of a layer, as the fold kernel sees it.  ids are sorted ascending
// and distinct; bucket[b] is the first index whose id >= b * kFoldEventsPerCta
// for b in [0, nb], with bucket[nb] == count.
struct EltDesc {
  const int32_t *ids;
  const double *losses;
  const int32_t *bucket;
  int32_t nb;
  int32_t count;
  double deductible;
  double limit;
};

// Zero-skip bitmap layout.  Event e maps to bit (e & 31) of word
// umulhi(e, mul) = floor(e * mul / 2^32).  With mul = 2^27 that is one bit
// per event (word e >> 5).  When the catalog has more events than the shared
// memory budget has bits, mul = floor(2^32 * words / events) spreads the
// events evenly over the words, and the few events of a word whose low five
// bits coincide share a bit.  A set bit means "some event of this bit may
// have a nonzero loss"; a clear bit proves every event of it has loss exactly
// zero, so skipping it leaves an exact sum unchanged.  The word index is one
// multiply-high (FMA pipe) and the bit index needs no arithmetic.
struct BitmapLayout {
  uint32_t mul;
  int32_t words;  // 32-bit words, a multiple of 4
};

__host__ __device__ inline uint32_t bitmap_word(uint32_t e, uint32_t mul) {
#ifdef __CUDA_ARCH__
  return __umulhi(e, mul);
#else
  return (uint32_t)(((uint64_t)e * mul) >> 32);
#endif
}

// ------------------------------------------------ 128-bit fixed point
// A non-negative value v is held as the unsigned 128-bit integer
// round(v / 2^q); sums of such integers are exact and independent of order.
struct U128 {
  unsigned long long lo, hi;
};

__device__ __forceinline__ void add128(U128 &a, unsigned long long lo, unsigned long long hi) {
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(a.hi) : "l"(lo), "l"(hi));
}

// x: finite, >= 0.  The caller picks q so that x / 2^q < 2^127.  Values whose
// last mantissa bit is worth at least 2^q convert exactly; smaller ones round
// to the nearest multiple of 2^q (ties up).
__device__ __forceinline__ U128 to_fixed(double x, int q) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  int E = (int)(b >> 52);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (E == 0)
    E = 1;  // subnormal
  else
    m |= 1ull << 52;
  U128 r{0ull, 0ull};
  if (m == 0) return r;
  int s = E - 1075 - q;  // x = m * 2^(E-1075) = (m << s) * 2^q
  if (s >= 64) {
    r.hi = m << (s - 64);
  } else if (s > 0) {
    r.lo = m << s;
    r.hi = m >> (64 - s);
  } else if (s == 0) {
    r.lo = m;
  } else {
    int rs = -s;
    if (rs <= 53) r.lo = (m + (1ull << (rs - 1))) >> rs;
  }
  return r;
}

// Correctly rounded binary64 value of a * 2^q.
__device__ __forceinline__ double from_fixed(U128 a, int q) {
  if ((a.hi | a.lo) == 0ull) return 0.0;
  int lz = a.hi ? __clzll((long long)a.hi) : 64 + __clzll((long long)a.lo);
  unsigned long long top, rest;
  if (lz == 0) {
    top = a.hi;
    rest = a.lo;
  } else if (lz < 64) {
    top = (a.hi << lz) | (a.lo >> (64 - lz));
    rest = a.lo << lz;
  } else if (lz == 64) {
    top = a.lo;
    rest = 0ull;
  } else {
    top = a.lo << (lz - 64);
    rest = 0ull;
  }
  top |= (rest != 0ull) ? 1ull : 0ull;  // sticky bit keeps round-to-nearest-even exact
  double d = __ull2double_rn(top);
  return ldexp(d, q + 64 - lz);
}

// The same value computed with integer instructions only (B300 issues FP64
// at a small fraction of its integer rate): round the 128-bit integer to 53
// significant bits, nearest-even, and assemble the binary64 bit pattern.
// Results that would be subnormal or overflow take the FP64 path above.
__device__ __forceinline__ double from_fixed_int(U128 a, int q) {
  if ((a.hi | a.lo) == 0ull) return 0.0;
  const int lz = a.hi ? __clzll((long long)a.hi) : 64 + __clzll((long long)a.lo);
  unsigned long long top, rest;
  if (lz == 0) {
    top = a.hi;
    rest = a.lo;
  } else if (lz < 64) {
    top = (a.hi << lz) | (a.lo >> (64 - lz));
    rest = a.lo << lz;
  } else if (lz == 64) {
    top = a.lo;
    rest = 0ull;
  } else {
    top = a.lo << (lz - 64);
    rest = 0ull;
  }
  unsigned long long mant = top >> 11;           // 53 bits, bit 52 set
  const unsigned long long low = top & 0x7FFull;  // the 11 bits below
  const bool half = low == 0x400ull && rest == 0ull;
  const bool up = low > 0x400ull || (low == 0x400ull && rest != 0ull) || (half && (mant & 1ull));
  mant += up ? 1ull : 0ull;
  int e2 = 127 - lz + q;  // value in [2^e2, 2^(e2+1)) before rounding
  if (mant == (1ull << 53)) {
    mant >>= 1;
    ++e2;
  }
  const int biased = e2 + 1023;
  if (biased <= 0 || biased >= 2047) return from_fixed(a, q);
  return __longlong_as_double((long long)(((unsigned long long)biased << 52) |
                                          (mant & 0xFFFFFFFFFFFFFull)));
}

// from_fixed_int for an integer of at most 53 significant bits (every single
// table entry: to_fixed keeps one binary64 mantissa), which converts without
// rounding: the same bits as from_fixed_int, with no rounding logic and no
// branches on the common path.
__device__ __forceinline__ double from_fixed_exact(U128 a, int q) {
  const bool h = a.hi != 0ull;
  const int lzh = __clzll((long long)a.hi), lzl = __clzll((long long)a.lo);
  const int lz = h ? lzh : 64 + lzl;
  // the 64 bits from the leading one down ((lo >> (63 - lzh)) >> 1 is lo >> (64 - lzh), 0 for lzh = 0)
  const unsigned long long top = h ? (a.hi << lzh) | ((a.lo >> (63 - lzh)) >> 1) : a.lo << (lzl & 63);
  const int biased = 127 - lz + q + 1023;
  if ((a.hi | a.lo) == 0ull) return 0.0;
  if (biased <= 0 || biased >= 2047) return from_fixed(a, q);
  return __longlong_as_double((long long)(((unsigned long long)biased << 52) | ((top >> 11) & 0xFFFFFFFFFFFFFull)));
}

// a >= b for 128-bit unsigned integers.
__device__ __forceinline__ bool ge128(U128 a, U128 b) {
  return a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo);
}

__device__ __forceinline__ U128 sub128(U128 a, U128 b) {
  U128 r = a;
  asm("sub.cc.u64 %0, %0, %2;\n\tsubc.u64 %1, %1, %3;" : "+l"(r.lo), "+l"(r.hi) : "l"(b.lo), "l"(b.hi));
  return r;
}

// Aggregate terms of a layer on the 128-bit fixed-point grid of its table.
// exact = 1 when AggR and AggL lie exactly on that grid (or AggL is beyond
// any trial sum), so min(max(S - AggR, 0), AggL) is computed exactly in
// integers and rounded once; otherwise the FP64 clamp is used.
struct AggFixed {
  U128 ret;
  U128 lim;
  int exact;
};

// Trial loss from the exact trial sum S (Section III step 4).
__device__ __forceinline__ double trial_loss(U128 S, int q, const AggFixed &af, double agg_ret,
                                             double agg_lim) {
  if (af.exact) {
    U128 d{0ull, 0ull};
    if (ge128(S, af.ret)) d = sub128(S, af.ret);
    if (ge128(d, af.lim)) d = af.lim;
    return from_fixed_int(d, q);
  }
  const double Sv = from_fixed(S, q);
  return fmin(fmax(__dsub_rn(Sv, agg_ret), 0.0), agg_lim);
}

__device__ __forceinline__ U128 shfl_xor_u128(U128 v, int m) {
  U128 r;
  r.lo = __shfl_xor_sync(0xFFFFFFFFu, v.lo, m);
  r.hi = __shfl_xor_sync(0xFFFFFFFFu, v.hi, m);
  return r;
}

__device__ __forceinline__ U128 warp_sum_u128(U128 v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    U128 o = shfl_xor_u128(v, m);
    add128(v, o.lo, o.hi);
  }
  return v;
}

// SM count of the current device (queried once per device; 148 on B300), for
// grids sized in multiples of the SMs.
int current_sm_count();

// --------------------------------------------------------- launchers
// Each returns cudaSuccess or the launch error.
// f64_out (nullable) gets every event's binary64 value; with inexact given,
// zeros are written as +0 and inexact is set when some value is not exactly
// on the fixed-point grid of q.
cudaError_t launch_fold(const EltDesc *d_elts, int n_elts, int32_t catalog, double occ_ret,
                        double occ_lim, int q, void *table, uint32_t *bitmap,
                        BitmapLayout bm, bool fp32, double *f64_out, cudaStream_t s,
                        unsigned int *inexact = nullptr);

struct YltLaunch {
  int blocks;
  int threads;          // 1024 (64 registers a thread) or 768 (85)
  size_t smem;
  int unroll;           // 16-byte id loads in flight per lane
  int lanes_per_trial;  // 16 or 32: a warp sums 32 / lanes_per_trial trials at once
  int prefetch;         // 1: bulk-prefetch the next trials' ids into L2
};

// Launch-shape choice for the YLT kernel (0 = the planner's default).
struct YltShape {
  int unroll = 0;
  int lanes_per_trial = 0;
  int prefetch = -1;  // 0 off, 1 on, -1 the planner's choice
  int threads = 0;    // threads per CTA (1024 or 768; 0 = the planner's choice)
};

// Per-layer constants and output of one YLT kernel launch.
struct LayerOut {
  int q;             // fixed-point exponent of the layer's table
  AggFixed af;       // aggregate terms on the table's grid
  double agg_ret;
  double agg_lim;
  double *ylt;       // device output, one value per trial
};

// coff/chunks: the chunked YET layout written by launch_pad_ids (layout 1:
// 6 ids of 21 bits per chunk, layout 0: 4 plain ids) or by the compact
// builder (layout 2: per trial, 6 packed ids or 8 difference-coded ids, the
// choice in bit 62 of the trial's offset); sentinel = catalog size (its
// table entry is zero).  entry_bytes = 16 for FP64 layers (128-bit
// fixed-point entries) or 8 for FP32-table layers (64-bit entries whose trial
// sums stay below 2^64); G layers' tables interleaved (entry_bytes x G <= 32
// bytes per event, one L2 sector) with the union of their bitmaps.
cudaError_t launch_ylt_group(const int64_t *coff, const int4 *chunks, int layout, int64_t n_trials,
                             const void *table, int entry_bytes, const uint32_t *bitmap, BitmapLayout bm,
                             int32_t sentinel, int G, const LayerOut *outs, const YltLaunch &cfg,
                             cudaStream_t s);

// Pick the launch shape of the YLT kernel for a bitmap of bm.words words and
// trials of mean_chunks 16-byte chunks and a (possibly interleaved) table of
// table_bytes; fields of hint force the unroll (1/2), the lanes per trial
// (16/32) or the L2 prefetch (0/1).  entry_bytes x G <= 32.
cudaError_t plan_ylt(int device, const BitmapLayout &bm, double mean_chunks, int layout, int entry_bytes,
                     int G, size_t table_bytes, YltShape hint, YltLaunch *out);

// Up to four layers' tables and bitmaps for launch_interleave.
struct Tables4 {
  const void *t[4];
};
struct Bitmaps4 {
  const uint32_t *b[4];
};
cudaError_t launch_interleave(const Tables4 &in, int entry_bytes, int G, int64_t entries, void *out,
                              const Bitmaps4 &bin, int32_t words, uint32_t *bout, cudaStream_t s);

// Compact (sorted, difference-coded) id stream for YLT passes (compact.cu).
constexpr int64_t kCompactOffsetMask = ((int64_t)1 << 62) - 1;
int4 delta_sentinel_chunk(int32_t sentinel);  // 8 empty slots after the sentinel id
// Reorder each trial's ids (6-per-chunk layout coff/chunks) into sorted (raw
// CSR layout) so that every group of 8 ascends, and write count_flag[t] =
// chunk count | (1 << 62 when the trial is difference-coded).
cudaError_t launch_compact_sort(const int64_t *raw_off, const int64_t *coff, const int4 *chunks, int64_t n_trials,
                                uint32_t *sorted, int64_t *count_flag, cudaStream_t s);
// Exclusive scan of count_flag (n_trials + 1 entries of room) into dcoff
// (flag kept, n_trials + 1 entries) and, in place, the plain offsets; bsum
// is scratch of kCompactScanScratch entries.
constexpr int kCompactScanScratch = 1025;
cudaError_t launch_compact_scan(int64_t *count_plain, int64_t n_trials, int64_t *dcoff, int64_t *bsum,
                                cudaStream_t s);
// Write the compact stream at dcoff (offsets with the flag in bit 62), plus
// kChunkTail tail chunks.
cudaError_t launch_compact_encode(const int64_t *raw_off, const int64_t *coff, const int4 *chunks, int64_t n_trials,
                                  const uint32_t *sorted, const int64_t *dcoff, int4 *dchunks, cudaStream_t s);

// ELT ingest (ingest.cu): check the entries of n_elts ELTs (CSR by d_off,
// device), group each ELT by fold bucket into s_ids / s_losses (same CSR) and
// write the bucket index bucket[j][0..nb]; per ELT the largest loss (as
// binary64 bits) and id; bad[0..2] count ids outside the catalog, losses not
// finite and >= 0, and ids repeated within an ELT.  seen, count and the
// maxima start zeroed (max_id at -1).
cudaError_t launch_elt_ingest(const int64_t *d_off, int n_elts, int64_t total, const int32_t *d_raw_ids,
                              const double *d_raw_losses, int32_t catalog, int nb, uint32_t *seen,
                              int64_t seen_words, int32_t *count, int32_t *cursor, int32_t *bucket,
                              unsigned long long *max_loss, int *max_id, unsigned long long *bad,
                              int32_t *s_ids, double *s_losses, cudaStream_t s);

cudaError_t launch_pad_ids(const int32_t *src, const int64_t *off, const int64_t *coff,
                           int64_t n_trials, int4 *dst, int32_t catalog, bool packed,
                           unsigned long long *bad_count, cudaStream_t s);

cudaError_t launch_check_ts(const int64_t *offsets, int64_t n_trials, const float *ts,
                            unsigned long long *bad_count, cudaStream_t s);

// Year Event Loss Table of one layer: per-occurrence increments into
// yelt[raw_off[t] + k] (nullable), each trial's largest increment into
// occ_max[t] (nullable), and the trial loss into L.ylt[t] (nullable).
// With yelt, comb (required) is the layer's table with each event's binary64
// value interleaved (launch_yelt_comb), so one gather brings both; while
// *inexact (device) is 0 the binary64 values are exactly the entries' and an
// in-layer increment is read instead of converted.
cudaError_t launch_yelt(const int64_t *coff, const int4 *chunks, const int64_t *raw_off, bool packed,
                        int64_t n_trials, const void *table, int entry_bytes, const uint32_t *bitmap,
                        BitmapLayout bm, int32_t sentinel, const LayerOut &L, double *yelt, double *occ_max,
                        int device, cudaStream_t s, const ulonglong2 *comb = nullptr,
                        const unsigned int *inexact = nullptr);

// Interleave n_events table entries (entry_bytes 16 or 8) with their binary64
// values table64[e]: comb holds {lo, hi} {value, 0} per event for 16-byte
// entries (32 bytes: one sector) and {entry, value} for 8-byte entries.
cudaError_t launch_yelt_comb(const void *table, int entry_bytes, const double *table64, int64_t n_events,
                             ulonglong2 *comb, cudaStream_t s);

// PML/TVaR on the device.  ws must hold select_workspace_bytes(n_rp) bytes
// per layer; the batch form reads n_layers YLTs of n values each (layer-major)
// and writes 2*n_rp values per layer (PML then TVaR).
size_t select_workspace_bytes(int n_rp);
// Upper bound of select_workspace_bytes() for any n_rp <= kMaxReturnPeriods.
constexpr size_t kSelectWorkspaceMax = 32 * 1024;
// Record the message of a failed call that has no context (read back with
// ara_last_error(NULL)).
void set_context_free_error(const char *msg);
// q_count (>= n when given) sets the fixed-point scale of the tail sums as
// if that many values were summed: the tail form (ara_pml_tvar_tail) passes
// the full YLT's trial count, so its sums use the scale the full YLT's would.
cudaError_t launch_pml_tvar(const double *ylt, int64_t n, const int64_t *k, int n_rp,
                            void *ws, double *out_pml_tvar /* device, 2*n_rp */,
                            unsigned int *err_flag, int device, cudaStream_t s, int64_t q_count = 0);
cudaError_t launch_pml_tvar_batch(const double *ylts, int n_layers, int64_t n, const int64_t *k,
                                  int n_rp, void *ws, double *out, unsigned int *err_flag,
                                  int device, cudaStream_t s, int64_t q_count = 0);

// The k largest of n values (tail.cu): tau (device) is the k-th largest, as
// the selection wrote it; out gets the values above tau in index order, then
// copies of tau, k in all.  scratch holds kTailScratch entries.
constexpr int kTailScratch = 1024;
cudaError_t launch_ylt_tail(const double *y, int64_t n, int64_t k, const double *tau, int64_t *scratch,
                            double *out, cudaStream_t s);

}  // namespace ara
