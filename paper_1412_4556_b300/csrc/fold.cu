// Per-layer pre-pass: fold the layer's ELT terms and occurrence terms into
// one table over the catalog.
//
// Algorithm 1 (Section III), steps 1-3, depend only on the event id, so for
// every catalog event e the occurrence-net loss
//     o(e) = FT2( sum over the layer's ELTs j, in layer order, of FT1_j(DAT_j[e]) )
// is computed once here instead of once per occurrence.  DAT_j[e] is the
// ELT's loss for e, or 0 when e is absent (Section IV-B, direct access
// tables); an absent ELT adds FT1_j(0) = +0.0, which leaves the running sum's
// bits unchanged, so only the present entries are added -- in layer order --
// and the result is bit-identical to the sequential per-event ELT loop.
//
// One CTA owns kFoldEventsPerCta consecutive catalog events and keeps their
// running sums in shared memory.  Each ELT is stored sorted by event id with
// a bucket index, so the CTA finds its slice of every ELT with two loads.
// Outputs per event: the fixed-point table entry used by the YLT kernel, one
// bit of the zero-skip bitmap, and (optionally) the FP64 value.  FP64 layers
// store round(o / 2^q) as a 128-bit integer (exact for every value the grid
// can hold).  Reduced-precision layers run the same steps in binary32 (the
// paper's choice of binary32 wherever it can, Section IV-B) and store 64-bit
// entries on a grid chosen so that no trial sum reaches 2^64: half the table
// bytes; rounding to that grid moves a trial sum by less than its length x
// 2^(q-1), far below the binary32 rounding of the values themselves.
#include <algorithm>
#include <type_traits>

#include "ara_internal.cuh"
#include "fold_batch.h"

namespace ara {

__device__ __forceinline__ double elt_terms(double loss, double deductible, double limit) {
  // FT1 read as deductible then limit: min(max(l - D, 0), Lim)
  return fmin(fmax(__dsub_rn(loss, deductible), 0.0), limit);
}

// FP32 variant (reduced-precision layers): losses and terms rounded to
// binary32, the same operations in binary32.
__device__ __forceinline__ float elt_terms32(double loss, double deductible, double limit) {
  return fminf(fmaxf(__fsub_rn(__double2float_rn(loss), __double2float_rn(deductible)), 0.f),
               __double2float_rn(limit));
}

// ELT entries staged in shared memory per round (a bucket of a typical layer
// fits in one round).
constexpr int kStage = 1024;

// Shared memory of one fold CTA: the running sums of its events and one
// round of staged ELT entries.
template <typename Real>
struct FoldSmem {
  Real x[kFoldEventsPerCta];
  uint16_t st_off[kStage];
  Real st_val[kStage];
};

// One CTA's fold of catalog events [b * kFoldEventsPerCta, ...).  FP32 = true:
// combine and apply occurrence terms in binary32 (the table then holds
// binary32 values, exactly representable in the fixed-point grid).  s_dyn:
// 2 * n_elts + 1 ints of dynamic shared memory.
template <bool FP32>
__device__ __forceinline__ void fold_body(
    FoldSmem<typename std::conditional<FP32, float, double>::type> &sm, int32_t *s_dyn, int b,
    const EltDesc *__restrict__ elts, int n_elts, int32_t catalog, double occ_ret, double occ_lim, int q,
    void *__restrict__ table, uint32_t *__restrict__ bitmap, uint32_t bm_mul, double *__restrict__ f64_out,
    unsigned int *__restrict__ inexact, int stride) {
  using Real = typename std::conditional<FP32, float, double>::type;
  Real *x = sm.x;
  uint16_t *st_off = sm.st_off;
  Real *st_val = sm.st_val;
  int32_t *seg = s_dyn;                // prefix sums of slice lengths
  int32_t *first = s_dyn + n_elts + 1;  // slice start inside ELT j

  const int tid = threadIdx.x;
  const int32_t e0 = b * kFoldEventsPerCta;

  for (int i = tid; i < kFoldEventsPerCta; i += kFoldThreads) x[i] = Real(0);
  for (int j = tid; j < n_elts; j += kFoldThreads) {
    const EltDesc d = elts[j];
    int32_t a = d.count, z = d.count;
    if (b < d.nb) {
      a = d.bucket[b];
      z = d.bucket[b + 1];
    }
    first[j] = a;
    seg[j + 1] = z - a;
  }
  __syncthreads();
  if (tid == 0) {
    seg[0] = 0;
    for (int j = 0; j < n_elts; ++j) seg[j + 1] += seg[j];
  }
  __syncthreads();
  const int32_t total = seg[n_elts];

  for (int32_t base = 0; base < total; base += kStage) {
    const int32_t end = min(total, base + kStage);
    for (int32_t f = base + tid; f < end; f += kFoldThreads) {
      int lo = 0, hi = n_elts;  // find j with seg[j] <= f < seg[j+1]
      while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (seg[mid] <= f) lo = mid; else hi = mid;
      }
      const EltDesc &d = elts[lo];
      const int32_t i = first[lo] + (f - seg[lo]);
      st_off[f - base] = (uint16_t)(d.ids[i] - e0);
      if constexpr (FP32)
        st_val[f - base] = elt_terms32(d.losses[i], d.deductible, d.limit);
      else
        st_val[f - base] = elt_terms(d.losses[i], d.deductible, d.limit);
    }
    __syncthreads();
    // Apply the staged entries ELT by ELT, in layer order.  Within one ELT
    // the event ids are distinct, so its entries touch distinct sums.
    int j = 0;
    while (seg[j + 1] <= base) ++j;
    for (; j < n_elts && seg[j] < end; ++j) {
      const int32_t lo = max(seg[j], base), hi = min(seg[j + 1], end);
      if (lo >= hi) continue;  // uniform across the CTA
      for (int32_t f = lo + tid; f < hi; f += kFoldThreads) {
        const int o = st_off[f - base];
        if constexpr (FP32)
          x[o] = __fadd_rn(x[o], st_val[f - base]);
        else
          x[o] = __dadd_rn(x[o], st_val[f - base]);
      }
      __syncthreads();
    }
    __syncthreads();
  }

  for (int i = tid; i < kFoldEventsPerCta; i += kFoldThreads) {
    const int32_t e = e0 + i;
    if (e >= catalog) break;
    // FT2 read as occurrence retention then limit: min(max(x - OccR, 0), OccL)
    double o;
    if constexpr (FP32)
      o = (double)fminf(fmaxf(__fsub_rn(x[i], __double2float_rn(occ_ret)), 0.f),
                        __double2float_rn(occ_lim));
    else
      o = fmin(fmax(__dsub_rn(x[i], occ_ret), 0.0), occ_lim);
    if (inexact) {
      o = o == 0.0 ? 0.0 : o;  // +0: what the conversion of a zero entry gives
      const U128 v = to_fixed(o, q);
      if (__double_as_longlong(from_fixed_exact(v, q)) != __double_as_longlong(o)) atomicOr(inexact, 1u);
    }
    if (f64_out) f64_out[e] = o;
    if (table) {
      const U128 v = to_fixed(o, q);
      if constexpr (FP32)
        static_cast<unsigned long long *>(table)[(size_t)e * stride] = v.lo;  // v.hi = 0 on this grid
      else
        static_cast<ulonglong2 *>(table)[(size_t)e * stride] = make_ulonglong2(v.lo, v.hi);
      if ((v.lo | v.hi) != 0ull) {
        atomicOr(bitmap + bitmap_word((uint32_t)e, bm_mul), 1u << (e & 31));
      }
    }
  }
}


template <bool FP32>
__global__ void __launch_bounds__(kFoldThreads)
fold_kernel(const EltDesc *__restrict__ elts, int n_elts, int32_t catalog, double occ_ret,
            double occ_lim, int q, void *__restrict__ table, uint32_t *__restrict__ bitmap,
            uint32_t bm_mul, double *__restrict__ f64_out, unsigned int *__restrict__ inexact) {
  using Real = typename std::conditional<FP32, float, double>::type;
  __shared__ FoldSmem<Real> sm;
  // sized by the layer (n_elts + 1 and n_elts entries), so that a CTA of a
  // typical layer needs little shared memory and the whole grid is resident
  extern __shared__ int32_t s_dyn[];
  fold_body<FP32>(sm, s_dyn, blockIdx.x, elts, n_elts, catalog, occ_ret, occ_lim, q, table, bitmap, bm_mul,
                  f64_out, inexact, 1);
}

// Many layers' folds in one launch (grid.y = layer): the CTAs of all the
// layers are resident together, where one launch per layer leaves each
// layer's short dependent chains to run on an otherwise idle GPU.
__global__ void __launch_bounds__(kFoldThreads)
fold_batch_kernel(const FoldJob *__restrict__ jobs, int32_t catalog) {
  __shared__ __align__(16) unsigned char raw[sizeof(FoldSmem<double>)];
  extern __shared__ int32_t s_dyn[];
  const FoldJob j = jobs[blockIdx.y];
  if (j.fp32)
    fold_body<true>(*reinterpret_cast<FoldSmem<float> *>(raw), s_dyn, blockIdx.x, j.elts, j.n_elts, catalog,
                    j.occ_ret, j.occ_lim, j.q, j.table, j.bitmap, j.bm_mul, nullptr, nullptr, j.stride);
  else
    fold_body<false>(*reinterpret_cast<FoldSmem<double> *>(raw), s_dyn, blockIdx.x, j.elts, j.n_elts, catalog,
                     j.occ_ret, j.occ_lim, j.q, j.table, j.bitmap, j.bm_mul, nullptr, nullptr, j.stride);
}

// Before a batch of folds: every layer's bitmap cleared and its sentinel
// entry (id = catalog) zeroed at the layer's entry width.
__global__ void fold_clear_kernel(const FoldJob *__restrict__ jobs, int32_t catalog, int32_t words) {
  const FoldJob j = jobs[blockIdx.y];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) j.bitmap[i] = 0u;
  const int per = j.fp32 ? 1 : 2;  // 64-bit words of one entry
  if (blockIdx.x == 0 && (int)threadIdx.x < per)
    static_cast<unsigned long long *>(j.table)[(size_t)catalog * j.stride * per + threadIdx.x] = 0ull;
}

cudaError_t launch_fold(const EltDesc *d_elts, int n_elts, int32_t catalog, double occ_ret,
                        double occ_lim, int q, void *table, uint32_t *bitmap,
                        BitmapLayout bm, bool fp32, double *f64_out, cudaStream_t s, unsigned int *inexact) {
  if (catalog <= 0) return cudaSuccess;
  const int blocks = (catalog + kFoldEventsPerCta - 1) / kFoldEventsPerCta;
  const size_t dyn = (2 * (size_t)n_elts + 1) * sizeof(int32_t);  // at most 8 KB (kMaxLayerElts)
  if (fp32)
    fold_kernel<true><<<blocks, kFoldThreads, dyn, s>>>(d_elts, n_elts, catalog, occ_ret, occ_lim, q,
                                                         table, bitmap, bm.mul, f64_out, inexact);
  else
    fold_kernel<false><<<blocks, kFoldThreads, dyn, s>>>(d_elts, n_elts, catalog, occ_ret, occ_lim, q,
                                                          table, bitmap, bm.mul, f64_out, inexact);
  return cudaGetLastError();
}

cudaError_t launch_fold_batch(const FoldJob *d_jobs, int n_jobs, int max_elts, int32_t catalog, int32_t words,
                              cudaStream_t s) {
  if (catalog <= 0 || n_jobs <= 0) return cudaSuccess;
  const int sms = current_sm_count();
  fold_clear_kernel<<<dim3((unsigned)std::max(1, sms / 4), (unsigned)n_jobs), 256, 0, s>>>(d_jobs, catalog, words);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int blocks = (catalog + kFoldEventsPerCta - 1) / kFoldEventsPerCta;
  const size_t dyn = (2 * (size_t)max_elts + 1) * sizeof(int32_t);
  fold_batch_kernel<<<dim3((unsigned)blocks, (unsigned)n_jobs), kFoldThreads, dyn, s>>>(d_jobs, catalog);
  return cudaGetLastError();
}

}  // namespace ara
