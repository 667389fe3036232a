// Device-side ingest of Event Loss Tables (Section III: an ELT is a set of
// (event id, loss) pairs; Section IV-B: losses are found by event id).
//
// For the fold pre-pass every ELT is grouped by fold bucket (kFoldEventsPerCta
// consecutive catalog events): a counting sort by bucket -- count, scan,
// scatter -- so the CTA that folds a bucket finds the bucket's entries of
// each ELT with two loads.  Entries inside a bucket keep no particular
// order: an ELT holds each event at most once, so each catalog event gets at
// most one addition per ELT and the fold's sums do not depend on that order.
// The same pass checks every id against the catalog, every loss (finite,
// >= 0) and every ELT for a repeated event (one bit per catalog event and
// ELT), and records each ELT's largest loss and largest id.
#include "ara_internal.cuh"

namespace ara {

namespace {

// The ELT of entry i: largest j with off[j] <= i (off has n_elts + 1 entries).
__device__ __forceinline__ int elt_of(const int64_t *off, int n_elts, int64_t i) {
  int lo = 0, hi = n_elts;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void elt_count_kernel(const int64_t *__restrict__ off, int n_elts, const int32_t *__restrict__ ids,
                                 const double *__restrict__ losses, int32_t catalog, int nb,
                                 uint32_t *__restrict__ seen, int64_t seen_words, int32_t *__restrict__ count,
                                 unsigned long long *__restrict__ max_loss, int *__restrict__ max_id,
                                 unsigned long long *__restrict__ bad) {
  const int64_t total = off[n_elts];
  const int lane = threadIdx.x & 31;
  unsigned long long n_range = 0, n_loss = 0, n_dup = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // Warp-uniform loop: a warp takes 32 consecutive entries, which almost
  // always belong to one ELT, so the per-ELT maxima are reduced in the warp
  // before one atomic (thousands of entries share each ELT's address).
  for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < total; w0 += stride) {
    const int64_t i = w0 + lane;
    const bool in = i < total;
    int j = -1;
    unsigned long long lbits = 0ull;
    int e = -1;
    if (in) {
      j = elt_of(off, n_elts, i);
      e = ids[i];
      const double l = losses[i];
      if (e < 0 || e >= catalog) {
        ++n_range;
        e = -1;
      } else {
        if (!(l >= 0.0) || isinf(l)) ++n_loss;  // NaN, negative or infinite
        else lbits = (unsigned long long)__double_as_longlong(l);
        const uint32_t bit = 1u << (e & 31);
        if (atomicOr(&seen[(size_t)j * (size_t)seen_words + (e >> 5)], bit) & bit) ++n_dup;
        atomicAdd(&count[(size_t)j * (size_t)(nb + 1) + e / kFoldEventsPerCta], 1);
      }
    }
    const int j0 = __shfl_sync(0xFFFFFFFFu, j, 0);
    if (__all_sync(0xFFFFFFFFu, j == j0 || !in) && j0 >= 0) {
      unsigned long long mb = lbits;
      int me = e;
      for (int m = 16; m > 0; m >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xFFFFFFFFu, mb, m);
        const int oe = __shfl_xor_sync(0xFFFFFFFFu, me, m);
        mb = ob > mb ? ob : mb;
        me = oe > me ? oe : me;
      }
      if (lane == 0) {
        if (mb) atomicMax(&max_loss[j0], mb);
        if (me >= 0) atomicMax(&max_id[j0], me);
      }
    } else if (in && j >= 0) {
      if (lbits) atomicMax(&max_loss[j], lbits);
      if (e >= 0) atomicMax(&max_id[j], e);
    }
  }
  if (n_range) atomicAdd(&bad[0], n_range);
  if (n_loss) atomicAdd(&bad[1], n_loss);
  if (n_dup) atomicAdd(&bad[2], n_dup);
}

// One CTA per ELT: exclusive scan of its bucket counts into the bucket index
// (bucket[j][b] = first sorted position of bucket b, relative to the ELT),
// and the same offsets as the scatter cursors.
__global__ void elt_scan_kernel(int nb, const int32_t *__restrict__ count, int32_t *__restrict__ bucket,
                                int32_t *__restrict__ cursor) {
  __shared__ int32_t s_carry;
  __shared__ int32_t s_warp[32];
  const int j = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int32_t *c = count + (size_t)j * (size_t)(nb + 1);
  int32_t *bk = bucket + (size_t)j * (size_t)(nb + 1);
  int32_t *cur = cursor + (size_t)j * (size_t)(nb + 1);
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < nb + 1; base += blockDim.x) {
    const int b = base + tid;
    const int32_t v = b < nb ? c[b] : 0;
    int32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    int32_t warp_off = 0;
    for (int w = 0; w < wid; ++w) warp_off += s_warp[w];
    const int32_t excl = s_carry + warp_off + incl - v;
    if (b < nb + 1) {
      bk[b] = excl;
      cur[b] = excl;
    }
    __syncthreads();
    if (tid == blockDim.x - 1) s_carry = excl + v;
    __syncthreads();
  }
}

__global__ void elt_scatter_kernel(const int64_t *__restrict__ off, int n_elts, const int32_t *__restrict__ ids,
                                   const double *__restrict__ losses, int32_t catalog, int nb,
                                   int32_t *__restrict__ cursor, int32_t *__restrict__ s_ids,
                                   double *__restrict__ s_losses) {
  const int64_t total = off[n_elts];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int32_t e = ids[i];
    if (e < 0 || e >= catalog) continue;  // reported by the count pass
    const int j = elt_of(off, n_elts, i);
    const int32_t pos = atomicAdd(&cursor[(size_t)j * (size_t)(nb + 1) + e / kFoldEventsPerCta], 1);
    s_ids[off[j] + pos] = e;
    s_losses[off[j] + pos] = losses[i];
  }
}

}  // namespace

cudaError_t launch_elt_ingest(const int64_t *d_off, int n_elts, int64_t total, const int32_t *d_raw_ids,
                              const double *d_raw_losses, int32_t catalog, int nb, uint32_t *seen,
                              int64_t seen_words, int32_t *count, int32_t *cursor, int32_t *bucket,
                              unsigned long long *max_loss, int *max_id, unsigned long long *bad,
                              int32_t *s_ids, double *s_losses, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t want = (total + threads - 1) / threads;
  const int64_t cap = (int64_t)current_sm_count() * 16;
  const int blocks = (int)(want < cap ? want : cap);
  elt_count_kernel<<<blocks, threads, 0, s>>>(d_off, n_elts, d_raw_ids, d_raw_losses, catalog, nb, seen,
                                             seen_words, count, max_loss, max_id, bad);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  elt_scan_kernel<<<n_elts, 1024, 0, s>>>(nb, count, bucket, cursor);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  elt_scatter_kernel<<<blocks, threads, 0, s>>>(d_off, n_elts, d_raw_ids, d_raw_losses, catalog, nb, cursor, s_ids,
                                               s_losses);
  return cudaGetLastError();
}

}  // namespace ara
