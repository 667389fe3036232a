// The k largest values of a Year Loss Table, for the exchange between trial
// shards.  Section IV-C splits the trials of one analysis over several GPUs;
// PML and TVaR at return period RP read only the floor(N / RP) largest of
// the N trial losses, and the k largest values of a union of shards lie in
// the union of each shard's k largest.  So shards that send their
// floor(N_total / RP_min) largest values send everything the portfolio-wide
// PML and TVaR need, instead of whole YLTs.
//
// tau = the k-th largest value (found by the selection of select.cu); the
// output holds the values above tau in index order, then k - count copies
// of tau.  Values compare as binary64 bit patterns, as in the selection
// (trial losses are finite and >= 0, so the patterns order like the values).
#include <algorithm>

#include "ara_internal.cuh"

namespace ara {

namespace {

constexpr int kTailThreads = 1024;

__device__ __forceinline__ unsigned long long key_of(double v) {
  return (unsigned long long)__double_as_longlong(v);
}

// Block b counts the values above tau in [b * per, (b + 1) * per).
__global__ void __launch_bounds__(kTailThreads)
tail_count_kernel(const double *__restrict__ y, int64_t n, int64_t per, const double *__restrict__ tau_p,
                  int64_t *__restrict__ bcnt) {
  __shared__ int64_t s_warp[kTailThreads / 32];
  const unsigned long long tau = key_of(*tau_p);
  const int64_t a = (int64_t)blockIdx.x * per, e = min(a + per, n);
  int64_t c = 0;
  for (int64_t i = a + threadIdx.x; i < e; i += kTailThreads) c += key_of(y[i]) > tau;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t sum = 0;
    for (int w = 0; w < kTailThreads / 32; ++w) sum += s_warp[w];
    bcnt[blockIdx.x] = sum;
  }
}

// One CTA: the block counts (nb <= kTailThreads) become block offsets in
// place; the slots after the last value above tau get copies of tau.
__global__ void __launch_bounds__(kTailThreads)
tail_offsets_kernel(int64_t *bcnt, int nb, const double *__restrict__ tau_p, int64_t k, double *__restrict__ out) {
  __shared__ int64_t s_warp[kTailThreads / 32];
  __shared__ int64_t s_total;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t own = tid < nb ? bcnt[tid] : 0;
  int64_t incl = own;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  int64_t run = incl - own;
  for (int w = 0; w < wid; ++w) run += s_warp[w];
  if (tid == kTailThreads - 1) s_total = run + own;
  __syncthreads();
  if (tid < nb) bcnt[tid] = run;
  const double tau = *tau_p;
  for (int64_t j = s_total + tid; j < k; j += kTailThreads) out[j] = tau;
}

// Block b writes its values above tau from offset boff[b], in index order.
__global__ void __launch_bounds__(kTailThreads)
tail_write_kernel(const double *__restrict__ y, int64_t n, int64_t per, const double *__restrict__ tau_p,
                  const int64_t *__restrict__ boff, int64_t k, double *__restrict__ out) {
  __shared__ int s_warp[kTailThreads / 32];
  const unsigned long long tau = key_of(*tau_p);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t a = (int64_t)blockIdx.x * per, e = min(a + per, n);
  int64_t base = boff[blockIdx.x];
  for (int64_t t0 = a; t0 < e; t0 += kTailThreads) {
    const int64_t i = t0 + tid;
    const double v = i < e ? y[i] : 0.0;
    const bool f = i < e && key_of(v) > tau;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, f);
    if (lane == 0) s_warp[wid] = __popc(bal);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < kTailThreads / 32; ++w) {
      const int c = s_warp[w];
      off += w < wid ? c : 0;
      tot += c;
    }
    const int64_t pos = base + off + __popc(bal & ((1u << lane) - 1u));
    if (f && pos < k) out[pos] = v;  // pos < k always holds when tau is the k-th largest
    base += tot;
    __syncthreads();  // s_warp is rewritten by the next tile
  }
}

}  // namespace

cudaError_t launch_ylt_tail(const double *y, int64_t n, int64_t k, const double *tau, int64_t *scratch,
                            double *out, cudaStream_t s) {
  int64_t nb = (n + kTailThreads - 1) / kTailThreads;
  // four blocks per SM, and no more block counts than the offsets kernel's
  // threads (and the scratch) hold
  const int64_t cap = std::min<int64_t>((int64_t)current_sm_count() * 4, std::min(kTailThreads, kTailScratch));
  if (nb > cap) nb = cap;
  if (nb < 1) nb = 1;
  const int64_t per = (n + nb - 1) / nb > 0 ? (n + nb - 1) / nb : 1;
  nb = (n + per - 1) / per > 0 ? (n + per - 1) / per : 1;
  tail_count_kernel<<<(unsigned)nb, kTailThreads, 0, s>>>(y, n, per, tau, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tail_offsets_kernel<<<1, kTailThreads, 0, s>>>(scratch, (int)nb, tau, k, out);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  tail_write_kernel<<<(unsigned)nb, kTailThreads, 0, s>>>(y, n, per, tau, scratch, k, out);
  return cudaGetLastError();
}

}  // namespace ara
