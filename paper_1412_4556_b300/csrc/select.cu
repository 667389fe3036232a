// PML and TVaR from a Year Loss Table (Section III names both as risk
// measures computed from the analysis' output; their definitions below are
// the readings of the Introduction's and Section III's wording).
//
// For each return period r with k_r = floor(n / RP_r):
//   PML_r  = the k_r-th largest trial loss
//   TVaR_r = (sum of the k_r largest trial losses) / k_r
//
// Trial losses are finite and >= 0, so their binary64 bit patterns order like
// the values.  An MSD radix selection (8 passes of 8 bits) finds the exact
// k_r-th largest key tau_r for every r at once: each pass histograms the keys
// that share the prefix chosen so far, and the last CTA to finish a pass
// picks the next digit ("last block done" counter, no waiting).  A threshold
// is known early when its bucket holds a single key (the next pass records
// it), when at least k_r keys tie at the largest (counted in the second
// pass), or when all its remaining candidates are one key (from the fourth
// pass on); once all of a YLT's thresholds are known its remaining passes
// return at once.  A final pass sums the keys above tau_r exactly in 128-bit
// fixed point and adds (k_r - count) copies of tau_r, so ties at the
// threshold are handled exactly; one rounding to binary64 and one division
// give TVaR.
#include "ara_internal.cuh"

namespace ara {

struct SelState {
  unsigned long long prefix[kMaxReturnPeriods];
  long long k_rem[kMaxReturnPeriods];
  long long k[kMaxReturnPeriods];
  unsigned long long cnt_gt[kMaxReturnPeriods];
  unsigned long long acc_lo[kMaxReturnPeriods];
  unsigned long long acc_hi[kMaxReturnPeriods];
  unsigned long long max_key;
  unsigned int done_pass;
  unsigned int done_sum;
  // Early finish: once the bucket a threshold lies in holds a single key
  // (state 1), the next pass records that key (found, per distinct prefix)
  // and the threshold is known (state 2); when every return period is known
  // the remaining passes return at once.
  unsigned long long found[kMaxReturnPeriods];
  unsigned int rstate[kMaxReturnPeriods];
  unsigned int all_done;
  // Keys equal to the largest (counted in the second pass): when at least k
  // losses tie at the top (trials capped at AggL), the k-th largest is the
  // largest, and ties never leave a bucket with a single key.
  unsigned long long cnt_max;
  // From the fourth pass on: the smallest and largest key matching each
  // distinct prefix; equal, they say every candidate is the same loss (a
  // tie below the top), which is then the threshold.
  unsigned long long smin[kMaxReturnPeriods], smax[kMaxReturnPeriods];
  unsigned int hist[kMaxReturnPeriods][256];
};

size_t select_workspace_bytes(int) { return sizeof(SelState); }
static_assert(sizeof(SelState) <= kSelectWorkspaceMax, "selection workspace outgrew its bound");

struct KArgs {
  long long k[kMaxReturnPeriods];
};

__global__ void select_init_kernel(SelState *states, KArgs ka, int n_rp) {
  SelState *st = states + blockIdx.x;
  const int tid = threadIdx.x;
  unsigned int *h = &st->hist[0][0];
  for (int i = tid; i < kMaxReturnPeriods * 256; i += blockDim.x) h[i] = 0u;
  if (tid < kMaxReturnPeriods) {
    const long long k = tid < n_rp ? ka.k[tid] : 1;
    st->prefix[tid] = 0ull;
    st->k_rem[tid] = k;
    st->k[tid] = k;
    st->cnt_gt[tid] = 0ull;
    st->acc_lo[tid] = 0ull;
    st->acc_hi[tid] = 0ull;
    st->found[tid] = 0ull;
    st->rstate[tid] = 0u;
    st->smin[tid] = ~0ull;
    st->smax[tid] = 0ull;
  }
  if (tid == 0) {
    st->max_key = 0ull;
    st->done_pass = 0u;
    st->done_sum = 0u;
    st->all_done = 0u;
    st->cnt_max = 0ull;
  }
}

// FAST: at most four return periods, whose distinct prefixes are compared in
// registers; otherwise they are read from shared memory.
template <bool FAST>
__global__ void __launch_bounds__(kSelectThreads, 4)
select_pass_kernel(const double *__restrict__ ylts, int64_t n, int n_rp, int pass,
                   SelState *states, unsigned int *err) {
  const double *__restrict__ y = ylts + (size_t)blockIdx.y * (size_t)n;
  SelState *st = states + blockIdx.y;
  if (pass > 0 && st->all_done) return;  // every threshold of this layer is known
  __shared__ unsigned int sh[kMaxReturnPeriods][256];
  __shared__ unsigned long long s_prefix[kMaxReturnPeriods];
  __shared__ unsigned long long s_pre[kMaxReturnPeriods];  // distinct prefixes, above the current digit
  __shared__ int s_slot[kMaxReturnPeriods];                // return period -> its prefix's histogram (-1: known)
  __shared__ unsigned int s_state[kMaxReturnPeriods];
  __shared__ int s_nslots;
  __shared__ unsigned int s_find;  // slots whose bucket holds one key, to be recorded
  __shared__ bool s_last;
  const int tid = threadIdx.x;
  for (int i = tid; i < n_rp * 256; i += blockDim.x) (&sh[0][0])[i] = 0u;
  if (tid < n_rp) {
    s_prefix[tid] = st->prefix[tid];
    s_state[tid] = st->rstate[tid];
  }
  __syncthreads();
  const int shift = 56 - 8 * pass;
  // Return periods whose thresholds share the prefix chosen so far (all of
  // them in the first pass) count into one histogram, so a key takes at most
  // one shared-memory atomic: the distinct prefixes select disjoint keys.
  if (tid == 0) {
    int ns = 0;
    unsigned int find = 0u;
    for (int r = 0; r < n_rp; ++r) {
      if (s_state[r] == 2u) {
        s_slot[r] = -1;
        continue;
      }
      const unsigned long long pr = pass == 0 ? 0ull : s_prefix[r] >> (shift + 8);
      int sl = -1;
      for (int q = 0; q < ns; ++q)
        if (s_pre[q] == pr) sl = q;
      if (sl < 0) {
        s_pre[ns] = pr;
        sl = ns++;
      }
      s_slot[r] = sl;
      if (s_state[r] == 1u) find |= 1u << sl;
    }
    s_nslots = ns;
    s_find = find;
  }
  __syncthreads();
  const int ns = s_nslots;
  const unsigned int find = s_find;
  unsigned long long pre[4] = {0ull, 0ull, 0ull, 0ull};
  if constexpr (FAST) {
#pragma unroll
    for (int q = 0; q < 4; ++q) pre[q] = q < ns ? s_pre[q] : ~0ull;
  }
  unsigned long long local_max = 0ull;
  bool bad = false;
  const unsigned long long max_key = pass == 1 ? st->max_key : ~0ull;
  unsigned int n_max = 0u;  // pass 1: keys equal to the largest
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  auto take = [&](double v) {
    const unsigned long long key = (unsigned long long)__double_as_longlong(v);
    const unsigned int d = (unsigned int)(key >> shift) & 255u;
    if (pass == 1) n_max += key == max_key ? 1u : 0u;
    if (pass == 0) {
      bad |= key >= 0x7FF0000000000000ull;  // negative, infinite or NaN
      local_max = key > local_max ? key : local_max;
      atomicAdd(&sh[0][d], 1u);
      return;
    }
    const unsigned long long kp = key >> (shift + 8);
    int sl = -1;
    if constexpr (FAST) {
#pragma unroll
      for (int q = 0; q < 4; ++q) sl = kp == pre[q] ? q : sl;
    } else {
      for (int q = 0; q < ns; ++q) sl = kp == s_pre[q] ? q : sl;
    }
    if (sl >= 0) {
      atomicAdd(&sh[sl][d], 1u);
      if ((find >> sl) & 1u) st->found[sl] = key;  // the bucket's only key
      if (pass >= 3) {
        atomicMin(&st->smin[sl], key);
        atomicMax(&st->smax[sl], key);
      }
    }
  };
  // Four independent loads in flight per thread: one load at a time leaves
  // a pass over a many-layer batch (hundreds of MB) latency-bound.
  int64_t i = (int64_t)blockIdx.x * blockDim.x + tid;
  for (; i + 3 * stride < n; i += 4 * stride) {
    const double v0 = y[i], v1 = y[i + stride], v2 = y[i + 2 * stride], v3 = y[i + 3 * stride];
    take(v0);
    take(v1);
    take(v2);
    take(v3);
  }
  for (; i < n; i += stride) take(y[i]);
  if (pass == 0) {
    for (int m = 16; m > 0; m >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, local_max, m);
      local_max = o > local_max ? o : local_max;
    }
    if ((tid & 31) == 0 && local_max) atomicMax(&st->max_key, local_max);
    if (__any_sync(0xFFFFFFFFu, bad) && (tid & 31) == 0) atomicOr(err, 1u);
  }
  if (pass == 1) {
    const unsigned int w = __reduce_add_sync(0xFFFFFFFFu, n_max);
    if ((tid & 31) == 0 && w) atomicAdd(&st->cnt_max, (unsigned long long)w);
  }
  __syncthreads();
  for (int i = tid; i < n_rp * 256; i += blockDim.x) {
    const int sl = s_slot[i >> 8];
    const unsigned int c = sl >= 0 ? sh[sl][i & 255] : 0u;
    if (c) atomicAdd(&st->hist[0][0] + i, c);
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&st->done_pass, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // Pick the next digit of every return period: the merged counts come into
  // shared memory at once, then two return periods at a time (256 threads
  // each) thread i holds the count of digit 255 - i (descending), a scan over
  // its 256 threads gives the counts of keys above each digit, and the one
  // thread whose range contains rank k_rem records the digit.
  __shared__ long long s_warp[kSelectThreads / 32];
  __shared__ long long s_krem[kMaxReturnPeriods];
  const int lane = tid & 31, wid = tid >> 5;
  unsigned int *cnt = &sh[0][0];  // the block's histogram is merged: reuse its space
  for (int i = tid; i < n_rp * 256; i += blockDim.x) cnt[i] = __ldcg(&st->hist[0][0] + i);
  if (tid < n_rp) {
    s_krem[tid] = st->k_rem[tid];
    if (s_state[tid] == 1u) {  // recorded during this pass: the threshold is that key
      st->prefix[tid] = __ldcg(&st->found[s_slot[tid]]);
      st->rstate[tid] = 2u;
    } else if (pass == 1 && s_state[tid] == 0u && __ldcg(&st->cnt_max) >= (unsigned long long)st->k[tid]) {
      st->prefix[tid] = __ldcg(&st->max_key);  // at least k losses tie at the largest
      st->rstate[tid] = 2u;
      s_state[tid] = 2u;
    } else if (pass >= 3 && s_state[tid] == 0u) {
      const unsigned long long lo = __ldcg(&st->smin[s_slot[tid]]), hi = __ldcg(&st->smax[s_slot[tid]]);
      if (lo == hi) {  // every candidate is the same loss
        st->prefix[tid] = lo;
        st->rstate[tid] = 2u;
        s_state[tid] = 2u;
      }
    }
  }
  __syncthreads();
  const int half = tid >> 8, b = tid & 255;
  for (int r0 = 0; r0 < n_rp; r0 += 2) {
    const int r = r0 + half;
    const bool act = r < n_rp && s_state[r] == 0u;
    const long long k_rem = act ? s_krem[r] : 0;
    const long long h = act ? (long long)cnt[r * 256 + 255 - b] : 0;
    long long incl = h;
    for (int o = 1; o < 32; o <<= 1) {
      const long long v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    for (int w = half * 8; w < wid; ++w) incl += s_warp[w];
    const long long excl = incl - h;
    if (act && excl < k_rem && k_rem <= incl) {
      st->k_rem[r] = k_rem - excl;
      st->prefix[r] = s_prefix[r] | ((unsigned long long)(255 - b) << shift);
      if (h == 1 && pass < 7) st->rstate[r] = 1u;  // a single key left in its bucket
    }
    __syncthreads();
  }
  for (int i = tid; i < n_rp * 256; i += blockDim.x) (&st->hist[0][0])[i] = 0u;
  if (tid < kMaxReturnPeriods) {
    st->smin[tid] = ~0ull;
    st->smax[tid] = 0ull;
  }
  if (tid == 0) {
    st->done_pass = 0u;
    bool all = true;
    for (int r = 0; r < n_rp; ++r) all = all && st->rstate[r] == 2u;
    if (all) st->all_done = 1u;
  }
}

__device__ __forceinline__ int select_q(unsigned long long max_key, int64_t n) {
  // Largest value < 2^e1; n values sum to < 2^(e1 + ceil(log2 n)); keep the
  // fixed-point integer below 2^127.
  const int e1 = (int)(max_key >> 52) - 1022;
  const int lg = n > 1 ? 64 - __clzll((long long)(n - 1)) : 0;
  return e1 + lg + 1 - 127;
}

// PML and TVaR of every return period from the merged counts and sums: the
// (k - count) copies of the threshold complete the tail sum exactly, then one
// rounding to binary64 and one division.  Run by one thread, after every
// CTA's contribution is in.
__device__ void finish_pml_tvar(SelState *st, int n_rp, int q, double *out) {
  for (int j = 0; j < n_rp; ++j) {
    const unsigned long long tj = st->prefix[j];
    const double tau_v = __longlong_as_double((long long)tj);
    const unsigned long long m = (unsigned long long)(st->k[j] - (long long)__ldcg(&st->cnt_gt[j]));
    U128 total{__ldcg(&st->acc_lo[j]), __ldcg(&st->acc_hi[j])};
    const U128 ft = to_fixed(tau_v, q);
    const unsigned long long plo = ft.lo * m;
    const unsigned long long phi = __umul64hi(ft.lo, m) + ft.hi * m;
    add128(total, plo, phi);
    out[j] = tau_v;
    out[n_rp + j] = __ddiv_rn(from_fixed(total, q), (double)st->k[j]);
  }
  st->done_sum = 0u;
}

// grid.y = return period index, grid.z = layer (more than four return periods).
__global__ void __launch_bounds__(kSelectThreads)
select_sum_kernel(const double *__restrict__ ylts, int64_t n, int64_t q_count, int n_rp, SelState *states,
                  double *outs) {
  const double *__restrict__ y = ylts + (size_t)blockIdx.z * (size_t)n;
  SelState *st = states + blockIdx.z;
  double *out = outs + (size_t)blockIdx.z * 2 * (size_t)n_rp;
  __shared__ unsigned long long s_lo[kSelectThreads / 32], s_hi[kSelectThreads / 32],
      s_cnt[kSelectThreads / 32];
  __shared__ bool s_last;
  const int r = blockIdx.y;
  const int tid = threadIdx.x;
  const unsigned long long tau = st->prefix[r];
  const unsigned long long max_key = st->max_key;
  const int q = select_q(max_key, q_count);
  U128 acc{0ull, 0ull};
  unsigned long long cnt = 0ull;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + tid; i < n; i += stride) {
    const double v = y[i];
    const unsigned long long key = (unsigned long long)__double_as_longlong(v);
    if (key > tau) {
      const U128 f = to_fixed(v, q);
      add128(acc, f.lo, f.hi);
      ++cnt;
    }
  }
  acc = warp_sum_u128(acc);
  for (int m = 16; m > 0; m >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, m);
  if ((tid & 31) == 0) {
    s_lo[tid >> 5] = acc.lo;
    s_hi[tid >> 5] = acc.hi;
    s_cnt[tid >> 5] = cnt;
  }
  __syncthreads();
  if (tid == 0) {
    U128 b{0ull, 0ull};
    unsigned long long c = 0ull;
    for (int w = 0; w < kSelectThreads / 32; ++w) {
      add128(b, s_lo[w], s_hi[w]);
      c += s_cnt[w];
    }
    if (c) {
      atomicAdd(&st->cnt_gt[r], c);
      // 128-bit atomic add from two 64-bit ones: the carry out of the low
      // word goes into the high word, so the total is exact modulo 2^128.
      const unsigned long long old = atomicAdd(&st->acc_lo[r], b.lo);
      const unsigned long long carry = (old + b.lo < old) ? 1ull : 0ull;
      atomicAdd(&st->acc_hi[r], b.hi + carry);
    }
    __threadfence();
    s_last = atomicAdd(&st->done_sum, 1u) == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!s_last || tid != 0) return;
  __threadfence();
  finish_pml_tvar(st, n_rp, q, out);
}

// The same sums for R <= 4 return periods in one sweep: each CTA reads its
// part of the layer's losses once and adds every loss above the lowest
// threshold to the sums of the return periods it exceeds (grid.y = layer).
template <int R>
__global__ void __launch_bounds__(kSelectThreads, 2)
select_sum_rp_kernel(const double *__restrict__ ylts, int64_t n, int64_t q_count, SelState *states,
                     double *outs) {
  const double *__restrict__ y = ylts + (size_t)blockIdx.y * (size_t)n;
  SelState *st = states + blockIdx.y;
  double *out = outs + (size_t)blockIdx.y * 2 * R;
  __shared__ unsigned long long s_lo[R][kSelectThreads / 32], s_hi[R][kSelectThreads / 32],
      s_cnt[R][kSelectThreads / 32];
  __shared__ bool s_last;
  const int tid = threadIdx.x;
  unsigned long long tau[R];
  unsigned long long tmin = ~0ull;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    tau[r] = st->prefix[r];
    tmin = tau[r] < tmin ? tau[r] : tmin;
  }
  const int q = select_q(st->max_key, q_count);
  U128 acc[R];
  unsigned long long cnt[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    acc[r] = U128{0ull, 0ull};
    cnt[r] = 0ull;
  }
  auto take = [&](double v) {
    const unsigned long long key = (unsigned long long)__double_as_longlong(v);
    if (key > tmin) {
      const U128 f = to_fixed(v, q);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (key > tau[r]) {
          add128(acc[r], f.lo, f.hi);
          ++cnt[r];
        }
    }
  };
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + tid;
  for (; i + 3 * stride < n; i += 4 * stride) {
    const double v0 = y[i], v1 = y[i + stride], v2 = y[i + 2 * stride], v3 = y[i + 3 * stride];
    take(v0);
    take(v1);
    take(v2);
    take(v3);
  }
  for (; i < n; i += stride) take(y[i]);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    acc[r] = warp_sum_u128(acc[r]);
    for (int m = 16; m > 0; m >>= 1) cnt[r] += __shfl_xor_sync(0xFFFFFFFFu, cnt[r], m);
    if ((tid & 31) == 0) {
      s_lo[r][tid >> 5] = acc[r].lo;
      s_hi[r][tid >> 5] = acc[r].hi;
      s_cnt[r][tid >> 5] = cnt[r];
    }
  }
  __syncthreads();
  if (tid == 0) {
    for (int r = 0; r < R; ++r) {
      U128 b{0ull, 0ull};
      unsigned long long c = 0ull;
      for (int w = 0; w < kSelectThreads / 32; ++w) {
        add128(b, s_lo[r][w], s_hi[r][w]);
        c += s_cnt[r][w];
      }
      if (c) {
        atomicAdd(&st->cnt_gt[r], c);
        const unsigned long long old = atomicAdd(&st->acc_lo[r], b.lo);
        const unsigned long long carry = (old + b.lo < old) ? 1ull : 0ull;
        atomicAdd(&st->acc_hi[r], b.hi + carry);
      }
    }
    __threadfence();
    s_last = atomicAdd(&st->done_sum, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last || tid != 0) return;
  __threadfence();
  finish_pml_tvar(st, R, q, out);
}

cudaError_t launch_pml_tvar_batch(const double *ylts, int n_layers, int64_t n, const int64_t *k,
                                  int n_rp, void *ws, double *out, unsigned int *err_flag,
                                  int device, cudaStream_t s, int64_t q_count) {
  if (q_count < n) q_count = n;
  SelState *st = reinterpret_cast<SelState *>(ws);
  KArgs ka;
  for (int i = 0; i < kMaxReturnPeriods; ++i) ka.k[i] = i < n_rp ? (long long)k[i] : 1;
  select_init_kernel<<<n_layers, 256, 0, s>>>(st, ka, n_rp);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  int sms = 0;
  err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (err != cudaSuccess) return err;
  // One wave: four 512-thread CTAs are resident per SM (32 registers), and a
  // grid one CTA larger than that runs a second wave as long as the first
  // (measured on 64 layers of 1e6 losses: 640 CTAs took 0.31 ms a pass).
  int64_t blocks = (n + kSelectThreads - 1) / kSelectThreads;
  int64_t cap = (int64_t)sms * 4 / n_layers;
  if (cap < 1) cap = 1;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  for (int pass = 0; pass < 8; ++pass) {
    if (n_rp <= 4)
      select_pass_kernel<true><<<dim3((unsigned)blocks, (unsigned)n_layers), kSelectThreads, 0, s>>>(
          ylts, n, n_rp, pass, st, err_flag);
    else
      select_pass_kernel<false><<<dim3((unsigned)blocks, (unsigned)n_layers), kSelectThreads, 0, s>>>(
          ylts, n, n_rp, pass, st, err_flag);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (n_rp <= 4) {
    // two CTAs per SM (at most 64 registers a thread)
    int64_t bs = (n + kSelectThreads - 1) / kSelectThreads;
    int64_t cap2 = (int64_t)sms * 2 / n_layers;
    if (cap2 < 1) cap2 = 1;
    if (bs > cap2) bs = cap2;
    if (bs < 1) bs = 1;
    const dim3 grid((unsigned)bs, (unsigned)n_layers);
    switch (n_rp) {
      case 1: select_sum_rp_kernel<1><<<grid, kSelectThreads, 0, s>>>(ylts, n, q_count, st, out); break;
      case 2: select_sum_rp_kernel<2><<<grid, kSelectThreads, 0, s>>>(ylts, n, q_count, st, out); break;
      case 3: select_sum_rp_kernel<3><<<grid, kSelectThreads, 0, s>>>(ylts, n, q_count, st, out); break;
      default: select_sum_rp_kernel<4><<<grid, kSelectThreads, 0, s>>>(ylts, n, q_count, st, out); break;
    }
    return cudaGetLastError();
  }
  int64_t bx = (blocks + n_rp - 1) / n_rp;
  if (bx < 1) bx = 1;
  select_sum_kernel<<<dim3((unsigned)bx, (unsigned)n_rp, (unsigned)n_layers), kSelectThreads, 0, s>>>(
      ylts, n, q_count, n_rp, st, out);
  return cudaGetLastError();
}

cudaError_t launch_pml_tvar(const double *ylt, int64_t n, const int64_t *k, int n_rp, void *ws,
                            double *out, unsigned int *err_flag, int device, cudaStream_t s, int64_t q_count) {
  return launch_pml_tvar_batch(ylt, 1, n, k, n_rp, ws, out, err_flag, device, s, q_count);
}

}  // namespace ara
