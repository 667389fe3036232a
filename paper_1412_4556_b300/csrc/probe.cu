// Measured ceilings of the YLT kernel's inner loop.  Per occurrence the
// kernel tests one bit of a shared-memory bitmap at a random word and, when
// the event may have a nonzero loss, gathers its table entry from a table
// that L2 holds (Section IV-B: a direct access table costs one memory access
// per lookup).  Neither rate has a datasheet figure, so these
// microbenchmarks measure them on the device at hand, together with the
// binary64 add rate that an FP64 running sum would need:
//
//  * probe_gather_kernel: rows of row_bytes at random positions of a table
//    of table_bytes (warmed into L2 first), each row read by lanes_per_row
//    lanes of load_bytes each in one warp instruction, 4 rows in flight per
//    lane group, with the kernel's cache policy (no L1 allocation, L2
//    evict-last);
//  * probe_smem_kernel: random 32-bit words of the largest shared-memory
//    array a CTA can hold, 8 lookups in flight per thread;
//  * probe_dadd_kernel: 8 independent chains of binary64 adds per thread.
//
// Random positions come from a linear congruential step per lane group
// (Knuth's MMIX constants), its high bits scaled to the range with one
// multiply-high; nothing reads HBM but the table's first touch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "ara.h"
#include "ara_ctx.h"
#include "ara_internal.cuh"

using namespace ara;

namespace {

__device__ __forceinline__ uint64_t lcg(uint64_t s) { return s * 6364136223846793005ull + 1442695040888963407ull; }

__device__ __forceinline__ uint64_t seed_of(uint64_t g, uint64_t u) {
  // SplitMix64 finaliser of (group, stream): distinct, well-mixed starts
  uint64_t z = g * 0x9E3779B97F4A7C15ull + u * 0xD1B54A32D192ED03ull + 0x632BE59BD9B4E019ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <int LB>
struct Load;
template <>
struct Load<8> {
  static __device__ __forceinline__ uint64_t get(const char *p, uint64_t pol) {
    uint64_t a;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(a) : "l"(p), "l"(pol));
    return a;
  }
};
template <>
struct Load<16> {
  static __device__ __forceinline__ uint64_t get(const char *p, uint64_t pol) {
    uint64_t a, b;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
                 : "=l"(a), "=l"(b)
                 : "l"(p), "l"(pol));
    return a ^ b;
  }
};
template <>
struct Load<32> {
  static __device__ __forceinline__ uint64_t get(const char *p, uint64_t pol) {
    uint64_t a, b, c, d;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u64 {%0, %1, %2, %3}, [%4], %5;"
                 : "=l"(a), "=l"(b), "=l"(c), "=l"(d)
                 : "l"(p), "l"(pol));
    return a ^ b ^ c ^ d;
  }
};

constexpr int kInFlight = 4;

template <int LB>
__global__ void probe_gather_kernel(const char *__restrict__ table, uint32_t rows, uint32_t row_bytes,
                                    int lanes_per_row, int iters, unsigned long long *sink) {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t group = tid / (uint32_t)lanes_per_row;
  const uint32_t part = tid % (uint32_t)lanes_per_row;
  uint64_t s[kInFlight];
#pragma unroll
  for (int u = 0; u < kInFlight; ++u) s[u] = seed_of(group, u);
  uint64_t acc = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kInFlight; ++u) {
      s[u] = lcg(s[u]);
      const uint32_t r = __umulhi((uint32_t)(s[u] >> 32), rows);
      acc ^= Load<LB>::get(table + (size_t)r * row_bytes + (size_t)part * LB, pol);
    }
  }
  if (acc == 0x9E3779B97F4A7C15ull) sink[0] = acc;  // keeps the loads; never true for a zeroed table
}

constexpr int kSmemLookups = 8;

__global__ void probe_smem_kernel(uint32_t words, int iters, unsigned long long *sink) {
  extern __shared__ uint32_t s_words[];
  for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) s_words[i] = i * 2654435761u;
  __syncthreads();
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t s[kSmemLookups];
#pragma unroll
  for (int u = 0; u < kSmemLookups; ++u) s[u] = seed_of(tid, u);
  uint32_t acc = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kSmemLookups; ++u) {
      s[u] = lcg(s[u]);
      acc ^= s_words[__umulhi((uint32_t)(s[u] >> 32), words)];
    }
  }
  if (acc == 0x12345678u) sink[0] = acc;
}

constexpr int kDaddChains = 8;

__global__ void probe_dadd_kernel(double x, int iters, double *sink) {
  double a[kDaddChains];
#pragma unroll
  for (int u = 0; u < kDaddChains; ++u) a[u] = (double)(threadIdx.x + u);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kDaddChains; ++u) a[u] = __dadd_rn(a[u], x);
  }
  double t = 0.0;
#pragma unroll
  for (int u = 0; u < kDaddChains; ++u) t = __dadd_rn(t, a[u]);
  if (t == -1.0) sink[0] = t;
}

// Best-of-reps milliseconds of `launch` on stream s (the first run warms up).
template <typename F>
cudaError_t time_best(cudaStream_t s, int reps, F launch, float *best) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  *best = 1e30f;
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(a, s);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && r > 0) *best = std::min(*best, ms);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return e;
}

struct ProbeScope {
  cudaStream_t s = nullptr;
  void *buf = nullptr;
  ~ProbeScope() {
    if (s) cudaStreamSynchronize(s);
    if (buf) cudaFree(buf);
    if (s) cudaStreamDestroy(s);
  }
};

ara_status probe_fail(cudaError_t e, const char *what) {
  cudaGetLastError();
  return fail_free(e == cudaErrorMemoryAllocation ? ARA_E_NOMEM : ARA_E_CUDA, "%s: %s", what,
                   cudaGetErrorString(e));
}

}  // namespace

extern "C" {

ara_status ara_probe_gather(int device, int64_t table_bytes, int32_t load_bytes, int32_t lanes_per_row,
                            int32_t threads_per_cta, int32_t ctas_per_sm, double *rows_per_s,
                            double *sectors_per_s) {
  if (!rows_per_s || !sectors_per_s) return fail_free(ARA_E_INVALID_ARG, "NULL output");
  if (load_bytes != 8 && load_bytes != 16 && load_bytes != 32)
    return fail_free(ARA_E_INVALID_ARG, "load_bytes must be 8, 16 or 32");
  if (lanes_per_row != 1 && lanes_per_row != 2 && lanes_per_row != 4 && lanes_per_row != 8)
    return fail_free(ARA_E_INVALID_ARG, "lanes_per_row must be 1, 2, 4 or 8");
  const int64_t row_bytes = (int64_t)load_bytes * lanes_per_row;
  if (row_bytes > 128) return fail_free(ARA_E_INVALID_ARG, "a row is at most one 128-byte line");
  if (table_bytes < row_bytes * 1024 || table_bytes > ((int64_t)1 << 34))
    return fail_free(ARA_E_INVALID_ARG, "table_bytes must lie in [1024 rows, 16 GiB]");
  if (threads_per_cta < 32 || threads_per_cta > 1024 || threads_per_cta % 32 || ctas_per_sm < 1 || ctas_per_sm > 32)
    return fail_free(ARA_E_INVALID_ARG, "threads_per_cta a multiple of 32 in [32, 1024], ctas_per_sm in [1, 32]");
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return probe_fail(e, "cudaSetDevice");
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
    return probe_fail(e, "SM count");
  ProbeScope ps;
  if ((e = cudaStreamCreateWithFlags(&ps.s, cudaStreamNonBlocking)) != cudaSuccess) return probe_fail(e, "stream");
  const uint32_t rows = (uint32_t)std::min<int64_t>(table_bytes / row_bytes, 0xFFFFFFFFll);
  if ((e = cudaMalloc(&ps.buf, (size_t)rows * (size_t)row_bytes + 8)) != cudaSuccess) return probe_fail(e, "table");
  if ((e = cudaMemsetAsync(ps.buf, 0, (size_t)rows * (size_t)row_bytes + 8, ps.s)) != cudaSuccess)
    return probe_fail(e, "memset");
  const char *table = static_cast<const char *>(ps.buf);
  unsigned long long *sink = reinterpret_cast<unsigned long long *>(static_cast<char *>(ps.buf) +
                                                                    (size_t)rows * (size_t)row_bytes);
  const int blocks = sms * ctas_per_sm;
  const int iters = 256;
  auto launch = [&]() -> cudaError_t {
    if (load_bytes == 8)
      probe_gather_kernel<8><<<blocks, threads_per_cta, 0, ps.s>>>(table, rows, (uint32_t)row_bytes, lanes_per_row,
                                                                   iters, sink);
    else if (load_bytes == 16)
      probe_gather_kernel<16><<<blocks, threads_per_cta, 0, ps.s>>>(table, rows, (uint32_t)row_bytes, lanes_per_row,
                                                                    iters, sink);
    else
      probe_gather_kernel<32><<<blocks, threads_per_cta, 0, ps.s>>>(table, rows, (uint32_t)row_bytes, lanes_per_row,
                                                                    iters, sink);
    return cudaGetLastError();
  };
  float ms = 0.f;
  if ((e = time_best(ps.s, 5, launch, &ms)) != cudaSuccess) return probe_fail(e, "gather probe");
  const double loads = (double)blocks * threads_per_cta * iters * kInFlight;
  const double rws = loads / lanes_per_row;
  *rows_per_s = rws / (ms * 1e-3);
  *sectors_per_s = rws * (double)std::max<int64_t>(1, row_bytes / 32) / (ms * 1e-3);
  return ARA_OK;
}

ara_status ara_probe_smem_lookup(int device, double *lookups_per_s) {
  if (!lookups_per_s) return fail_free(ARA_E_INVALID_ARG, "NULL output");
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return probe_fail(e, "cudaSetDevice");
  int sms = 0, optin = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device)) != cudaSuccess)
    return probe_fail(e, "device attributes");
  const size_t smem = (size_t)optin / 16 * 16;
  if ((e = cudaFuncSetAttribute(probe_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return probe_fail(e, "shared memory size");
  ProbeScope ps;
  if ((e = cudaStreamCreateWithFlags(&ps.s, cudaStreamNonBlocking)) != cudaSuccess) return probe_fail(e, "stream");
  if ((e = cudaMalloc(&ps.buf, 64)) != cudaSuccess) return probe_fail(e, "sink");
  const int threads = kYltThreads, iters = 512;
  auto launch = [&]() -> cudaError_t {
    probe_smem_kernel<<<sms, threads, smem, ps.s>>>((uint32_t)(smem / 4), iters,
                                                    static_cast<unsigned long long *>(ps.buf));
    return cudaGetLastError();
  };
  float ms = 0.f;
  if ((e = time_best(ps.s, 5, launch, &ms)) != cudaSuccess) return probe_fail(e, "shared-memory probe");
  *lookups_per_s = (double)sms * threads * iters * kSmemLookups / (ms * 1e-3);
  return ARA_OK;
}

ara_status ara_probe_fp64_add(int device, double *adds_per_s) {
  if (!adds_per_s) return fail_free(ARA_E_INVALID_ARG, "NULL output");
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return probe_fail(e, "cudaSetDevice");
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
    return probe_fail(e, "SM count");
  ProbeScope ps;
  if ((e = cudaStreamCreateWithFlags(&ps.s, cudaStreamNonBlocking)) != cudaSuccess) return probe_fail(e, "stream");
  if ((e = cudaMalloc(&ps.buf, 64)) != cudaSuccess) return probe_fail(e, "sink");
  const int threads = 256, per_sm = 8, iters = 512;
  auto launch = [&]() -> cudaError_t {
    probe_dadd_kernel<<<sms * per_sm, threads, 0, ps.s>>>(0.5, iters, static_cast<double *>(ps.buf));
    return cudaGetLastError();
  };
  float ms = 0.f;
  if ((e = time_best(ps.s, 5, launch, &ms)) != cudaSuccess) return probe_fail(e, "FP64 add probe");
  *adds_per_s = (double)sms * per_sm * threads * iters * kDaddChains / (ms * 1e-3);
  return ARA_OK;
}

}  // extern "C"
