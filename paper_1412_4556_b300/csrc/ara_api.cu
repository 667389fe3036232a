// Host side of the C ABI in include/ara.h: argument validation, device
// buffers owned by the context, and the launch sequence of each call.
//
// Device memory layout of a context (all buffers library-owned):
//   YET       raw offsets int64[N+1]; chunk offsets int64[N+1]; id chunks
//             int4[Mc + kChunkTail]: trial t at chunks [coff[t], coff[t+1]),
//             6 ids of 21 bits per chunk when the catalog fits (else 4 plain
//             ids), gaps and tail filled with the sentinel id (the catalog
//             size); ts float32[M] or none; staging for host ids
//   ELT pool  one block per ara_load_elts call: ids int32 (sorted by id per
//             ELT), losses f64 (same order), fold bucket index int32
//   layer     EltDesc[J]; fixed-point table 16 B x catalog; zero-skip bitmap
//   scratch   YLT staging for host outputs, PML/TVaR workspace, error words
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <numeric>
#include <utility>
#include <string>
#include <vector>

#include "ara.h"
#include "ara_ctx.h"
#include "ara_internal.cuh"

using namespace ara;


namespace ara {

thread_local std::string g_create_error;

ara_status fail(ara_ctx *c, ara_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return st;
}

ara_status cuda_fail(ara_ctx *c, cudaError_t e, const char *what) {
  ara_status st = (e == cudaErrorMemoryAllocation) ? ARA_E_NOMEM : ARA_E_CUDA;
  cudaGetLastError();  // clear a sticky launch error where possible
  return fail(c, st, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// Common entry of the ABI calls on a context: a context attached to a pricing
// service is used by the service's thread alone, so other calls are refused
// without touching its state (the message goes to ara_last_error(NULL)).
#define ARA_ENTER(c)                                                                     \
  do {                                                                                   \
    if (!(c)) return ARA_E_INVALID_ARG;                                                  \
    if ((c)->service)                                                                    \
      return ara::fail_free(ARA_E_STATE, "the context is attached to a pricing service"); \
    (c)->err.clear();                                                                    \
  } while (0)

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device memory of a GPU other than the current one.  Every entry point makes
// the context's device current before it looks at pointers, so such an array
// belongs to another GPU: it is not a host array (a host-to-device copy from
// it fails) and this device's kernels cannot read it (unmapped peer memory
// would fault), so the entry points reject it with ARA_E_INVALID_ARG.
bool foreign_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  int dev = -1;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice && a.device != dev;
}

ara_status reject_foreign(ara_ctx *c, std::initializer_list<std::pair<const void *, const char *>> ptrs) {
  for (const auto &pn : ptrs)
    if (foreign_device_ptr(pn.first))
      return fail(c, ARA_E_INVALID_ARG, "%s is memory of another GPU than the context's (device %d)", pn.second,
                  c->device);
  return ARA_OK;
}

int current_sm_count() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    cudaGetLastError();
    dev = 0;
  }
  const int slot = dev < kMaxDev ? dev : kMaxDev - 1;
  int sms = cache[slot].load(std::memory_order_relaxed);
  if (sms > 0 && dev < kMaxDev) return sms;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    sms = 1;
  }
  if (dev < kMaxDev) cache[slot].store(sms, std::memory_order_relaxed);
  return sms;
}

bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }
bool limit_ok(double v) { return !std::isnan(v) && v >= 0.0; }

// Timing helpers: record an event pair around a launch when enabled.
struct TimedLaunch {
  ara_ctx *c;
  int ch;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  TimedLaunch(ara_ctx *c_, int ch_, cudaStream_t s_) : c(c_), ch(ch_), s(s_) {
    if (c->timing && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
      cudaEventRecord(a, s);
  }
  void done() {
    if (a && b) {
      cudaEventRecord(b, s);
      c->chan[ch].events.emplace_back(a, b);
      a = b = nullptr;
    }
  }
  ~TimedLaunch() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Choose the zero-skip bitmap layout that fits the shared-memory budget of
// the YLT kernel: one bit per event when the catalog fits, otherwise the
// events spread evenly over every word of the budget (see BitmapLayout).
BitmapLayout plan_bitmap(int32_t events, size_t smem_bytes) {
  const uint64_t max_words = (uint64_t)(smem_bytes / 16) * 4;  // whole uint4s
  const uint64_t E = (uint64_t)std::max<int32_t>(events, 1);
  BitmapLayout bm;
  const uint64_t exact_words = (E + 31) / 32;
  if (exact_words <= max_words) {
    bm.mul = 1u << 27;  // word e >> 5
    bm.words = (int32_t)((exact_words + 3) / 4 * 4);
  } else {
    bm.words = (int32_t)max_words;
    bm.mul = (uint32_t)(((uint64_t)max_words << 32) / E);  // word(E-1) < max_words
  }
  return bm;
}

size_t ylt_smem_budget(int device) {
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
      optin <= 0) {
    cudaGetLastError();
    optin = 48 * 1024;
  }
  return (size_t)optin;
}

// Fixed-point exponent for a layer: any trial sum is at most upper * lmax;
// keep the integer below 2^(bits - 1): 2^127 for the 128-bit entries of FP64
// layers, 2^63 for the 64-bit entries of FP32-table layers (each entry then
// rounds to the grid, adding at most lmax / 2 grid steps to the sum).
bool choose_q(double upper, int64_t lmax, int bits, int *q) {
  if (!(upper > 0.0) || lmax <= 0) {
    *q = 0;
    return true;
  }
  const double bound = upper * (double)lmax;
  if (!std::isfinite(bound)) return false;
  int e = 0;
  std::frexp(bound, &e);  // bound < 2^e
  *q = e + 1 - bits;
  return true;
}

// v (finite, >= 0) as the integer v / 2^q, when that is exact and below
// 2^127; false otherwise.
bool to_fixed_exact(double v, int q, U128 *out) {
  *out = U128{0ull, 0ull};
  if (v == 0.0) return true;
  int e = 0;
  const double m = std::frexp(v, &e);                     // v = m * 2^e, m in [0.5, 1)
  const uint64_t mi = (uint64_t)std::ldexp(m, 53);         // v = mi * 2^(e - 53)
  const int sh = e - 53 - q;                               // v / 2^q = mi * 2^sh
  if (sh < 0) {
    if (-sh >= 64 || (mi & ((1ull << -sh) - 1)) != 0ull) return false;
    out->lo = mi >> -sh;
    return true;
  }
  if (sh + 53 > 127) return false;
  if (sh >= 64) {
    out->hi = mi << (sh - 64);
  } else if (sh > 0) {
    out->lo = mi << sh;
    out->hi = mi >> (64 - sh);
  } else {
    out->lo = mi;
  }
  return true;
}

// The layer's aggregate terms on its fixed-point grid (see AggFixed).
AggFixed agg_terms_fixed(double agg_ret, double agg_lim, int q) {
  AggFixed af{{0ull, 0ull}, {~0ull, ~0ull}, 0};
  const bool ret_ok = to_fixed_exact(agg_ret, q, &af.ret);
  bool lim_ok = true;
  if (std::isfinite(agg_lim) && agg_lim < std::ldexp(1.0, 127 + q)) {
    lim_ok = to_fixed_exact(agg_lim, q, &af.lim);
  }  // else: no trial sum reaches AggL, the clamp never binds
  af.exact = (ret_ok && lim_ok) ? 1 : 0;
  return af;
}

YltStream ylt_stream(const ara_ctx *c, int G) {
  if (G == 1 && c->compact_version == c->yet_version && c->d_dchunks)
    return YltStream{c->d_dcoff, c->d_dchunks, 2, c->h_dcoff.data()};
  return YltStream{c->d_coff, c->d_chunks, c->packed ? 1 : 0, c->h_coff.data()};
}

ara_status enqueue_fold(ara_ctx *c, const LayerRec &L, cudaStream_t s) {
  ARA_CUDA(c, cudaMemsetAsync(L.d_bitmap, 0, (size_t)L.bm.words * 4, s), "cudaMemsetAsync(bitmap)");
  // The sentinel entry (id = catalog) must read zero at this layer's entry
  // width; a buffer used before at the other width may hold data there.
  ARA_CUDA(c, cudaMemsetAsync(reinterpret_cast<unsigned char *>(L.d_table) + (size_t)c->catalog * L.entry_bytes(), 0,
                              (size_t)L.entry_bytes(), s),
           "cudaMemsetAsync(sentinel entry)");
  TimedLaunch tl(c, ARA_TIMING_FOLD, s);
  ARA_CUDA(c, launch_fold(L.d_desc, (int)L.elts.size(), c->catalog, L.occ_ret, L.occ_lim, L.q,
                          L.d_table, L.d_bitmap, L.bm, L.precision == ARA_FP32_TABLE, nullptr, s),
           "fold kernel launch");
  tl.done();
  return ARA_OK;
}

ara_status fold_layer(ara_ctx *c, LayerRec &L, cudaStream_t s) {
  int q = 0;
  if (!choose_q(L.upper, std::max<int64_t>(c->max_trial_len, 1), L.entry_bytes() * 8 - 1, &q))
    return fail(c, ARA_E_INVALID_ARG,
                "layer loss bound x longest trial overflows binary64; losses too large");
  if (L.table_catalog != c->catalog || !L.d_table) {
    if (L.d_table) cudaFree(L.d_table);
    if (L.d_bitmap) cudaFree(L.d_bitmap);
    L.d_table = nullptr;
    L.d_bitmap = nullptr;
    L.table_catalog = 0;
    // One extra entry for the sentinel id (= catalog) that pads trials; it
    // stays zero because the fold only writes entries below the catalog size.
    L.bm = plan_bitmap(c->catalog + 1, ylt_smem_budget(c->device));
    ARA_CUDA(c, cudaMalloc(&L.d_table, ((size_t)c->catalog + 1) * sizeof(ulonglong2)),
             "cudaMalloc(layer table)");
    ARA_CUDA(c, cudaMalloc(&L.d_bitmap, (size_t)L.bm.words * 4), "cudaMalloc(layer bitmap)");
    ARA_CUDA(c, cudaMemsetAsync(L.d_table + c->catalog, 0, sizeof(ulonglong2), s), "cudaMemsetAsync(table)");
    L.table_catalog = c->catalog;
  }
  L.q = q;
  L.agg_fx = agg_terms_fixed(L.agg_ret, L.agg_lim, q);
  ara_status st = enqueue_fold(c, L, s);
  if (st) return st;
  L.folded_version = c->yet_version;
  return ARA_OK;
}

void free_layer(LayerRec &L) {
  if (L.d_desc) cudaFree(L.d_desc);
  if (L.d_table) cudaFree(L.d_table);
  if (L.d_bitmap) cudaFree(L.d_bitmap);
  L = LayerRec();
}

void free_buffers(LayerBuffers &B) {
  if (B.d_desc) cudaFree(B.d_desc);
  if (B.d_table) cudaFree(B.d_table);
  if (B.d_bitmap) cudaFree(B.d_bitmap);
  B = LayerBuffers();
}

// Hand a layer's buffers to the pool (or free them when the pool is full).
void recycle_layer(ara_ctx *c, LayerRec &L) {
  LayerBuffers B;
  B.d_desc = L.d_desc;
  B.desc_cap = L.desc_cap;
  B.d_table = L.d_table;
  B.d_bitmap = L.d_bitmap;
  B.table_catalog = L.table_catalog;
  B.bm = L.bm;
  L = LayerRec();
  if (c->pool.size() < c->pool_max) {
    c->pool.push_back(B);
  } else {
    cudaStreamSynchronize(c->stream);
    free_buffers(B);
  }
}

// Take pooled buffers that fit (descriptor capacity and catalog size).
bool take_pooled(ara_ctx *c, int32_t n_elts, LayerRec &L) {
  for (size_t i = c->pool.size(); i-- > 0;) {
    LayerBuffers &B = c->pool[i];
    if (B.desc_cap >= n_elts && B.table_catalog == c->catalog && B.d_table) {
      L.d_desc = B.d_desc;
      L.desc_cap = B.desc_cap;
      L.d_table = B.d_table;
      L.d_bitmap = B.d_bitmap;
      L.table_catalog = B.table_catalog;
      L.bm = B.bm;
      c->pool.erase(c->pool.begin() + (long)i);
      return true;
    }
  }
  return false;
}

ara_status reserve_layers(ara_ctx *c, size_t count, cudaStream_t s) {
  size_t fitting = 0;
  for (const LayerBuffers &B : c->pool)
    if (B.table_catalog == c->catalog && B.d_table) ++fitting;
  while (fitting < count && c->pool.size() < c->pool_max) {
    LayerBuffers B;
    B.bm = plan_bitmap(c->catalog + 1, ylt_smem_budget(c->device));
    B.desc_cap = 64;
    cudaError_t e = cudaMalloc(&B.d_desc, (size_t)B.desc_cap * sizeof(EltDesc));
    if (e == cudaSuccess) e = cudaMalloc(&B.d_table, ((size_t)c->catalog + 1) * sizeof(ulonglong2));
    if (e == cudaSuccess) e = cudaMalloc(&B.d_bitmap, (size_t)B.bm.words * 4);
    // the sentinel entry (id = catalog) stays zero for the buffers' lifetime
    if (e == cudaSuccess) e = cudaMemsetAsync(B.d_table + c->catalog, 0, sizeof(ulonglong2), s);
    if (e != cudaSuccess) {
      free_buffers(B);
      return cuda_fail(c, e, "reserve layer buffers");
    }
    B.table_catalog = c->catalog;
    c->pool.push_back(B);
    ++fitting;
  }
  return ARA_OK;
}

ara_status get_layer(ara_ctx *c, int32_t layer, LayerRec **out) {
  if (layer < 0 || layer >= (int32_t)c->layers.size() || !c->layers[layer].live)
    return fail(c, ARA_E_NOT_FOUND, "unknown layer handle %d", layer);
  *out = &c->layers[layer];
  return ARA_OK;
}


ara_status fail_free(ara_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_create_error = buf;
  return st;
}

ara_status check_layer_args(const ara_ctx *c, int32_t n_elts, const int32_t *handles, double occ_ret,
                            double occ_lim, double agg_ret, double agg_lim, int32_t precision) {
  if (!handles) return fail_free(ARA_E_INVALID_ARG, "elt_handles is NULL");
  if (n_elts < 1 || n_elts > kMaxLayerElts)
    return fail_free(ARA_E_INVALID_ARG, "a layer covers 1..%d ELTs (got %d)", kMaxLayerElts, n_elts);
  if (precision != ARA_FP64 && precision != ARA_FP32_TABLE)
    return fail_free(ARA_E_INVALID_ARG, "precision must be ARA_FP64 or ARA_FP32_TABLE (got %d)", precision);
  if (!finite_nonneg(occ_ret) || !finite_nonneg(agg_ret))
    return fail_free(ARA_E_INVALID_ARG, "retentions must be finite and >= 0");
  if (!limit_ok(occ_lim) || !limit_ok(agg_lim))
    return fail_free(ARA_E_INVALID_ARG, "limits must be >= 0 (inf allowed)");
  std::vector<int32_t> sorted(handles, handles + n_elts);
  std::sort(sorted.begin(), sorted.end());
  for (size_t i = 0; i < sorted.size(); ++i) {
    if (sorted[i] < 0 || sorted[i] >= (int32_t)c->elts.size())
      return fail_free(ARA_E_NOT_FOUND, "unknown ELT handle %d", sorted[i]);
    if (i && sorted[i] == sorted[i - 1])
      return fail_free(ARA_E_INVALID_ARG, "ELT handle %d appears twice in the layer", sorted[i]);
  }
  return ARA_OK;
}

ara_status tail_counts(int64_t n, const double *rps, int32_t n_rp, int64_t *k) {
  if (n_rp < 1 || n_rp > kMaxReturnPeriods || !rps)
    return fail_free(ARA_E_INVALID_ARG, "need 1..%d return periods", kMaxReturnPeriods);
  for (int32_t r = 0; r < n_rp; ++r) {
    if (!(rps[r] >= 1.0)) return fail_free(ARA_E_INVALID_ARG, "return period %d must be >= 1", r);
    const double kk = std::floor((double)n / rps[r]);
    if (kk < 1.0)
      return fail_free(ARA_E_INVALID_ARG, "return period %g exceeds the %lld trials", rps[r], (long long)n);
    k[r] = (int64_t)kk;
  }
  return ARA_OK;
}

size_t layer_bitmap_bytes(const ara_ctx *c) {
  return (size_t)plan_bitmap(c->catalog + 1, ylt_smem_budget(c->device)).words * 4;
}

ara_status define_layer_on(ara_ctx *c, int32_t n_elts, const int32_t *handles, double occ_ret,
                           double occ_lim, double agg_ret, double agg_lim, int32_t precision,
                           cudaStream_t s, int32_t *layer_out, EltDesc *stage) {
  std::vector<int32_t> el(handles, handles + n_elts);
  LayerRec L;
  L.live = true;
  L.elts = el;
  L.occ_ret = occ_ret;
  L.occ_lim = occ_lim;
  L.agg_ret = agg_ret;
  L.agg_lim = agg_lim;
  L.precision = precision;
  // Upper bound of any per-event value: FT1 <= min(loss, limit), summed over
  // the ELTs, capped by the occurrence limit.
  double up = 0.0;
  std::vector<EltDesc> desc((size_t)n_elts);
  for (int32_t j = 0; j < n_elts; ++j) {
    const EltMeta &m = c->elts[(size_t)el[(size_t)j]];
    up += std::min(m.max_loss, m.limit);
    desc[(size_t)j] = EltDesc{m.d_ids, m.d_losses, m.d_bucket, m.nb, m.count, m.deductible, m.limit};
  }
  L.upper = std::min(up * (1.0 + 1e-12), occ_lim);
  if (!take_pooled(c, n_elts, L)) {
    L.desc_cap = std::max<int32_t>(n_elts, 64);
    ARA_CUDA(c, cudaMalloc(&L.d_desc, (size_t)L.desc_cap * sizeof(EltDesc)), "cudaMalloc(layer ELT list)");
  }
  // A copy from pageable memory returns once the data is staged, so `desc`
  // may go out of scope; the stream orders it after earlier users of d_desc.
  if (stage) std::copy(desc.begin(), desc.end(), stage);
  cudaError_t e = cudaMemcpyAsync(L.d_desc, stage ? stage : desc.data(), desc.size() * sizeof(EltDesc),
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    free_layer(L);
    return cuda_fail(c, e, "upload layer ELT list");
  }
  ara_status st = fold_layer(c, L, s);
  if (st != ARA_OK) {
    free_layer(L);
    return st;
  }
  int32_t id = -1;
  for (size_t i = 0; i < c->layers.size(); ++i)
    if (!c->layers[i].live) {
      id = (int32_t)i;
      break;
    }
  if (id < 0) {
    id = (int32_t)c->layers.size();
    c->layers.emplace_back();
  }
  L.gen = ++c->layer_gen;
  c->layers[(size_t)id] = L;
  *layer_out = id;
  return ARA_OK;
}

std::vector<LayerGroup> group_in_order(const std::vector<LayerRec *> &Ls, int g16, int g8) {
  std::vector<LayerGroup> out;
  for (const int eb : {16, 8}) {
    std::vector<int32_t> idx;
    for (size_t i = 0; i < Ls.size(); ++i)
      if (Ls[i]->entry_bytes() == eb) idx.push_back((int32_t)i);
    const int gmax = eb == 16 ? g16 : g8;
    for (size_t p = 0; p < idx.size();) {
      int G = (int)std::min<size_t>((size_t)gmax, idx.size() - p);
      if (G == 3) G = 2;
      out.push_back(LayerGroup{eb, std::vector<int32_t>(idx.begin() + (long)p, idx.begin() + (long)p + G)});
      p += (size_t)G;
    }
  }
  return out;
}

ara_status group_by_overlap(ara_ctx *c, const std::vector<LayerRec *> &Ls, int g16, int g8, cudaStream_t s,
                            std::vector<LayerGroup> *out) {
  out->clear();
  if (Ls.empty()) return ARA_OK;
  // Up to 128 layers every bitmap word takes part; beyond that a strided
  // sample of the words (every stride-th 64-bit word: overlaps estimated on
  // a sample), and each layer is compared with at most kWindow candidates,
  // the next ones in density order, so the host work stays near 1e8 word
  // operations however many layers a plan has.
  constexpr size_t kWindow = 64;
  const size_t full64 = (size_t)Ls[0]->bm.words / 2;  // bitmaps hold a multiple of 4 words
  const size_t stride = Ls.size() <= 128 ? 1 : (Ls.size() + 127) / 128;
  const size_t words64 = (full64 + stride - 1) / stride;
  std::vector<uint64_t> bits(Ls.size() * words64);
  for (size_t i = 0; i < Ls.size(); ++i) {
    uint64_t *dst = bits.data() + i * words64;
    if (stride == 1)
      ARA_CUDA(c, cudaMemcpyAsync(dst, Ls[i]->d_bitmap, words64 * 8, cudaMemcpyDeviceToHost, s),
               "copy zero-skip bitmap");
    else
      ARA_CUDA(c, cudaMemcpy2DAsync(dst, 8, Ls[i]->d_bitmap, 8 * stride, 8, words64, cudaMemcpyDeviceToHost, s),
               "copy zero-skip bitmap sample");
  }
  ARA_CUDA(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
  auto row = [&](size_t i) { return bits.data() + i * words64; };
  std::vector<int64_t> pop(Ls.size(), 0);
  for (size_t i = 0; i < Ls.size(); ++i)
    for (size_t w = 0; w < words64; ++w) pop[i] += __builtin_popcountll(row(i)[w]);
  std::vector<uint64_t> uni(words64);
  for (const int eb : {16, 8}) {
    const int gmax = eb == 16 ? g16 : g8;
    std::vector<int32_t> left;
    for (size_t i = 0; i < Ls.size(); ++i)
      if (Ls[i]->entry_bytes() == eb) left.push_back((int32_t)i);
    std::stable_sort(left.begin(), left.end(), [&](int32_t a, int32_t b) { return pop[(size_t)a] > pop[(size_t)b]; });
    while (!left.empty()) {
      std::vector<int32_t> g{left.front()};
      left.erase(left.begin());
      std::copy(row((size_t)g[0]), row((size_t)g[0]) + words64, uni.begin());
      while ((int)g.size() < gmax && !left.empty()) {
        size_t best = 0;
        int64_t best_ov = -1;
        for (size_t k = 0; k < std::min(left.size(), kWindow); ++k) {
          const uint64_t *b = row((size_t)left[k]);
          int64_t ov = 0;
          for (size_t w = 0; w < words64; ++w) ov += __builtin_popcountll(uni[w] & b[w]);
          if (ov > best_ov) {
            best_ov = ov;
            best = k;
          }
        }
        const uint64_t *b = row((size_t)left[best]);
        for (size_t w = 0; w < words64; ++w) uni[w] |= b[w];
        g.push_back(left[best]);
        left.erase(left.begin() + (long)best);
      }
      if (g.size() == 3) {  // no 3-layer pass: 2 + 1
        out->push_back(LayerGroup{eb, {g[0], g[1]}});
        out->push_back(LayerGroup{eb, {g[2]}});
      } else {
        out->push_back(LayerGroup{eb, g});
      }
    }
  }
  return ARA_OK;
}

ara_status layers_ylt_on(ara_ctx *c, const int32_t *layers, int32_t n_layers, int64_t n_trials,
                         double *dst, cudaStream_t s, ulonglong2 *pair_table, uint32_t *pair_bitmap,
                         const std::vector<LayerGroup> *groups, const std::vector<GroupTable> *tables) {
  std::vector<LayerRec *> Ls((size_t)n_layers);
  for (int32_t i = 0; i < n_layers; ++i) {
    ara_status st = get_layer(c, layers[i], &Ls[(size_t)i]);
    if (st) return st;
  }
  for (LayerRec *L : Ls)
    if (L->folded_version != c->yet_version) {
      ara_status st = fold_layer(c, *L, s);
      if (st) return st;
    }
  const BitmapLayout bm = Ls[0]->bm;  // every layer of a catalog shares the layout
  const size_t entries = (size_t)c->catalog + 1;
  // By default FP64 layers go two to a pass (2 x 16-byte entries per event)
  // and FP32-table layers four to a pass (4 x 8 bytes): one 32-byte L2
  // sector per gather.
  const std::vector<LayerGroup> in_order = groups ? std::vector<LayerGroup>() : group_in_order(Ls, 2, 4);
  size_t gi = 0;
  for (const LayerGroup &grp : groups ? *groups : in_order) {
    const GroupTable pre = tables && gi < tables->size() ? (*tables)[gi] : GroupTable{nullptr, nullptr};
    ++gi;
    const int eb = grp.eb;
    const int G = (int)grp.idx.size();
    if (!((eb == 16 && (G == 1 || G == 2)) || (eb == 8 && (G == 1 || G == 2 || G == 4))))
      return fail(c, ARA_E_INVALID_ARG, "a pass of %d layers of %d-byte entries", G, eb);
    LayerOut outs[4];
    Tables4 tabs{};
    Bitmaps4 bms{};
    for (int g = 0; g < G; ++g) {
      const int32_t i = grp.idx[(size_t)g];
      if (i < 0 || i >= n_layers || Ls[(size_t)i]->entry_bytes() != eb)
        return fail(c, ARA_E_INVALID_ARG, "pass layer position %d", i);
      const LayerRec *L = Ls[(size_t)i];
      outs[g] = LayerOut{L->q, L->agg_fx, L->agg_ret, L->agg_lim, dst + (size_t)i * (size_t)n_trials};
      tabs.t[g] = L->d_table;
      bms.b[g] = L->d_bitmap;
    }
    const void *table = tabs.t[0];
    const uint32_t *bitmap = bms.b[0];
    if (G > 1 && pre.table) {
      table = pre.table;
      bitmap = pre.bitmap;
    } else if (G > 1) {
      ARA_CUDA(c, launch_interleave(tabs, eb, G, (int64_t)entries, pair_table, bms, bm.words, pair_bitmap, s),
               "interleave layer tables");
      table = pair_table;
      bitmap = pair_bitmap;
    }
    const YltStream ys = ylt_stream(c, G);
    const double mean_chunks = (double)ys.h_coff[(size_t)n_trials] / (double)n_trials;
    YltLaunch cfg;
    ARA_CUDA(c, plan_ylt(c->device, bm, mean_chunks, ys.layout, eb, G, entries * (size_t)(eb * G),
                         c->tuned[eb == 8 ? 1 : 0][G], &cfg),
             "plan YLT launch");
    TimedLaunch tl(c, ARA_TIMING_YLT, s);
    ARA_CUDA(c, launch_ylt_group(ys.coff, ys.chunks, ys.layout, n_trials, table, eb, bitmap, bm, c->catalog,
                                 G, outs, cfg, s),
             "YLT kernel launch");
    tl.done();
  }
  return ARA_OK;
}

}  // namespace ara

void ara::set_context_free_error(const char *msg) { g_create_error = msg ? msg : ""; }

// ======================================================================= ABI
extern "C" {

const char *ara_status_string(ara_status s) {
  switch (s) {
    case ARA_OK: return "ARA_OK";
    case ARA_E_INVALID_ARG: return "ARA_E_INVALID_ARG";
    case ARA_E_EVENT_RANGE: return "ARA_E_EVENT_RANGE";
    case ARA_E_DUP_EVENT: return "ARA_E_DUP_EVENT";
    case ARA_E_NOMEM: return "ARA_E_NOMEM";
    case ARA_E_CUDA: return "ARA_E_CUDA";
    case ARA_E_TIMEOUT: return "ARA_E_TIMEOUT";
    case ARA_E_NOT_FOUND: return "ARA_E_NOT_FOUND";
    case ARA_E_STATE: return "ARA_E_STATE";
    case ARA_E_CANCELLED: return "ARA_E_CANCELLED";
    default: return "ARA_E_UNKNOWN";
  }
}

ara_status ara_create(ara_ctx **out, int device) {
  if (!out) {
    g_create_error = "ara_create: out is NULL";
    return ARA_E_INVALID_ARG;
  }
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    g_create_error = std::string("ara_create: no usable CUDA device (") +
                     (e != cudaSuccess ? cudaGetErrorString(e) : "device count is 0") + ")";
    return ARA_E_CUDA;
  }
  if (device < 0 || device >= n) {
    g_create_error = "ara_create: device index out of range";
    return ARA_E_INVALID_ARG;
  }
  ara_ctx *c = new (std::nothrow) ara_ctx();
  if (!c) {
    g_create_error = "ara_create: out of host memory";
    return ARA_E_NOMEM;
  }
  c->device = device;
  e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
  for (cudaEvent_t &ev : c->load_ev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_counter, 4 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_sel_ws, select_workspace_bytes(kMaxReturnPeriods));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_sel_out, 2 * kMaxReturnPeriods * sizeof(double));
  if (e != cudaSuccess) {
    g_create_error = std::string("ara_create: ") + cudaGetErrorString(e);
    cudaGetLastError();
    ara_destroy(c);
    return e == cudaErrorMemoryAllocation ? ARA_E_NOMEM : ARA_E_CUDA;
  }
  c->stream = c->own_stream;
  *out = c;
  return ARA_OK;
}

void ara_destroy(ara_ctx *c) {
  if (!c) return;
  if (c->service) ara_service_destroy(c->service);
  while (!c->plans.empty()) ara_plan_destroy(c->plans.back());
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  for (auto &L : c->layers) free_layer(L);
  for (auto &B : c->pool) free_buffers(B);
  for (void *p : c->elt_blocks) cudaFree(p);
  cudaFree(c->d_offsets);
  cudaFree(c->d_coff);
  cudaFree(c->d_chunks);
  cudaFree(c->d_dcoff);
  cudaFree(c->d_dchunks);
  cudaFree(c->d_cflag);
  cudaFree(c->d_raw);
  cudaFreeHost(c->h_off_stage);
  cudaFree(c->d_ts);
  cudaFree(c->d_ylt_stage);
  cudaFree(c->d_yelt_stage);
  cudaFree(c->d_elt_scratch);
  cudaFree(c->d_sel_in);
  cudaFree(c->d_sel_ws);
  cudaFree(c->d_sel_out);
  cudaFree(c->d_tail_scratch);
  cudaFree(c->d_evt64);
  cudaFree(c->d_evt64_inexact);
  cudaFree(c->d_yelt_comb);
  cudaFree(c->d_tail);
  cudaFree(c->d_sel_ws_batch);
  cudaFree(c->d_sel_out_batch);
  cudaFree(c->d_pair_table);
  cudaFree(c->d_pair_bitmap);
  cudaFree(c->d_counter);
  cudaFree(c->d_err);
  for (auto &ch : c->chan)
    for (auto &ev : ch.events) {
      cudaEventDestroy(ev.first);
      cudaEventDestroy(ev.second);
    }
  for (cudaEvent_t ev : c->load_ev)
    if (ev) cudaEventDestroy(ev);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  cudaGetLastError();
  delete c;
}

const char *ara_last_error(const ara_ctx *c) {
  // An attached service's thread owns c->err; refusals go to the thread's slot.
  return c && !c->service ? c->err.c_str() : g_create_error.c_str();
}

ara_status ara_set_stream(ara_ctx *c, void *stream) {
  ARA_ENTER(c);
  c->stream = stream ? (cudaStream_t)stream : c->own_stream;
  return ARA_OK;
}

ara_status ara_load_yet(ara_ctx *c, int32_t catalog, int64_t n_trials, const int64_t *offsets,
                        const int32_t *ids, const float *ts) {
  ARA_ENTER(c);
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (ara_status st_ptr = reject_foreign(c, {{offsets, "trial_offsets"}, {ids, "event_ids"}, {ts, "timestamps"}})) return st_ptr;
  if (catalog < 1) return fail(c, ARA_E_INVALID_ARG, "catalog_size must be >= 1 (got %d)", catalog);
  if (n_trials < 0 || n_trials > (int64_t)1 << 40)
    return fail(c, ARA_E_INVALID_ARG, "n_trials out of range (got %lld)", (long long)n_trials);
  if (!offsets) return fail(c, ARA_E_INVALID_ARG, "trial_offsets is NULL");
  cudaStream_t s = c->stream;
  // The id copy (the bulk of the bytes) starts first; the offsets are
  // checked and the chunk layout computed on the host while it runs.
  const bool dev_off = is_device_ptr(offsets);
  int64_t M_claimed = 0;
  if (dev_off) {
    ARA_CUDA(c, cudaMemcpyAsync(&M_claimed, offsets + n_trials, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
             "copy trial_offsets");
    ARA_CUDA(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
  } else {
    M_claimed = offsets[n_trials];
  }
  if (M_claimed < 0) return fail(c, ARA_E_INVALID_ARG, "trial_offsets[n_trials] must be >= 0");
  if (M_claimed > 0 && !ids)
    return fail(c, ARA_E_INVALID_ARG, "event_ids is NULL but offsets hold %lld events", (long long)M_claimed);
  // The ids go to a staging buffer the loaded YET does not use, so a failed
  // check below still leaves the previous YET loaded.
  // Host ids are copied in up to kLoadPieces pieces on the copy stream; the
  // trials a piece completes are chunked while the later pieces are copied.
  // The first piece starts now, the others once the offsets are checked.
  const bool dev_ids = M_claimed > 0 && is_device_ptr(ids);
  int np = 0;      // pieces of the host id copy (0: none)
  int issued = 0;  // pieces whose copy has been issued
  int64_t step = 0;
  auto piece_end = [&](int i) { return i + 1 == np ? M_claimed : step * (i + 1); };
  auto issue_piece = [&](int i) {
    ++issued;
    return cudaMemcpyAsync(c->d_raw + step * i, ids + step * i, (size_t)(piece_end(i) - step * i) * sizeof(int32_t),
                           cudaMemcpyHostToDevice, c->copy_stream);
  };
  // Errors below wait for the id copies before returning (the caller may free ids).
  auto wait_copies = [&]() {
    if (issued > 0) cudaStreamSynchronize(c->copy_stream);
  };
  if (M_claimed > 0 && !dev_ids) {
    ARA_CUDA(c, ensure(&c->d_raw, &c->cap_raw, (size_t)M_claimed), "allocate YET buffers");
    ARA_CUDA(c, cudaEventRecord(c->load_ev[kLoadPieces], s), "cudaEventRecord");
    ARA_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->load_ev[kLoadPieces], 0), "cudaStreamWaitEvent");
    np = (int)std::min<int64_t>(kLoadPieces, std::max<int64_t>(1, M_claimed >> kLoadPieceShift));
    step = M_claimed / np;
    const cudaError_t e = issue_piece(0);
    if (e != cudaSuccess) {
      wait_copies();
      return cuda_fail(c, e, "copy event_ids");
    }
  }
  std::vector<int64_t> h((size_t)n_trials + 1);
  if (dev_off) {
    cudaError_t e = cudaMemcpyAsync(h.data(), offsets, h.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      wait_copies();
      return cuda_fail(c, e, "copy trial_offsets");
    }
  } else {
    std::memcpy(h.data(), offsets, h.size() * sizeof(int64_t));
  }
  auto fail_sync = [&](ara_status st, const char *msg) {
    wait_copies();
    cudaStreamSynchronize(s);
    cudaGetLastError();
    return fail(c, st, "%s", msg);
  };
  if (h[0] != 0) return fail_sync(ARA_E_INVALID_ARG, "trial_offsets[0] must be 0");
  int64_t lmax = 0;
  for (int64_t t = 0; t < n_trials; ++t) {
    const int64_t d = h[t + 1] - h[t];
    if (d < 0) {
      char msg[128];
      snprintf(msg, sizeof(msg), "trial_offsets decreases at trial %lld", (long long)t);
      return fail_sync(ARA_E_INVALID_ARG, msg);
    }
    lmax = std::max(lmax, d);
  }
  const int64_t M = h[n_trials];
  if (M != M_claimed) return fail_sync(ARA_E_INVALID_ARG, "trial_offsets changed while being read");
  if (lmax > ((int64_t)1 << 31) - 1024)
    return fail_sync(ARA_E_INVALID_ARG, "a trial holds more than 2^31-1024 events");
  // ELTs already loaded must still fit the new catalog.
  for (size_t j = 0; j < c->elts.size(); ++j)
    if (c->elts[j].max_id >= catalog) {
      char msg[160];
      snprintf(msg, sizeof(msg), "loaded ELT %zu holds event id %d outside the new catalog of %d", j,
               c->elts[j].max_id, catalog);
      return fail_sync(ARA_E_EVENT_RANGE, msg);
    }
  // Chunked layout: every trial rounded up to whole 16-byte chunks.
  const bool packed = catalog <= kPackedIdLimit;
  const int64_t ipc = packed ? 6 : 4;
  std::vector<int64_t> hp((size_t)n_trials + 1);
  hp[0] = 0;
  for (int64_t t = 0; t < n_trials; ++t)
    hp[(size_t)t + 1] = hp[(size_t)t] + (h[(size_t)t + 1] - h[(size_t)t] + ipc - 1) / ipc;
  const int64_t Mc = hp[(size_t)n_trials];
  // The YET is replaced in place (it can be several GB): from here on a
  // failure leaves the context without a YET.
  c->yet_loaded = false;
  c->yet_version++;
  cudaError_t e = ensure(&c->d_offsets, &c->cap_offsets, (size_t)n_trials + 1);
  if (e == cudaSuccess) e = ensure(&c->d_coff, &c->cap_coff, (size_t)n_trials + 1);
  if (e == cudaSuccess) e = ensure(&c->d_chunks, &c->cap_chunks, (size_t)Mc + kChunkTail);
  if (e == cudaSuccess && ts) e = ensure(&c->d_ts, &c->cap_ts, (size_t)std::max<int64_t>(M, 1));
  if (e != cudaSuccess) {
    wait_copies();
    cudaStreamSynchronize(s);
    return cuda_fail(c, e, "allocate YET buffers");
  }
  if (np > 0) {
    // The offsets go between the first id piece and the second, from pinned
    // memory, so that neither they nor the chunking wait for the whole id copy.
    const size_t n1 = (size_t)n_trials + 1;
    e = ensure_pinned(&c->h_off_stage, &c->cap_off_stage, 2 * n1);
    if (e == cudaSuccess) {
      std::memcpy(c->h_off_stage, h.data(), n1 * sizeof(int64_t));
      std::memcpy(c->h_off_stage + n1, hp.data(), n1 * sizeof(int64_t));
      e = cudaMemcpyAsync(c->d_offsets, c->h_off_stage, n1 * sizeof(int64_t), cudaMemcpyHostToDevice,
                          c->copy_stream);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->d_coff, c->h_off_stage + n1, n1 * sizeof(int64_t), cudaMemcpyHostToDevice,
                          c->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->load_ev[0], c->copy_stream);
    for (int i = 1; i < np && e == cudaSuccess; ++i) {
      e = issue_piece(i);
      if (e == cudaSuccess) e = cudaEventRecord(c->load_ev[i], c->copy_stream);
    }
  } else {
    e = cudaMemcpyAsync(c->d_offsets, h.data(), h.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->d_coff, hp.data(), hp.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  }
  const int32_t *src = (M > 0 && !dev_ids) ? c->d_raw : ids;
  if (e == cudaSuccess && ts && M > 0)
    e = cudaMemcpyAsync(c->d_ts, ts, (size_t)M * sizeof(float), cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counter, 0, 2 * sizeof(unsigned long long), s);
  // Piece i completes the trials whose ids end at or before piece_end(i).
  int64_t t_done = 0;
  for (int i = 0; i < std::max(np, 1) && e == cudaSuccess; ++i) {
    const bool last = i + 1 >= np;
    int64_t t_next = n_trials;
    if (np > 0) {
      e = cudaStreamWaitEvent(s, c->load_ev[i], 0);
      if (!last) t_next = std::upper_bound(h.begin() + 1, h.end(), piece_end(i)) - (h.begin() + 1);
    }
    if (e == cudaSuccess && (t_next > t_done || last))
      e = launch_pad_ids_range(src, c->d_offsets, c->d_coff, t_done, t_next, last, c->d_chunks, catalog,
                               packed, c->d_counter, s);
    t_done = t_next;
  }
  if (e == cudaSuccess && ts) e = launch_check_ts(c->d_offsets, n_trials, c->d_ts, c->d_counter + 1, s);
  unsigned long long bad[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(bad, c->d_counter, sizeof(bad), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    wait_copies();
    return cuda_fail(c, e, "load YET");
  }
  if (bad[0]) return fail(c, ARA_E_EVENT_RANGE, "%llu event ids lie outside [0, %d)", bad[0], catalog);
  if (bad[1])
    return fail(c, ARA_E_INVALID_ARG,
                "%llu time-stamps are non-finite or out of ascending order within a trial", bad[1]);
  c->has_ts = ts != nullptr;
  c->yet_loaded = true;
  c->catalog = catalog;
  c->n_trials = n_trials;
  c->n_occ = M;
  c->max_trial_len = lmax;
  c->h_offsets.swap(h);
  c->h_coff.swap(hp);
  c->packed = packed;
  return ARA_OK;
}

ara_status ara_compact_yet(ara_ctx *c) {
  ARA_ENTER(c);
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (!c->yet_loaded) return fail(c, ARA_E_STATE, "no YET loaded");
  if (!c->packed || c->compact_version == c->yet_version) return ARA_OK;  // nothing to do
  const int64_t n = c->n_trials, M = c->n_occ;
  cudaStream_t s = c->stream;
  ARA_CUDA(c, ensure(&c->d_raw, &c->cap_raw, (size_t)std::max<int64_t>(M, 1)), "compact YET scratch");
  ARA_CUDA(c, ensure(&c->d_cflag, &c->cap_cflag, (size_t)n + 1 + kCompactScanScratch), "compact YET scratch");
  c->compact_version = -1;
  ARA_CUDA(c, ensure(&c->d_dcoff, &c->cap_dcoff, (size_t)n + 1), "compact YET offsets");
  ARA_CUDA(c, launch_compact_sort(c->d_offsets, c->d_coff, c->d_chunks, n, reinterpret_cast<uint32_t *>(c->d_raw),
                                  c->d_cflag, s),
           "reorder trials");
  ARA_CUDA(c, launch_compact_scan(c->d_cflag, n, c->d_dcoff, c->d_cflag + n + 1, s), "scan chunk counts");
  int64_t total = 0;
  ARA_CUDA(c, cudaMemcpyAsync(&total, c->d_cflag + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "copy chunk total");
  ARA_CUDA(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
  ARA_CUDA(c, ensure(&c->d_dchunks, &c->cap_dchunks, (size_t)total + kChunkTail), "compact YET chunks");
  ARA_CUDA(c, launch_compact_encode(c->d_offsets, c->d_coff, c->d_chunks, n, reinterpret_cast<const uint32_t *>(c->d_raw),
                                    c->d_dcoff, c->d_dchunks, s),
           "encode compact YET");
  std::vector<int64_t> plain((size_t)n + 1);
  ARA_CUDA(c, cudaMemcpyAsync(plain.data(), c->d_cflag, plain.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s),
           "copy compact offsets");
  ARA_CUDA(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
  c->h_dcoff.swap(plain);
  c->compact_version = c->yet_version;
  return ARA_OK;
}

ara_status ara_load_elts(ara_ctx *c, int32_t n_elts, const int64_t *off, const int32_t *ids,
                         const double *losses, const double *ded, const double *lim,
                         int32_t *first_handle) {
  ARA_ENTER(c);
  if (!c->yet_loaded) return fail(c, ARA_E_STATE, "load the YET before ELTs (ids are checked against its catalog)");
  if (n_elts < 1) return fail(c, ARA_E_INVALID_ARG, "n_elts must be >= 1");
  if (!off || !ded || !lim || !first_handle) return fail(c, ARA_E_INVALID_ARG, "NULL argument");
  if ((int64_t)c->elts.size() + n_elts > ((int64_t)1 << 30))
    return fail(c, ARA_E_INVALID_ARG, "ELT pool is full");
  for (const void *p : {(const void *)off, (const void *)ids, (const void *)losses, (const void *)ded,
                        (const void *)lim})
    if (p && is_device_ptr(p)) return fail(c, ARA_E_INVALID_ARG, "ELT arrays must be host pointers");
  if (off[0] != 0) return fail(c, ARA_E_INVALID_ARG, "elt_offsets[0] must be 0");
  for (int32_t j = 0; j < n_elts; ++j) {
    if (off[j + 1] < off[j]) return fail(c, ARA_E_INVALID_ARG, "elt_offsets decreases at ELT %d", j);
    if (off[j + 1] - off[j] > (int64_t)c->catalog)
      return fail(c, ARA_E_DUP_EVENT, "ELT %d has more entries than catalog events", j);
    if (!finite_nonneg(ded[j])) return fail(c, ARA_E_INVALID_ARG, "deductible of ELT %d must be finite and >= 0", j);
    if (!limit_ok(lim[j])) return fail(c, ARA_E_INVALID_ARG, "limit of ELT %d must be >= 0 (inf allowed)", j);
  }
  const int64_t total = off[n_elts];
  if (total > 0 && (!ids || !losses)) return fail(c, ARA_E_INVALID_ARG, "event_ids/losses NULL");
  if (total > ((int64_t)1 << 31) - 1)
    return fail(c, ARA_E_INVALID_ARG, "one call loads at most 2^31-1 ELT entries (got %lld)", (long long)total);
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  // The entries go to the device as given; the device checks them, groups
  // each ELT by fold bucket and finds each ELT's largest loss and id.
  const int nb = (c->catalog + kFoldEventsPerCta - 1) / kFoldEventsPerCta;
  const size_t nbk = (size_t)n_elts * (size_t)(nb + 1);
  const int64_t seen_words = ((int64_t)c->catalog + 31) / 32;
  const size_t n_ids_b = ((size_t)total * 4 + 15) / 16 * 16;
  const size_t n_loss_b = (size_t)total * 8;
  const size_t n_bk_b = nbk * 4;
  // scratch: raw ids | raw losses | offsets | seen bits | counts | cursors | maxima | error counts
  const size_t sc_ids = 0, sc_loss = sc_ids + n_ids_b, sc_off = sc_loss + (n_loss_b + 15) / 16 * 16;
  const size_t sc_seen = sc_off + ((size_t)(n_elts + 1) * 8 + 15) / 16 * 16;
  const size_t sc_cnt = sc_seen + ((size_t)n_elts * (size_t)seen_words * 4 + 15) / 16 * 16;
  const size_t sc_cur = sc_cnt + (nbk * 4 + 15) / 16 * 16;
  const size_t sc_maxl = sc_cur + (nbk * 4 + 15) / 16 * 16;
  const size_t sc_maxi = sc_maxl + (size_t)n_elts * 8;
  const size_t sc_bad = sc_maxi + ((size_t)n_elts * 4 + 15) / 16 * 16;
  const size_t sc_total = sc_bad + 3 * 8;
  ARA_CUDA(c, ensure(&c->d_elt_scratch, &c->cap_elt_scratch, sc_total), "ELT ingest scratch");
  unsigned char *sc = c->d_elt_scratch;
  char *blk = nullptr;
  ARA_CUDA(c, cudaMalloc(&blk, std::max<size_t>(n_ids_b + n_loss_b + n_bk_b, 16)), "cudaMalloc(ELT pool)");
  cudaStream_t s = c->stream;
  std::vector<unsigned long long> h_maxl((size_t)n_elts);
  std::vector<int> h_maxi((size_t)n_elts);
  unsigned long long h_bad[3] = {0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(sc + sc_off, off, (size_t)(n_elts + 1) * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && total > 0)
    e = cudaMemcpyAsync(sc + sc_ids, ids, (size_t)total * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && total > 0)
    e = cudaMemcpyAsync(sc + sc_loss, losses, (size_t)total * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc + sc_seen, 0, sc_cnt - sc_seen, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc + sc_cnt, 0, sc_cur - sc_cnt, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc + sc_maxl, 0, (size_t)n_elts * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc + sc_maxi, 0xFF, (size_t)n_elts * 4, s);  // -1
  if (e == cudaSuccess) e = cudaMemsetAsync(sc + sc_bad, 0, 3 * 8, s);
  int32_t *d_bucket = reinterpret_cast<int32_t *>(blk + n_ids_b + n_loss_b);
  if (e == cudaSuccess && total == 0) e = cudaMemsetAsync(d_bucket, 0, n_bk_b, s);
  if (e == cudaSuccess)
    e = launch_elt_ingest(reinterpret_cast<const int64_t *>(sc + sc_off), n_elts, total,
                          reinterpret_cast<const int32_t *>(sc + sc_ids), reinterpret_cast<const double *>(sc + sc_loss),
                          c->catalog, nb, reinterpret_cast<uint32_t *>(sc + sc_seen), seen_words,
                          reinterpret_cast<int32_t *>(sc + sc_cnt), reinterpret_cast<int32_t *>(sc + sc_cur), d_bucket,
                          reinterpret_cast<unsigned long long *>(sc + sc_maxl), reinterpret_cast<int *>(sc + sc_maxi),
                          reinterpret_cast<unsigned long long *>(sc + sc_bad), reinterpret_cast<int32_t *>(blk),
                          reinterpret_cast<double *>(blk + n_ids_b), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_maxl.data(), sc + sc_maxl, (size_t)n_elts * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_maxi.data(), sc + sc_maxi, (size_t)n_elts * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_bad, sc + sc_bad, sizeof(h_bad), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(blk);
    return cuda_fail(c, e, "upload ELTs");
  }
  if (h_bad[0] || h_bad[1] || h_bad[2]) {
    cudaFree(blk);
    if (h_bad[0]) return fail(c, ARA_E_EVENT_RANGE, "%llu ELT event ids lie outside [0, %d)", h_bad[0], c->catalog);
    if (h_bad[2]) return fail(c, ARA_E_DUP_EVENT, "%llu event ids repeat within an ELT", h_bad[2]);
    return fail(c, ARA_E_INVALID_ARG, "%llu ELT losses are not finite and >= 0", h_bad[1]);
  }
  c->elt_blocks.push_back(blk);
  *first_handle = (int32_t)c->elts.size();
  for (int32_t j = 0; j < n_elts; ++j) {
    EltMeta m;
    m.count = (int32_t)(off[j + 1] - off[j]);
    m.deductible = ded[j];
    m.limit = lim[j];
    unsigned long long bits = h_maxl[(size_t)j];
    double mx = 0.0;
    std::memcpy(&mx, &bits, sizeof(mx));
    m.max_loss = mx;
    m.max_id = h_maxi[(size_t)j];
    m.nb = m.count ? nb : 0;
    m.d_ids = reinterpret_cast<const int32_t *>(blk) + off[j];
    m.d_losses = reinterpret_cast<const double *>(blk + n_ids_b) + off[j];
    m.d_bucket = d_bucket + (size_t)j * (size_t)(nb + 1);
    c->elts.push_back(m);
  }
  return ARA_OK;
}

ara_status ara_define_layer(ara_ctx *c, int32_t n_elts, const int32_t *handles, double occ_ret,
                            double occ_lim, double agg_ret, double agg_lim, int32_t precision,
                            int32_t *layer_out) {
  ARA_ENTER(c);
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (!c->yet_loaded) return fail(c, ARA_E_STATE, "no YET loaded");
  if (!layer_out) return fail(c, ARA_E_INVALID_ARG, "NULL argument");
  ara_status st = check_layer_args(c, n_elts, handles, occ_ret, occ_lim, agg_ret, agg_lim, precision);
  if (st) return fail(c, st, "%s", ara_last_error(nullptr));
  return define_layer_on(c, n_elts, handles, occ_ret, occ_lim, agg_ret, agg_lim, precision, c->stream,
                         layer_out);
}

ara_status ara_release_layer(ara_ctx *c, int32_t layer) {
  ARA_ENTER(c);
  LayerRec *L = nullptr;
  ara_status st = get_layer(c, layer, &L);
  if (st) return st;
  recycle_layer(c, *L);
  return ARA_OK;
}

ara_status ara_layer_event_table(ara_ctx *c, int32_t layer, double *out) {
  ARA_ENTER(c);
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (ara_status st_ptr = reject_foreign(c, {{out, "out"}})) return st_ptr;
  LayerRec *L = nullptr;
  ara_status st = get_layer(c, layer, &L);
  if (st) return st;
  if (!out) return fail(c, ARA_E_INVALID_ARG, "out is NULL");
  cudaStream_t s = c->stream;
  const bool dev = is_device_ptr(out);
  double *dst = out;
  if (!dev) {
    ARA_CUDA(c, ensure(&c->d_ylt_stage, &c->cap_ylt_stage, (size_t)c->catalog), "stage buffer");
    dst = c->d_ylt_stage;
  }
  ARA_CUDA(c, launch_fold(L->d_desc, (int)L->elts.size(), c->catalog, L->occ_ret, L->occ_lim, 0,
                          nullptr, nullptr, L->bm, L->precision == ARA_FP32_TABLE, dst, s),
           "fold kernel launch");
  if (!dev) {
    ARA_CUDA(c, cudaMemcpyAsync(out, dst, (size_t)c->catalog * sizeof(double), cudaMemcpyDeviceToHost, s),
             "copy event table");
    ARA_CUDA(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
  }
  return ARA_OK;
}

ara_status ara_layer_ylt(ara_ctx *c, int32_t layer, int64_t n_trials, double *ylt_out,
                         void *cuda_stream) {
  ARA_ENTER(c);
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (ara_status st_ptr = reject_foreign(c, {{ylt_out, "ylt_out"}})) return st_ptr;
  if (!c->yet_loaded) return fail(c, ARA_E_STATE, "no YET loaded");
  LayerRec *L = nullptr;
  ara_status st = get_layer(c, layer, &L);
  if (st) return st;
  if (n_trials < 0 || n_trials > c->n_trials)
    return fail(c, ARA_E_INVALID_ARG, "n_trials %lld outside [0, %lld]", (long long)n_trials,
                (long long)c->n_trials);
  if (n_trials > 0 && !ylt_out) return fail(c, ARA_E_INVALID_ARG, "ylt_out is NULL");
  if (n_trials == 0) return ARA_OK;
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : c->stream;
  if (L->folded_version != c->yet_version) {
    st = fold_layer(c, *L, s);
    if (st) return st;
  }
  const bool dev = is_device_ptr(ylt_out);
  double *dst = ylt_out;
  if (!dev) {
    ARA_CUDA(c, ensure(&c->d_ylt_stage, &c->cap_ylt_stage, (size_t)n_trials), "stage buffer");
    dst = c->d_ylt_stage;
  }
  const YltStream ys = ylt_stream(c, 1);
  const double mean_chunks = (double)ys.h_coff[(size_t)n_trials] / (double)n_trials;
  YltLaunch cfg;
  ARA_CUDA(c, plan_ylt(c->device, L->bm, mean_chunks, ys.layout, L->entry_bytes(), 1,
                       ((size_t)c->catalog + 1) * (size_t)L->entry_bytes(),
                       c->tuned[L->entry_bytes() == 8 ? 1 : 0][1], &cfg),
           "plan YLT launch");
  const LayerOut out{L->q, L->agg_fx, L->agg_ret, L->agg_lim, dst};
  TimedLaunch tl(c, ARA_TIMING_YLT, s);
  ARA_CUDA(c, launch_ylt_group(ys.coff, ys.chunks, ys.layout, n_trials, L->d_table, L->entry_bytes(),
                               L->d_bitmap, L->bm, c->catalog, 1, &out, cfg, s),
           "YLT kernel launch");
  tl.done();
  if (!dev) {
    ARA_CUDA(c, cudaMemcpyAsync(ylt_out, dst, (size_t)n_trials * sizeof(double), cudaMemcpyDeviceToHost, s),
             "copy YLT");
    ARA_CUDA(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
  }
  return ARA_OK;
}

namespace {

// Device input for the selection: ylt itself, or a copy of a host array.
ara_status selection_input(ara_ctx *c, const double *ylt, int64_t n, const double **src) {
  *src = ylt;
  if (!is_device_ptr(ylt)) {
    ARA_CUDA(c, ensure(&c->d_sel_in, &c->cap_sel_in, (size_t)n), "selection input buffer");
    ARA_CUDA(c, cudaMemcpyAsync(c->d_sel_in, ylt, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, c->stream),
             "copy YLT");
    *src = c->d_sel_in;
  }
  return ARA_OK;
}

// PML/TVaR of m values at ranks k[0..n_rp), fixed-point scale of q_count values.
ara_status pml_tvar_ranks(ara_ctx *c, const double *vals, int64_t m, const int64_t *k, int32_t n_rp,
                          int64_t q_count, double *pml_out, double *tvar_out) {
  cudaStream_t s = c->stream;
  const double *src = nullptr;
  ara_status st = selection_input(c, vals, m, &src);
  if (st) return st;
  ARA_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(unsigned int), s), "cudaMemsetAsync");
  TimedLaunch tl(c, ARA_TIMING_PML, s);
  ARA_CUDA(c, launch_pml_tvar(src, m, k, n_rp, c->d_sel_ws, c->d_sel_out, c->d_err, c->device, s, q_count),
           "PML/TVaR kernels");
  tl.done();
  double out[2 * kMaxReturnPeriods];
  unsigned int bad = 0;
  ARA_CUDA(c, cudaMemcpyAsync(out, c->d_sel_out, 2 * (size_t)n_rp * sizeof(double), cudaMemcpyDeviceToHost, s),
           "copy PML/TVaR");
  ARA_CUDA(c, cudaMemcpyAsync(&bad, c->d_err, sizeof(bad), cudaMemcpyDeviceToHost, s), "copy flag");
  ARA_CUDA(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
  if (bad) return fail(c, ARA_E_INVALID_ARG, "trial losses must be finite and >= 0");
  for (int32_t r = 0; r < n_rp; ++r) {
    pml_out[r] = out[r];
    tvar_out[r] = out[n_rp + r];
  }
  return ARA_OK;
}

// k_r = floor(n / RP_r) for every return period, each in [1, k_max].
ara_status ranks_of(ara_ctx *c, int64_t n, const double *rps, int32_t n_rp, int64_t k_max, int64_t *k) {
  if (n_rp < 1 || n_rp > kMaxReturnPeriods || !rps)
    return fail(c, ARA_E_INVALID_ARG, "need 1..%d return periods", kMaxReturnPeriods);
  for (int32_t r = 0; r < n_rp; ++r) {
    if (!(rps[r] >= 1.0)) return fail(c, ARA_E_INVALID_ARG, "return period %d must be >= 1", r);
    const double kk = std::floor((double)n / rps[r]);
    if (kk < 1.0) return fail(c, ARA_E_INVALID_ARG, "return period %g exceeds the %lld trials", rps[r], (long long)n);
    if (kk > (double)k_max)
      return fail(c, ARA_E_INVALID_ARG, "return period %g needs the %.0f largest losses; the tail holds %lld", rps[r],
                  kk, (long long)k_max);
    k[r] = (int64_t)kk;
  }
  return ARA_OK;
}

}  // namespace

ara_status ara_pml_tvar(ara_ctx *c, const double *ylt, int64_t n, const double *rps, int32_t n_rp,
                        double *pml_out, double *tvar_out) {
  ARA_ENTER(c);
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (ara_status st_ptr = reject_foreign(c, {{ylt, "ylt"}})) return st_ptr;
  if (n < 1 || !ylt) return fail(c, ARA_E_INVALID_ARG, "need n >= 1 trial losses");
  if (!pml_out || !tvar_out) return fail(c, ARA_E_INVALID_ARG, "NULL output array");
  int64_t k[kMaxReturnPeriods];
  ara_status st = ranks_of(c, n, rps, n_rp, n, k);
  if (st) return st;
  return pml_tvar_ranks(c, ylt, n, k, n_rp, n, pml_out, tvar_out);
}

}  // extern "C"

namespace {

// The queued form's results: the selection's outputs, or quiet NaNs when the
// losses failed their check (which the synchronous form reports as a status).
__global__ void pml_tvar_out_kernel(const double *__restrict__ sel_out, const unsigned int *__restrict__ err, int n,
                                    double *__restrict__ out) {
  const int i = threadIdx.x;
  if (i < n) out[i] = *err ? __longlong_as_double(0x7FF8000000000000LL) : sel_out[i];
}

cudaError_t launch_pml_tvar_out(const double *sel_out, const unsigned int *err, int n, double *out, cudaStream_t s) {
  pml_tvar_out_kernel<<<1, 2 * kMaxReturnPeriods, 0, s>>>(sel_out, err, n, out);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

ara_status ara_pml_tvar_async(ara_ctx *c, const double *ylt, int64_t n, const double *rps, int32_t n_rp,
                              double *out) {
  ARA_ENTER(c);
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (ara_status st_ptr = reject_foreign(c, {{ylt, "ylt"}, {out, "out"}})) return st_ptr;
  if (n < 1 || !ylt) return fail(c, ARA_E_INVALID_ARG, "need n >= 1 trial losses");
  if (!out) return fail(c, ARA_E_INVALID_ARG, "NULL output array");
  if (!is_device_ptr(ylt) || !is_device_ptr(out))
    return fail(c, ARA_E_INVALID_ARG, "ylt and out must be device memory");
  int64_t k[kMaxReturnPeriods];
  ara_status st = ranks_of(c, n, rps, n_rp, n, k);
  if (st) return st;
  cudaStream_t s = c->stream;
  ARA_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(unsigned int), s), "cudaMemsetAsync");
  TimedLaunch tl(c, ARA_TIMING_PML, s);
  ARA_CUDA(c, launch_pml_tvar(ylt, n, k, n_rp, c->d_sel_ws, c->d_sel_out, c->d_err, c->device, s, n),
           "PML/TVaR kernels");
  tl.done();
  ARA_CUDA(c, launch_pml_tvar_out(c->d_sel_out, c->d_err, 2 * n_rp, out, s), "PML/TVaR output");
  return ARA_OK;
}

ara_status ara_ylt_tail(ara_ctx *c, const double *ylt, int64_t n, int64_t k, double *tail_out) {
  ARA_ENTER(c);
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (ara_status st_ptr = reject_foreign(c, {{ylt, "ylt"}, {tail_out, "tail_out"}})) return st_ptr;
  if (n < 1 || !ylt) return fail(c, ARA_E_INVALID_ARG, "need n >= 1 trial losses");
  if (k < 1 || k > n) return fail(c, ARA_E_INVALID_ARG, "k = %lld outside [1, %lld]", (long long)k, (long long)n);
  if (!tail_out) return fail(c, ARA_E_INVALID_ARG, "tail_out is NULL");
  cudaStream_t s = c->stream;
  const double *src = nullptr;
  ara_status st = selection_input(c, ylt, n, &src);
  if (st) return st;
  const bool dev = is_device_ptr(tail_out);
  double *dst = tail_out;
  if (!dev) {
    ARA_CUDA(c, ensure(&c->d_tail, &c->cap_tail, (size_t)k), "tail output buffer");
    dst = c->d_tail;
  }
  ARA_CUDA(c, ensure(&c->d_tail_scratch, &c->cap_tail_scratch, (size_t)kTailScratch), "tail scratch");
  ARA_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(unsigned int), s), "cudaMemsetAsync");
  // The selection's PML at rank k is the threshold tau (d_sel_out[0]).
  ARA_CUDA(c, launch_pml_tvar(src, n, &k, 1, c->d_sel_ws, c->d_sel_out, c->d_err, c->device, s), "select tau");
  ARA_CUDA(c, launch_ylt_tail(src, n, k, c->d_sel_out, c->d_tail_scratch, dst, s), "tail kernels");
  if (!dev)
    ARA_CUDA(c, cudaMemcpyAsync(tail_out, dst, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, s), "copy tail");
  unsigned int bad = 0;
  ARA_CUDA(c, cudaMemcpyAsync(&bad, c->d_err, sizeof(bad), cudaMemcpyDeviceToHost, s), "copy flag");
  ARA_CUDA(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
  if (bad) return fail(c, ARA_E_INVALID_ARG, "trial losses must be finite and >= 0");
  return ARA_OK;
}

ara_status ara_pml_tvar_tail(ara_ctx *c, const double *tail, int64_t m, int64_t n_total, const double *rps,
                             int32_t n_rp, double *pml_out, double *tvar_out) {
  ARA_ENTER(c);
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (ara_status st_ptr = reject_foreign(c, {{tail, "tail"}})) return st_ptr;
  if (m < 1 || !tail) return fail(c, ARA_E_INVALID_ARG, "need m >= 1 tail values");
  if (n_total < m) return fail(c, ARA_E_INVALID_ARG, "n_total %lld < m %lld", (long long)n_total, (long long)m);
  if (!pml_out || !tvar_out) return fail(c, ARA_E_INVALID_ARG, "NULL output array");
  int64_t k[kMaxReturnPeriods];
  ara_status st = ranks_of(c, n_total, rps, n_rp, m, k);
  if (st) return st;
  return pml_tvar_ranks(c, tail, m, k, n_rp, n_total, pml_out, tvar_out);
}

ara_status ara_layers_ylt(ara_ctx *c, int32_t n_layers, const int32_t *layers, int64_t n_trials,
                          double *ylt_out, void *cuda_stream) {
  ARA_ENTER(c);
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (ara_status st_ptr = reject_foreign(c, {{ylt_out, "ylt_out"}})) return st_ptr;
  if (!c->yet_loaded) return fail(c, ARA_E_STATE, "no YET loaded");
  if (n_layers < 1 || !layers) return fail(c, ARA_E_INVALID_ARG, "need n_layers >= 1 layer handles");
  if (n_trials < 0 || n_trials > c->n_trials)
    return fail(c, ARA_E_INVALID_ARG, "n_trials %lld outside [0, %lld]", (long long)n_trials,
                (long long)c->n_trials);
  if (n_trials > 0 && !ylt_out) return fail(c, ARA_E_INVALID_ARG, "ylt_out is NULL");
  LayerRec *first = nullptr;
  for (int32_t i = 0; i < n_layers; ++i) {
    ara_status st = get_layer(c, layers[i], &first);
    if (st) return st;
  }
  if (n_trials == 0) return ARA_OK;
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : c->stream;
  const bool dev = is_device_ptr(ylt_out);
  double *dst = ylt_out;
  const size_t total = (size_t)n_layers * (size_t)n_trials;
  if (!dev) {
    ARA_CUDA(c, ensure(&c->d_ylt_stage, &c->cap_ylt_stage, total), "stage buffer");
    dst = c->d_ylt_stage;
  }
  if (n_layers > 1) {
    const size_t entries = (size_t)c->catalog + 1;
    const BitmapLayout bm = plan_bitmap(c->catalog + 1, ylt_smem_budget(c->device));
    ARA_CUDA(c, ensure(&c->d_pair_table, &c->cap_pair_table, 2 * entries), "pair table");
    ARA_CUDA(c, ensure(&c->d_pair_bitmap, &c->cap_pair_bitmap, (size_t)bm.words), "pair bitmap");
  }
  ara_status st = layers_ylt_on(c, layers, n_layers, n_trials, dst, s, c->d_pair_table, c->d_pair_bitmap);
  if (st) return st;
  if (!dev) {
    ARA_CUDA(c, cudaMemcpyAsync(ylt_out, dst, total * sizeof(double), cudaMemcpyDeviceToHost, s), "copy YLTs");
    ARA_CUDA(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
  }
  return ARA_OK;
}

ara_status ara_layer_yelt(ara_ctx *c, int32_t layer, int64_t n_trials, double *yelt_out,
                          double *occ_max_out, void *cuda_stream) {
  ARA_ENTER(c);
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (ara_status st_ptr = reject_foreign(c, {{yelt_out, "yelt_out"}, {occ_max_out, "occ_max_out"}})) return st_ptr;
  if (!c->yet_loaded) return fail(c, ARA_E_STATE, "no YET loaded");
  LayerRec *L = nullptr;
  ara_status st = get_layer(c, layer, &L);
  if (st) return st;
  if (n_trials < 0 || n_trials > c->n_trials)
    return fail(c, ARA_E_INVALID_ARG, "n_trials %lld outside [0, %lld]", (long long)n_trials,
                (long long)c->n_trials);
  if (n_trials == 0) return ARA_OK;
  const int64_t M = c->h_offsets[(size_t)n_trials];
  if (M > 0 && !yelt_out && !occ_max_out) return fail(c, ARA_E_INVALID_ARG, "no output given");
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : c->stream;
  if (L->folded_version != c->yet_version) {
    st = fold_layer(c, *L, s);
    if (st) return st;
  }
  const bool ydev = yelt_out && is_device_ptr(yelt_out);
  const bool odev = occ_max_out && is_device_ptr(occ_max_out);
  double *ydst = ydev ? yelt_out : nullptr;
  double *odst = odev ? occ_max_out : nullptr;
  if (yelt_out && !ydev) {
    ARA_CUDA(c, ensure(&c->d_yelt_stage, &c->cap_yelt_stage, (size_t)M), "YELT stage buffer");
    ydst = c->d_yelt_stage;
  }
  if (occ_max_out && !odev) {
    ARA_CUDA(c, ensure(&c->d_ylt_stage, &c->cap_ylt_stage, (size_t)n_trials), "stage buffer");
    odst = c->d_ylt_stage;
  }
  const LayerOut out{L->q, L->agg_fx, L->agg_ret, L->agg_lim, nullptr};
  if (ydst) {
    // The layer's table in binary64 (the event table), with a flag set when
    // some value is not exactly on the table's grid: in-layer increments are
    // then read from it instead of converted one by one.
    ARA_CUDA(c, ensure(&c->d_evt64, &c->cap_evt64, (size_t)c->catalog + 1), "binary64 event table");
    ARA_CUDA(c, ensure(&c->d_evt64_inexact, &c->cap_evt64_inexact, 1), "binary64 event table flag");
    ARA_CUDA(c, cudaMemsetAsync(c->d_evt64 + c->catalog, 0, sizeof(double), s), "cudaMemsetAsync");
    ARA_CUDA(c, cudaMemsetAsync(c->d_evt64_inexact, 0, sizeof(unsigned int), s), "cudaMemsetAsync");
    ARA_CUDA(c, launch_fold(L->d_desc, (int)L->elts.size(), c->catalog, L->occ_ret, L->occ_lim, L->q, nullptr,
                            nullptr, L->bm, L->precision == ARA_FP32_TABLE, c->d_evt64, s, c->d_evt64_inexact),
             "binary64 event table");
    // ... interleaved with the layer's entries, so the kernel's one gather per
    // occurrence brings both
    ARA_CUDA(c, ensure(&c->d_yelt_comb, &c->cap_yelt_comb, ((size_t)c->catalog + 1) * (L->entry_bytes() == 16 ? 2 : 1)),
             "YELT event table");
    ARA_CUDA(c, launch_yelt_comb(L->d_table, L->entry_bytes(), c->d_evt64, (int64_t)c->catalog + 1, c->d_yelt_comb, s),
             "YELT event table");
  }
  TimedLaunch tl(c, ARA_TIMING_YELT, s);
  ARA_CUDA(c, launch_yelt(c->d_coff, c->d_chunks, c->d_offsets, c->packed, n_trials, L->d_table,
                          L->entry_bytes(), L->d_bitmap, L->bm, c->catalog, out, ydst, odst, c->device, s,
                          ydst ? c->d_yelt_comb : nullptr, c->d_evt64_inexact),
           "YELT kernel launch");
  tl.done();
  if (yelt_out && !ydev)
    ARA_CUDA(c, cudaMemcpyAsync(yelt_out, ydst, (size_t)M * sizeof(double), cudaMemcpyDeviceToHost, s),
             "copy YELT");
  if (occ_max_out && !odev)
    ARA_CUDA(c, cudaMemcpyAsync(occ_max_out, odst, (size_t)n_trials * sizeof(double), cudaMemcpyDeviceToHost, s),
             "copy occurrence maxima");
  if ((yelt_out && !ydev) || (occ_max_out && !odev))
    ARA_CUDA(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
  return ARA_OK;
}

ara_status ara_rpl_report(ara_ctx *c, int32_t layer, int64_t n_trials, const double *rps, int32_t n_rp,
                          double *aep_out, double *aep_tvar_out, double *oep_out, double *oep_tvar_out) {
  ARA_ENTER(c);
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (!c->yet_loaded) return fail(c, ARA_E_STATE, "no YET loaded");
  LayerRec *L = nullptr;
  ara_status st = get_layer(c, layer, &L);
  if (st) return st;
  if (n_trials < 1 || n_trials > c->n_trials)
    return fail(c, ARA_E_INVALID_ARG, "n_trials %lld outside [1, %lld]", (long long)n_trials,
                (long long)c->n_trials);
  if (!aep_out || !aep_tvar_out || !oep_out || !oep_tvar_out)
    return fail(c, ARA_E_INVALID_ARG, "NULL output array");
  int64_t k[kMaxReturnPeriods];
  if (tail_counts(n_trials, rps, n_rp, k) != ARA_OK) return fail(c, ARA_E_INVALID_ARG, "%s", ara_last_error(nullptr));
  cudaStream_t s = c->stream;
  if (L->folded_version != c->yet_version) {
    st = fold_layer(c, *L, s);
    if (st) return st;
  }
  // [0, n): trial losses (AEP); [n, 2n): largest increment per trial (OEP)
  ARA_CUDA(c, ensure(&c->d_sel_in, &c->cap_sel_in, 2 * (size_t)n_trials), "report buffer");
  const LayerOut out{L->q, L->agg_fx, L->agg_ret, L->agg_lim, c->d_sel_in};
  TimedLaunch tl(c, ARA_TIMING_YELT, s);
  ARA_CUDA(c, launch_yelt(c->d_coff, c->d_chunks, c->d_offsets, c->packed, n_trials, L->d_table,
                          L->entry_bytes(), L->d_bitmap, L->bm, c->catalog, out, nullptr, c->d_sel_in + n_trials,
                          c->device, s),
           "YELT kernel launch");
  tl.done();
  ARA_CUDA(c, ensure(&c->d_sel_ws_batch, &c->cap_sel_ws_batch, 2 * select_workspace_bytes(kMaxReturnPeriods)),
           "selection workspace");
  ARA_CUDA(c, ensure(&c->d_sel_out_batch, &c->cap_sel_out_batch, 4 * (size_t)n_rp), "selection output");
  ARA_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(unsigned int), s), "cudaMemsetAsync");
  ARA_CUDA(c, launch_pml_tvar_batch(c->d_sel_in, 2, n_trials, k, n_rp, c->d_sel_ws_batch, c->d_sel_out_batch,
                                    c->d_err, c->device, s),
           "PML/TVaR kernels");
  std::vector<double> res(4 * (size_t)n_rp);
  ARA_CUDA(c, cudaMemcpyAsync(res.data(), c->d_sel_out_batch, res.size() * sizeof(double), cudaMemcpyDeviceToHost, s),
           "copy report");
  ARA_CUDA(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
  for (int32_t r = 0; r < n_rp; ++r) {
    aep_out[r] = res[(size_t)r];
    aep_tvar_out[r] = res[(size_t)n_rp + r];
    oep_out[r] = res[2 * (size_t)n_rp + r];
    oep_tvar_out[r] = res[3 * (size_t)n_rp + r];
  }
  return ARA_OK;
}

ara_status ara_pml_tvar_batch(ara_ctx *c, const double *ylt, int32_t n_layers, int64_t n,
                              const double *rps, int32_t n_rp, double *pml_out, double *tvar_out) {
  ARA_ENTER(c);
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (ara_status st_ptr = reject_foreign(c, {{ylt, "ylt"}})) return st_ptr;
  if (n < 1 || !ylt || n_layers < 1) return fail(c, ARA_E_INVALID_ARG, "need n_layers >= 1 and n >= 1 trial losses");
  if (n_layers > 65535) return fail(c, ARA_E_INVALID_ARG, "at most 65535 layers per call");
  if (n_rp < 1 || n_rp > kMaxReturnPeriods || !rps || !pml_out || !tvar_out)
    return fail(c, ARA_E_INVALID_ARG, "need 1..%d return periods and output arrays", kMaxReturnPeriods);
  int64_t k[kMaxReturnPeriods];
  for (int32_t r = 0; r < n_rp; ++r) {
    if (!(rps[r] >= 1.0)) return fail(c, ARA_E_INVALID_ARG, "return period %d must be >= 1", r);
    const double kk = std::floor((double)n / rps[r]);
    if (kk < 1.0) return fail(c, ARA_E_INVALID_ARG, "return period %g exceeds the %lld trials", rps[r], (long long)n);
    k[r] = (int64_t)kk;
  }
  cudaStream_t s = c->stream;
  const size_t total = (size_t)n_layers * (size_t)n;
  const double *src = ylt;
  if (!is_device_ptr(ylt)) {
    ARA_CUDA(c, ensure(&c->d_sel_in, &c->cap_sel_in, total), "selection input buffer");
    ARA_CUDA(c, cudaMemcpyAsync(c->d_sel_in, ylt, total * sizeof(double), cudaMemcpyHostToDevice, s),
             "copy YLTs");
    src = c->d_sel_in;
  }
  ARA_CUDA(c, ensure(&c->d_sel_ws_batch, &c->cap_sel_ws_batch,
                     (size_t)n_layers * select_workspace_bytes(kMaxReturnPeriods)),
           "selection workspace");
  ARA_CUDA(c, ensure(&c->d_sel_out_batch, &c->cap_sel_out_batch, (size_t)n_layers * 2 * (size_t)n_rp),
           "selection output");
  ARA_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(unsigned int), s), "cudaMemsetAsync");
  TimedLaunch tl(c, ARA_TIMING_PML, s);
  ARA_CUDA(c, launch_pml_tvar_batch(src, n_layers, n, k, n_rp, c->d_sel_ws_batch, c->d_sel_out_batch,
                                    c->d_err, c->device, s),
           "PML/TVaR kernels");
  tl.done();
  std::vector<double> out((size_t)n_layers * 2 * (size_t)n_rp);
  unsigned int bad = 0;
  ARA_CUDA(c, cudaMemcpyAsync(out.data(), c->d_sel_out_batch, out.size() * sizeof(double),
                              cudaMemcpyDeviceToHost, s),
           "copy PML/TVaR");
  ARA_CUDA(c, cudaMemcpyAsync(&bad, c->d_err, sizeof(bad), cudaMemcpyDeviceToHost, s), "copy flag");
  ARA_CUDA(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
  if (bad) return fail(c, ARA_E_INVALID_ARG, "trial losses must be finite and >= 0");
  for (int32_t l = 0; l < n_layers; ++l)
    for (int32_t r = 0; r < n_rp; ++r) {
      pml_out[(size_t)l * n_rp + r] = out[(size_t)l * 2 * n_rp + r];
      tvar_out[(size_t)l * n_rp + r] = out[(size_t)l * 2 * n_rp + n_rp + r];
    }
  return ARA_OK;
}

ara_status ara_set_kernel_timing(ara_ctx *c, int32_t enable) {
  ARA_ENTER(c);
  for (auto &ch : c->chan) {
    for (auto &ev : ch.events) {
      cudaEventSynchronize(ev.second);
      cudaEventDestroy(ev.first);
      cudaEventDestroy(ev.second);
    }
    ch.events.clear();
    ch.launches = 0;
    ch.total_ms = 0.0;
  }
  c->timing = enable != 0;
  return ARA_OK;
}

ara_status ara_kernel_timing(ara_ctx *c, int32_t channel, int64_t *launches, double *total_ms) {
  ARA_ENTER(c);
  if (channel < 0 || channel > ARA_TIMING_YELT || !launches || !total_ms)
    return fail(c, ARA_E_INVALID_ARG, "bad timing channel or NULL output");
  TimingChannel &ch = c->chan[channel];
  for (auto &ev : ch.events) {
    ARA_CUDA(c, cudaEventSynchronize(ev.second), "cudaEventSynchronize");
    float ms = 0.f;
    ARA_CUDA(c, cudaEventElapsedTime(&ms, ev.first, ev.second), "cudaEventElapsedTime");
    ch.total_ms += ms;
    ch.launches += 1;
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  ch.events.clear();
  *launches = ch.launches;
  *total_ms = ch.total_ms;
  return ARA_OK;
}

}  // extern "C"
