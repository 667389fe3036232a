// Internal state of a context (struct ara_ctx) and the host helpers shared by
// the C ABI (ara_api.cu) and the pricing service (service.cu).
#pragma once

#include <cuda_runtime.h>

#include <initializer_list>
#include <string>
#include <utility>
#include <vector>

#include "ara.h"
#include "ara_internal.cuh"
#include "yet_load.cuh"

namespace ara {

struct EltMeta {
  int32_t count = 0;
  double deductible = 0.0;
  double limit = 0.0;
  double max_loss = 0.0;
  int32_t max_id = -1;
  const int32_t *d_ids = nullptr;
  const double *d_losses = nullptr;
  const int32_t *d_bucket = nullptr;
  int32_t nb = 0;
};

struct LayerRec {
  bool live = false;
  uint64_t gen = 0;  // distinct for every definition (plans detect redefinition)
  std::vector<int32_t> elts;
  double occ_ret = 0, occ_lim = 0, agg_ret = 0, agg_lim = 0;
  int32_t precision = ARA_FP64;
  EltDesc *d_desc = nullptr;
  int32_t desc_cap = 0;
  ulonglong2 *d_table = nullptr;
  uint32_t *d_bitmap = nullptr;
  int32_t table_catalog = 0;
  BitmapLayout bm{0u, 0};
  int q = 0;
  AggFixed agg_fx{{0ull, 0ull}, {0ull, 0ull}, 0};
  int64_t folded_version = -1;
  double upper = 0.0;  // upper bound of any per-event table value
  // Table entry width: 128-bit entries for FP64 layers, 64-bit entries (the
  // first half of the same buffer) for FP32-table layers.
  int entry_bytes() const { return precision == ARA_FP32_TABLE ? 8 : 16; }
};

// Device buffers of a released layer, kept for the next layer (defining and
// releasing layers then needs no cudaMalloc/cudaFree, which would stall the
// device).  Reuse is ordered by the context's stream.
struct LayerBuffers {
  EltDesc *d_desc = nullptr;
  int32_t desc_cap = 0;
  ulonglong2 *d_table = nullptr;
  uint32_t *d_bitmap = nullptr;
  int32_t table_catalog = 0;
  BitmapLayout bm{0u, 0};
};

constexpr size_t kLayerPoolMax = 64;

struct TimingChannel {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
  int64_t launches = 0;
  double total_ms = 0.0;
};

}  // namespace ara

struct ara_ctx {
  using EltMeta = ara::EltMeta;
  using LayerRec = ara::LayerRec;
  using LayerBuffers = ara::LayerBuffers;
  using TimingChannel = ara::TimingChannel;
  using EltDesc = ara::EltDesc;

  int device = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  // host-to-device YET id copies run here, in pieces, each followed by an
  // event; load_ev[kLoadPieces] orders the copies after the work on stream
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t load_ev[ara::kLoadPieces + 1] = {};
  std::string err;
  // YET
  int64_t yet_version = 0;
  uint64_t layer_gen = 0;           // last LayerRec::gen handed out
  bool yet_loaded = false;
  int32_t catalog = 0;
  int64_t n_trials = 0;
  int64_t n_occ = 0;
  int64_t max_trial_len = 0;
  std::vector<int64_t> h_offsets;   // raw CSR offsets
  std::vector<int64_t> h_coff;      // chunk offsets
  int64_t *d_offsets = nullptr;     // raw offsets
  size_t cap_offsets = 0;
  int64_t *d_coff = nullptr;        // chunk offsets
  size_t cap_coff = 0;
  int4 *d_chunks = nullptr;         // id chunks + sentinel tail
  size_t cap_chunks = 0;
  bool packed = false;              // 6 ids of 21 bits per chunk
  // compact id stream for YLT passes (ara_compact_yet): valid while
  // compact_version == yet_version
  int64_t compact_version = -1;
  std::vector<int64_t> h_dcoff;     // chunk offsets (without flags)
  int64_t *d_dcoff = nullptr;       // chunk offsets, bit 62 = difference-coded trial
  size_t cap_dcoff = 0;
  int4 *d_dchunks = nullptr;
  size_t cap_dchunks = 0;
  int64_t *d_cflag = nullptr;       // per-trial chunk count and flag (scratch)
  size_t cap_cflag = 0;
  int32_t *d_raw = nullptr;         // staging for ids copied from the host
  size_t cap_raw = 0;
  int64_t *h_off_stage = nullptr;   // pinned: raw then chunk offsets, copied between id pieces
  size_t cap_off_stage = 0;
  float *d_ts = nullptr;
  size_t cap_ts = 0;
  bool has_ts = false;
  // ELT pool
  std::vector<EltMeta> elts;
  std::vector<void *> elt_blocks;
  // layers
  std::vector<LayerRec> layers;
  std::vector<LayerBuffers> pool;
  // scratch
  double *d_ylt_stage = nullptr;
  size_t cap_ylt_stage = 0;
  double *d_yelt_stage = nullptr;           // per-occurrence output for host callers
  size_t cap_yelt_stage = 0;
  unsigned char *d_elt_scratch = nullptr;   // ELT ingest: raw entries, counts, checks
  size_t cap_elt_scratch = 0;
  double *d_sel_in = nullptr;
  size_t cap_sel_in = 0;
  void *d_sel_ws = nullptr;
  double *d_sel_out = nullptr;
  unsigned char *d_sel_ws_batch = nullptr;  // per-layer selection states
  size_t cap_sel_ws_batch = 0;
  double *d_sel_out_batch = nullptr;
  size_t cap_sel_out_batch = 0;
  double *d_evt64 = nullptr;                // ara_layer_yelt: the layer's table in binary64
  ulonglong2 *d_yelt_comb = nullptr;  // the YELT's interleaved entry + binary64 table
  size_t cap_yelt_comb = 0;
  size_t cap_evt64 = 0;
  unsigned int *d_evt64_inexact = nullptr;  // set when that table is not exact
  size_t cap_evt64_inexact = 0;
  int64_t *d_tail_scratch = nullptr;        // ara_ylt_tail: block counts
  size_t cap_tail_scratch = 0;
  double *d_tail = nullptr;                 // ara_ylt_tail: output for host callers
  size_t cap_tail = 0;
  ulonglong2 *d_pair_table = nullptr;       // two layers' tables interleaved
  size_t cap_pair_table = 0;
  uint32_t *d_pair_bitmap = nullptr;        // union of their bitmaps
  size_t cap_pair_bitmap = 0;
  ara::YltShape tuned[2][5];                // YLT launch shape chosen by the autotuner: [entry 8 B][G]
  unsigned long long *d_counter = nullptr;  // validation counters
  unsigned int *d_err = nullptr;            // PML/TVaR input check flag
  // timing
  bool timing = false;
  TimingChannel chan[4];
  // pricing service that owns the context while attached (service.cu)
  ara_service *service = nullptr;
  // live pricing plans (plan.cu), destroyed with the context
  std::vector<ara_plan *> plans;
  size_t pool_max = ara::kLayerPoolMax;     // released layers kept for reuse
};

namespace ara {

ara_status fail(ara_ctx *c, ara_status st, const char *fmt, ...);
ara_status cuda_fail(ara_ctx *c, cudaError_t e, const char *what);

#define ARA_CUDA(ctx, expr, what)                                 \
  do {                                                            \
    cudaError_t _e = (expr);                                      \
    if (_e != cudaSuccess) return ara::cuda_fail((ctx), _e, (what)); \
  } while (0)

bool is_device_ptr(const void *p);
// ARA_E_INVALID_ARG (message naming the argument) when one of the pointers is
// device memory of a GPU other than the current one (the context's).
ara_status reject_foreign(ara_ctx *c, std::initializer_list<std::pair<const void *, const char *>> ptrs);

template <typename T>
cudaError_t ensure(T **buf, size_t *cap, size_t count) {
  if (*cap >= count && *buf) return cudaSuccess;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc((void **)buf, (count > 0 ? count : 1) * sizeof(T));
  if (e == cudaSuccess) *cap = count > 0 ? count : 1;
  return e;
}

// The same for pinned host memory (page-locked, so copies from it are
// asynchronous).
template <typename T>
cudaError_t ensure_pinned(T **buf, size_t *cap, size_t count) {
  if (*cap >= count && *buf) return cudaSuccess;
  if (*buf) cudaFreeHost(*buf);
  *buf = nullptr;
  *cap = 0;
  cudaError_t e = cudaMallocHost((void **)buf, (count > 0 ? count : 1) * sizeof(T));
  if (e == cudaSuccess) *cap = count > 0 ? count : 1;
  return e;
}

// Message into the calling thread's context-free error slot (read with
// ara_last_error(NULL)); returns st.
ara_status fail_free(ara_status st, const char *fmt, ...);

// The id stream a YLT pass of G layers reads: the compact one when it is
// current and G == 1 (measured on B300: 3% faster for one-layer passes,
// 5-10% slower for multi-layer passes, whose gathers dominate and which run
// without the L2 prefetch), else the stored-order chunks.
struct YltStream {
  const int64_t *coff;
  const int4 *chunks;
  int layout;               // as launch_ylt_group
  const int64_t *h_coff;    // host copy of the chunk offsets (no flags)
};
YltStream ylt_stream(const ara_ctx *c, int G);

ara_status fold_layer(ara_ctx *c, LayerRec &L, cudaStream_t s);
// The device work of fold_layer for a layer whose buffers exist and whose
// grid (q) is set: queue only memsets and the fold kernel.
ara_status enqueue_fold(ara_ctx *c, const LayerRec &L, cudaStream_t s);
void recycle_layer(ara_ctx *c, LayerRec &L);
ara_status get_layer(ara_ctx *c, int32_t layer, LayerRec **out);
// Fill the pool with buffers for `count` layers of the loaded catalog (within
// pool_max), so that defining that many layers allocates nothing.
ara_status reserve_layers(ara_ctx *c, size_t count, cudaStream_t s);

// Checks of ara_define_layer that need no device work (terms, handles);
// the message goes to ara_last_error(NULL) so that any thread may call it.
ara_status check_layer_args(const ara_ctx *c, int32_t n_elts, const int32_t *handles, double occ_ret,
                            double occ_lim, double agg_ret, double agg_lim, int32_t precision);

// Return periods -> k = floor(n / RP) per period (each >= 1); message to
// ara_last_error(NULL) on failure.
ara_status tail_counts(int64_t n, const double *rps, int32_t n_rp, int64_t *k);

// Device bytes of a layer's zero-skip bitmap for the loaded catalog.
size_t layer_bitmap_bytes(const ara_ctx *c);

// ara_define_layer after check_layer_args, its device work queued on stream s.
// stage: NULL, or pinned host memory for n_elts ELT descriptors that stays
// untouched until the stream has run the upload (the copy is then fully
// asynchronous; from pageable memory the driver may wait on the stream).
ara_status define_layer_on(ara_ctx *c, int32_t n_elts, const int32_t *handles, double occ_ret,
                           double occ_lim, double agg_ret, double agg_lim, int32_t precision,
                           cudaStream_t s, int32_t *layer_out, EltDesc *stage = nullptr);

// The layers of one YLT pass: their entry width (16 FP64, 8 FP32-table) and
// their positions in a layer list (1 or 2 layers of 16 bytes, 1, 2 or 4 of 8
// bytes: at most one 32-byte sector per event).
struct LayerGroup {
  int eb;
  std::vector<int32_t> idx;
};

// Passes over the layers Ls in list order, g16 FP64 layers or g8 FP32-table
// layers to a pass (a group of three splits 2 + 1).
std::vector<LayerGroup> group_in_order(const std::vector<LayerRec *> &Ls, int g16, int g8);

// Passes whose layers share most of their possibly nonzero events: layers
// taken densest first, each pass filled with the layers whose zero-skip
// bitmaps overlap its union most (bitmaps copied to the host on stream s;
// among the next 64 layers in density order, on a sample of the bitmap words
// beyond 128 layers).  A pass gathers one table row for every occurrence
// that any of its layers needs, so overlapping layers gather fewer rows.
// g16 / g8 as above.
ara_status group_by_overlap(ara_ctx *c, const std::vector<LayerRec *> &Ls, int g16, int g8, cudaStream_t s,
                            std::vector<LayerGroup> *out);

// The kernels of ara_layers_ylt on stream s: device output dst (layer-major),
// pair_table / pair_bitmap scratch of 2 * (catalog + 1) entries and of the
// layers' bitmap size.  Layers must be folded for the loaded YET.  groups:
// the passes to run (positions in layers), or NULL for group_in_order(2, 4).
// tables: for each group of groups, an interleaved table and union bitmap
// already written for it (by a plan's folds), used instead of interleaving
// the layers' tables into pair_table (NULL entries: interleave as usual).
struct GroupTable {
  const void *table;
  const uint32_t *bitmap;
};
ara_status layers_ylt_on(ara_ctx *c, const int32_t *layers, int32_t n_layers, int64_t n_trials,
                         double *dst, cudaStream_t s, ulonglong2 *pair_table, uint32_t *pair_bitmap,
                         const std::vector<LayerGroup> *groups = nullptr,
                         const std::vector<GroupTable> *tables = nullptr);

}  // namespace ara
