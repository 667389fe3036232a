// Pricing plans: the whole batched step for a fixed list of layers -- every
// layer's ELT fold, the grouped YLT passes over the YET and the batched
// PML/TVaR selection -- captured once into a CUDA graph and replayed with one
// launch (Section III: a Program or Portfolio is a set of Layers, each priced
// by Algorithm 1).  A plan groups its layers into passes whose layers share
// most of their nonzero events (a pass gathers one table row for every
// occurrence any of its layers needs).  Before capture an optional autotuner
// times the YLT kernel's launch shapes (lanes per trial, i.e. trials summed
// side by side per warp, id loads per lane, and the L2 prefetch of the id
// stream) and the group size (layers per pass) on the plan's own layers and
// trials, and the captured passes use the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "ara.h"
#include "ara_ctx.h"
#include "ara_internal.cuh"
#include "fold_batch.h"

using namespace ara;

struct ara_plan {
  ara_ctx *c = nullptr;
  std::vector<int32_t> layers;
  std::vector<uint64_t> gens;
  int64_t n_trials = 0;
  int64_t yet_version = -1;
  int32_t n_rp = 0;
  int64_t k[kMaxReturnPeriods] = {};
  cudaStream_t cap = nullptr;  // capture stream
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double *d_ylt = nullptr;           // [n_layers][n_trials]
  ulonglong2 *d_pair = nullptr;      // interleaved tables of one pass
  uint32_t *d_pair_bm = nullptr;     // their union bitmap
  unsigned char *d_ws = nullptr;     // selection state per layer
  double *d_out = nullptr;           // PML then TVaR per layer
  unsigned int *d_err = nullptr;
  double *h_out = nullptr;           // pinned copy of d_out
  unsigned int *h_err = nullptr;     // pinned copy of d_err
  FoldJob *d_jobs = nullptr;         // every layer's fold, launched as one batch
  int max_elts = 0;
  // Per pass over several layers: its interleaved table and union bitmap,
  // written by the folds directly (no interleave step in the graph).
  std::vector<ara::GroupTable> gtables;
  std::vector<void *> gbufs;
  std::vector<ara::LayerGroup> groups;  // the YLT passes (positions in layers)
  std::vector<int32_t> pass_info;    // kPassInfo per pass: entry bytes, layers, lanes per trial, unroll, prefetch,
                                     // threads per CTA, the layers' positions (-1 padded to 4)
};

namespace {

constexpr int kPassInfo = 10;

void free_plan(ara_plan *p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cap) {
    cudaStreamSynchronize(p->cap);
    cudaStreamDestroy(p->cap);
  }
  cudaFree(p->d_ylt);
  cudaFree(p->d_pair);
  cudaFree(p->d_pair_bm);
  cudaFree(p->d_ws);
  cudaFree(p->d_out);
  cudaFree(p->d_err);
  cudaFree(p->d_jobs);
  for (void *b : p->gbufs) cudaFree(b);
  cudaFreeHost(p->h_out);
  cudaFreeHost(p->h_err);
  cudaGetLastError();
  delete p;
}

// Time the YLT kernel of one pass in every launch shape on the first n trials
// and keep the fastest in the context (ara_layers_ylt then uses it too).
ara_status tune_pass(ara_plan *p, const LayerGroup &ps, int64_t n) {
  ara_ctx *c = p->c;
  const int G = (int)ps.idx.size();
  LayerOut outs[4];
  Tables4 tabs{};
  Bitmaps4 bms{};
  for (int g = 0; g < G; ++g) {
    const LayerRec &L = c->layers[(size_t)p->layers[(size_t)ps.idx[(size_t)g]]];
    outs[g] = LayerOut{L.q, L.agg_fx, L.agg_ret, L.agg_lim, p->d_ylt + (size_t)g * (size_t)n};
    tabs.t[g] = L.d_table;
    bms.b[g] = L.d_bitmap;
  }
  const BitmapLayout bm = c->layers[(size_t)p->layers[(size_t)ps.idx[0]]].bm;
  const void *table = tabs.t[0];
  const uint32_t *bitmap = bms.b[0];
  if (G > 1) {
    ARA_CUDA(c, launch_interleave(tabs, ps.eb, G, (int64_t)c->catalog + 1, p->d_pair, bms, bm.words, p->d_pair_bm,
                                  p->cap),
             "interleave layer tables");
    table = p->d_pair;
    bitmap = p->d_pair_bm;
  }
  const YltStream ys = ylt_stream(c, G);
  const double mean_chunks = (double)ys.h_coff[(size_t)n] / (double)n;
  cudaEvent_t a = nullptr, b = nullptr;
  ARA_CUDA(c, cudaEventCreate(&a), "cudaEventCreate");
  cudaError_t e = cudaEventCreate(&b);
  if (e != cudaSuccess) {
    cudaEventDestroy(a);
    return cuda_fail(c, e, "cudaEventCreate");
  }
  const size_t table_bytes = ((size_t)c->catalog + 1) * (size_t)(ps.eb * G);
  YltShape best{};
  float best_ms = 1e30f;
  // every shape: lanes per trial 16/32 x id loads 1/2 x L2 prefetch off/on x 1024/768 threads
  for (int shape = 0; shape < 16 && e == cudaSuccess; ++shape) {
      YltShape hint;
      hint.lanes_per_trial = (shape & 8) ? 32 : 16;
      hint.unroll = (shape & 4) ? 2 : 1;
      hint.prefetch = (shape & 2) ? 1 : 0;
      hint.threads = (shape & 1) ? 768 : 1024;
      YltLaunch cfg;
      e = plan_ylt(c->device, bm, mean_chunks, ys.layout, ps.eb, G, table_bytes, hint, &cfg);
      float ms = 1e30f;
      for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // first run warms L2 and the clocks
        e = cudaEventRecord(a, p->cap);
        if (e == cudaSuccess)
          e = launch_ylt_group(ys.coff, ys.chunks, ys.layout, n, table, ps.eb, bitmap, bm, c->catalog, G,
                               outs, cfg, p->cap);
        if (e == cudaSuccess) e = cudaEventRecord(b, p->cap);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        if (e == cudaSuccess && rep > 0) ms = std::min(ms, t);
      }
      if (e != cudaSuccess) break;
      if (ms < best_ms) {
        best_ms = ms;
        best = YltShape{cfg.unroll, cfg.lanes_per_trial, cfg.prefetch, cfg.threads};
      }
    }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune YLT launch shapes");
  c->tuned[ps.eb == 8 ? 1 : 0][G] = best;
  return ARA_OK;
}

// Milliseconds of the passes `groups` over the first n trials (best of two
// after a warm-up run; one after the warm-up beyond 64 passes).
ara_status time_groups(ara_plan *p, const std::vector<LayerGroup> &groups, int64_t n, float *ms_out) {
  ara_ctx *c = p->c;
  cudaEvent_t a = nullptr, b = nullptr;
  ARA_CUDA(c, cudaEventCreate(&a), "cudaEventCreate");
  cudaError_t e = cudaEventCreate(&b);
  ara_status st = e == cudaSuccess ? ARA_OK : cuda_fail(c, e, "cudaEventCreate");
  float best = 1e30f;
  const int reps = groups.size() > 64 ? 2 : 3;
  for (int rep = 0; rep < reps && st == ARA_OK; ++rep) {
    if ((e = cudaEventRecord(a, p->cap)) != cudaSuccess) {
      st = cuda_fail(c, e, "cudaEventRecord");
      break;
    }
    st = layers_ylt_on(c, p->layers.data(), (int32_t)p->layers.size(), n, p->d_ylt, p->cap, p->d_pair,
                       p->d_pair_bm, &groups);
    float t = 0.f;
    if (st == ARA_OK && ((e = cudaEventRecord(b, p->cap)) != cudaSuccess ||
                         (e = cudaEventSynchronize(b)) != cudaSuccess ||
                         (e = cudaEventElapsedTime(&t, a, b)) != cudaSuccess))
      st = cuda_fail(c, e, "time YLT passes");
    if (st == ARA_OK && rep > 0) best = std::min(best, t);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  *ms_out = best;
  return st;
}

// The plan's passes with the autotuner: for each entry width, every group
// size the kernel has (FP64: 2 or 1 layers per pass; FP32 tables: 4, 2 or
// 1), layers grouped by overlap, launch shapes tuned per group size on the
// first n trials, and the whole set of passes of that width timed on the
// first min(n, 2^18) trials; the fastest group size per width is kept.
ara_status choose_groups(ara_plan *p, const std::vector<LayerRec *> &Ls, int64_t n, std::vector<LayerGroup> *out) {
  ara_ctx *c = p->c;
  out->clear();
  bool tuned[2][5] = {};
  // Only the group sizes the plan keeps leave their tuned launch shapes in
  // the context (the others were tuned on this plan's passes alone).
  YltShape before[2][5];
  for (int a = 0; a < 2; ++a)
    for (int g = 0; g < 5; ++g) before[a][g] = c->tuned[a][g];
  for (const int eb : {16, 8}) {
    std::vector<LayerGroup> best;
    float best_ms = 1e30f;
    for (const int gm : eb == 16 ? std::vector<int>{2, 1} : std::vector<int>{4, 2, 1}) {
      std::vector<LayerGroup> all, mine;
      ara_status st = group_by_overlap(c, Ls, gm, gm, p->cap, &all);
      if (st) return st;
      for (const LayerGroup &g : all)
        if (g.eb == eb) mine.push_back(g);
      if (mine.empty()) break;
      for (const LayerGroup &g : mine) {
        const int G = (int)g.idx.size();
        if (tuned[eb == 8][G]) continue;
        tuned[eb == 8][G] = true;
        if ((st = tune_pass(p, g, n)) != ARA_OK) return st;
      }
      float ms = 0.f;
      if ((st = time_groups(p, mine, std::min<int64_t>(n, 1 << 18), &ms)) != ARA_OK) return st;
      if (ms < best_ms) {
        best_ms = ms;
        best = mine;
      }
    }
    out->insert(out->end(), best.begin(), best.end());
  }
  bool kept[2][5] = {};
  for (const LayerGroup &g : *out) kept[g.eb == 8][g.idx.size()] = true;
  for (int a = 0; a < 2; ++a)
    for (int g = 0; g < 5; ++g)
      if (!kept[a][g]) c->tuned[a][g] = before[a][g];
  return ARA_OK;
}

}  // namespace

extern "C" {

ara_status ara_plan_create(ara_ctx *c, const int32_t *layers, int32_t n_layers, int64_t n_trials,
                           const double *rps, int32_t n_rp, int32_t autotune, ara_plan **out) {
  if (out) *out = nullptr;
  if (!c || !out) return fail_free(ARA_E_INVALID_ARG, "NULL argument");
  if (c->service) return fail_free(ARA_E_STATE, "the context is attached to a pricing service");
  c->err.clear();
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (!c->yet_loaded) return fail(c, ARA_E_STATE, "no YET loaded");
  if (n_layers < 1 || n_layers > 65535 || !layers) return fail(c, ARA_E_INVALID_ARG, "need 1..65535 layer handles");
  if (n_trials < 1 || n_trials > c->n_trials)
    return fail(c, ARA_E_INVALID_ARG, "n_trials %lld outside [1, %lld]", (long long)n_trials, (long long)c->n_trials);
  ara_plan *p = new ara_plan();
  p->c = c;
  p->n_trials = n_trials;
  p->n_rp = n_rp;
  if (tail_counts(n_trials, rps, n_rp, p->k) != ARA_OK) {
    delete p;
    return fail(c, ARA_E_INVALID_ARG, "%s", ara_last_error(nullptr));
  }
  for (int32_t i = 0; i < n_layers; ++i) {
    LayerRec *L = nullptr;
    ara_status st = get_layer(c, layers[i], &L);
    if (st) {
      delete p;
      return st;
    }
    p->layers.push_back(layers[i]);
    p->gens.push_back(L->gen);
  }
  auto bail = [&](ara_status st) {
    free_plan(p);
    return st;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaStreamCreate"));
  // Layers not yet folded for this YET are folded now (their grids are set
  // here; the graph re-runs the folds with the same grids).
  for (const int32_t h : p->layers) {
    LayerRec &L = c->layers[(size_t)h];
    if (L.folded_version != c->yet_version) {
      ara_status st = fold_layer(c, L, c->stream);
      if (st) return bail(st);
    }
  }
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaStreamSynchronize"));
  p->yet_version = c->yet_version;
  const size_t nl = (size_t)n_layers;
  const BitmapLayout bm = c->layers[(size_t)p->layers[0]].bm;
  if ((e = cudaMalloc(&p->d_ylt, nl * (size_t)n_trials * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_pair, 2 * ((size_t)c->catalog + 1) * sizeof(ulonglong2))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_pair_bm, (size_t)bm.words * 4)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_ws, nl * select_workspace_bytes(kMaxReturnPeriods))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_out, nl * 2 * (size_t)n_rp * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_err, sizeof(unsigned int))) != cudaSuccess ||
      (e = cudaMallocHost(&p->h_out, nl * 2 * (size_t)n_rp * sizeof(double))) != cudaSuccess ||
      (e = cudaMallocHost(&p->h_err, sizeof(unsigned int))) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(c, ARA_E_NOMEM, "plan buffers: %s", cudaGetErrorString(e)));
  }
  std::vector<LayerRec *> Ls;
  for (const int32_t h : p->layers) Ls.push_back(&c->layers[(size_t)h]);
  ara_status gst = ARA_OK;
  const bool timing_was = c->timing;  // the autotuner's launches stay off the timing channels
  c->timing = false;
  if (autotune)
    gst = choose_groups(p, Ls, std::min<int64_t>(n_trials, 1 << 20), &p->groups);
  else
    gst = group_by_overlap(c, Ls, 2, 4, p->cap, &p->groups);
  c->timing = timing_was;
  if (gst) return bail(gst);
  for (const LayerGroup &ps : p->groups) {
    const int G = (int)ps.idx.size();
    const YltStream ys = ylt_stream(c, G);
    const double mean_chunks = (double)ys.h_coff[(size_t)n_trials] / (double)n_trials;
    YltLaunch cfg;
    e = plan_ylt(c->device, bm, mean_chunks, ys.layout, ps.eb, G, ((size_t)c->catalog + 1) * (size_t)(ps.eb * G),
                 c->tuned[ps.eb == 8][G], &cfg);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "plan YLT launch"));
    p->pass_info.insert(p->pass_info.end(), {ps.eb, G, cfg.lanes_per_trial, cfg.unroll, cfg.prefetch, cfg.threads});
    for (int g = 0; g < 4; ++g) p->pass_info.push_back(g < G ? ps.idx[(size_t)g] : -1);
  }
  // The folds of every layer as one batch (the layers' folds at creation
  // fixed their exponents).  A layer of a pass over several layers is folded
  // straight into that pass's interleaved table and union bitmap, so the
  // graph has no interleave step; the others write their own table.
  std::vector<FoldJob> jobs;
  for (const LayerRec *L : Ls) {
    jobs.push_back(FoldJob{L->d_desc, (int32_t)L->elts.size(), L->q, L->occ_ret, L->occ_lim, L->d_table, L->d_bitmap,
                           L->bm.mul, L->precision == ARA_FP32_TABLE ? 1 : 0, 1});
    p->max_elts = std::max(p->max_elts, (int)L->elts.size());
  }
  {
    // ARA_PLAN_INTERLEAVE=1 keeps the interleave step (the path taken when the
    // pass tables cannot be allocated), for tests and measurements.
    const char *force = std::getenv("ARA_PLAN_INTERLEAVE");
    bool ok = !(force && std::atoi(force));
    std::vector<ara::GroupTable> gt;
    for (const LayerGroup &ps : p->groups) {
      const int G = (int)ps.idx.size();
      if (G < 2 || !ok) {
        gt.push_back(ara::GroupTable{nullptr, nullptr});
        continue;
      }
      void *tab = nullptr, *gbm = nullptr;
      if (cudaMalloc(&tab, ((size_t)c->catalog + 1) * (size_t)(ps.eb * G)) != cudaSuccess ||
          cudaMalloc(&gbm, (size_t)bm.words * 4) != cudaSuccess) {
        cudaGetLastError();
        if (tab) cudaFree(tab);
        ok = false;  // not enough memory: interleave in the graph instead
        gt.push_back(ara::GroupTable{nullptr, nullptr});
        continue;
      }
      p->gbufs.push_back(tab);
      p->gbufs.push_back(gbm);
      gt.push_back(ara::GroupTable{tab, static_cast<const uint32_t *>(gbm)});
      for (int g = 0; g < G; ++g) {
        FoldJob &j = jobs[(size_t)ps.idx[(size_t)g]];
        j.table = static_cast<unsigned char *>(tab) + (size_t)g * (size_t)ps.eb;
        j.bitmap = static_cast<uint32_t *>(gbm);
        j.stride = G;
      }
    }
    if (ok) {
      p->gtables = gt;
    } else {  // back to the layers' own tables and the interleave step
      for (size_t i = 0; i < jobs.size(); ++i) {
        jobs[i].table = Ls[i]->d_table;
        jobs[i].bitmap = Ls[i]->d_bitmap;
        jobs[i].stride = 1;
      }
    }
  }
  // The batch's CTAs run layer after layer (blockIdx.y): the layers of one
  // pass go next to each other, so the halves of each interleaved row are
  // written while its L2 line is still there.
  {
    std::vector<FoldJob> ordered;
    for (const LayerGroup &ps : p->groups)
      for (const int32_t i : ps.idx) ordered.push_back(jobs[(size_t)i]);
    if (ordered.size() == jobs.size()) jobs.swap(ordered);
  }
  if ((e = cudaMalloc(&p->d_jobs, jobs.size() * sizeof(FoldJob))) != cudaSuccess ||
      (e = cudaMemcpy(p->d_jobs, jobs.data(), jobs.size() * sizeof(FoldJob), cudaMemcpyHostToDevice)) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(c, ARA_E_NOMEM, "plan fold list: %s", cudaGetErrorString(e)));
  }
  // Capture: folds, grouped YLT passes, batched selection, result copies.
  const bool timing = c->timing;
  c->timing = false;
  e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
  ara_status st = e == cudaSuccess ? ARA_OK : cuda_fail(c, e, "cudaStreamBeginCapture");
  if (st == ARA_OK && (e = launch_fold_batch(p->d_jobs, n_layers, p->max_elts, c->catalog, bm.words, p->cap)) !=
                          cudaSuccess)
    st = cuda_fail(c, e, "fold kernels");
  if (st == ARA_OK)
    st = layers_ylt_on(c, p->layers.data(), n_layers, n_trials, p->d_ylt, p->cap, p->d_pair, p->d_pair_bm,
                       &p->groups, p->gtables.empty() ? nullptr : &p->gtables);
  if (st == ARA_OK && (e = cudaMemsetAsync(p->d_err, 0, sizeof(unsigned int), p->cap)) != cudaSuccess)
    st = cuda_fail(c, e, "cudaMemsetAsync");
  if (st == ARA_OK && (e = launch_pml_tvar_batch(p->d_ylt, n_layers, n_trials, p->k, n_rp, p->d_ws, p->d_out,
                                                  p->d_err, c->device, p->cap)) != cudaSuccess)
    st = cuda_fail(c, e, "PML/TVaR kernels");
  if (st == ARA_OK && (e = cudaMemcpyAsync(p->h_out, p->d_out, nl * 2 * (size_t)n_rp * sizeof(double),
                                           cudaMemcpyDeviceToHost, p->cap)) != cudaSuccess)
    st = cuda_fail(c, e, "copy PML/TVaR");
  if (st == ARA_OK && (e = cudaMemcpyAsync(p->h_err, p->d_err, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                                           p->cap)) != cudaSuccess)
    st = cuda_fail(c, e, "copy flag");
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(p->cap, &g);
  c->timing = timing;
  if (st == ARA_OK && e != cudaSuccess) st = cuda_fail(c, e, "cudaStreamEndCapture");
  p->graph = g;
  if (st != ARA_OK) return bail(st);
  e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaGraphInstantiate"));
  c->plans.push_back(p);
  *out = p;
  return ARA_OK;
}

ara_status ara_plan_run(ara_plan *p, double *ylt_out, double *pml_out, double *tvar_out, void *cuda_stream) {
  if (!p) return fail_free(ARA_E_INVALID_ARG, "NULL plan");
  ara_ctx *c = p->c;
  if (c->service) return fail_free(ARA_E_STATE, "the context is attached to a pricing service");
  c->err.clear();
  ARA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (c->yet_version != p->yet_version) return fail(c, ARA_E_STATE, "the YET was reloaded after the plan was made");
  for (size_t i = 0; i < p->layers.size(); ++i) {
    const int32_t h = p->layers[i];
    if (h >= (int32_t)c->layers.size() || !c->layers[(size_t)h].live || c->layers[(size_t)h].gen != p->gens[i])
      return fail(c, ARA_E_STATE, "layer %d was released or redefined after the plan was made", h);
  }
  if (ara_status st = reject_foreign(c, {{ylt_out, "ylt_out"}})) return st;
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : c->stream;
  ARA_CUDA(c, cudaGraphLaunch(p->exec, s), "cudaGraphLaunch");
  const size_t total = p->layers.size() * (size_t)p->n_trials;
  if (ylt_out)
    ARA_CUDA(c, cudaMemcpyAsync(ylt_out, p->d_ylt, total * sizeof(double), cudaMemcpyDefault, s), "copy YLTs");
  if (pml_out || tvar_out || (ylt_out && !is_device_ptr(ylt_out))) {
    ARA_CUDA(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (*p->h_err) return fail(c, ARA_E_INVALID_ARG, "trial losses must be finite and >= 0");
    const int32_t n_rp = p->n_rp;
    for (size_t l = 0; l < p->layers.size(); ++l)
      for (int32_t r = 0; r < n_rp; ++r) {
        if (pml_out) pml_out[l * (size_t)n_rp + (size_t)r] = p->h_out[l * 2 * (size_t)n_rp + (size_t)r];
        if (tvar_out) tvar_out[l * (size_t)n_rp + (size_t)r] = p->h_out[l * 2 * (size_t)n_rp + (size_t)(n_rp + r)];
      }
  }
  return ARA_OK;
}

ara_status ara_plan_passes(const ara_plan *p, int32_t max_passes, int32_t *info, int32_t *n_passes) {
  if (!p || !n_passes) return fail_free(ARA_E_INVALID_ARG, "NULL argument");
  const int32_t n = (int32_t)(p->pass_info.size() / kPassInfo);
  *n_passes = n;
  if (info)
    for (int32_t i = 0; i < std::min(n, max_passes); ++i)
      for (int j = 0; j < kPassInfo; ++j) info[kPassInfo * i + j] = p->pass_info[(size_t)(kPassInfo * i + j)];
  return ARA_OK;
}

ara_status ara_plan_kernel_launches(const ara_plan *p, int32_t *n_kernels) {
  if (!p || !n_kernels) return fail_free(ARA_E_INVALID_ARG, "NULL argument");
  size_t n = 0;
  cudaError_t e = cudaGraphGetNodes(p->graph, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  if (e == cudaSuccess && n) e = cudaGraphGetNodes(p->graph, nodes.data(), &n);
  int32_t k = 0;
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
    cudaGraphNodeType t;
    e = cudaGraphNodeGetType(nodes[i], &t);
    if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail_free(ARA_E_CUDA, "plan graph nodes: %s", cudaGetErrorString(e));
  }
  *n_kernels = k;
  return ARA_OK;
}

void ara_plan_destroy(ara_plan *p) {
  if (!p) return;
  ara_ctx *c = p->c;
  cudaSetDevice(c->device);
  c->plans.erase(std::remove(c->plans.begin(), c->plans.end(), p), c->plans.end());
  free_plan(p);
}

}  // extern "C"
