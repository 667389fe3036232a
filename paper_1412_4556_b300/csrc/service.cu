// Ad hoc pricing service: a scheduler thread that admits layer-pricing
// requests by device memory and batches them onto overlapping slots
// (Section I: real-time pricing of a contract; Section III: each request is a
// Layer priced by Algorithm 1 over a prefix of the YET, then PML/TVaR).
//
// Threads: callers submit/wait/cancel under `mu`; the scheduler thread alone
// touches the context and launches work; a host function queued behind each
// slot's work marks the slot complete.  Each slot owns a stream and the
// scratch of one batch (YLTs, paired tables, selection state, pinned copies),
// grown on demand and kept, so a steady request mix allocates nothing.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <limits>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ara.h"
#include "ara_ctx.h"
#include "ara_internal.cuh"

using namespace ara;

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxSlots = 16;
constexpr int kMaxBatch = 64;

enum class ReqState { kQueued, kRunning, kDone };

struct Req {
  int64_t ticket = 0;
  std::vector<int32_t> elts;
  double occ_ret = 0, occ_lim = 0, agg_ret = 0, agg_lim = 0;
  int32_t precision = ARA_FP64;
  int64_t n_trials = 0;
  double deadline = std::numeric_limits<double>::infinity();  // service seconds
  double *ylt_out = nullptr;
  size_t bytes = 0;  // device footprint charged against the budget
  ReqState state = ReqState::kQueued;
  int32_t layer = -1;
  size_t ylt_off = 0;  // offset of its YLT in the slot's pinned copy
  ara_result res{};
};

struct Slot {
  ara_service *svc = nullptr;
  int index = 0;
  cudaStream_t s = nullptr;
  bool busy = false;
  bool complete = false;  // set by the host function behind the batch
  std::vector<Req *> reqs;
  std::vector<int32_t> layers;
  int64_t n = 0;
  size_t extra_bytes = 0;  // paired-table scratch charged to the batch
  ara_status launch_status = ARA_OK;
  std::string launch_message;
  double *d_ylt = nullptr;
  size_t cap_ylt = 0;
  ulonglong2 *d_pair = nullptr;
  size_t cap_pair = 0;
  uint32_t *d_pair_bm = nullptr;
  size_t cap_pair_bm = 0;
  unsigned char *d_ws = nullptr;
  size_t cap_ws = 0;
  double *d_out = nullptr;
  size_t cap_out = 0;
  unsigned int *d_err = nullptr;
  size_t cap_err = 0;
  double *h_out = nullptr;  // pinned
  size_t cap_h_out = 0;
  double *h_ylt = nullptr;  // pinned
  size_t cap_h_ylt = 0;
  unsigned int *h_err = nullptr;  // pinned
  EltDesc *h_desc = nullptr;      // pinned ELT lists of the batch's layers
  size_t cap_h_desc = 0;
};

void free_slot(Slot &sl) {
  if (sl.s) {
    cudaStreamSynchronize(sl.s);
    cudaStreamDestroy(sl.s);
  }
  cudaFree(sl.d_ylt);
  cudaFree(sl.d_pair);
  cudaFree(sl.d_pair_bm);
  cudaFree(sl.d_ws);
  cudaFree(sl.d_out);
  cudaFree(sl.d_err);
  cudaFreeHost(sl.h_out);
  cudaFreeHost(sl.h_ylt);
  cudaFreeHost(sl.h_err);
  cudaFreeHost(sl.h_desc);
  sl = Slot();
}

void set_message(ara_result &r, const char *msg) {
  std::snprintf(r.message, sizeof(r.message), "%s", msg ? msg : "");
}

}  // namespace

struct ara_service {
  ara_ctx *c = nullptr;
  ara_service_config cfg{};
  std::mutex mu;
  std::condition_variable work_cv;  // scheduler: new request, slot done, stop
  std::condition_variable done_cv;  // waiters: a request ended
  std::thread worker;
  bool stop = false;
  Clock::time_point t0;
  int64_t next_ticket = 1;
  std::unordered_map<int64_t, std::unique_ptr<Req>> reqs;
  std::deque<Req *> queue;
  std::vector<std::unique_ptr<Slot>> slots;
  int64_t bytes_in_flight = 0;
  int64_t admitted = 0;
  int64_t in_flight = 0;
  size_t pair_bytes = 0;   // paired table + union bitmap of one slot
  size_t fixed_layer_bytes = 0;  // table + bitmap of one layer
  size_t saved_pool_max = 0;
  ara_service_stats stats{};

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

  // Footprint of one request: its layer buffers, its YLT, its selection state.
  size_t request_bytes(int32_t n_elts, int64_t n) const {
    return fixed_layer_bytes + (size_t)std::max<int32_t>(n_elts, 64) * sizeof(EltDesc) +
           (size_t)n * sizeof(double) + select_workspace_bytes(kMaxReturnPeriods) +
           2 * kMaxReturnPeriods * sizeof(double);
  }

  // End a request (mu held).
  void end(Req *r, ara_status st, const char *msg) {
    r->state = ReqState::kDone;
    r->res.status = st;
    r->res.t_done = now();
    set_message(r->res, st ? msg : "");
    if (st == ARA_OK) {
      ++stats.completed;
    } else {
      ++stats.failed;
      if (st == ARA_E_CANCELLED) ++stats.cancelled;
      if (st == ARA_E_TIMEOUT) ++stats.timed_out;
    }
    done_cv.notify_all();
  }

  void run();
  bool form_batch(Slot &slot, std::vector<Req *> &batch);
  void launch(Slot &slot, std::vector<Req *> &batch);
  void finish(Slot &slot);
};

namespace {

void CUDART_CB on_slot_done(void *p) {
  Slot *sl = static_cast<Slot *>(p);
  std::lock_guard<std::mutex> lk(sl->svc->mu);
  sl->complete = true;
  sl->svc->work_cv.notify_one();
}

}  // namespace

// Take the oldest queued request and the queued requests that share its trial
// count, in arrival order, while they fit in the memory budget (mu held).
bool ara_service::form_batch(Slot &slot, std::vector<Req *> &batch) {
  batch.clear();
  if (queue.empty()) return false;
  const int64_t n = queue.front()->n_trials;
  int64_t add_total = 0;
  for (auto it = queue.begin(); it != queue.end() && (int)batch.size() < cfg.max_batch;) {
    Req *r = *it;
    if (r->n_trials != n) {
      ++it;
      continue;
    }
    const int64_t add = (int64_t)r->bytes + (batch.size() == 1 ? (int64_t)pair_bytes : 0);
    if (bytes_in_flight + add_total + add > cfg.memory_budget) break;
    batch.push_back(r);
    add_total += add;
    it = queue.erase(it);
  }
  if (batch.empty()) return false;
  slot.extra_bytes = batch.size() > 1 ? pair_bytes : 0;
  bytes_in_flight += add_total;
  const double t = now();
  for (Req *r : batch) {
    r->state = ReqState::kRunning;
    r->res.t_start = t;
    r->res.slot = slot.index;
    r->res.batch_size = (int32_t)batch.size();
  }
  in_flight += (int64_t)batch.size();
  ++stats.batches;
  stats.max_batch_seen = std::max<int64_t>(stats.max_batch_seen, (int64_t)batch.size());
  stats.max_in_flight = std::max(stats.max_in_flight, in_flight);
  stats.max_bytes_in_flight = std::max(stats.max_bytes_in_flight, bytes_in_flight);
  slot.busy = true;
  slot.complete = false;
  int64_t busy = 0;
  for (auto &s : slots) busy += s->busy ? 1 : 0;
  stats.max_slots_busy = std::max(stats.max_slots_busy, busy);
  return true;
}

// Queue a batch's work on the slot's stream (scheduler thread, mu not held).
void ara_service::launch(Slot &slot, std::vector<Req *> &batch) {
  slot.reqs.clear();
  slot.layers.clear();
  slot.launch_status = ARA_OK;
  slot.launch_message.clear();
  slot.n = batch.front()->n_trials;
  std::vector<std::pair<Req *, std::pair<ara_status, std::string>>> failed;
  size_t n_desc = 0;
  for (Req *r : batch) n_desc += r->elts.size();
  // A failed allocation leaves h_desc NULL: the uploads then go from pageable memory.
  if (ensure_pinned(&slot.h_desc, &slot.cap_h_desc, n_desc) != cudaSuccess) cudaGetLastError();
  size_t desc_off = 0;
  for (Req *r : batch) {
    bool inject = false;
    {
      std::lock_guard<std::mutex> lk(mu);
      ++admitted;
      inject = cfg.fail_every > 0 && admitted % cfg.fail_every == 0;
    }
    if (inject) {
      failed.push_back({r, {ARA_E_NOMEM, "injected allocation failure"}});
      continue;
    }
    c->err.clear();
    EltDesc *stage = slot.h_desc ? slot.h_desc + desc_off : nullptr;
    desc_off += r->elts.size();
    const ara_status st = define_layer_on(c, (int32_t)r->elts.size(), r->elts.data(), r->occ_ret, r->occ_lim,
                                          r->agg_ret, r->agg_lim, r->precision, slot.s, &r->layer, stage);
    if (st) {
      failed.push_back({r, {st, c->err}});
      continue;
    }
    slot.reqs.push_back(r);
    slot.layers.push_back(r->layer);
  }
  if (!failed.empty()) {
    std::lock_guard<std::mutex> lk(mu);
    for (auto &f : failed) {
      bytes_in_flight -= (int64_t)f.first->bytes;
      --in_flight;
      end(f.first, f.second.first, f.second.second.c_str());
    }
  }
  auto cuda_error = [&](cudaError_t e, const char *what) {
    slot.launch_status = ARA_E_CUDA;
    slot.launch_message = std::string(what) + ": " + cudaGetErrorString(e);
  };
  const int32_t nl = (int32_t)slot.reqs.size();
  if (nl > 0) {
    const int64_t n = slot.n;
    const int32_t n_rp = cfg.n_return_periods;
    int64_t kk[kMaxReturnPeriods];
    size_t ylt_total = 0;
    for (Req *r : slot.reqs)
      if (r->ylt_out) {
        r->ylt_off = ylt_total;
        ylt_total += (size_t)n;
      }
    cudaError_t e = cudaSuccess;
    const size_t entries = (size_t)c->catalog + 1;
    const BitmapLayout bm = c->layers[(size_t)slot.layers[0]].bm;
    if (tail_counts(n, cfg.return_periods, n_rp, kk) != ARA_OK) {
      slot.launch_status = ARA_E_INVALID_ARG;
      slot.launch_message = ara_last_error(nullptr);
    } else if ((e = ensure(&slot.d_ylt, &slot.cap_ylt, (size_t)nl * (size_t)n)) != cudaSuccess ||
               (nl > 1 && (e = ensure(&slot.d_pair, &slot.cap_pair, 2 * entries)) != cudaSuccess) ||
               (nl > 1 && (e = ensure(&slot.d_pair_bm, &slot.cap_pair_bm, (size_t)bm.words)) != cudaSuccess) ||
               (e = ensure(&slot.d_ws, &slot.cap_ws, (size_t)nl * select_workspace_bytes(kMaxReturnPeriods))) !=
                   cudaSuccess ||
               (e = ensure(&slot.d_out, &slot.cap_out, (size_t)nl * 2 * (size_t)n_rp)) != cudaSuccess ||
               (e = ensure(&slot.d_err, &slot.cap_err, 1)) != cudaSuccess ||
               (e = ensure_pinned(&slot.h_out, &slot.cap_h_out, (size_t)nl * 2 * (size_t)n_rp)) != cudaSuccess ||
               (ylt_total > 0 && (e = ensure_pinned(&slot.h_ylt, &slot.cap_h_ylt, ylt_total)) != cudaSuccess)) {
      slot.launch_status = ARA_E_NOMEM;
      slot.launch_message = std::string("slot buffers: ") + cudaGetErrorString(e);
      cudaGetLastError();
    } else {
      c->err.clear();
      const ara_status st =
          layers_ylt_on(c, slot.layers.data(), nl, n, slot.d_ylt, slot.s, slot.d_pair, slot.d_pair_bm);
      if (st) {
        slot.launch_status = st;
        slot.launch_message = c->err;
      } else if ((e = cudaMemsetAsync(slot.d_err, 0, sizeof(unsigned int), slot.s)) != cudaSuccess) {
        cuda_error(e, "cudaMemsetAsync");
      } else if ((e = launch_pml_tvar_batch(slot.d_ylt, nl, n, kk, n_rp, slot.d_ws, slot.d_out, slot.d_err,
                                            c->device, slot.s)) != cudaSuccess) {
        cuda_error(e, "PML/TVaR kernels");
      } else if ((e = cudaMemcpyAsync(slot.h_out, slot.d_out, (size_t)nl * 2 * (size_t)n_rp * sizeof(double),
                                      cudaMemcpyDeviceToHost, slot.s)) != cudaSuccess ||
                 (e = cudaMemcpyAsync(slot.h_err, slot.d_err, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                                      slot.s)) != cudaSuccess) {
        cuda_error(e, "copy results");
      } else {
        for (int32_t i = 0; i < nl && e == cudaSuccess; ++i) {
          Req *r = slot.reqs[(size_t)i];
          if (r->ylt_out)
            e = cudaMemcpyAsync(slot.h_ylt + r->ylt_off, slot.d_ylt + (size_t)i * (size_t)n,
                                (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, slot.s);
        }
        if (e != cudaSuccess) cuda_error(e, "copy YLT");
      }
    }
  }
  // The host function runs after everything queued above, also when part of
  // it failed to launch; a batch with nothing to do completes at once.
  cudaError_t e = cudaLaunchHostFunc(slot.s, on_slot_done, &slot);
  if (e != cudaSuccess) {
    if (slot.launch_status == ARA_OK) cuda_error(e, "cudaLaunchHostFunc");
    cudaStreamSynchronize(slot.s);
    cudaGetLastError();
    std::lock_guard<std::mutex> lk(mu);
    slot.complete = true;
  }
}

// Publish a completed batch: results, YLT copies, released layers, memory.
void ara_service::finish(Slot &slot) {
  const int32_t nl = (int32_t)slot.reqs.size();
  const int32_t n_rp = cfg.n_return_periods;
  ara_status st = slot.launch_status;
  std::string msg = slot.launch_message;
  if (st == ARA_OK && nl > 0) {
    const cudaError_t e = cudaStreamQuery(slot.s);
    if (e != cudaSuccess && e != cudaErrorNotReady) {
      st = ARA_E_CUDA;
      msg = std::string("batch: ") + cudaGetErrorString(e);
    } else if (*slot.h_err) {
      st = ARA_E_INVALID_ARG;
      msg = "a trial loss was not finite or negative";
    }
  }
  for (int32_t i = 0; i < nl; ++i) {
    Req *r = slot.reqs[(size_t)i];
    if (st == ARA_OK) {
      r->res.n_return_periods = n_rp;
      for (int32_t q = 0; q < n_rp; ++q) {
        r->res.pml[q] = slot.h_out[(size_t)i * 2 * n_rp + q];
        r->res.tvar[q] = slot.h_out[(size_t)i * 2 * n_rp + n_rp + q];
      }
      if (r->ylt_out) std::memcpy(r->ylt_out, slot.h_ylt + r->ylt_off, (size_t)slot.n * sizeof(double));
    }
    LayerRec *L = nullptr;
    if (r->layer >= 0 && get_layer(c, r->layer, &L) == ARA_OK) recycle_layer(c, *L);
    r->layer = -1;
  }
  std::lock_guard<std::mutex> lk(mu);
  for (Req *r : slot.reqs) {
    bytes_in_flight -= (int64_t)r->bytes;
    --in_flight;
    end(r, st, msg.c_str());
  }
  bytes_in_flight -= (int64_t)slot.extra_bytes;
  slot.extra_bytes = 0;
  slot.reqs.clear();
  slot.busy = false;
  slot.complete = false;
}

void ara_service::run() {
  cudaSetDevice(c->device);
  std::vector<Req *> batch;
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    bool progressed = false;
    for (auto &sp : slots) {
      Slot &sl = *sp;
      if (sl.busy && sl.complete) {
        lk.unlock();
        finish(sl);
        lk.lock();
        progressed = true;
      }
    }
    // Requests whose deadline passed before they started.
    double wake = std::numeric_limits<double>::infinity();
    const double t = now();
    for (auto it = queue.begin(); it != queue.end();) {
      if ((*it)->deadline <= t) {
        end(*it, ARA_E_TIMEOUT, "deadline passed before the request started");
        it = queue.erase(it);
      } else {
        wake = std::min(wake, (*it)->deadline);
        ++it;
      }
    }
    bool any_busy = false;
    for (auto &sp : slots) any_busy = any_busy || sp->busy;
    if (stop && queue.empty() && !any_busy) break;
    Slot *free_slot = nullptr;
    for (auto &sp : slots)
      if (!sp->busy) {
        free_slot = sp.get();
        break;
      }
    if (free_slot && form_batch(*free_slot, batch)) {
      lk.unlock();
      launch(*free_slot, batch);
      lk.lock();
      continue;
    }
    if (progressed) continue;
    if (std::isfinite(wake)) {
      work_cv.wait_for(lk, std::chrono::duration<double>(std::max(wake - now(), 0.0) + 1e-5));
    } else {
      work_cv.wait(lk);
    }
  }
}

// ======================================================================= ABI

extern "C" {

ara_status ara_service_create(ara_ctx *c, const ara_service_config *cfg, ara_service **out) {
  if (out) *out = nullptr;
  if (!c || !cfg || !out) return fail_free(ARA_E_INVALID_ARG, "NULL argument");
  if (c->service) return fail_free(ARA_E_STATE, "a service is already attached to the context");
  if (!c->yet_loaded) return fail_free(ARA_E_STATE, "no YET loaded");
  if (cfg->slots < 1 || cfg->slots > kMaxSlots)
    return fail_free(ARA_E_INVALID_ARG, "slots must be 1..%d (got %d)", kMaxSlots, cfg->slots);
  if (cfg->max_batch < 1 || cfg->max_batch > kMaxBatch)
    return fail_free(ARA_E_INVALID_ARG, "max_batch must be 1..%d (got %d)", kMaxBatch, cfg->max_batch);
  if (cfg->memory_budget < 0) return fail_free(ARA_E_INVALID_ARG, "memory_budget must be >= 0");
  if (cfg->fail_every < 0) return fail_free(ARA_E_INVALID_ARG, "fail_every must be >= 0");
  int64_t k[kMaxReturnPeriods];
  ara_status st = tail_counts(1 << 30, cfg->return_periods, cfg->n_return_periods, k);
  if (st) return st;
  cudaError_t e = cudaSetDevice(c->device);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail_free(ARA_E_CUDA, "service start: %s", cudaGetErrorString(e));
  std::unique_ptr<ara_service> svc(new ara_service());
  svc->c = c;
  svc->cfg = *cfg;
  if (svc->cfg.memory_budget == 0) {
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return fail_free(ARA_E_CUDA, "cudaMemGetInfo: %s", cudaGetErrorString(e));
    svc->cfg.memory_budget = (int64_t)(free_b / 4);
  }
  const size_t table_bytes = ((size_t)c->catalog + 1) * sizeof(ulonglong2);
  svc->fixed_layer_bytes = table_bytes + layer_bitmap_bytes(c);
  svc->pair_bytes = 2 * table_bytes + layer_bitmap_bytes(c);
  for (int i = 0; i < cfg->slots; ++i) {
    std::unique_ptr<Slot> sl(new Slot());
    sl->svc = svc.get();
    sl->index = i;
    e = cudaStreamCreateWithFlags(&sl->s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl->h_err, sizeof(unsigned int));
    if (e != cudaSuccess) {
      free_slot(*sl);
      for (auto &o : svc->slots) free_slot(*o);
      return fail_free(ARA_E_CUDA, "slot setup: %s", cudaGetErrorString(e));
    }
    svc->slots.push_back(std::move(sl));
  }
  svc->stats.memory_budget = svc->cfg.memory_budget;
  svc->saved_pool_max = c->pool_max;
  c->pool_max = std::max(c->pool_max, (size_t)cfg->slots * (size_t)cfg->max_batch + 8);
  // Reserve up front what a full load of requests over all loaded trials
  // needs (as far as the budget covers it), so that requests do not wait on
  // cudaMalloc: layer buffers in the context's pool, and each slot's YLT,
  // selection and paired-table scratch, and pinned room for one YLT over all
  // loaded trials (a request that asks for its YLT would otherwise pin pages
  // inside the scheduler thread, which holds up every other launch; batches
  // with several such requests grow it on first use).
  const size_t per = svc->request_bytes(64, c->n_trials);
  const size_t n_res = std::min<size_t>((size_t)cfg->slots * (size_t)cfg->max_batch,
                                        (size_t)svc->cfg.memory_budget / std::max<size_t>(per, 1));
  const size_t per_slot = std::min<size_t>((size_t)cfg->max_batch, std::max<size_t>(n_res, 1));
  st = reserve_layers(c, n_res, c->stream);
  for (auto &sp : svc->slots) {
    if (st != ARA_OK) break;
    Slot &sl = *sp;
    e = ensure(&sl.d_ylt, &sl.cap_ylt, per_slot * (size_t)c->n_trials);
    if (e == cudaSuccess) e = ensure(&sl.d_ws, &sl.cap_ws, per_slot * select_workspace_bytes(kMaxReturnPeriods));
    if (e == cudaSuccess) e = ensure(&sl.d_out, &sl.cap_out, per_slot * 2 * kMaxReturnPeriods);
    if (e == cudaSuccess) e = ensure(&sl.d_err, &sl.cap_err, 1);
    if (e == cudaSuccess) e = ensure_pinned(&sl.h_out, &sl.cap_h_out, per_slot * 2 * kMaxReturnPeriods);
    if (e == cudaSuccess) e = ensure_pinned(&sl.h_ylt, &sl.cap_h_ylt, (size_t)c->n_trials);
    if (e == cudaSuccess && per_slot > 1) e = ensure(&sl.d_pair, &sl.cap_pair, 2 * ((size_t)c->catalog + 1));
    if (e == cudaSuccess && per_slot > 1) e = ensure(&sl.d_pair_bm, &sl.cap_pair_bm, layer_bitmap_bytes(c) / 4);
    if (e != cudaSuccess) st = fail_free(ARA_E_NOMEM, "service reservation: %s", cudaGetErrorString(e));
  }
  if (st == ARA_OK && (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    st = fail_free(ARA_E_CUDA, "service reservation: %s", cudaGetErrorString(e));
  if (st != ARA_OK) {
    cudaGetLastError();
    c->pool_max = svc->saved_pool_max;
    for (auto &o : svc->slots) free_slot(*o);
    return st;
  }
  svc->t0 = Clock::now();
  c->service = svc.get();
  ara_service *raw = svc.get();
  try {
    svc->worker = std::thread([raw] { raw->run(); });
  } catch (...) {
    c->service = nullptr;
    c->pool_max = svc->saved_pool_max;
    for (auto &o : svc->slots) free_slot(*o);
    return fail_free(ARA_E_NOMEM, "could not start the scheduler thread");
  }
  *out = svc.release();
  return ARA_OK;
}

ara_status ara_service_submit(ara_service *svc, const ara_request *rq, int64_t *ticket) {
  if (ticket) *ticket = 0;
  if (!svc || !rq || !ticket) return fail_free(ARA_E_INVALID_ARG, "NULL argument");
  ara_ctx *c = svc->c;
  ara_status st = check_layer_args(c, rq->n_elts, rq->elt_handles, rq->occ_ret, rq->occ_lim, rq->agg_ret,
                                   rq->agg_lim, rq->precision);
  if (st) return st;
  if (rq->n_trials < 1 || rq->n_trials > c->n_trials)
    return fail_free(ARA_E_INVALID_ARG, "n_trials %lld outside [1, %lld]", (long long)rq->n_trials,
                     (long long)c->n_trials);
  if (!(rq->deadline_s >= 0.0)) return fail_free(ARA_E_INVALID_ARG, "deadline_s must be >= 0");
  int64_t k[kMaxReturnPeriods];
  st = tail_counts(rq->n_trials, svc->cfg.return_periods, svc->cfg.n_return_periods, k);
  if (st) return st;
  std::unique_ptr<Req> r(new Req());
  r->elts.assign(rq->elt_handles, rq->elt_handles + rq->n_elts);
  r->occ_ret = rq->occ_ret;
  r->occ_lim = rq->occ_lim;
  r->agg_ret = rq->agg_ret;
  r->agg_lim = rq->agg_lim;
  r->precision = rq->precision;
  r->n_trials = rq->n_trials;
  r->ylt_out = rq->ylt_out;
  r->bytes = svc->request_bytes(rq->n_elts, rq->n_trials);
  if ((int64_t)r->bytes > svc->cfg.memory_budget)
    return fail_free(ARA_E_NOMEM, "request needs %zu device bytes, above the service budget of %lld", r->bytes,
                     (long long)svc->cfg.memory_budget);
  r->res.slot = -1;
  std::lock_guard<std::mutex> lk(svc->mu);
  if (svc->stop) return fail_free(ARA_E_STATE, "the service is shutting down");
  r->ticket = svc->next_ticket++;
  r->res.t_submit = svc->now();
  if (rq->deadline_s > 0.0) r->deadline = r->res.t_submit + rq->deadline_s;
  *ticket = r->ticket;
  svc->queue.push_back(r.get());
  svc->reqs[r->ticket] = std::move(r);
  ++svc->stats.submitted;
  svc->work_cv.notify_one();
  return ARA_OK;
}

ara_status ara_service_wait(ara_service *svc, int64_t ticket, double timeout_s, ara_result *out) {
  if (!svc || !out) return fail_free(ARA_E_INVALID_ARG, "NULL argument");
  if (!(timeout_s >= 0.0)) return fail_free(ARA_E_INVALID_ARG, "timeout_s must be >= 0");
  std::unique_lock<std::mutex> lk(svc->mu);
  auto it = svc->reqs.find(ticket);
  if (it == svc->reqs.end()) return fail_free(ARA_E_NOT_FOUND, "unknown ticket %lld", (long long)ticket);
  Req *r = it->second.get();
  const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                        std::chrono::duration<double>(std::min(timeout_s, 1e7)));
  while (r->state != ReqState::kDone) {
    if (svc->done_cv.wait_until(lk, until) == std::cv_status::timeout && r->state != ReqState::kDone)
      return fail_free(ARA_E_TIMEOUT, "request %lld has not ended", (long long)ticket);
  }
  *out = r->res;
  svc->reqs.erase(it);
  return ARA_OK;
}

ara_status ara_service_cancel(ara_service *svc, int64_t ticket) {
  if (!svc) return fail_free(ARA_E_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(svc->mu);
  auto it = svc->reqs.find(ticket);
  if (it == svc->reqs.end()) return fail_free(ARA_E_NOT_FOUND, "unknown ticket %lld", (long long)ticket);
  Req *r = it->second.get();
  if (r->state != ReqState::kQueued)
    return fail_free(ARA_E_STATE, "request %lld already started", (long long)ticket);
  svc->queue.erase(std::find(svc->queue.begin(), svc->queue.end(), r));
  svc->end(r, ARA_E_CANCELLED, "cancelled");
  return ARA_OK;
}

ara_status ara_service_get_stats(ara_service *svc, ara_service_stats *out) {
  if (!svc || !out) return fail_free(ARA_E_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(svc->mu);
  *out = svc->stats;
  out->queued = (int64_t)svc->queue.size();
  out->in_flight = svc->in_flight;
  out->bytes_in_flight = svc->bytes_in_flight;
  return ARA_OK;
}

void ara_service_destroy(ara_service *svc) {
  if (!svc) return;
  {
    std::lock_guard<std::mutex> lk(svc->mu);
    for (Req *r : svc->queue) svc->end(r, ARA_E_CANCELLED, "service destroyed");
    svc->queue.clear();
    svc->stop = true;
    svc->work_cv.notify_one();
  }
  if (svc->worker.joinable()) svc->worker.join();
  ara_ctx *c = svc->c;
  cudaSetDevice(c->device);
  for (auto &sp : svc->slots) free_slot(*sp);
  cudaGetLastError();
  c->pool_max = svc->saved_pool_max;
  c->service = nullptr;
  delete svc;
}

}  // extern "C"
