/*
 * ara.h -- C ABI of the B300 Year Loss Table engine for Aggregate Risk
 * Analysis (Varghese & Barker, "Are Clouds Ready to Accelerate Ad hoc
 * Financial Simulations?", arXiv 1412.4556).
 *
 * The calls follow the paper's problem statement (Section III):
 *   - the Year Event Table (YET): trials of (event id, time-stamp) pairs in
 *     ascending time-stamp order                        -> ara_load_yet
 *   - Event Loss Tables (ELTs): (event id, loss) pairs plus financial terms
 *     FT1 (read as a deductible and a limit)            -> ara_load_elts
 *   - a Layer: ELTs plus occurrence terms FT2 = (OccR, OccL) and aggregate
 *     terms FT3 = (AggR, AggL)                          -> ara_define_layer
 *   - Algorithm 1: the Year Loss Table (one loss per trial) -> ara_layer_ylt
 *   - PML and TVaR derived from the YLT                 -> ara_pml_tvar
 *
 * Conventions for every call:
 *   - Plain pointers and sizes.  A pointer argument documented "host or
 *     device" may point to host memory (pageable or pinned) or to device
 *     memory of the context's GPU; the library tells them apart with
 *     cudaPointerGetAttributes.
 *   - The library COPIES every input; the caller keeps ownership of its
 *     arrays and may free them when the call returns.  Outputs are
 *     allocated by the caller.
 *   - No call aborts the process or traps on the device.  Every failure is a
 *     negative status; ara_last_error(ctx) holds a one-line message.  On
 *     failure, the context's previous state (loaded YET, ELTs, layers) is
 *     unchanged unless the description says otherwise.
 *   - Calls on one context are not thread-safe; serialise them.
 *   - Work runs on the context's stream (a library-owned stream, or the one
 *     given to ara_set_stream).  Calls that write host memory return after
 *     the data is in place; calls that only write device memory return once
 *     the work is queued.
 */
#ifndef ARA_H_
#define ARA_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ARA_API __attribute__((visibility("default")))
#else
#define ARA_API
#endif

typedef struct ara_ctx ara_ctx;
typedef int32_t ara_status;

#define ARA_OK 0
#define ARA_E_INVALID_ARG (-1) /* bad size, pointer, term or ordering */
#define ARA_E_EVENT_RANGE (-2) /* an event id outside [0, catalog_size) */
#define ARA_E_DUP_EVENT (-3)   /* an event id repeated within one ELT */
#define ARA_E_NOMEM (-4)       /* device or host allocation failed */
#define ARA_E_CUDA (-5)        /* a CUDA runtime call failed */
#define ARA_E_TIMEOUT (-6)     /* a bounded wait ran out */
#define ARA_E_NOT_FOUND (-7)   /* unknown ELT or layer handle */
#define ARA_E_STATE (-8)       /* call order: e.g. no YET loaded yet */
#define ARA_E_CANCELLED (-9)   /* a service request cancelled before it started */

/* Precision of a layer's per-event table (ara_define_layer). */
#define ARA_FP64 0        /* FP64 event losses, exact integer trial sums */
#define ARA_FP32_TABLE 1  /* ELT terms, combination and occurrence terms in FP32;
                             trial sums still exact (at least FP64) */

/* Timing channels for ara_kernel_timing. */
#define ARA_TIMING_YLT 0  /* the per-trial gather/sum kernel */
#define ARA_TIMING_FOLD 1 /* the per-layer ELT fold (pre-pass) kernel */
#define ARA_TIMING_PML 2  /* the PML/TVaR selection kernels, summed */
#define ARA_TIMING_YELT 3 /* the Year Event Loss Table kernel (ara_layer_yelt, ara_rpl_report) */

/* ------------------------------------------------------------------ setup */

/* Create a context on CUDA device `device` with its own stream.
 * *out receives the context (NULL on failure).  ARA_E_CUDA if the device
 * cannot be used (for instance when no GPU is present). */
ARA_API ara_status ara_create(ara_ctx **out, int device);

/* Free every device and host resource of the context (an attached pricing
 * service is destroyed first).  NULL is a no-op. */
ARA_API void ara_destroy(ara_ctx *ctx);

/* Message of the last failed call on ctx ("" if none).  The pointer stays
 * valid until the next call on ctx.  ctx == NULL gives the message of the
 * last failed call that takes no context (ara_create,
 * ara_pml_tvar_noalloc, the ara_service_* calls) on the calling thread, as
 * does a ctx that a pricing service owns. */
ARA_API const char *ara_last_error(const ara_ctx *ctx);

/* Static name of a status code ("ARA_OK", "ARA_E_INVALID_ARG", ...). */
ARA_API const char *ara_status_string(ara_status status);

/* Run later work on `cuda_stream` (a cudaStream_t of the context's device);
 * NULL restores the context's own stream.  The caller keeps ownership of
 * the stream and must keep it alive while the context uses it. */
ARA_API ara_status ara_set_stream(ara_ctx *ctx, void *cuda_stream);

/* ------------------------------------------------ Year Event Table (YET) */

/* Load the YET (Section III: trials T_i = {(E_ik, t_ik)} in ascending
 * time-stamp order; "about one million trials of about one thousand
 * events") as CSR arrays, replacing any YET loaded before.
 *   catalog_size  number of catalog events; ids must lie in [0, catalog_size)
 *   n_trials      number of trials N >= 0
 *   trial_offsets int64[N+1], host or device: trial t owns positions
 *                 [trial_offsets[t], trial_offsets[t+1]); [0] == 0 and the
 *                 sequence is nondecreasing; M = trial_offsets[N] occurrences
 *   event_ids     int32[M], host or device, in stored (time-stamp) order;
 *                 may be NULL when M == 0.  A trial may repeat an event.
 *   timestamps    float32[M], host or device, or NULL.  When given they must
 *                 be finite and nondecreasing within each trial; they are
 *                 kept on the device but the trial loss does not read them
 *                 (the stored order already is the time order).
 * Errors: ARA_E_INVALID_ARG (sizes, offsets, time-stamp order),
 * ARA_E_EVENT_RANGE (an id outside the catalog, or an already loaded ELT
 * holding an id outside the new catalog), ARA_E_NOMEM, ARA_E_CUDA.  Errors
 * found in the sizes, the offsets or the ELT check leave the previous YET
 * loaded; once the copy has started (it replaces the previous YET in place,
 * since it can be several GB), a failure leaves the context with no YET.
 * Layers already defined are re-folded against the new YET on their next
 * use.  The call returns when the YET is on the device (the caller may then
 * free its arrays).  Host ids go up in pieces of at least 2^24 ids on a copy
 * stream of the context's, each piece's completed trials being laid out
 * while later pieces copy; from pinned host memory the copies run
 * asynchronously to the host's checks of the offsets. */
ARA_API ara_status ara_load_yet(ara_ctx *ctx, int32_t catalog_size, int64_t n_trials,
                        const int64_t *trial_offsets, const int32_t *event_ids,
                        const float *timestamps);

/* Prepare the loaded YET for repeated pricing.  A trial's loss does not
 * depend on the order of its events (Algorithm 1 sums them; the engine sums
 * exactly), so one-layer YLT passes may read each trial's ids reordered (so
 * that every group of 8 ascends in small steps) and stored as differences:
 * 8 ids per 16 bytes instead of 6, a quarter fewer bytes read from HBM by
 * every later one-layer pass (ara_layer_ylt, and the odd layer of
 * ara_layers_ylt, plans and service batches; passes over several layers keep
 * the stored layout, which measured faster for them).  Trials whose ids are
 * far apart (short trials over a large catalog) keep the stored layout.
 * Results are bit for bit those of the stored layout; the Year Event Loss
 * Table keeps reading the stored (time) order.  Takes a few milliseconds
 * and about 2 bytes per occurrence of device memory; a later ara_load_yet
 * drops it.  No-op for catalogs above 2^21 - 1 events or when already
 * prepared.
 * Errors: ARA_E_STATE (no YET), ARA_E_NOMEM, ARA_E_CUDA. */
ARA_API ara_status ara_compact_yet(ara_ctx *ctx);

/* ------------------------------------------------- Event Loss Tables (ELT) */

/* Append n_elts ELTs to the context's pool (Section III: ELT = {(E_i, l_i)}
 * plus financial terms FT1; an ELT typically holds 10^4-10^5 events).  All
 * arrays are host pointers.
 *   elt_offsets int64[n_elts+1]: ELT j owns positions [off[j], off[j+1]);
 *               off[0] == 0, nondecreasing (an empty ELT is allowed)
 *   event_ids   int32[off[n_elts]]: distinct within one ELT, each in
 *               [0, catalog_size) of the loaded YET
 *   losses      double[off[n_elts]]: finite and >= 0
 *   deductibles double[n_elts]: finite and >= 0
 *   limits      double[n_elts]: >= 0; +inf means "no limit"
 *   first_elt_handle (out): handle of the first new ELT; the others follow
 *               contiguously.  Handles stay valid until ara_destroy.
 * The entries are checked, and grouped for the fold, on the device; one call
 * takes at most 2^31 - 1 entries.
 * Requires a loaded YET (ARA_E_STATE otherwise).  Errors:
 * ARA_E_INVALID_ARG, ARA_E_EVENT_RANGE, ARA_E_DUP_EVENT, ARA_E_NOMEM,
 * ARA_E_CUDA; on error no ELT of the call is added. */
ARA_API ara_status ara_load_elts(ara_ctx *ctx, int32_t n_elts, const int64_t *elt_offsets,
                         const int32_t *event_ids, const double *losses,
                         const double *deductibles, const double *limits,
                         int32_t *first_elt_handle);

/* ------------------------------------------------------------------ layers */

/* Define a layer (Section III: L = {E = {ELT_1..ELT_j}, FT2, FT3}).
 *   n_elts, elt_handles  the layer's ELTs; their order is the order in
 *                        which the per-ELT net losses are summed.  An ELT
 *                        may not appear twice.  n_elts >= 1.
 *   occ_ret, occ_lim     FT2: occurrence retention and limit, applied to
 *                        each event's loss combined across the ELTs
 *   agg_ret, agg_lim     FT3: aggregate retention and limit, on a trial's
 *                        running total of occurrence-net losses
 *   precision            ARA_FP64, or ARA_FP32_TABLE: losses and terms are
 *                        rounded to binary32 and the ELT combination and
 *                        occurrence terms run in binary32 (Section IV-B uses
 *                        binary32 arithmetic wherever it can); the trial sum
 *                        and aggregate terms keep full precision
 *   layer_out (out)      the layer handle
 * Retentions must be finite and >= 0, limits >= 0 (+inf allowed).  The
 * per-layer pre-pass (folding the ELT terms and the occurrence terms into
 * one per-event table) is queued on the context's stream.
 * Errors: ARA_E_INVALID_ARG, ARA_E_NOT_FOUND, ARA_E_STATE (no YET),
 * ARA_E_NOMEM, ARA_E_CUDA. */
ARA_API ara_status ara_define_layer(ara_ctx *ctx, int32_t n_elts, const int32_t *elt_handles,
                            double occ_ret, double occ_lim, double agg_ret, double agg_lim,
                            int32_t precision, int32_t *layer_out);

/* Release a layer; its handle becomes invalid.  Its device buffers are kept
 * for reuse by later layers, ordered by the context's stream: work queued on
 * other streams that reads the layer must be complete before this call. */
ARA_API ara_status ara_release_layer(ara_ctx *ctx, int32_t layer);

/* The layer's per-event table as FP64: out[e] = FT2(sum_j FT1(DAT_j[e]))
 * for every catalog event e (the occurrence-net loss of one occurrence of
 * e).  out: double[catalog_size], host or device.  Bit-identical to a
 * sequential FP64 loop over the layer's ELTs in layer order. */
ARA_API ara_status ara_layer_event_table(ara_ctx *ctx, int32_t layer, double *out);

/* Year Loss Table of one layer (Algorithm 1) over the first n_trials trials
 * of the loaded YET (0 <= n_trials <= loaded N).
 *   ylt_out     double[n_trials], host or device: ylt_out[t] =
 *               min(max(S_t - AggR, 0), AggL), S_t the sum of the trial's
 *               occurrence-net event losses (0 for an empty trial)
 *   cuda_stream stream for this call only, or NULL for the context's stream
 * FP64 layers sum each trial exactly in 128-bit fixed point and round once
 * to binary64; the result is independent of launch shape and summation
 * order.  Errors: ARA_E_INVALID_ARG, ARA_E_NOT_FOUND, ARA_E_STATE,
 * ARA_E_NOMEM, ARA_E_CUDA. */
ARA_API ara_status ara_layer_ylt(ara_ctx *ctx, int32_t layer, int64_t n_trials, double *ylt_out,
                         void *cuda_stream);

/* PML and TVaR from a YLT of n trial losses (Section III names both as read
 * from the YLT).  For each return period RP_r: k = floor(n / RP_r);
 * PML_r = the k-th largest trial loss; TVaR_r = mean of the k largest.
 *   ylt             double[n], host or device; finite and >= 0
 *   return_periods  double[n_rp], host; each RP >= 1 with floor(n/RP) >= 1
 *   pml_out, tvar_out  double[n_rp], host
 * The k-th largest is found by an exact radix selection on the device and
 * the tail sum is exact before one final rounding.  Errors:
 * ARA_E_INVALID_ARG (bad RP, NaN/negative/inf loss), ARA_E_NOMEM, ARA_E_CUDA. */
ARA_API ara_status ara_pml_tvar(ara_ctx *ctx, const double *ylt, int64_t n,
                        const double *return_periods, int32_t n_rp, double *pml_out,
                        double *tvar_out);

/* ara_pml_tvar queued on the context's stream, for a caller that keeps the
 * results on the device (pricing layer after layer without waiting for each):
 *   ylt             double[n], DEVICE memory; finite and >= 0
 *   return_periods  double[n_rp], host; as for ara_pml_tvar
 *   out             double[2 * n_rp], DEVICE memory: PML_0..PML_{n_rp-1}, then
 *                   TVaR_0..TVaR_{n_rp-1}, written in the stream's order
 * Returns once the work is queued: the host does not wait.  Same definitions
 * and bits as ara_pml_tvar.  Losses that fail the check (NaN, negative or
 * infinite) cannot be reported by the return status: every output is then a
 * quiet NaN.  Errors found on the host: ARA_E_INVALID_ARG (bad RP, host
 * pointers), ARA_E_CUDA. */
ARA_API ara_status ara_pml_tvar_async(ara_ctx *ctx, const double *ylt, int64_t n,
                                      const double *return_periods, int32_t n_rp, double *out);

/* The k largest of a YLT's n trial losses, for the exchange between trial
 * shards (Section IV-C spreads one analysis' trials over several GPUs).  PML
 * and TVaR at return period RP read only the floor(N / RP) largest of N
 * losses, and the k largest of a union of shards lie in the union of each
 * shard's k largest: shards that send their floor(N_total / RP_min) largest
 * send all that ara_pml_tvar_tail needs, instead of whole YLTs.
 *   ylt       double[n], host or device; finite and >= 0
 *   k         1 <= k <= n
 *   tail_out  double[k], host or device, caller-owned: the values above the
 *             k-th largest value tau, in index order, then copies of tau
 *             (k values in all; the same on every run)
 * Errors: ARA_E_INVALID_ARG (sizes, NaN/negative/inf loss; tail_out is then
 * unspecified), ARA_E_NOMEM, ARA_E_CUDA. */
ARA_API ara_status ara_ylt_tail(ara_ctx *ctx, const double *ylt, int64_t n, int64_t k, double *tail_out);

/* PML and TVaR of a YLT of n_total trial losses from m values of it that
 * include its floor(n_total / RP) largest for every return period given
 * (for example the concatenated ara_ylt_tail outputs of its shards): the
 * same definitions as ara_pml_tvar with k = floor(n_total / RP_r), and the
 * same bits as ara_pml_tvar on the whole YLT (the tail sum is exact, on the
 * fixed-point scale the whole YLT would use).
 *   tail      double[m], host or device; finite and >= 0
 *   n_total   trial count of the whole YLT, >= m
 * Errors: ARA_E_INVALID_ARG (bad RP, floor(n_total / RP) above m,
 * NaN/negative/inf value), ARA_E_NOMEM, ARA_E_CUDA. */
ARA_API ara_status ara_pml_tvar_tail(ara_ctx *ctx, const double *tail, int64_t m, int64_t n_total,
                                     const double *return_periods, int32_t n_rp, double *pml_out,
                                     double *tvar_out);

/* Year Loss Tables of several layers over the first n_trials trials
 * (Section III: a Program covers several Layers, a Portfolio several
 * Programs; each layer's YLT is Algorithm 1 for that layer).
 *   layers       n_layers layer handles
 *   ylt_out      double[n_layers][n_trials], host or device, layer-major:
 *                ylt_out[i * n_trials + t] is trial t of layers[i]
 *   cuda_stream  stream for this call only, or NULL for the context's stream
 * Layers are priced two at a time: their tables are interleaved so one L2
 * sector serves both, and one pass over the YET feeds both.  Each value is
 * identical to ara_layer_ylt's for the same layer.  Errors as ara_layer_ylt. */
ARA_API ara_status ara_layers_ylt(ara_ctx *ctx, int32_t n_layers, const int32_t *layers,
                                  int64_t n_trials, double *ylt_out, void *cuda_stream);

/* PML and TVaR of n_layers YLTs of n trials each, as ara_pml_tvar for each
 * layer.  ylt: double[n_layers][n] (host or device, layer-major);
 * return_periods: double[n_rp] (host); pml_out, tvar_out: double[n_layers][n_rp]
 * (host).  Errors as ara_pml_tvar. */
ARA_API ara_status ara_pml_tvar_batch(ara_ctx *ctx, const double *ylt, int32_t n_layers, int64_t n,
                                      const double *return_periods, int32_t n_rp, double *pml_out,
                                      double *tvar_out);

/* Year Event Loss Table of one layer over the first n_trials trials
 * (Section III, step 4: the aggregate terms act on the running sum after
 * every event; the YELT keeps each event's share of the trial loss).  For
 * occurrence k of trial t (stored order), with P_k the running sum of
 * occurrence-net losses and a_k = min(max(P_k - AggR, 0), AggL), a_0 = 0:
 *   yelt_out[offsets[t] + k] = a_k - a_{k-1}     (>= 0; a trial's entries sum
 *                                                 to its YLT entry up to rounding)
 *   occ_max_out[t] = max_k (a_k - a_{k-1})       (0 for an empty trial: the
 *                                                 trial's occurrence loss for OEP)
 *   yelt_out     double[offsets[n_trials]], host or device, CSR by the YET's
 *                trial offsets; NULL if not wanted
 *   occ_max_out  double[n_trials], host or device; NULL if not wanted
 *   cuda_stream  stream for this call, or NULL for the context's stream
 * FP64 layers: the running sums are exact integers on the layer's grid; each
 * entry is rounded once.  With yelt_out, the context keeps (catalog_size + 1)
 * doubles of device scratch for the layer's table in binary64, rebuilt by
 * each call.  Errors as ara_layer_ylt. */
ARA_API ara_status ara_layer_yelt(ara_ctx *ctx, int32_t layer, int64_t n_trials, double *yelt_out,
                                  double *occ_max_out, void *cuda_stream);

/* Return Period Loss report of one layer over the first n_trials trials
 * (Section III names RPL reports beside PML and TVaR): for each return
 * period RP, k = floor(n_trials / RP),
 *   aep_out[r], aep_tvar_out[r]  k-th largest trial loss and mean of the k
 *                                largest (aggregate exceedance: equal to
 *                                ara_pml_tvar of the layer's YLT)
 *   oep_out[r], oep_tvar_out[r]  the same over the trials' largest
 *                                increments (occurrence exceedance)
 * return_periods: double[n_rp] (host, 1..16 values, RP >= 1 and k >= 1);
 * outputs: double[n_rp] each (host).  Errors as ara_layer_ylt and
 * ara_pml_tvar. */
ARA_API ara_status ara_rpl_report(ara_ctx *ctx, int32_t layer, int64_t n_trials,
                                  const double *return_periods, int32_t n_rp, double *aep_out,
                                  double *aep_tvar_out, double *oep_out, double *oep_tvar_out);

/* Allocation-free variant of ara_pml_tvar.  The paper has no counterpart:
 * this exists for callers that cannot call cudaMalloc -- a service whose
 * pooling allocator already owns the device memory it may use, or a
 * latency-critical request path that forbids allocation after start-up
 * because cudaMalloc/cudaFree can stall the whole device.  It needs no
 * context (creating one allocates) and allocates nothing: its selection
 * workspace is a fixed static device array of about 33 KB that every GPU
 * loading the library keeps until the process exits.
 *   ylt             double[n], DEVICE memory of the current device; finite, >= 0
 *   return_periods  double[n_rp], host; 1 <= n_rp <= 16 (the array's limit;
 *                   more is rejected with ARA_E_INVALID_ARG)
 *   pml_out, tvar_out  double[n_rp], host or device
 *   cuda_stream     stream to run on (NULL = the legacy default stream)
 * Same definitions and results as ara_pml_tvar.  Returns after the outputs
 * are written.  The first call on each device looks up the array's device
 * address; make that first call before any stream capture.  Every call
 * shares the one array: calls whose work overlaps on the GPU (other threads
 * or streams) race and must be serialised by the caller.  Errors as
 * ara_pml_tvar; the message is read with ara_last_error(NULL). */
ARA_API ara_status ara_pml_tvar_noalloc(const double *ylt, int64_t n, const double *return_periods,
                                        int32_t n_rp, double *pml_out, double *tvar_out,
                                        void *cuda_stream);

/* ------------------------------------------------------------ pricing plans */
/*
 * A plan prices a fixed list of layers (Section III: a Program or Portfolio
 * is a set of Layers) as one CUDA graph: every layer's ELT fold (the
 * pre-pass of ara_define_layer), the grouped passes of ara_layers_ylt over
 * the first n_trials trials, and the PML/TVaR selection of
 * ara_pml_tvar_batch.  ara_plan_run replays it with one graph launch and
 * gives the same values as those calls.  The plan groups its layers into
 * passes whose layers share most of their possibly nonzero events (each pass
 * gathers one table row per occurrence that any of its layers needs): layers
 * are taken densest first and each pass is filled with the layers whose
 * zero-skip bitmaps overlap its union most.  Without autotune a pass holds 2
 * FP64 or 4 FP32-table layers.  With autotune != 0, plan creation first
 * times the YLT kernel's launch shapes (lanes per trial -- the trials a warp
 * sums side by side --, id loads per lane, whether the id stream is
 * prefetched into L2, and 1024- or 768-thread CTAs) on the first
 * min(n_trials, 2^20) trials and, per entry width, the group size (FP64: 2
 * or 1 layers per pass; FP32 tables: 4, 2 or 1) by timing the whole set of
 * passes on the first min(n_trials, 2^18) trials, all on the plan's own
 * layers, and keeps the fastest; the launch shapes also serve later
 * ara_layers_ylt / ara_layer_ylt calls on the context.
 * The plan owns its output buffers and, for each pass over several layers,
 * that pass's interleaved table ((catalog + 1) x entry bytes x layers) and
 * union bitmap, into which its folds write directly (when these cannot be
 * allocated the graph interleaves the layers' own tables instead).  A plan
 * stops working (ARA_E_STATE from
 * ara_plan_run) when the YET is reloaded or one of its layers is released;
 * ara_destroy destroys the context's plans.
 */
typedef struct ara_plan ara_plan;

/* layers: n_layers handles (1..65535); return_periods: double[n_rp] (host,
 * 1..16 values, floor(n_trials / RP) >= 1).  Errors: ARA_E_INVALID_ARG,
 * ARA_E_NOT_FOUND, ARA_E_STATE (no YET, or a service owns the context),
 * ARA_E_NOMEM, ARA_E_CUDA. */
ARA_API ara_status ara_plan_create(ara_ctx *ctx, const int32_t *layers, int32_t n_layers, int64_t n_trials,
                                   const double *return_periods, int32_t n_rp, int32_t autotune,
                                   ara_plan **out);

/* Replay the plan on cuda_stream (NULL = the context's stream).
 *   ylt_out   NULL, or double[n_layers][n_trials] (host or device)
 *   pml_out, tvar_out  NULL, or double[n_layers][n_rp] (host)
 * Returns once the outputs are written (host outputs), or once the work is
 * queued (device or no outputs).  Errors: ARA_E_STATE, ARA_E_CUDA. */
ARA_API ara_status ara_plan_run(ara_plan *plan, double *ylt_out, double *pml_out, double *tvar_out,
                                void *cuda_stream);

/* The plan's YLT passes: *n_passes receives their number and, for the first
 * max_passes, info[10*i .. 10*i+9] = entry bytes (16 FP64, 8 FP32-table),
 * layers in the pass (G), lanes per trial, id loads per lane, L2 prefetch
 * (1/0), threads per CTA, and the positions in the plan's layer list of the
 * pass's G layers (then -1 up to four). */
ARA_API ara_status ara_plan_passes(const ara_plan *plan, int32_t max_passes, int32_t *info,
                                   int32_t *n_passes);

/* The number of kernel launches one ara_plan_run replays (the kernel nodes
 * of the plan's graph: the folds, the YLT passes, any interleave of tables,
 * the selection), in *n_kernels.  Errors: ARA_E_INVALID_ARG, ARA_E_CUDA. */
ARA_API ara_status ara_plan_kernel_launches(const ara_plan *plan, int32_t *n_kernels);

ARA_API void ara_plan_destroy(ara_plan *plan);

/* ---------------------------------------------------------- pricing service */
/*
 * Ad hoc pricing (Section I: an underwriter quotes a contract while on the
 * phone, so a layer must be priced in real time).  Each request is one Layer
 * (Section III) over ELTs already loaded into the context, priced by
 * Algorithm 1 over a prefix of the loaded YET, with PML and TVaR at the
 * service's return periods.  The YET and the ELT pool stay on the device.
 *
 * A scheduler thread owned by the service admits queued requests in arrival
 * order while a slot is free and the in-flight requests' device memory stays
 * within the budget, and batches the requests that share the oldest queued
 * request's trial count (up to max_batch) into one slot: their layers are
 * folded, priced two per pass over the YET, and their PML/TVaR computed in
 * one batched selection, all on the slot's own stream, so batches of
 * different slots overlap on the device.  Requests that arrive meanwhile are
 * queued and join the next batch that a free slot takes (continuous
 * batching).  A request's results do not depend on the other requests of its
 * batch: they are identical to pricing it alone.
 *
 * While a service is attached, the context is used by the scheduler thread
 * alone: every other call on the context returns ARA_E_STATE (ara_destroy
 * destroys the service first).  The service calls may be made from any
 * thread; their error messages are read with ara_last_error(NULL) on the
 * calling thread.  Requests use the ELTs and the YET loaded before
 * ara_service_create.
 */
typedef struct ara_service ara_service;

typedef struct {
  int32_t slots;             /* batches in flight at once, 1..16; each has a stream */
  int32_t max_batch;         /* requests per batch, 1..64 */
  int64_t memory_budget;     /* device bytes that in-flight requests may hold
                                (layer tables, YLTs, selection state); 0 = a
                                quarter of the free device memory at creation */
  int32_t n_return_periods;  /* 1..16 */
  double return_periods[16]; /* each >= 1 */
  int32_t fail_every;        /* fault injection for tests: when > 0, every
                                fail_every-th admitted request ends with
                                ARA_E_NOMEM as if its allocation had failed,
                                and the rest of its batch proceeds; 0 = off */
} ara_service_config;

typedef struct {
  int32_t n_elts;              /* 1..1024 */
  const int32_t *elt_handles;  /* host; copied at submit; order = summation order */
  double occ_ret, occ_lim, agg_ret, agg_lim;  /* as ara_define_layer */
  int32_t precision;           /* ARA_FP64 or ARA_FP32_TABLE */
  int64_t n_trials;            /* trials 0..n_trials-1 of the loaded YET; floor(n_trials / RP) >= 1 */
  double deadline_s;           /* > 0: a request not started this many seconds
                                  after submit ends with ARA_E_TIMEOUT; 0 = none */
  double *ylt_out;             /* optional host double[n_trials] that receives
                                  the YLT; must stay valid until the request
                                  ends (ara_service_wait returns it or
                                  ara_service_destroy runs); NULL = not wanted */
} ara_request;

typedef struct {
  ara_status status;     /* ARA_OK, or why the request failed */
  int32_t batch_size;    /* requests priced in its batch */
  int32_t slot;          /* slot that priced it (-1 if it never started) */
  int32_t n_return_periods;
  double pml[16], tvar[16];
  double t_submit, t_start, t_done;  /* seconds since the service started */
  char message[160];     /* failure message, empty on success */
} ara_result;

typedef struct {
  int64_t submitted, completed, failed, cancelled, timed_out, batches;
  int64_t queued, in_flight;         /* now */
  int64_t max_in_flight;             /* most requests in flight at once */
  int64_t max_batch_seen;            /* largest batch formed */
  int64_t bytes_in_flight, max_bytes_in_flight, memory_budget;
  int64_t max_slots_busy;            /* most slots busy at once */
} ara_service_stats;

/* Attach a service to ctx (a YET must be loaded: ARA_E_STATE otherwise) and
 * start its scheduler thread.  Waits for the context's queued work first.
 * Errors: ARA_E_INVALID_ARG (config), ARA_E_STATE (no YET, or a service is
 * already attached), ARA_E_NOMEM, ARA_E_CUDA. */
ARA_API ara_status ara_service_create(ara_ctx *ctx, const ara_service_config *config,
                                      ara_service **out);

/* Queue one request; *ticket identifies it (> 0).  The request is checked
 * here: ARA_E_INVALID_ARG (terms, sizes, a return period above n_trials),
 * ARA_E_NOT_FOUND (ELT handle), ARA_E_NOMEM (its device footprint exceeds
 * the whole budget), ARA_E_STATE (service shutting down). */
ARA_API ara_status ara_service_submit(ara_service *svc, const ara_request *request, int64_t *ticket);

/* Wait up to timeout_s seconds (>= 0) for a request to end.  ARA_OK: *out
 * holds its result (out->status says whether it succeeded) and the ticket is
 * retired.  ARA_E_TIMEOUT: still queued or running (the wait changed
 * nothing).  ARA_E_NOT_FOUND: unknown or retired ticket. */
ARA_API ara_status ara_service_wait(ara_service *svc, int64_t ticket, double timeout_s, ara_result *out);

/* Cancel a queued request: it ends with ARA_E_CANCELLED.  ARA_E_STATE if it
 * already started or ended; ARA_E_NOT_FOUND for an unknown ticket. */
ARA_API ara_status ara_service_cancel(ara_service *svc, int64_t ticket);

/* Counters since creation (host copy). */
ARA_API ara_status ara_service_get_stats(ara_service *svc, ara_service_stats *out);

/* Stop the scheduler: queued requests end with ARA_E_CANCELLED, batches on
 * the device are waited for, the service's buffers are freed and the
 * context is detached (usable again).  Results not collected are dropped. */
ARA_API void ara_service_destroy(ara_service *svc);

/* ------------------------------------------------------------- measurement */

/* Record CUDA events around every kernel launch of the timing channels
 * (enable != 0) or stop recording (enable == 0).  Enabling clears the
 * totals. */
ARA_API ara_status ara_set_kernel_timing(ara_ctx *ctx, int32_t enable);

/* Launch count and summed device time (milliseconds) of one timing channel
 * since timing was enabled.  Waits for the recorded events. */
ARA_API ara_status ara_kernel_timing(ara_ctx *ctx, int32_t channel, int64_t *launches,
                             double *total_ms);

/* Ceilings of the YLT kernel's inner loop, measured on a device (they are
 * not part of the method: a benchmark states the kernels' rates against
 * them).  Per occurrence the YLT kernel tests one bit of a shared-memory
 * bitmap at a random word and, when the event may have a nonzero loss,
 * gathers its entry from a per-event table held in L2 (Section IV-B: one
 * memory access per direct-access-table lookup); an FP64 running sum would
 * need one binary64 add per occurrence.  Each call allocates and frees its
 * own device buffers on a stream of its own, runs a warm-up launch and
 * returns the best of five timed launches; messages go to
 * ara_last_error(NULL).  Errors: ARA_E_INVALID_ARG, ARA_E_NOMEM, ARA_E_CUDA.
 *
 * ara_probe_gather: rows of load_bytes x lanes_per_row bytes (at most one
 * 128-byte line) at random positions of a table of table_bytes, warmed into
 * L2 by the first launch; each row is read by lanes_per_row lanes of one
 * warp instruction, load_bytes (8, 16 or 32) each, four rows in flight per
 * lane group, with the YLT kernel's cache policy (no L1 allocation, L2
 * evict-last); grid = SM count x ctas_per_sm CTAs of threads_per_cta
 * threads.  *rows_per_s: rows read per second; *sectors_per_s: 32-byte
 * sectors per second (a row of fewer than 32 bytes counts one). */
ARA_API ara_status ara_probe_gather(int device, int64_t table_bytes, int32_t load_bytes,
                                    int32_t lanes_per_row, int32_t threads_per_cta,
                                    int32_t ctas_per_sm, double *rows_per_s, double *sectors_per_s);

/* Random 32-bit shared-memory reads per second over the whole device: one
 * CTA of 1024 threads per SM holding the largest shared array a CTA may
 * have, eight independent lookups in flight per thread. */
ARA_API ara_status ara_probe_smem_lookup(int device, double *lookups_per_s);

/* Binary64 adds per second over the whole device: eight independent chains
 * of round-to-nearest adds per thread, eight CTAs of 256 threads per SM. */
ARA_API ara_status ara_probe_fp64_add(int device, double *adds_per_s);

#ifdef __cplusplus
}
#endif

#endif /* ARA_H_ */
