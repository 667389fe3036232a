/*
 * FP64 reference ("oracle") for the Year Loss Table of Aggregate Risk Analysis.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  It shares no code, header or
 * constant with the CUDA engine, and the engine never calls it.
 *
 * It follows Varghese & Barker, "Are Clouds Ready to Accelerate Ad hoc
 * Financial Simulations?" (arXiv 1412.4556), Section III, Algorithm 1, in
 * the paper's loop order:
 *
 *   for each layer L; for each trial T of the YET; for each event E of T
 *     (stored = ascending time-stamp order); for each ELT of L (layer order):
 *       l_E  = DAT_ELT[E]                 lookup (Sec. III step 1; Sec. IV-B:
 *                                          direct access table, 0 when absent)
 *       l_E  = FT1(l_E)                   ELT financial terms (step 2)
 *       x   += l_E                        combine across the layer's ELTs
 *     o  = FT2(x)                         occurrence terms (step 3)
 *     P += o;  a = FT3(P)                 aggregate terms on the running
 *                                          cumulative sum (step 4)
 *   YLT[T] = a                            trial (year) loss
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes of the repository):
 *   R1  FT1 = (deductible D, limit Lim):  min(max(l - D, 0), Lim).
 *       Secondary uncertainty (named in step 2, never defined) is the
 *       identity.  PARITY UNPINNED for secondary uncertainty: it is not built.
 *   R2  FT2 = (OccR, OccL), applied to each event's combined loss:
 *       min(max(x - OccR, 0), OccL)  (the printed formula drops max's 0).
 *   R3  FT3 = (AggR, AggL), applied to the running sum P of occurrence-net
 *       losses of the trial: min(max(P - AggR, 0), AggL); P restarts at 0
 *       for every trial; the trial loss is the clamp after the last event.
 *   R4  An empty trial has loss 0.
 *   R5  PML(RP) = y(k), TVaR(RP) = (y(1) + ... + y(k)) / k with y sorted
 *       descending and k = floor(N / RP) >= 1; the sum runs in descending
 *       order in FP64.
 *   R6  ELTs are summed in layer order, events in stored order.
 *   R11 The Year Event Loss Table (YELT) holds, for every occurrence, the
 *       increment of the aggregate-clamped running loss (inc_k = a_k -
 *       a_{k-1}); a trial's occurrence loss for the occurrence exceedance
 *       (OEP) report is its largest increment (0 for an empty trial), and a
 *       Return Period Loss (Sec. III, reports) is the PML-style k-th largest
 *       value of the YLT (aggregate, AEP) or of those maxima (OEP).
 *
 * All arithmetic is IEEE binary64 with round-to-nearest; the hot path has no
 * multiplications, and the file is built with -ffp-contract=off.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_E_ARG -1
#define ORACLE_E_RANGE -2
#define ORACLE_E_NOMEM -4

/* Sec. III step 2, reading R1: ELT terms on one event loss. */
static double ft1(double loss, double deductible, double limit) {
  double v = loss - deductible;
  if (v < 0.0) v = 0.0;
  if (v > limit) v = limit;
  return v;
}

/* Sec. III step 3, reading R2: occurrence retention then occurrence limit. */
static double ft2(double x, double occ_ret, double occ_lim) {
  double v = x - occ_ret;
  if (v < 0.0) v = 0.0;
  if (v > occ_lim) v = occ_lim;
  return v;
}

/* Sec. III step 4, reading R3: aggregate terms on the cumulative sum. */
static double ft3(double p, double agg_ret, double agg_lim) {
  double v = p - agg_ret;
  if (v < 0.0) v = 0.0;
  if (v > agg_lim) v = agg_lim;
  return v;
}

/* A layer as the oracle sees it: one dense direct access table per ELT. */
typedef struct {
  int32_t catalog;
  int32_t n_elts;
  double *dats;          /* n_elts x catalog, row j = DAT of the layer's j-th ELT */
  const double *ded;     /* n_elts */
  const double *lim;     /* n_elts */
  double occ_ret, occ_lim, agg_ret, agg_lim;
  double *memo;          /* optional: combined ELT loss x(e) per event (R6) */
} layer_t;

/* Sec. IV-B's direct access table of an ELT: a dense array over event ids
 * holding the ELT's loss for present events and 0 elsewhere. */
static int build_dats(layer_t *L, const int64_t *elt_off, const int32_t *elt_ids,
                      const double *elt_losses) {
  size_t n = (size_t)L->n_elts * (size_t)L->catalog;
  L->dats = (double *)calloc(n ? n : 1, sizeof(double));
  if (!L->dats) return ORACLE_E_NOMEM;
  for (int32_t j = 0; j < L->n_elts; ++j) {
    double *dat = L->dats + (size_t)j * (size_t)L->catalog;
    for (int64_t i = elt_off[j]; i < elt_off[j + 1]; ++i) {
      int32_t e = elt_ids[i];
      if (e < 0 || e >= L->catalog) return ORACLE_E_RANGE;
      dat[e] = elt_losses[i];
    }
  }
  return ORACLE_OK;
}

/* Steps 1-2 for one event: the loss combined across the layer's ELTs. */
static double combined_elt_loss(const layer_t *L, int32_t e) {
  double x = 0.0;
  for (int32_t j = 0; j < L->n_elts; ++j) {
    double l = L->dats[(size_t)j * (size_t)L->catalog + (size_t)e];
    x = x + ft1(l, L->ded[j], L->lim[j]);
  }
  return x;
}

/* Steps 1-4 for one trial.  Optional per-event outputs (length = count):
 * occ[k] occurrence-net loss, agg[k] aggregate-clamped running loss,
 * inc[k] = agg[k] - agg[k-1] (the per-event increment). */
static double trial_loss(const layer_t *L, const int32_t *ids, int64_t count, double *presum,
                         double *occ, double *agg, double *inc) {
  double p = 0.0, a = 0.0, prev = 0.0;
  for (int64_t k = 0; k < count; ++k) {
    int32_t e = ids[k];
    double x = L->memo ? L->memo[e] : combined_elt_loss(L, e);
    double o = ft2(x, L->occ_ret, L->occ_lim);
    p = p + o;
    a = ft3(p, L->agg_ret, L->agg_lim);
    if (occ) occ[k] = o;
    if (agg) agg[k] = a;
    if (inc) inc[k] = a - prev;
    prev = a;
  }
  if (presum) *presum = p;
  return a; /* R4: 0.0 when count == 0 */
}

typedef struct {
  const layer_t *L;
  const int64_t *offsets;
  const int32_t *ids;
  const int64_t *sel;
  int64_t first, last; /* range over sel (or over trials when sel is NULL) */
  double *ylt;
  double *presum;
} job_t;

static void *run_job(void *arg) {
  job_t *J = (job_t *)arg;
  for (int64_t i = J->first; i < J->last; ++i) {
    int64_t t = J->sel ? J->sel[i] : i;
    int64_t a = J->offsets[t], b = J->offsets[t + 1];
    double s = 0.0;
    J->ylt[i] = trial_loss(J->L, J->ids + a, b - a, &s, NULL, NULL, NULL);
    if (J->presum) J->presum[i] = s;
  }
  return NULL;
}

static int check_yet(int32_t catalog, int64_t n_trials, const int64_t *offsets,
                     const int32_t *ids) {
  if (catalog < 0 || n_trials < 0 || !offsets) return ORACLE_E_ARG;
  if (offsets[0] != 0) return ORACLE_E_ARG;
  for (int64_t t = 0; t < n_trials; ++t)
    if (offsets[t + 1] < offsets[t]) return ORACLE_E_ARG;
  for (int64_t i = 0; i < offsets[n_trials]; ++i)
    if (ids[i] < 0 || ids[i] >= catalog) return ORACLE_E_RANGE;
  return ORACLE_OK;
}

typedef struct {
  layer_t *L;
  int32_t first, last; /* event range */
} memo_job_t;

static void *run_memo_job(void *arg) {
  memo_job_t *J = (memo_job_t *)arg;
  for (int32_t e = J->first; e < J->last; ++e) J->L->memo[e] = combined_elt_loss(J->L, e);
  return NULL;
}

static int init_layer(layer_t *L, int32_t catalog, int32_t n_elts, const int64_t *elt_off,
                      const int32_t *elt_ids, const double *elt_losses, const double *ded,
                      const double *lim, double occ_ret, double occ_lim, double agg_ret,
                      double agg_lim, int memoise, int32_t n_threads) {
  memset(L, 0, sizeof(*L));
  if (n_elts < 0) return ORACLE_E_ARG;
  L->catalog = catalog;
  L->n_elts = n_elts;
  L->ded = ded;
  L->lim = lim;
  L->occ_ret = occ_ret;
  L->occ_lim = occ_lim;
  L->agg_ret = agg_ret;
  L->agg_lim = agg_lim;
  int rc = build_dats(L, elt_off, elt_ids, elt_losses);
  if (rc) return rc;
  if (memoise) {
    /* R6 memoised mode: x(e) is a pure function of the event, so computing it
     * once per catalog event with the same ELT loop gives the same bits. */
    L->memo = (double *)malloc((size_t)(catalog ? catalog : 1) * sizeof(double));
    if (!L->memo) return ORACLE_E_NOMEM;
    /* threads split the catalog; each event's ELT loop is the same sequential
     * loop whichever thread runs it */
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    if (catalog < 65536) n_threads = 1;
    pthread_t th[256];
    memo_job_t jobs[256];
    for (int32_t i = 0; i < n_threads; ++i) {
      jobs[i].L = L;
      jobs[i].first = (int32_t)((int64_t)catalog * i / n_threads);
      jobs[i].last = (int32_t)((int64_t)catalog * (i + 1) / n_threads);
    }
    int32_t started = 0;
    if (n_threads > 1)
      for (; started < n_threads; ++started)
        if (pthread_create(&th[started], NULL, run_memo_job, &jobs[started])) break;
    for (int32_t i = started; i < n_threads; ++i) run_memo_job(&jobs[i]);
    for (int32_t i = 0; i < started; ++i) pthread_join(th[i], NULL);
  }
  return ORACLE_OK;
}

static void free_layer(layer_t *L) {
  free(L->dats);
  free(L->memo);
}

/* Threads split the trial list; per-trial arithmetic is sequential, so the
 * results do not depend on the thread count. */
static void run_trials(const layer_t *L, const int64_t *offsets, const int32_t *ids, const int64_t *sel,
                       int64_t n, int32_t n_threads, double *ylt_out, double *presum_out) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  if (n < n_threads) n_threads = n > 0 ? (int32_t)n : 1;
  pthread_t th[256];
  job_t jobs[256];
  for (int32_t i = 0; i < n_threads; ++i) {
    jobs[i].L = L;
    jobs[i].offsets = offsets;
    jobs[i].ids = ids;
    jobs[i].sel = sel;
    jobs[i].first = n * i / n_threads;
    jobs[i].last = n * (i + 1) / n_threads;
    jobs[i].ylt = ylt_out;
    jobs[i].presum = presum_out;
  }
  int32_t started = 0;
  if (n_threads > 1)
    for (; started < n_threads; ++started)
      if (pthread_create(&th[started], NULL, run_job, &jobs[started])) break;
  for (int32_t i = started; i < n_threads; ++i) run_job(&jobs[i]);
  for (int32_t i = 0; i < started; ++i) pthread_join(th[i], NULL);
}

static int check_sel(int64_t n_trials, const int64_t *sel, int64_t n_sel) {
  if (sel)
    for (int64_t i = 0; i < n_sel; ++i)
      if (sel[i] < 0 || sel[i] >= n_trials) return ORACLE_E_ARG;
  return ORACLE_OK;
}

/*
 * One layer's YLT (Algorithm 1) over the trials listed in sel[0..n_sel) (or
 * over all n_trials trials when sel is NULL, n_sel ignored).
 *   offsets int64[n_trials+1], ids int32[offsets[n_trials]]  -- CSR YET
 *   elt_off int64[n_elts+1], elt_ids int32, elt_losses f64   -- the layer's
 *       ELTs in layer (summation) order; ids distinct within one ELT
 *   ded, lim f64[n_elts]                                     -- FT1 per ELT
 *   mode 0 = literal (ELT loop per occurrence), 1 = memoised (R6)
 *   ylt_out f64[n_sel or n_trials]; presum_out (nullable): sum before FT3.
 */
int ara_oracle_layer_ylt(int32_t catalog, int64_t n_trials, const int64_t *offsets,
                         const int32_t *ids, int32_t n_elts, const int64_t *elt_off,
                         const int32_t *elt_ids, const double *elt_losses, const double *ded,
                         const double *lim, double occ_ret, double occ_lim, double agg_ret,
                         double agg_lim, int32_t mode, int32_t n_threads, const int64_t *sel,
                         int64_t n_sel, double *ylt_out, double *presum_out) {
  int rc = check_yet(catalog, n_trials, offsets, ids);
  if (!rc) rc = check_sel(n_trials, sel, n_sel);
  if (rc) return rc;
  layer_t L;
  rc = init_layer(&L, catalog, n_elts, elt_off, elt_ids, elt_losses, ded, lim, occ_ret,
                  occ_lim, agg_ret, agg_lim, mode == 1, n_threads);
  if (!rc) run_trials(&L, offsets, ids, sel, sel ? n_sel : n_trials, n_threads, ylt_out, presum_out);
  free_layer(&L);
  return rc;
}

/*
 * The YLTs of n_layers layers (Algorithm 1's outer loop over the layers of a
 * Program, each layer's trials priced as ara_oracle_layer_ylt does), with the
 * YET checked once.  Layer i has n_elts[i] ELTs in the arrays elt_off[i],
 * elt_ids[i], elt_losses[i], ded[i], lim[i] and the terms occ_ret[i],
 * occ_lim[i], agg_ret[i], agg_lim[i]; its outputs are
 * ylt_out[i * n .. i * n + n) and (nullable) presum_out[same], n = n_sel or
 * n_trials.  Same bits as one ara_oracle_layer_ylt call per layer.
 */
int ara_oracle_layers_ylt(int32_t catalog, int64_t n_trials, const int64_t *offsets,
                          const int32_t *ids, int32_t n_layers, const int32_t *n_elts,
                          const int64_t *const *elt_off, const int32_t *const *elt_ids,
                          const double *const *elt_losses, const double *const *ded,
                          const double *const *lim, const double *occ_ret, const double *occ_lim,
                          const double *agg_ret, const double *agg_lim, int32_t mode,
                          int32_t n_threads, const int64_t *sel, int64_t n_sel, double *ylt_out,
                          double *presum_out) {
  if (n_layers < 0) return ORACLE_E_ARG;
  int rc = check_yet(catalog, n_trials, offsets, ids);
  if (!rc) rc = check_sel(n_trials, sel, n_sel);
  if (rc) return rc;
  const int64_t n = sel ? n_sel : n_trials;
  for (int32_t i = 0; i < n_layers; ++i) {
    layer_t L;
    rc = init_layer(&L, catalog, n_elts[i], elt_off[i], elt_ids[i], elt_losses[i], ded[i], lim[i],
                    occ_ret[i], occ_lim[i], agg_ret[i], agg_lim[i], mode == 1, n_threads);
    if (!rc)
      run_trials(&L, offsets, ids, sel, n, n_threads, ylt_out + (size_t)i * (size_t)n,
                 presum_out ? presum_out + (size_t)i * (size_t)n : NULL);
    free_layer(&L);
    if (rc) return rc;
  }
  return ORACLE_OK;
}

typedef struct {
  const layer_t *L;
  const int64_t *offsets;
  const int32_t *ids;
  const int64_t *sel;
  const int64_t *out_off;
  int64_t first, last;
  double *inc, *occ_max, *ylt, *presum;
} yelt_job_t;

static void *run_yelt_job(void *arg) {
  yelt_job_t *J = (yelt_job_t *)arg;
  for (int64_t i = J->first; i < J->last; ++i) {
    int64_t t = J->sel ? J->sel[i] : i;
    int64_t a = J->offsets[t], b = J->offsets[t + 1];
    double *inc = J->inc + J->out_off[i];
    double s = 0.0;
    J->ylt[i] = trial_loss(J->L, J->ids + a, b - a, &s, NULL, NULL, inc);
    double m = 0.0; /* R11: 0 for an empty trial */
    for (int64_t k = 0; k < b - a; ++k)
      if (inc[k] > m) m = inc[k];
    J->occ_max[i] = m;
    if (J->presum) J->presum[i] = s;
  }
  return NULL;
}

/*
 * Year Event Loss Table of one layer (reading R11) over the trials listed in
 * sel[0..n_sel) (all trials when sel is NULL): the increments of every
 * selected trial, concatenated in list order (trial i's at
 * inc_out[out_off[i] .. out_off[i+1]), out_off int64[n+1] built by the
 * caller from the trial lengths), each trial's largest increment
 * (occ_max_out) and trial loss (ylt_out), and optionally its pre-aggregate
 * sum.  Arguments otherwise as ara_oracle_layer_ylt.
 */
int ara_oracle_layer_yelt(int32_t catalog, int64_t n_trials, const int64_t *offsets,
                          const int32_t *ids, int32_t n_elts, const int64_t *elt_off,
                          const int32_t *elt_ids, const double *elt_losses, const double *ded,
                          const double *lim, double occ_ret, double occ_lim, double agg_ret,
                          double agg_lim, int32_t mode, int32_t n_threads, const int64_t *sel,
                          int64_t n_sel, const int64_t *out_off, double *inc_out,
                          double *occ_max_out, double *ylt_out, double *presum_out) {
  int rc = check_yet(catalog, n_trials, offsets, ids);
  if (rc) return rc;
  int64_t n = sel ? n_sel : n_trials;
  if (!out_off || out_off[0] != 0) return ORACLE_E_ARG;
  for (int64_t i = 0; i < n; ++i) {
    int64_t t = sel ? sel[i] : i;
    if (t < 0 || t >= n_trials) return ORACLE_E_ARG;
    if (out_off[i + 1] - out_off[i] != offsets[t + 1] - offsets[t]) return ORACLE_E_ARG;
  }
  layer_t L;
  rc = init_layer(&L, catalog, n_elts, elt_off, elt_ids, elt_losses, ded, lim, occ_ret,
                  occ_lim, agg_ret, agg_lim, mode == 1, n_threads);
  if (rc) {
    free_layer(&L);
    return rc;
  }
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  if (n < n_threads) n_threads = n > 0 ? (int32_t)n : 1;
  pthread_t th[256];
  yelt_job_t jobs[256];
  for (int32_t i = 0; i < n_threads; ++i) {
    yelt_job_t J = {&L, offsets, ids, sel, out_off, n * i / n_threads, n * (i + 1) / n_threads,
                    inc_out, occ_max_out, ylt_out, presum_out};
    jobs[i] = J;
  }
  int32_t started = 0;
  if (n_threads > 1)
    for (; started < n_threads; ++started)
      if (pthread_create(&th[started], NULL, run_yelt_job, &jobs[started])) break;
  for (int32_t i = started; i < n_threads; ++i) run_yelt_job(&jobs[i]);
  for (int32_t i = 0; i < started; ++i) pthread_join(th[i], NULL);
  free_layer(&L);
  return ORACLE_OK;
}

/* Per-event trace of one trial (steps 3-4): occurrence-net loss, clamped
 * running aggregate and increment for every event; returns the trial loss in
 * *trial_loss and the pre-aggregate sum in *presum. */
int ara_oracle_trial_trace(int32_t catalog, int64_t count, const int32_t *ids, int32_t n_elts,
                           const int64_t *elt_off, const int32_t *elt_ids,
                           const double *elt_losses, const double *ded, const double *lim,
                           double occ_ret, double occ_lim, double agg_ret, double agg_lim,
                           double *occ, double *agg, double *inc, double *trial_loss_out,
                           double *presum) {
  for (int64_t k = 0; k < count; ++k)
    if (ids[k] < 0 || ids[k] >= catalog) return ORACLE_E_RANGE;
  layer_t L;
  int rc = init_layer(&L, catalog, n_elts, elt_off, elt_ids, elt_losses, ded, lim, occ_ret,
                      occ_lim, agg_ret, agg_lim, 0, 1);
  if (rc) {
    free_layer(&L);
    return rc;
  }
  *trial_loss_out = trial_loss(&L, ids, count, presum, occ, agg, inc);
  free_layer(&L);
  return ORACLE_OK;
}

/* Steps 1-3 for every catalog event: FT2(sum_j FT1(DAT_j[e])), the
 * occurrence-net loss of one occurrence of e, for all e in [0, catalog). */
int ara_oracle_event_table(int32_t catalog, int32_t n_elts, const int64_t *elt_off,
                           const int32_t *elt_ids, const double *elt_losses, const double *ded,
                           const double *lim, double occ_ret, double occ_lim, double *out) {
  layer_t L;
  int rc = init_layer(&L, catalog, n_elts, elt_off, elt_ids, elt_losses, ded, lim, occ_ret,
                      occ_lim, 0.0, 0.0, 0, 1);
  if (rc) {
    free_layer(&L);
    return rc;
  }
  for (int32_t e = 0; e < catalog; ++e) out[e] = ft2(combined_elt_loss(&L, e), occ_ret, occ_lim);
  free_layer(&L);
  return ORACLE_OK;
}

static int cmp_desc(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x < y) - (x > y);
}

/* Reading R5: PML and TVaR from a YLT of n trial losses. */
int ara_oracle_pml_tvar(const double *ylt, int64_t n, const double *rps, int32_t n_rp,
                        double *pml_out, double *tvar_out) {
  if (n < 1 || n_rp < 0) return ORACLE_E_ARG;
  for (int32_t r = 0; r < n_rp; ++r) {
    if (!(rps[r] >= 1.0)) return ORACLE_E_ARG;
    if (floor((double)n / rps[r]) < 1.0) return ORACLE_E_ARG;
  }
  double *y = (double *)malloc((size_t)n * sizeof(double));
  if (!y) return ORACLE_E_NOMEM;
  memcpy(y, ylt, (size_t)n * sizeof(double));
  qsort(y, (size_t)n, sizeof(double), cmp_desc);
  for (int32_t r = 0; r < n_rp; ++r) {
    int64_t k = (int64_t)floor((double)n / rps[r]);
    double s = 0.0;
    for (int64_t i = 0; i < k; ++i) s = s + y[i];
    pml_out[r] = y[k - 1];
    tvar_out[r] = s / (double)k;
  }
  free(y);
  return ORACLE_OK;
}
