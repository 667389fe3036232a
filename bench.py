#!/usr/bin/env python3
"""Benchmark of the Year Loss Table hot path (Varghese & Barker, arXiv 1412.4556).

One step = one pass of the whole path over the paper-scale workload
(catalog 2,000,000 events; one layer over 16 ELTs of 20,000 events;
1,000,000 trials of Poisson(1000) events, about 1e9 occurrences, each an
int32 event id and a float32 time-stamp):

    ara_define_layer  (per-layer ELT fold pre-pass on the device)
    ara_layer_ylt     (per-trial gather + exact sum + aggregate terms)
    ara_pml_tvar      (PML and TVaR at return periods 100 / 250 / 500)

The YET and the ELT pool are resident in HBM when the timed region starts
(the paper's pre-processing stage); the id stream is larger than L2, so every
step reads it from HBM.  ``e2e`` repeats the step through the same C ABI with
host buffers: the YET (ids and time-stamps), the ELTs and the layer go
host->device and the YLT, PML and TVaR come back, inside the timed region.

The default line also carries, each with its own clock record:
  parity    every trial's loss and PML/TVaR against the FP64 oracle;
  batched   64 FP64 layers over the same YET priced as one CUDA graph
            (speed-up over the plain per-layer path, error against the oracle);
  mixed     the same 64 layers with FP32 tables;
  service   a seeded stream of layer-pricing requests at 50/s (p50/p99).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl engine|reference]

Under torchrun (N > 1) every rank prices its own shard of 1,000,000 trials
(weak scaling); each shard's largest losses are all-gathered for the
portfolio-wide PML/TVaR.  ``--impl reference`` times the FP64 CPU oracle (the
only reference this path has) on the same workload.
"""
from __future__ import annotations

import argparse
import concurrent.futures
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import ara_synth as S  # noqa: E402

METRIC = "YLT trial-events/s & HBM GB/s vs roofline; layer-request p50/p99 latency"
UNIT = "trial-events/s"
PAPER_1GPU_TRIAL_EVENTS_PER_S = 1e9 / 19.93  # Tesla M2050, Section IV-C (context only)
WORKLOAD = ("paper-scale plain ARA, FP64: catalog 2,000,000 events; 1 layer over 16 ELTs x 20,000 "
            "events (lognormal(12,1.5) losses, D~U[5e3,5e4], Lim~U[1e6,1e7]); 1,000,000 trials x "
            "Poisson(1000) events (int32 ids + float32 time-stamps); OccR 1e5, OccL 2e7, AggR 5e5, "
            "AggL 1e8; RP 100/250/500")


def paper_config(N: int, M: int, C: int, elts: int, world: int, k_tail: int = 0) -> dict:
    """The workload's config dict, the same for the engine and reference arms."""
    return {"workload": WORKLOAD, "n_trials_per_gpu": N, "occurrences_per_gpu": M, "catalog": C,
            "elts": elts, "return_periods": [100, 250, 500],
            "l2": "inputs larger than L2: the 2-4 GB YET id stream is re-read from HBM every step",
            "parallelism": (f"trial shards x{world}; each rank sends its {k_tail} largest trial losses "
                            "(ara_ylt_tail, NCCL all-gather) and rank 0 prices the union "
                            "(ara_pml_tvar_tail)") if world > 1 else "1 GPU"}


def compact(eng, args):
    """Prepare the resident YET for repeated pricing (ara_compact_yet:
    reordered, difference-coded ids, same results); returns the milliseconds
    it took."""
    if args.no_compact:
        return None
    t = time.perf_counter()
    eng.compact_yet()
    return (time.perf_counter() - t) * 1e3


def yet_layout(compact_ms):
    return ("stored order, 6 packed ids per 16 bytes" if compact_ms is None else
            "ara_compact_yet: 8 difference-coded ids per 16 bytes, each group of 8 ascending (prepared once "
            "before timing, %.1f ms)" % compact_ms)


# ------------------------------------------------------------ distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), ws, int(os.environ.get("LOCAL_RANK", "0"))


def shard_seed(seed: int, rank: int) -> int:
    """Each rank prices its own independent block of trials."""
    return S.sub_seed(seed, "rank", rank) if rank else seed


def tail_size(n_per_rank: int, world: int, return_periods) -> int:
    """Largest losses each trial shard sends for the portfolio-wide PML/TVaR:
    floor(N_total / RP_min) (all of its own when that is more), since the
    k largest of the whole YLT lie among every shard's k largest."""
    n_total = n_per_rank * world
    return max(1, min(n_per_rank, int(math.floor(n_total / min(return_periods)))))


def merge_shard_tails(parts):
    """The union of the ranks' tails (rank order), the input of
    ara_pml_tvar_tail."""
    return np.concatenate([np.asarray(p, dtype=np.float64) for p in parts])


def shard_step(eng, handles, layer, ylt_out, k_tail, tail_out, gather_out, n_per_rank, rank, world, rps,
               all_gather):
    """One step of a trial shard under torchrun: fold the layer, price this
    rank's trials, send its k_tail largest losses (ara_ylt_tail) through
    all_gather(gather_out, tail_out), and on rank 0 price the union as the
    whole YLT of n_per_rank * world trials (ara_pml_tvar_tail).  Returns
    (PML, TVaR) on rank 0, None elsewhere."""
    L = eng.define_layer(handles, layer.occ_ret, layer.occ_lim, layer.agg_ret, layer.agg_lim)
    eng.layer_ylt(L, out=ylt_out)
    eng.ylt_tail(ylt_out, k_tail, out=tail_out)
    all_gather(gather_out, tail_out)
    res = eng.pml_tvar_tail(gather_out, n_per_rank * world, rps) if rank == 0 else None
    eng.release_layer(L)
    return res


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []            # (monotonic time, csv line)
        self.window = (0.0, float("inf"))

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def wait_first_sample(self, timeout_s: float = 5.0):
        t0 = time.monotonic()
        while self.proc and not self.lines and time.monotonic() - t0 < timeout_s:
            time.sleep(0.05)

    def mark(self, start: float, end: float):
        self.window = (start, end)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lo, hi = self.window
        inside = [x for x in self.lines if lo <= x[0] <= hi]
        nearest = False
        if not inside and self.lines and lo > 0.0:
            # a timed region shorter than the 200 ms sampling period: take the
            # samples read within 0.3 s after it (they cover its last moments)
            inside = [x for x in self.lines if lo <= x[0] <= hi + 0.3]
            nearest = bool(inside)
        for ts, ln in inside:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
               "samples": len(sm)}
        if nearest:
            out["note"] = "timed region shorter than the sampling period; samples from just after it"
        return out


# -------------------------------------------------------------- roofline
def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def kernel_source_digest(kernel_file: str = "ylt.cu") -> str:
    import hashlib
    h = hashlib.sha256()
    for f in (kernel_file, "ara_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1412_4556_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic_per_launch(occurrences: int, profile: str = "ylt_fp64_kernel_paper_scale.md",
                           kernel_file: str = "ylt.cu"):
    """DRAM bytes per launch from a committed ncu summary, scaled to this
    launch by occurrences; None when the kernel changed since the capture."""
    p = os.path.join(ROOT, "profiles", profile)
    try:
        text = open(p).read()
    except OSError:
        return None
    m = re.search(r"kernel_digest:\s*([0-9a-f]+)", text)
    b = re.search(r"dram_bytes_per_occurrence:\s*([0-9.eE+-]+)", text)
    if not m or not b or m.group(1) != kernel_source_digest(kernel_file):
        return None
    return float(b.group(1)) * occurrences


def measure_ceilings(device: int) -> dict:
    """Rates the YLT kernel's inner loop is built from, measured on this GPU
    (ara_probe_*): random reads of one row from an L2-resident table (16-byte
    rows from a 32 MB table: one FP64 layer; 32-byte rows from a 64 MB table:
    a pass over two FP64 or four FP32-table layers), random shared-memory
    lookups (the zero-skip bitmap test) and binary64 adds."""
    from paper_1412_4556_b300 import _native as nat
    mb = 1 << 20
    r16, _ = nat.ara_probe_gather(device, 32 * mb, 16, 1, 1024, 1)
    r32, _ = nat.ara_probe_gather(device, 64 * mb, 32, 1, 1024, 1)
    return {"gather16_rows_per_s": r16, "gather32_rows_per_s": r32,
            "smem_lookups_per_s": nat.ara_probe_smem_lookup(device),
            "fp64_adds_per_s": nat.ara_probe_fp64_add(device),
            "how": "ara_probe_gather (1024-thread CTAs, one per SM, 4 rows in flight per lane, evict-last), "
                   "ara_probe_smem_lookup, ara_probe_fp64_add: best of 5 launches"}


def l1tex_roofline(gathers: float, lookups: float, kernel_ms: float, rows_per_s: float, ceil: dict) -> dict:
    """The kernel against its L1TEX co-bound: each occurrence takes one random
    shared-memory lookup and each nonzero one a random L2 row read; both go
    through the SM's L1TEX pipe, so their measured times add up to a floor."""
    t_g = gathers / rows_per_s
    t_l = lookups / ceil["smem_lookups_per_s"]
    floor_ms = (t_g + t_l) * 1e3
    return {"bound": "l1tex", "unit": "ms", "kernel_ms": kernel_ms, "floor_ms": floor_ms,
            "frac": floor_ms / kernel_ms,
            "gathers_per_launch": gathers, "lookups_per_launch": lookups,
            "achieved_gathers_per_s": gathers / (kernel_ms / 1e3), "peak_gathers_per_s": rows_per_s,
            "achieved_lookups_per_s": lookups / (kernel_ms / 1e3), "peak_lookups_per_s": ceil["smem_lookups_per_s"],
            "note": "floor = algorithmic gathers (occurrences whose event has a nonzero table value) / measured "
                    "random L2 row rate + occurrences / measured random shared-memory lookup rate; the two share "
                    "the L1TEX pipe"}


def event_counts(ids: np.ndarray, catalog: int, threads: int = 16) -> np.ndarray:
    """Occurrences of every catalog event (threaded bincount)."""
    n = ids.size
    k = max(1, threads)
    parts = [(i * n // k, (i + 1) * n // k) for i in range(k)]
    with concurrent.futures.ThreadPoolExecutor(k) as ex:
        cs = list(ex.map(lambda p: np.bincount(ids[p[0]:p[1]], minlength=catalog), parts))
    return np.sum(cs, axis=0)


# ------------------------------------------------------------ CPU oracle
def sample_yet(yet, sel):
    """A YET of the trials sel (ascending indices) of yet, in CSR form."""
    lens = yet.offsets[sel + 1] - yet.offsets[sel]
    off = np.zeros(sel.size + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    src = np.arange(off[-1], dtype=np.int64) + np.repeat(yet.offsets[sel] - off[:-1], lens)
    return S.YET(yet.catalog_size, off, yet.ids[src], None)


def _time_oracle(w, sel, threads):
    """Seconds of one oracle call (literal Algorithm 1) on the trials sel and
    their occurrence count.  A sample of a tenth of the trials or less is
    priced as a YET of its own (built before the clock starts), so the
    oracle's per-call pass over its input covers the sample, not the whole
    YET; a larger one goes through the oracle's trial selection, and all the
    trials go through no selection at all."""
    import oracle
    layer = w.layers[0]
    occ = int((w.yet.offsets[sel + 1] - w.yet.offsets[sel]).sum())
    if sel.size * 10 <= w.yet.n_trials:
        y = sample_yet(w.yet, sel)
        t0 = time.perf_counter()
        oracle.layer_ylt(y, w.pool, layer, mode="literal", threads=threads)
    elif sel.size == w.yet.n_trials:
        t0 = time.perf_counter()
        oracle.layer_ylt(w.yet, w.pool, layer, mode="literal", threads=threads)
    else:
        t0 = time.perf_counter()
        oracle.layer_ylt(w.yet, w.pool, layer, trials=sel, mode="literal", threads=threads)
    return time.perf_counter() - t0, occ


def oracle_cost_model(w, threads, rng):
    """(fixed seconds per call, seconds per trial) of the oracle on this host,
    from two probes of 2,048 and 16,384 trials."""
    n = w.yet.n_trials
    sizes = [min(n, 2048), min(n, 16384)]
    times = [_time_oracle(w, np.sort(rng.choice(n, m, replace=False)), threads)[0] for m in sizes]
    if sizes[1] > sizes[0]:
        per_trial = max((times[1] - times[0]) / (sizes[1] - sizes[0]), 1e-8)
        fixed = max(times[0] - sizes[0] * per_trial, 0.0)
    else:
        per_trial, fixed = max(times[1] / max(sizes[1], 1), 1e-8), 0.0
    return fixed, per_trial


def oracle_sample(w, budget_s: float = 12.0, threads=None, model=None, rng=None):
    """Time the FP64 oracle (literal Algorithm 1) on a bounded trial sample
    sized to about budget_s seconds (all the trials when they fit)."""
    threads = threads or os.cpu_count() or 1
    rng = rng or np.random.default_rng(5)
    n = w.yet.n_trials
    fixed, per_trial = model or oracle_cost_model(w, threads, rng)
    k = int(min(n, max(256, (budget_s - fixed) / per_trial)))
    sel = np.arange(n) if k == n else np.sort(rng.choice(n, k, replace=False))
    dt, occ = _time_oracle(w, sel, threads)
    return {"value": occ / dt, "unit": UNIT, "cores": threads, "kind": "oracle", "seconds": dt,
            "trials": k, "occurrences": occ,
            "sample": f"{k} of {n} trials ({occ} trial-events), literal Algorithm 1 "
                      f"(16 direct-access-table lookups per event), {dt:.2f} s including the "
                      f"table build"}


def oracle_parity(w, g, pml_g, tvar_g) -> dict:
    """Every trial loss g (and PML/TVaR from g) against the FP64 oracle
    (memoised Algorithm 1 on all host cores, same bits as the literal loop)."""
    import oracle
    t = time.perf_counter()
    o, pre = oracle.layer_ylt(w.yet, w.pool, w.layers[0], mode="memo")
    pml_o, tvar_o = oracle.pml_tvar(o, w.return_periods)
    rep = oracle.compare_fp64(g, o, pre)
    rep["pml_tvar"] = oracle.compare_pml_tvar(pml_g, tvar_g, pml_o, tvar_o, w.return_periods, g.size,
                                              rep["max_abs_err"])
    rep["gate"] = "|g - o| / max(|o|, S_o) <= 1e-12 per trial (S_o: the oracle's pre-aggregate sum)"
    rep["plain_form"] = "|g - o| / |o| <= 1e-12 (reported, not gated)"
    rep["oracle_seconds"] = time.perf_counter() - t
    return rep


# --------------------------------------------------------------- engine arm
def run_engine(args):
    import torch
    from paper_1412_4556_b300 import ARA_TIMING_FOLD, ARA_TIMING_PML, ARA_TIMING_YLT, Engine

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    t_gen = time.perf_counter()
    # ranks share the host's cores while they draw their shards
    w = S.paper_scale(seed=shard_seed(S.DEFAULT_SEED, rank), n_trials=args.trials,
                      with_timestamps=not args.no_timestamps,
                      threads=max(1, (os.cpu_count() or 1) // world))
    gen_s = time.perf_counter() - t_gen
    layer = w.layers[0]
    rps = w.return_periods
    M, N, C = w.yet.n_occurrences, w.yet.n_trials, w.yet.catalog_size

    stream = torch.cuda.Stream(device=dev)
    eng = Engine(local, stream=stream)
    eng.load_yet_from(w.yet)
    compact_ms = compact(eng, args)
    first = eng.load_pool(w.pool)
    handles = [first + j for j in layer.elts]
    ylt_dev = torch.empty(N, dtype=torch.float64, device=dev)
    # PML then TVaR of the latest step, written in stream order (one GPU)
    res_dev = torch.empty(2 * len(rps), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    ceil = measure_ceilings(local)

    gather_buf = tail_dev = None
    k_tail = tail_size(N, world, rps)
    if world > 1:
        tail_dev = torch.empty(k_tail, dtype=torch.float64, device=dev)
        gather_buf = torch.empty(k_tail * world, dtype=torch.float64, device=dev)

    def all_gather(out, inp):
        import torch.distributed as dist
        with torch.cuda.stream(stream):
            dist.all_gather_into_tensor(out, inp)

    def step():
        if world > 1:
            # each shard sends its k_tail largest losses (not its whole YLT)
            return shard_step(eng, handles, layer, ylt_dev, k_tail, tail_dev, gather_buf, N, rank, world, rps,
                              all_gather)
        L = eng.define_layer(handles, layer.occ_ret, layer.occ_lim, layer.agg_ret, layer.agg_lim)
        eng.layer_ylt(L, out=ylt_dev)
        # queued without a host wait, so the next step's launches overlap this
        # one's kernels; the results stay in HBM (the e2e line reads them back
        # every step)
        eng.pml_tvar_async(ylt_dev, rps, res_dev)
        eng.release_layer(L)
        return None

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        clocks.wait_first_sample()
        for _ in range(args.warmup):
            step()
        eng.set_kernel_timing(True)
        barrier()
        t_start = time.monotonic()
        ev0.record(stream)
        for _ in range(args.steps):
            res = step()
        ev1.record(stream)
        barrier()
        t_end = time.monotonic()
        time.sleep(0.3)
        clocks.mark(t_start, t_end)
    ms_total = ev0.elapsed_time(ev1)
    if world == 1:
        r = res_dev.cpu().numpy()
        res = (r[:len(rps)], r[len(rps):])
    n_ylt, ylt_ms = eng.kernel_timing(ARA_TIMING_YLT)
    n_fold, fold_ms = eng.kernel_timing(ARA_TIMING_FOLD)
    n_pml, pml_ms = eng.kernel_timing(ARA_TIMING_PML)
    eng.set_kernel_timing(False)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms_total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    value = M * world / (ms_step / 1e3)

    # Roofline of the dominant kernel (the YLT gather/sum).
    ylt_avg_ms = ylt_ms / max(n_ylt, 1)
    alg_bytes = 4 * M + 8 * (N + 1) + 8 * N + 8 * C
    achieved = alg_bytes / (ylt_avg_ms / 1e3) / 1e9
    peak, peak_kind = measured_hbm_peak()
    traffic = ncu_traffic_per_launch(M)

    # The last step's YLT, for the parity check and the L1TEX co-bound (its
    # table's nonzero events and their occurrences).
    g = ylt_dev.cpu().numpy()
    L = eng.define_layer(handles, layer.occ_ret, layer.occ_lim, layer.agg_ret, layer.agg_lim)
    nonzero = eng.event_table(L) != 0.0
    eng.release_layer(L)
    eng.close()
    del eng
    torch.cuda.empty_cache()
    gathers = float(event_counts(w.yet.ids, C)[nonzero].sum())
    l1tex = l1tex_roofline(gathers, float(M), ylt_avg_ms, ceil["gather16_rows_per_s"], ceil)

    # End to end through the C ABI with host buffers (pinned), per step.
    e2e = run_e2e(args, w, local=local) if rank == 0 else None

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    parity = oracle_parity(w, g, res[0], res[1]) if world == 1 and not args.no_parity else None
    nested = {}
    if world == 1 and not args.no_nested:
        # a failure in one of the other configs is reported in its key and
        # does not take the headline line down with it
        def guarded(fn):
            try:
                return fn()
            except Exception as exc:  # noqa: BLE001
                return {"error": f"{type(exc).__name__}: {exc}"}
        bw = S.batched(yet=w.yet)
        nested["batched"] = guarded(lambda: batched_result(args, bw, mixed=False, ceil=ceil))
        nested["mixed"] = guarded(lambda: batched_result(args, bw, mixed=True, ceil=ceil))
        del bw
        nested["service"] = guarded(lambda: service_result(args, S.batched(n_layers=1, yet=w.yet), nested=True))
    cpu = oracle_sample(w, budget_s=args.cpu_budget) if world == 1 and not args.no_cpu else None
    if cpu:
        for key in ("seconds", "trials", "occurrences"):
            cpu.pop(key, None)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": value / PAPER_1GPU_TRIAL_EVENTS_PER_S,
        "vs_baseline_basis": "paper's best single GPU run (Tesla M2050, 19.93 s for 1e9 trial-events, "
                             "Section IV-C); other hardware, context only",
        "dtype": "f64", "data": "synthetic (seeded; stands in for the paper's proprietary industry data)",
        "config": paper_config(N, M, C, len(layer.elts), world, k_tail),
        "step": ("ara_define_layer (ELT fold) + ara_layer_ylt + ara_pml_tvar_async (PML/TVaR queued, results "
                 "kept in HBM; read back after the timed steps)") if world == 1 else
                "ara_define_layer (ELT fold) + ara_layer_ylt + ara_ylt_tail + all-gather + ara_pml_tvar_tail",
        "yet_layout": yet_layout(compact_ms),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "ylt_fp64_kernel", "kernel_ms": ylt_avg_ms,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "frac_of_nominal_8000_gbs": achieved / 8000.0,
                     "l1tex": l1tex},
        "ceilings": ceil,
        "breakdown_ms_per_step": {"fold": fold_ms / max(args.steps, 1), "ylt": ylt_ms / max(args.steps, 1),
                                  "pml_tvar": pml_ms / max(args.steps, 1)},
        "pml": list(map(float, res[0])), "tvar": list(map(float, res[1])),
        "parity": parity,
        "clocks": clocks.summary(),
        "e2e": e2e,
        # fold, YLT, selection (init + 8 passes + sum) and, on one GPU, the
        # copy of its results; with shards instead the tail (selection + 3
        # kernels) and the selection over the union
        "gpu_launches": args.steps * (1 + 1 + 10 + (13 if world > 1 else 1)),
        "cpu_baseline": cpu,
        "host_generation_s": gen_s,
    }
    line.update(nested)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_e2e(args, w, local: int):
    """Same step through the public C ABI with pinned host buffers: H2D of the
    YET (ids and, when the workload has them, time-stamps, which the load
    checks on the device) and the ELTs, the layer definition, the YLT and
    PML/TVaR back to host.  Also timed with the ids alone."""
    import torch
    from paper_1412_4556_b300 import Engine

    layer = w.layers[0]
    rps = w.return_periods
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    h_off, h_ids = pin(w.yet.offsets), pin(w.yet.ids)
    h_ts = pin(w.yet.ts) if w.yet.ts is not None else None
    p = w.pool
    h_eoff, h_eids, h_eloss = pin(p.offsets), pin(p.ids), pin(p.losses)
    h_ded, h_lim = pin(p.deductibles), pin(p.limits)
    h_ylt = torch.empty(w.yet.n_trials, dtype=torch.float64).pin_memory()
    eng = Engine(local)
    N, M = w.yet.n_trials, w.yet.n_occurrences

    def step(ts):
        eng.load_yet(w.yet.catalog_size, h_off.numpy(), h_ids.numpy(), None if ts is None else ts.numpy())
        first = eng.load_elts(h_eoff.numpy(), h_eids.numpy(), h_eloss.numpy(), h_ded.numpy(),
                              h_lim.numpy())
        L = eng.define_layer([first + j for j in layer.elts], layer.occ_ret, layer.occ_lim,
                             layer.agg_ret, layer.agg_lim)
        out = eng.layer_ylt(L, out=h_ylt.numpy())
        res = eng.pml_tvar(out, rps)
        eng.release_layer(L)
        return res

    def timed(ts):
        for _ in range(max(1, min(args.warmup, 2))):
            step(ts)
        torch.cuda.synchronize()
        k = max(1, min(args.steps, args.e2e_steps))
        t0 = time.perf_counter()
        for _ in range(k):
            step(ts)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / k, k

    dt, k = timed(h_ts)
    dt_ids, _ = timed(None) if h_ts is not None else (dt, k)
    eng.close()
    h2d_ids = 8 * (N + 1) + 4 * M + 8 * (p.n_elts + 1) + 12 * p.ids.size + 16 * p.n_elts
    h2d = h2d_ids + (4 * M if h_ts is not None else 0)
    d2h = 8 * N + 16 * len(rps)
    return {"value": M / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": dt * 1e3, "steps": k,
            "ids_only": {"value": M / dt_ids, "ms_per_step": dt_ids * 1e3, "h2d_bytes_per_step": int(h2d_ids)},
            "note": "pinned host buffers through ara_load_yet (ids and float32 time-stamps, both checked on the "
                    "device)/ara_load_elts/ara_define_layer/ara_layer_ylt(host out)/ara_pml_tvar; ids_only: the "
                    "same without the time-stamps"}


# ------------------------------------------------------- batched layers
BATCHED = ("batched layers, FP64: the paper-scale YET (1,000,000 trials x Poisson(1000), catalog "
           "2,000,000) shared by 64 layers of U{1..32} ELTs from a pool of 256 ELTs of U{10k..50k} "
           "events; per-layer OccR/OccL/AggR/AggL log-uniform over [1e4,1e6]/[1e6,1e8]/[1e5,1e7]/"
           "[1e7,1e9]; RP 100/250/500")


def batched_roofline(M, N, C, layers, table_bytes_per_event, ylt_ms, passes):
    """Roofline of the YLT passes of a many-layer step against the
    algorithmic minimum of the step: the YET read once (4 B per occurrence)
    plus each layer's table (table_bytes_per_event per catalog event), YLT
    (8 B per trial) and trial offsets."""
    alg = 4 * M + layers * (table_bytes_per_event * C + 8 * N) + 8 * (N + 1)
    achieved = alg / (ylt_ms / 1e3) / 1e9
    peak, peak_kind = measured_hbm_peak()
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "kernel": "ylt_fp64_kernel (%d grouped passes)" % passes, "kernel_ms": ylt_ms,
            "algorithmic_bytes_per_step": alg, "peak_kind": peak_kind,
            "frac_of_nominal_8000_gbs": achieved / 8000.0,
            "note": "the algorithmic minimum reads the YET once for all layers; the passes re-read it once "
                    "per pass and are bound by their L1TEX line requests (see l1tex), not by HBM"}


def batched_result(args, w, mixed: bool, ceil=None, oracle_trials: int = 2048) -> dict:
    """Config-2 step (config 3 with mixed=True: FP32 tables): one replay of a
    plan (a CUDA graph of the 64 ELT folds, the grouped YLT passes and the
    batched PML/TVaR).  Also times the same work as calls (ara_layers_ylt)
    and as the plain per-layer path (ara_layer_ylt per layer), and checks a
    sample of trials of every layer against the FP64 oracle."""
    import torch
    import oracle
    from paper_1412_4556_b300 import ARA_FP32_TABLE, ARA_FP64, ARA_TIMING_YLT, Engine, Plan

    prec = ARA_FP32_TABLE if mixed else ARA_FP64
    M, N, C = w.yet.n_occurrences, w.yet.n_trials, w.yet.catalog_size
    G = len(w.layers)
    stream = torch.cuda.Stream()
    eng = Engine(0, stream=stream)
    eng.load_yet_from(w.yet)
    compact_ms = compact(eng, args)
    first = eng.load_pool(w.pool)
    handles = [[first + j for j in L.elts] for L in w.layers]
    out = torch.empty((G, N), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    ceil = ceil or measure_ceilings(0)

    def define(p=prec):
        return [eng.define_layer(h, L.occ_ret, L.occ_lim, L.agg_ret, L.agg_lim, precision=p)
                for h, L in zip(handles, w.layers)]

    def step_batched():
        hs = define()
        eng.layers_ylt(hs, out=out)
        res = eng.pml_tvar_batch(out, w.return_periods)
        for h in hs:
            eng.release_layer(h)
        return res

    def step_plain(p=prec):
        hs = define(p)
        for i, h in enumerate(hs):
            eng.layer_ylt(h, out=out[i])
        res = eng.pml_tvar_batch(out, w.return_periods)
        for h in hs:
            eng.release_layer(h)
        return res

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        eng.set_kernel_timing(True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        n_k, k_ms = eng.kernel_timing(ARA_TIMING_YLT)
        eng.set_kernel_timing(False)
        return e0.elapsed_time(e1) / steps, k_ms / steps

    plan_layers = define()
    plan = Plan(eng, plan_layers, w.return_periods, autotune=not args.no_autotune)

    def step_plan():
        # one graph launch: 64 ELT folds, the grouped YLT passes, PML/TVaR
        return plan.run(ylt_out=out, stream=stream)

    steps = max(3, min(args.steps, 10))
    with ClockSampler(0) as clocks:
        clocks.wait_first_sample()
        t0 = time.monotonic()
        ms_g, _ = timed(step_plan, steps)
        t1 = time.monotonic()
        time.sleep(0.3)
        clocks.mark(t0, t1)
    y_plan = out.cpu().numpy()
    pml_plan, tvar_plan = eng.pml_tvar_batch(out, w.return_periods)
    ms_b, ylt_b = timed(step_batched, steps)
    ms_p, ylt_p = timed(step_plain, steps)
    ms_p64 = timed(lambda: step_plain(ARA_FP64), steps)[0] if mixed else ms_p
    passes = plan.passes()
    plan_launches = plan.kernel_launches()
    # nonzero events of every layer (for the passes' L1TEX floor)
    nz = np.stack([eng.event_table(h) != 0.0 for h in plan_layers])
    plan.close()
    for h in plan_layers:
        eng.release_layer(h)
    eng.close()
    value = G * M / (ms_g / 1e3)

    cnt = event_counts(w.yet.ids, C)
    gathers = 0.0
    for eb, g, _lpt, _u, _pf, _th, pos in passes:
        gathers += float(cnt[np.logical_or.reduce(nz[list(pos)])].sum())
    rows = ceil["gather32_rows_per_s"] if any(g > 1 for _, g, *_ in passes) else ceil["gather16_rows_per_s"]
    l1tex = l1tex_roofline(gathers, float(M) * len(passes), ylt_b, rows, ceil)
    l1tex["note"] = ("floor = for every pass, the occurrences whose event is nonzero in any of the pass's "
                     "layers / measured random 32-byte row rate (64 MB table) + its occurrences / measured "
                     "random shared-memory lookup rate")

    # a sample of trials of every layer against the FP64 oracle
    rng = np.random.default_rng(11)
    sel = np.sort(rng.choice(N, min(N, oracle_trials), replace=False))
    t = time.perf_counter()
    o, pre = oracle.layers_ylt(w.yet, w.pool, w.layers, trials=sel, mode="memo")
    o_s = time.perf_counter() - t
    worst = {}
    for i in range(G):
        rep = (oracle.compare_reduced if mixed else oracle.compare_fp64)(y_plan[i][sel], o[i], pre[i])
        for k, v in rep.items():
            if k == "trials":
                worst[k] = worst.get(k, 0) + v
            elif k.startswith("trials_over") or k == "bitwise_equal_trials":
                worst[k] = worst.get(k, 0) + v
            else:
                worst[k] = max(worst.get(k, 0.0), v)
    accuracy = {"vs": "FP64 oracle (memoised Algorithm 1)", "layers": G, "trials_per_layer": int(sel.size),
                **worst, "oracle_seconds": o_s,
                "gate": ("|g - o| <= max(1e-5 * max(|o|, S_o), 1 USD)" if mixed else
                         "|g - o| / max(|o|, S_o) <= 1e-12")}
    res = {
        "workload": ("mixed precision (FP32 tables): " if mixed else "") + BATCHED,
        "metric": "layer-trial-events/s", "value": value, "unit": "layer-trial-events/s",
        "ms_per_step": ms_g, "steps": steps, "warmup": args.warmup,
        "dtype": "f32 tables, exact trial sums" if mixed else "f64",
        "step": "ara_plan_run: one CUDA graph of the 64 layers' ELT folds (one batched launch, into each "
                "pass's interleaved table) + the grouped YLT passes + batched PML/TVaR "
                + ("(default launch shapes and group sizes: --no-autotune)" if args.no_autotune
                   else "(launch shapes and group sizes autotuned at plan creation)"),
        "yet_layout": yet_layout(compact_ms),
        "l2": "inputs larger than L2 (a 2-2.7 GB YET id stream per pass)",
        "ylt_kernels_ms_per_step": ylt_b,
        "passes": [{"entry_bytes": eb, "layers": list(pos), "lanes_per_trial": lpt, "unroll": u, "l2_prefetch": pf,
                    "threads": th} for eb, g, lpt, u, pf, th, pos in passes],
        "calls_per_step": {"ms_per_step": ms_b, "ylt_kernels_ms_per_step": ylt_b,
                           "step": "64 x ara_define_layer + ara_layers_ylt + ara_pml_tvar_batch"},
        "plain_per_layer": {"ms_per_step": ms_p, "ylt_kernels_ms_per_step": ylt_p,
                            "step": "64 x ara_define_layer + 64 x ara_layer_ylt + ara_pml_tvar_batch"},
        "speedup_vs_plain": ms_p / ms_g,
        "roofline": batched_roofline(M, N, C, G, 4 if mixed else 8, ylt_b, len(passes)),
        "accuracy": accuracy,
        "pml_tvar_sample": {"layer0_pml": pml_plan[0].tolist(), "layer0_tvar": tvar_plan[0].tolist()},
        "clocks": clocks.summary(),
        "gpu_launches_per_step": None,
    }
    res["roofline"]["l1tex"] = l1tex
    if mixed:
        res["plain_fp64_per_layer_ms_per_step"] = ms_p64
        res["speedup_vs_plain_fp64"] = ms_p64 / ms_g
    res["gpu_launches_per_step"] = plan_launches  # kernel nodes of the plan's graph
    return res


def run_batched(args):
    """The config-2 (or, with --workload mixed, config-3) line on its own."""
    w = S.batched(n_trials=args.trials)
    r = batched_result(args, w, mixed=args.workload == "mixed")
    line = {"metric": METRIC, "value": r["value"], "unit": r["unit"], "n_gpus": 1, "steps": r["steps"],
            "warmup": r["warmup"], "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": r["dtype"], "data": "synthetic (seeded)",
            "config": {"workload": r["workload"], "layers": len(w.layers), "n_trials": w.yet.n_trials,
                       "occurrences": w.yet.n_occurrences, "l2": r["l2"]},
            "gpu_launches": r["gpu_launches_per_step"] * r["steps"]}
    line.update({k: v for k, v in r.items() if k not in line and k not in ("workload", "gpu_launches_per_step")})
    print(json.dumps(line), flush=True)


SERVICE = ("ad hoc pricing service: paper-scale YET (catalog 2,000,000 events; 1,000,000 trials x "
           "Poisson(1000)) and a pool of 256 ELTs (10,000-50,000 events each) resident on the device; "
           "layer requests of 2-32 pool ELTs with batched-layer terms over a 100k/250k/1M-trial prefix, "
           "FP32 tables with exact trial sums; PML/TVaR at RP 100/250/500")


def service_result(args, w, nested: bool = False) -> dict:
    """Config-4 serving run: a seeded Poisson stream of layer-pricing requests
    played open-loop against the pricing service (continuous batching over
    slots, admission by device memory); requests/s and p50/p99 latency, then
    the same requests all at once (saturating) and, unless nested, at ten
    times the rate; 1% of the requests are checked against the oracle on
    every trial, with their PML/TVaR."""
    from paper_1412_4556_b300 import ARA_FP32_TABLE, Engine, Service
    import oracle

    rps = (100.0, 250.0, 500.0)
    n_req = args.nested_requests if nested else args.requests
    reqs = S.service_requests(n_requests=n_req, rate_per_s=args.rate)
    eng = Engine(0)
    eng.load_yet_from(w.yet)
    compact_ms = compact(eng, args)
    first = eng.load_pool(w.pool)
    sample = list(range(0, len(reqs), 100))

    def play(rate_scale, want=()):
        svc = Service(eng, rps, slots=args.slots, max_batch=args.max_batch)
        for rq in reqs[:max(args.warmup, 3)]:  # warm-up requests, not timed
            L = rq.layer
            svc.wait(svc.submit([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret, L.agg_lim,
                                rq.n_trials, precision=ARA_FP32_TABLE))
        tickets = []
        t0 = time.perf_counter()
        for i, rq in enumerate(reqs):
            if rate_scale is not None:
                delay = t0 + rq.arrival_s / rate_scale - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            L = rq.layer
            tickets.append(svc.submit([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret,
                                      L.agg_lim, rq.n_trials, precision=ARA_FP32_TABLE,
                                      want_ylt=i in want))
        res = [svc.wait(t) for t in tickets]
        st = svc.stats()
        svc.close()
        bad = [r for r in res if not r.ok]
        if bad:
            raise RuntimeError(f"{len(bad)} requests failed: {bad[0].status_name} {bad[0].message}")
        lat = np.array([r.latency for r in res]) * 1e3
        queue_ms = np.array([r.t_start - r.t_submit for r in res]) * 1e3
        run_ms = np.array([r.t_done - r.t_start for r in res]) * 1e3
        span = max(r.t_done for r in res) - min(r.t_submit for r in res)
        occ = sum(int(w.yet.offsets[rq.n_trials]) for rq in reqs)
        by_n = {}
        for n in sorted({rq.n_trials for rq in reqs}):
            ln = np.array([r.latency for r, rq in zip(res, reqs) if rq.n_trials == n]) * 1e3
            by_n[str(n)] = {"count": int(ln.size), "p50_ms": float(np.percentile(ln, 50)),
                            "p99_ms": float(np.percentile(ln, 99))}
        return res, {
            "offered_rate_per_s": None if rate_scale is None else args.rate * rate_scale,
            "latency_by_trials": by_n,
            "requests_per_s": len(res) / span, "layer_trial_events_per_s": occ / span,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            # the requests that return PML/TVaR only (not the sampled ones that also copy out their YLT)
            "p99_ms_pml_tvar_only": (float(np.percentile([x for i, x in enumerate(lat) if i not in want], 99))
                                     if want else None),
            "max_ms": float(lat.max()), "mean_batch": float(np.mean([r.batch_size for r in res])),
            "queue_p50_ms": float(np.percentile(queue_ms, 50)), "queue_p99_ms": float(np.percentile(queue_ms, 99)),
            "run_p50_ms": float(np.percentile(run_ms, 50)), "run_p99_ms": float(np.percentile(run_ms, 99)),
            "max_batch": st["max_batch_seen"], "max_in_flight": st["max_in_flight"],
            "max_slots_busy": st["max_slots_busy"], "max_device_bytes_in_flight": st["max_bytes_in_flight"],
        }

    # Device time of one request priced alone through the engine (define +
    # YLT + PML/TVaR on the device, GPU kept busy): the floor under latency.
    import torch
    stream = torch.cuda.Stream()
    eng.set_stream(stream)
    device_ms = {}
    for n in sorted({rq.n_trials for rq in reqs}):
        rq = next(r for r in reqs if r.n_trials == n)
        L = rq.layer
        out = torch.empty(n, dtype=torch.float64, device="cuda")

        def one():
            h = eng.define_layer([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret, L.agg_lim,
                                 precision=ARA_FP32_TABLE)
            eng.layer_ylt(h, n, out=out)
            eng.pml_tvar_batch(out.view(1, n), rps)
            eng.release_layer(h)
        for _ in range(5):
            one()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(20):
            one()
        torch.cuda.synchronize()
        device_ms[str(n)] = (time.perf_counter() - t) / 20 * 1e3
    eng.set_stream(None)

    with ClockSampler(0) as clocks:
        clocks.wait_first_sample()
        t0 = time.monotonic()
        res, paced = play(1.0, want=set(sample))
        t1 = time.monotonic()
        time.sleep(0.3)
        clocks.mark(t0, t1)
    _, saturating = play(None)
    fast = None if nested else play(10.0)[1]

    # 1% of the requests against the FP64 oracle (memoised Algorithm 1): every
    # trial of each sampled request (or --oracle-trials sampled trials), and
    # its PML/TVaR against the oracle's PML/TVaR of the oracle's YLT, within
    # the largest per-trial error plus rounding (both are 1-Lipschitz).
    g = np.random.default_rng(7)
    worst = {"max_err_over_bar": 0.0, "trials_over_bar": 0, "trials_over_plain_bar": 0, "max_rel_err": 0.0,
             "max_abs_err": 0.0}
    pml_tvar = {"requests_within_bound": 0, "max_pml_rel_err": 0.0, "max_tvar_rel_err": 0.0,
                "max_err_over_bound": 0.0}
    oracle_s, oracle_occ, checked = 0.0, 0, 0
    for i in sample:
        rq, r = reqs[i], res[i]
        n = rq.n_trials
        every = args.oracle_trials <= 0 or args.oracle_trials >= n
        sel = np.arange(n) if every else np.sort(g.choice(n, args.oracle_trials, replace=False))
        t = time.perf_counter()
        o, pre = oracle.layer_ylt(w.yet, w.pool, rq.layer, trials=sel, mode="memo")
        oracle_s += time.perf_counter() - t
        oracle_occ += int(np.sum(np.diff(w.yet.offsets)[sel]))
        checked += sel.size
        rep = oracle.compare_reduced(r.ylt[sel], o, pre)
        for k in worst:
            worst[k] = (worst[k] + rep[k]) if k.startswith("trials") else max(worst[k], rep[k])
        if every:
            p_o, t_o = oracle.pml_tvar(o, rps)
            pt = oracle.compare_pml_tvar(r.pml, r.tvar, p_o, t_o, rps, n, rep["max_abs_err"])
            pml_tvar["requests_within_bound"] += int(pt["within_bound"])
            pml_tvar["max_pml_rel_err"] = max(pml_tvar["max_pml_rel_err"], max(pt["pml_rel_err"]))
            pml_tvar["max_tvar_rel_err"] = max(pml_tvar["max_tvar_rel_err"], max(pt["tvar_rel_err"]))
            over = max(max(a / b if b > 0 else (0.0 if a == 0 else np.inf) for a, b in zip(pt[e], pt["bound"]))
                       for e in ("pml_abs_err", "tvar_abs_err"))
            pml_tvar["max_err_over_bound"] = max(pml_tvar["max_err_over_bound"], float(over))
    eng.close()
    import multiprocessing
    return {
        "workload": SERVICE, "requests": len(reqs), "arrival_rate_per_s": args.rate,
        "slots": args.slots, "max_batch": args.max_batch, "yet_layout": yet_layout(compact_ms),
        "requests_per_s_saturating": saturating["requests_per_s"],
        "latency_ms": {"p50": paced["p50_ms"], "p99": paced["p99_ms"], "at_rate_per_s": args.rate,
                       "p99_pml_tvar_only": paced["p99_ms_pml_tvar_only"],
                       "note": "p99 over every request; p99_pml_tvar_only leaves out the 1% sampled requests "
                               "that also copy their whole YLT to the host"},
        "alone_ms_by_trials": device_ms,
        "paced": paced, "paced_10x": fast, "saturating": saturating,
        "accuracy_1pct": {"vs": "FP64 oracle (memoised Algorithm 1)", "requests": len(sample),
                          "trials_checked": checked, **worst,
                          "pml_tvar_vs_oracle": pml_tvar,
                          "gate": "|g - o| <= max(1e-5 * max(|o|, S_o), 1 USD) per trial; PML/TVaR within "
                                  "the largest per-trial error + (k + 1) 2^-53 TVaR"},
        "cpu_baseline": {"value": oracle_occ / oracle_s, "unit": "layer-trial-events/s",
                         "cores": multiprocessing.cpu_count(), "kind": "oracle",
                         "sample": f"memoised oracle on {checked} trials of {len(sample)} requests"},
        "clocks": clocks.summary(),
    }


def run_service(args):
    """The config-4 line on its own (requests/s saturating is its value)."""
    w = S.batched(n_layers=1, n_trials=args.trials)
    r = service_result(args, w)
    line = {"metric": METRIC, "value": r["requests_per_s_saturating"], "unit": "requests/s", "n_gpus": 1,
            "steps": r["requests"], "warmup": max(args.warmup, 3),
            "ms_per_step": 1e3 / r["requests_per_s_saturating"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 tables, exact trial sums", "data": "synthetic (seeded)",
            "config": {"workload": r["workload"], "requests": r["requests"],
                       "arrival_rate_per_s": r["arrival_rate_per_s"], "slots": r["slots"],
                       "max_batch": r["max_batch"], "l2": "inputs larger than L2 (up to 4 GB of YET ids per request)"}}
    line.update({k: v for k, v in r.items() if k not in line and k != "workload"})
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ YELT arm
YELT_WORKLOAD = ("paper-scale Year Event Loss Table, FP64: the paper-scale YET and layer; step = "
                 "ara_define_layer + ara_layer_yelt (every occurrence's increment and each trial's "
                 "largest, device outputs) + ara_rpl_report (AEP/OEP return period losses, RP "
                 "100/250/500)")


def run_yelt(args):
    """Year Event Loss Table and RPL reports (per-occurrence output): each
    rank prices its own trials (weak scaling, no exchange)."""
    import torch
    from paper_1412_4556_b300 import ARA_TIMING_YELT, Engine

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = f"cuda:{local}"
    torch.cuda.set_device(dev)
    w = S.paper_scale(seed=shard_seed(S.DEFAULT_SEED, rank), n_trials=args.trials)
    layer = w.layers[0]
    rps = w.return_periods
    M, N, C = w.yet.n_occurrences, w.yet.n_trials, w.yet.catalog_size
    stream = torch.cuda.Stream(device=dev)
    eng = Engine(local, stream=stream)
    eng.load_yet_from(w.yet)
    first = eng.load_pool(w.pool)
    handles = [first + j for j in layer.elts]
    yelt = torch.empty(M, dtype=torch.float64, device=dev)
    occ_max = torch.empty(N, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()

    def define():
        return eng.define_layer(handles, layer.occ_ret, layer.occ_lim, layer.agg_ret, layer.agg_lim)

    def step():
        L = define()
        eng.layer_yelt(L, out=yelt, occ_max=occ_max, stream=stream)
        rep = eng.rpl_report(L, rps)
        eng.release_layer(L)
        return rep

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        clocks.wait_first_sample()
        for _ in range(args.warmup):
            step()
        barrier()
        t_start = time.monotonic()
        ev0.record(stream)
        for _ in range(args.steps):
            rep = step()
        ev1.record(stream)
        barrier()
        t_end = time.monotonic()
        # the YELT kernel alone (with its per-occurrence output), for the roofline
        L = define()
        eng.layer_yelt(L, out=yelt, occ_max=occ_max, stream=stream)
        eng.set_kernel_timing(True)
        for _ in range(args.steps):
            eng.layer_yelt(L, out=yelt, occ_max=occ_max, stream=stream)
        n_k, k_ms = eng.kernel_timing(ARA_TIMING_YELT)
        eng.set_kernel_timing(True)
        for _ in range(args.steps):
            eng.rpl_report(L, rps)
        n_r, r_ms = eng.kernel_timing(ARA_TIMING_YELT)
        eng.set_kernel_timing(False)
        eng.release_layer(L)
        torch.cuda.synchronize()
        time.sleep(0.3)
        clocks.mark(t_start, t_end)
    ms_total = ev0.elapsed_time(ev1)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms_total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    kern_ms = k_ms / max(n_k, 1)
    # ids read, increments written, per-trial maxima written, chunk and raw
    # offsets read, one FP64 table read
    alg_bytes = 4 * M + 8 * M + 8 * N + 16 * (N + 1) + 8 * C
    peak, peak_kind = measured_hbm_peak()
    eng.close()
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    achieved = alg_bytes / (kern_ms / 1e3) / 1e9
    line = {
        "metric": "YELT trial-events/s (per-occurrence increments + AEP/OEP report)",
        "value": M * world / (ms_step / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
        "config": {"workload": YELT_WORKLOAD, "n_trials_per_gpu": N, "occurrences_per_gpu": M,
                   "yelt_bytes_per_step": 8 * M,
                   "l2": "inputs larger than L2: the 2.67 GB id stream and the 8 GB YELT pass through HBM "
                         "every step"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": ncu_traffic_per_launch(M, "yelt_kernel_paper_scale.md", "yelt.cu"),
                     "kernel": "yelt_kernel",
                     "kernel_ms": kern_ms, "algorithmic_bytes_per_launch": alg_bytes,
                     "peak_kind": peak_kind, "frac_of_nominal_8000_gbs": achieved / 8000.0},
        "breakdown_ms": {"yelt_kernel_with_output": kern_ms,
                         "rpl_report_yelt_kernel": r_ms / max(n_r, 1)},
        "rpl": {k: v.tolist() for k, v in rep.items()},
        "clocks": clocks.summary(),
        # fold; binary64 fold, interleave, YELT kernel; report pass and the
        # AEP/OEP selection (init + 8 passes + sum)
        "gpu_launches": args.steps * (1 + 3 + 1 + 10),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------ oracle arm
def reference_step_trials(n: int, fixed: float, per_trial: float, steps: int, warmup: int,
                          budget_s: float) -> int:
    """Trials each reference step prices: all n when (steps + warmup) steps of
    them fit in budget_s seconds, else the largest sample that does."""
    per_step = budget_s / max(steps + warmup, 1)
    if fixed + n * per_trial <= per_step:
        return n
    return int(max(256, min(n, (per_step - fixed) / per_trial)))


def run_reference(args):
    """The oracle (literal Algorithm 1 on all host cores) timed on the engine
    arm's workload and config: each step prices the whole YET when the run
    fits the budget, else the same fixed trial sample every step; value and
    ms_per_step are the priced trials' own, measured, not extrapolated."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = S.paper_scale(n_trials=args.trials)
    N, C = w.yet.n_trials, w.yet.catalog_size
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(5)
    fixed, per_trial = oracle_cost_model(w, threads, rng)
    k = reference_step_trials(N, fixed, per_trial, args.steps, args.warmup, args.reference_budget)
    sel = np.arange(N) if k == N else np.sort(rng.choice(N, k, replace=False))
    for _ in range(args.warmup):
        _time_oracle(w, sel, threads)
    secs, occ = [], 0
    t_all = time.perf_counter()
    for _ in range(args.steps):
        dt, occ = _time_oracle(w, sel, threads)
        secs.append(dt)
    wall = time.perf_counter() - t_all
    ms_step = 1e3 * sum(secs) / len(secs)
    value = occ / (ms_step / 1e3)
    sample = (f"{k} of {N} trials ({occ} trial-events) per step, literal Algorithm 1 (16 direct-access-table "
              f"lookups per event), {threads} threads")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded; stands in for the paper's proprietary "
                                                      "industry data)", "impl": "reference",
        "config": paper_config(N, w.yet.n_occurrences, C, len(w.layers[0].elts), world,
                               tail_size(N, world, w.return_periods)),
        "step": "oracle: literal Algorithm 1 over the step's trials (FP64, threaded over trials)",
        "trials_per_step": k,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["engine", "reference"], default="engine")
    ap.add_argument("--workload", choices=["paper", "batched", "mixed", "service", "yelt"], default="paper",
                    help="paper: the single-layer paper-scale step with the other configs nested (default); "
                         "batched: 64 layers; mixed: 64 FP32-table layers; service: the pricing-request "
                         "stream; yelt: the Year Event Loss Table and RPL report")
    ap.add_argument("--requests", type=int, default=2000, help="service: requests in the stream")
    ap.add_argument("--nested-requests", type=int, default=500,
                    help="requests of the service run nested in the default line")
    ap.add_argument("--rate", type=float, default=50.0, help="service: Poisson arrival rate per s")
    ap.add_argument("--slots", type=int, default=4, help="service: batches in flight")
    ap.add_argument("--max-batch", type=int, default=16, help="service: requests per batch")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched/mixed: plan without timing launch shapes and group sizes (for profilers, "
                         "whose overhead would skew the timing)")
    ap.add_argument("--oracle-trials", type=int, default=0,
                    help="service: trials checked per sampled request (0: every trial)")
    ap.add_argument("--trials", type=int, default=1_000_000, help="trials per GPU")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work (cpu_baseline)")
    ap.add_argument("--reference-budget", type=float, default=240.0,
                    help="seconds the --impl reference run may take over all its steps")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-parity", action="store_true", help="skip the full oracle comparison")
    ap.add_argument("--no-nested", action="store_true",
                    help="default line without the nested batched/mixed/service runs")
    ap.add_argument("--no-timestamps", action="store_true", help="YET without time-stamps")
    ap.add_argument("--no-compact", action="store_true",
                    help="price from the stored-order id layout (skip ara_compact_yet)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "engine":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in ("batched", "mixed"):
        run_batched(args)
    elif args.workload == "service":
        run_service(args)
    elif args.workload == "yelt":
        run_yelt(args)
    else:
        run_engine(args)


if __name__ == "__main__":
    main()
