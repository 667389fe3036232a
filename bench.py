#!/usr/bin/env python3
"""Benchmark of the Year Loss Table hot path (Varghese & Barker, arXiv 1412.4556).

One step = one pass of the whole path over the paper-scale workload
(catalog 2,000,000 events; one layer over 16 ELTs of 20,000 events;
1,000,000 trials of Poisson(1000) events, about 1e9 occurrences):

    ara_define_layer  (per-layer ELT fold pre-pass on the device)
    ara_layer_ylt     (per-trial gather + exact sum + aggregate terms)
    ara_pml_tvar      (PML and TVaR at return periods 100 / 250 / 500)

The YET and the ELT pool are resident in HBM when the timed region starts
(the paper's pre-processing stage); the 4 GB id stream is larger than L2, so
every step reads it from HBM.  ``e2e`` repeats the step through the same C
ABI with host buffers: the YET, the ELTs and the layer go host->device and
the YLT, PML and TVaR come back, inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl engine|reference]

Under torchrun (N > 1) every rank prices its own shard of 1,000,000 trials
(weak scaling); the shards' YLTs are all-gathered for the portfolio-wide
PML/TVaR.  ``--impl reference`` times the FP64 CPU oracle (the only reference
this path has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
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
            "Poisson(1000) events; OccR 1e5, OccL 2e7, AggR 5e5, AggL 1e8; RP 100/250/500")


def compact(eng, args):
    """Prepare the resident YET for repeated pricing (ara_compact_yet:
    reordered, difference-coded ids, same results); returns the milliseconds
    it took."""
    if args.no_compact:
        return None
    t = time.perf_counter()
    eng.compact_yet()
    return (time.perf_counter() - t) * 1e3


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
    YET; a larger one goes through the oracle's trial selection."""
    import oracle
    layer = w.layers[0]
    occ = int((w.yet.offsets[sel + 1] - w.yet.offsets[sel]).sum())
    if sel.size * 10 <= w.yet.n_trials:
        y = sample_yet(w.yet, sel)
        t0 = time.perf_counter()
        oracle.layer_ylt(y, w.pool, layer, mode="literal", threads=threads)
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
    sized to about budget_s seconds."""
    threads = threads or os.cpu_count() or 1
    rng = rng or np.random.default_rng(5)
    n = w.yet.n_trials
    fixed, per_trial = model or oracle_cost_model(w, threads, rng)
    k = int(min(n, max(256, (budget_s - fixed) / per_trial)))
    sel = np.sort(rng.choice(n, k, replace=False))
    dt, occ = _time_oracle(w, sel, threads)
    return {"value": occ / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{k} of {n} trials ({occ} trial-events), literal Algorithm 1 "
                      f"(16 direct-access-table lookups per event), {dt:.2f} s including the "
                      f"table build"}


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

    w = S.paper_scale(seed=shard_seed(S.DEFAULT_SEED, rank), n_trials=args.trials)
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

    gather_buf = tail_dev = None
    k_tail = tail_size(N, world, rps)
    if world > 1:
        tail_dev = torch.empty(k_tail, dtype=torch.float64, device=dev)
        gather_buf = torch.empty(k_tail * world, dtype=torch.float64, device=dev)

    def step():
        L = eng.define_layer(handles, layer.occ_ret, layer.occ_lim, layer.agg_ret, layer.agg_lim)
        eng.layer_ylt(L, out=ylt_dev)
        if world > 1:
            # each shard sends its k_tail largest losses (not its whole YLT)
            import torch.distributed as dist
            eng.ylt_tail(ylt_dev, k_tail, out=tail_dev)
            with torch.cuda.stream(stream):
                dist.all_gather_into_tensor(gather_buf, tail_dev)
            res = eng.pml_tvar_tail(gather_buf, N * world, rps) if rank == 0 else None
        else:
            # queued without a host wait, so the next step's launches overlap
            # this one's kernels; the results stay in HBM (the e2e line reads
            # them back every step)
            eng.pml_tvar_async(ylt_dev, rps, res_dev)
            res = None
        eng.release_layer(L)
        return res

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

    # End to end through the C ABI with host buffers (pinned), per step.
    e2e = run_e2e(args, w, handles_count=len(layer.elts), local=local) if rank == 0 else None

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    cpu = oracle_sample(w, budget_s=args.cpu_budget) if world == 1 and not args.no_cpu else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": value / PAPER_1GPU_TRIAL_EVENTS_PER_S,
        "vs_baseline_basis": "paper's best single GPU run (Tesla M2050, 19.93 s for 1e9 trial-events, "
                             "Section IV-C); other hardware, context only",
        "dtype": "f64", "data": "synthetic (seeded; stands in for the paper's proprietary industry data)",
        "config": {"workload": WORKLOAD, "n_trials_per_gpu": N, "occurrences_per_gpu": M,
                   "catalog": C, "elts": len(layer.elts),
                   "step": ("ara_define_layer (ELT fold) + ara_layer_ylt + ara_pml_tvar_async (PML/TVaR "
                            "queued, results kept in HBM; read back after the timed steps)") if world == 1 else
                           "ara_define_layer (ELT fold) + ara_layer_ylt + ara_ylt_tail + all-gather + "
                           "ara_pml_tvar_tail",
                   "yet_layout": ("stored order, 6 packed ids per 16 bytes" if compact_ms is None else
                                  "ara_compact_yet: 8 difference-coded ids per 16 bytes, each group of 8 ascending (prepared once "
                                  "before timing, %.1f ms)" % compact_ms),
                   "l2": "inputs larger than L2: the 2-2.7 GB chunked YET id stream is re-read from HBM every step",
                   "parallelism": (f"trial shards x{world}; each rank sends its {k_tail} largest trial losses "
                                   "(ara_ylt_tail, NCCL all-gather) and rank 0 prices the union "
                                   "(ara_pml_tvar_tail)") if world > 1 else "1 GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "ylt_fp64_kernel", "kernel_ms": ylt_avg_ms,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "frac_of_nominal_8000_gbs": achieved / 8000.0},
        "breakdown_ms_per_step": {"fold": fold_ms / max(args.steps, 1), "ylt": ylt_ms / max(args.steps, 1),
                                  "pml_tvar": pml_ms / max(args.steps, 1)},
        "pml": list(map(float, res[0])), "tvar": list(map(float, res[1])),
        "clocks": clocks.summary(),
        "e2e": e2e,
        # fold, YLT, selection (init + 8 passes + sum) and, on one GPU, the
        # copy of its results; with shards instead the tail (selection + 3
        # kernels) and the selection over the union
        "gpu_launches": args.steps * (1 + 1 + 10 + (13 if world > 1 else 1)),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_e2e(args, w, handles_count: int, local: int):
    """Same step through the public C ABI with pinned host buffers: H2D of the
    YET and the ELTs, the layer definition, the YLT and PML/TVaR back to host."""
    import torch
    from paper_1412_4556_b300 import Engine

    layer = w.layers[0]
    rps = w.return_periods
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    h_off, h_ids = pin(w.yet.offsets), pin(w.yet.ids)
    p = w.pool
    h_eoff, h_eids, h_eloss = pin(p.offsets), pin(p.ids), pin(p.losses)
    h_ded, h_lim = pin(p.deductibles), pin(p.limits)
    h_ylt = torch.empty(w.yet.n_trials, dtype=torch.float64).pin_memory()
    eng = Engine(local)
    N, M = w.yet.n_trials, w.yet.n_occurrences

    def step():
        eng.load_yet(w.yet.catalog_size, h_off.numpy(), h_ids.numpy())
        first = eng.load_elts(h_eoff.numpy(), h_eids.numpy(), h_eloss.numpy(), h_ded.numpy(),
                              h_lim.numpy())
        L = eng.define_layer([first + j for j in layer.elts], layer.occ_ret, layer.occ_lim,
                             layer.agg_ret, layer.agg_lim)
        out = eng.layer_ylt(L, out=h_ylt.numpy())
        res = eng.pml_tvar(out, rps)
        eng.release_layer(L)
        return res

    for _ in range(max(1, min(args.warmup, 2))):
        step()
    torch.cuda.synchronize()
    k = max(1, min(args.steps, args.e2e_steps))
    t0 = time.perf_counter()
    for _ in range(k):
        step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / k
    eng.close()
    h2d = 8 * (N + 1) + 4 * M + 8 * (p.n_elts + 1) + 12 * p.ids.size + 16 * p.n_elts
    d2h = 8 * N + 16 * len(rps)
    return {"value": M / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": dt * 1e3, "steps": k,
            "note": "pinned host buffers through ara_load_yet/ara_load_elts/ara_define_layer/"
                    "ara_layer_ylt(host out)/ara_pml_tvar; YET ids validated on the device each step"}


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
                    "per pass and gather one 32-byte sector per occurrence any of a pass's layers needs, "
                    "which bounds them (L1TEX, not HBM)"}


def run_batched(args):
    """Config-2 step: define 64 layers (ELT folds), price them in pairs in one
    call (ara_layers_ylt), PML/TVaR for all (ara_pml_tvar_batch).  Also times
    the plain path (ara_layer_ylt once per layer) for comparison.  With
    --workload mixed the layers use FP32 tables (config 3) and the line
    reports their error against the FP64 path."""
    import torch
    from paper_1412_4556_b300 import ARA_FP32_TABLE, ARA_FP64, ARA_TIMING_YLT, Engine

    mixed = args.workload == "mixed"
    prec = ARA_FP32_TABLE if mixed else ARA_FP64

    w = S.batched(n_trials=args.trials)
    M, N = w.yet.n_occurrences, w.yet.n_trials
    G = len(w.layers)
    stream = torch.cuda.Stream()
    eng = Engine(0, stream=stream)
    eng.load_yet_from(w.yet)
    compact_ms = compact(eng, args)
    first = eng.load_pool(w.pool)
    handles = [[first + j for j in L.elts] for L in w.layers]
    out = torch.empty((G, N), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()

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

    def step_plain():
        hs = define()
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

    from paper_1412_4556_b300 import Plan
    plan_layers = define()
    plan = Plan(eng, plan_layers, w.return_periods, autotune=True)

    def step_plan():
        # one graph launch: 64 ELT folds, the grouped YLT passes, PML/TVaR
        return plan.run(ylt_out=out, stream=stream)

    steps = max(3, min(args.steps, 20))
    with ClockSampler(0) as clocks:
        clocks.wait_first_sample()
        t0 = time.monotonic()
        ms_g, ylt_g = timed(step_plan, steps)
        t1 = time.monotonic()
        time.sleep(0.3)
        clocks.mark(t0, t1)
    ms_b, ylt_b = timed(step_batched, steps)
    ms_p, ylt_p = timed(step_plain, steps)
    passes = plan.passes()
    plan.close()
    for h in plan_layers:
        eng.release_layer(h)
    value = G * M / (ms_g / 1e3)
    accuracy = None
    if mixed:
        # Error of the FP32-table YLTs and PML/TVaR against the FP64 path (which
        # matches the FP64 oracle within 1e-12 per trial in the parity tests).
        h32, h64 = define(ARA_FP32_TABLE), define(ARA_FP64)
        # pre-aggregate sums S (same layers with neutral aggregate terms): the
        # per-trial bar is |err| <= max(1e-5 * max(|y|, S), 1 USD)
        hpre = [eng.define_layer(h, L.occ_ret, L.occ_lim, 0.0, math.inf) for h, L in zip(handles, w.layers)]
        y32 = eng.layers_ylt(h32)
        y64 = eng.layers_ylt(h64)
        s64 = eng.layers_ylt(hpre)
        p32, t32 = eng.pml_tvar_batch(y32, w.return_periods)
        p64, t64 = eng.pml_tvar_batch(y64, w.return_periods)
        err = np.abs(y32 - y64)
        scale = np.maximum(np.abs(y64), s64)
        rel = err / np.maximum(scale, 1e-300)
        accuracy = {"max_rel_trial_err_vs_fp64": float(rel.max()),
                    "relative_to": "max(|y_fp64|, pre-aggregate sum S)",
                    "max_err_over_bound(1e-5 rel, 1 USD)": float(np.max(err / np.maximum(1e-5 * scale, 1.0))),
                    "max_abs_trial_err_usd": float(err.max()),
                    "max_rel_pml_err": float((np.abs(p32 - p64) / np.maximum(p64, 1.0)).max()),
                    "max_rel_tvar_err": float((np.abs(t32 - t64) / np.maximum(t64, 1.0)).max())}
        for h in h32 + h64 + hpre:
            eng.release_layer(h)
    line = {
        "metric": METRIC, "value": value, "unit": "layer-trial-events/s", "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms_g, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
        "config": {"workload": BATCHED, "layers": G, "n_trials": N, "occurrences": M,
                   "step": "ara_plan_run: one CUDA graph of 64 ELT folds + the grouped YLT passes + "
                           "batched PML/TVaR (launch shapes autotuned at plan creation)",
                   "yet_layout": ("stored order, 6 packed ids per 16 bytes" if compact_ms is None else
                                  "ara_compact_yet: 8 difference-coded ids per 16 bytes, each group of 8 ascending (prepared once "
                                  "before timing, %.1f ms)" % compact_ms),
                   "l2": "inputs larger than L2 (4 GB YET id stream per pass)"},
        "ylt_kernels_ms_per_step": ylt_b,
        "ylt_kernels_note": "CUDA events around the YLT launches of ara_layers_ylt (the graph replays the "
                            "same kernels in the same shapes)",
        "passes": [{"entry_bytes": eb, "layers": g, "lanes_per_trial": lpt, "unroll": u, "l2_prefetch": pf}
                   for eb, g, lpt, u, pf, _ in passes],
        "calls_per_step": {"ms_per_step": ms_b, "ylt_kernels_ms_per_step": ylt_b,
                           "value": G * M / (ms_b / 1e3),
                           "step": "64 x ara_define_layer + ara_layers_ylt + ara_pml_tvar_batch"},
        "plain_per_layer": {"ms_per_step": ms_p, "ylt_kernels_ms_per_step": ylt_p,
                            "value": G * M / (ms_p / 1e3),
                            "step": "64 x ara_define_layer + 64 x ara_layer_ylt + ara_pml_tvar_batch"},
        "speedup_vs_plain": ms_p / ms_g,
        "roofline": batched_roofline(M, N, w.yet.catalog_size, G, 4 if mixed else 8, ylt_b, len(passes)),
        "clocks": clocks.summary(),
    }
    if mixed:
        line["dtype"] = "f32 tables, exact trial sums"
        line["config"]["workload"] = "mixed precision (FP32 tables): " + BATCHED
        line["accuracy"] = accuracy
    print(json.dumps(line), flush=True)


SERVICE = ("ad hoc pricing service: paper-scale YET (catalog 2,000,000 events; 1,000,000 trials x "
           "Poisson(1000)) and a pool of 256 ELTs (10,000-50,000 events each) resident on the device; "
           "layer requests of 2-32 pool ELTs with batched-layer terms over a 100k/250k/1M-trial prefix, "
           "FP32 tables with exact trial sums; PML/TVaR at RP 100/250/500")


def run_service(args):
    """Config-4 serving run: a seeded Poisson stream of layer-pricing requests
    played open-loop against the pricing service (continuous batching over
    slots, admission by device memory); reports requests/s and p50/p99
    latency, then the same requests all at once (saturating) and at a higher
    rate; 1% of the requests are checked against the oracle on sampled trials."""
    from paper_1412_4556_b300 import ARA_FP32_TABLE, ARA_FP64, Engine, Service
    import oracle

    rps = (100.0, 250.0, 500.0)
    w = S.batched(n_layers=1, n_trials=args.trials)
    reqs = S.service_requests(n_requests=args.requests, rate_per_s=args.rate)
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
    _, fast = play(10.0)

    # 1% of the requests against the FP64 oracle (memoised Algorithm 1) on
    # sampled trials; PML/TVaR against the FP64 GPU path, which matches the
    # oracle within 1e-12 per trial in the parity tests.
    g = np.random.default_rng(7)
    worst_rel, worst_bound, worst_pml, worst_tvar, oracle_s, oracle_occ = 0.0, 0.0, 0.0, 0.0, 0.0, 0
    for i in sample:
        rq, r = reqs[i], res[i]
        sel = np.sort(g.choice(rq.n_trials, min(rq.n_trials, args.oracle_trials), replace=False))
        t = time.perf_counter()
        o, pre = oracle.layer_ylt(w.yet, w.pool, rq.layer, trials=sel, mode="memo")
        oracle_s += time.perf_counter() - t
        oracle_occ += int(np.sum(np.diff(w.yet.offsets)[sel]))
        err = np.abs(r.ylt[sel] - o)
        worst_rel = max(worst_rel, float(np.max(err / np.maximum(np.maximum(np.abs(o), pre), 1e-300))))
        worst_bound = max(worst_bound, float(np.max(err / np.maximum(1e-5 * np.maximum(np.abs(o), pre), 1.0))))
        L = rq.layer
        h = eng.define_layer([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret, L.agg_lim,
                             precision=ARA_FP64)
        p64, t64 = eng.pml_tvar(eng.layer_ylt(h, rq.n_trials), rps)
        eng.release_layer(h)
        worst_pml = max(worst_pml, float(np.max(np.abs(r.pml - p64) / np.maximum(p64, 1.0))))
        worst_tvar = max(worst_tvar, float(np.max(np.abs(r.tvar - t64) / np.maximum(t64, 1.0))))
    eng.close()
    import multiprocessing
    line = {
        "metric": METRIC, "value": saturating["requests_per_s"], "unit": "requests/s", "n_gpus": 1,
        "steps": len(reqs), "warmup": max(args.warmup, 3), "ms_per_step": 1e3 / saturating["requests_per_s"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 tables, exact trial sums", "data": "synthetic (seeded)",
        "config": {"workload": SERVICE, "requests": len(reqs), "arrival_rate_per_s": args.rate,
                   "slots": args.slots, "max_batch": args.max_batch,
                   "step": "one request: fold + YLT + PML/TVaR, host in and out",
                   "yet_layout": ("stored order, 6 packed ids per 16 bytes" if compact_ms is None else
                                  "ara_compact_yet: 8 difference-coded ids per 16 bytes, each group of 8 ascending (prepared once "
                                  "before timing, %.1f ms)" % compact_ms),
                   "l2": "inputs larger than L2 (up to 4 GB of YET ids per request)"},
        "latency_ms": {"p50": paced["p50_ms"], "p99": paced["p99_ms"], "at_rate_per_s": args.rate},
        "alone_ms_by_trials": device_ms,
        "paced": paced, "paced_10x": fast, "saturating": saturating,
        "accuracy_1pct": {"requests": len(sample), "trials_per_request": args.oracle_trials,
                          "max_rel_trial_err_vs_oracle": worst_rel,
                          "max_err_over_bound(1e-5 rel, 1 USD)": worst_bound,
                          "max_rel_pml_err_vs_fp64": worst_pml, "max_rel_tvar_err_vs_fp64": worst_tvar},
        "cpu_baseline": {"value": oracle_occ / oracle_s, "unit": "layer-trial-events/s",
                         "cores": multiprocessing.cpu_count(), "kind": "oracle",
                         "sample": f"memoised oracle on {args.oracle_trials} sampled trials of each of "
                                   f"{len(sample)} requests"},
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ oracle arm
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


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = S.paper_scale(n_trials=args.trials)
    M = w.yet.n_occurrences
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(5)
    model = oracle_cost_model(w, threads, rng)
    # Each timed step prices a fresh trial sample sized so that the whole run
    # stays within a few minutes; warm-up steps price 256 trials.
    per = max(0.25, min(args.cpu_budget, 150.0 / max(args.steps + args.warmup, 1)))
    for _ in range(args.warmup):
        oracle_sample(w, budget_s=0.0, threads=threads, model=model, rng=rng)
    vals, samples = [], []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        r = oracle_sample(w, budget_s=per, threads=threads, model=model, rng=rng)
        vals.append(r["value"])
        samples.append(r)
    wall = time.perf_counter() - t_all
    value = statistics.median(vals)
    ms_step = M / value * 1e3
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)", "impl": "reference",
        "config": {"workload": WORKLOAD, "n_trials_per_gpu": w.yet.n_trials, "occurrences_per_gpu": M,
                   "note": "each step times the oracle on a fresh bounded trial sample (about "
                           f"{per:.2f} s of it, so that the run ends within minutes; the oracle's fixed "
                           "cost per call, its table build, weighs more in short samples); "
                           "ms_per_step is extrapolated to the full workload from the median rate"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": samples[-1]["cores"], "kind": "oracle",
                         "sample": samples[-1]["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["engine", "reference"], default="engine")
    ap.add_argument("--workload", choices=["paper", "batched", "mixed", "service", "yelt"], default="paper",
                    help="paper: the single-layer paper-scale step (default); batched: 64 layers; "
                         "mixed: 64 FP32-table layers; service: the pricing-request stream; "
                         "yelt: the Year Event Loss Table and RPL report")
    ap.add_argument("--requests", type=int, default=2000, help="service: requests in the stream")
    ap.add_argument("--rate", type=float, default=50.0, help="service: Poisson arrival rate per s")
    ap.add_argument("--slots", type=int, default=4, help="service: batches in flight")
    ap.add_argument("--max-batch", type=int, default=16, help="service: requests per batch")
    ap.add_argument("--oracle-trials", type=int, default=2000, help="service: trials checked per sample")
    ap.add_argument("--trials", type=int, default=1_000_000, help="trials per GPU")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
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
