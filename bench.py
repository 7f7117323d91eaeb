"""Benchmark: measurements/s of the batched FP32 log-likelihood + gradient.

Workload (default ``c4``): 1024 independent series, N ~ U{2000..20000}
exposures each (11.29M measurements, 22.6M events), kernel = sum of two SHO
terms with one integral state per term (augmented dimension 6), per-series
hyperparameters; one step = log-likelihood and adjoint gradient w.r.t. the 7
natural parameters of every series, inputs resident in HBM.  The event stream
(~292 MB) is larger than the 129 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank takes a longest-processing-time share of
the series (no collective on the data path) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "measurements/sec for loglik+grad (batched FP32 vs plain FP64 filter, 1 GB300)"
UNIT = "measurements/s"

# Dominant kernel (k_grad, the reverse-time gradient): FP32 FLOPs per event it
# executes (fadd + fmul + 2 ffma, thread-level, predicated-on; the segment
# replay included), from ncu's FP32 instruction counters of one k_grad launch
# on 512 series of the c4 recipe (chunk length 256, segments of 64), captured
# with --clock-control none.
ALG_FLOPS_PER_EVENT = {"c4": 1440.2}
# DRAM bytes (read + write) per event of that k_grad launch, same capture;
# the traffic grows with the events (replay records, cached step scalars,
# partial elements, event stream), so a full launch is this x its events.
# Valid for the captured configuration only (chunk length 256, segments of 64).
TRAFFIC_PER_EVENT = {"c4": (347.1, 256, 64)}
FP32_LANES_PER_SM = 128

# Per workload: whether a step includes the gradient, and whether the
# parameter sets are per series (else every set applies to the one series).
WORKLOADS = {"c1": False, "c2": False, "c3": False, "c4": True, "c5": True, "c2i": True,
             "c2p": False, "c4h": True, "c4s": True}


def alg_bytes_per_meas(ck):
    """Algorithmic HBM bytes per measurement of one loglik+grad pass: two gaps
    (8 B), two tags (2 B) and y, yerr^2, 1/delta (12 B) read by the forward
    pass and again by the reverse sweep, plus a filter state (m and packed P,
    27 floats at state dimension 6) written and read back every ck events."""
    return 2 * 22 + 2 * 4 * 27 * 2 / ck


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def product_extra(gp, stream):
    """Log-likelihood throughput of the product-kernel path (quasi-periodic
    SHO x SHO + Matern-3/2 on instantaneous measurements, 410 series of the
    c2p recipe): FP32 chunked parallel-in-time, and the plain FP64 filter;
    and of its FP32 log-likelihood + gradient, chunked and per series."""
    import synth
    import torch
    wl = synth.c2p(n_series=410)
    theta = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    out = {"workload": "c2p, 410 series", "n_meas": int(wl.n_meas), "unit": UNIT,
           "work": "fp32, fp64: loglik (chunked parallel-in-time; plain per-series filter); "
                   "fp32_grad_*: loglik + gradient, per chunk or per series"}
    for prec in (32, 64):
        m = gp.Model.from_workload(wl, precision=prec)
        ll = torch.empty(wl.n_series, dtype=torch.float64, device="cuda")
        m.loglik(theta, out=ll)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            m.loglik(theta, out=ll)
        b.record(stream)
        torch.cuda.synchronize()
        out[f"fp{prec}"] = wl.n_meas / (a.elapsed_time(b) / 3 / 1e3)
        del m
    # loglik + gradient (FP32 forward-mode tangents): per chunk and parameter
    # against the combination's boundary adjoints, and per series and parameter
    for key, sched in (("fp32_grad_chunked", 0), ("fp32_grad_per_series", 3)):
        m = gp.Model.from_workload(wl, schedule=sched)
        ll = torch.empty(wl.n_series, dtype=torch.float64, device="cuda")
        g = torch.empty(wl.n_series, m.n_params, dtype=torch.float32, device="cuda")
        m.loglik_grad(theta, out=ll, grad=g)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            m.loglik_grad(theta, out=ll, grad=g)
        b.record(stream)
        torch.cuda.synchronize()
        out[key] = wl.n_meas / (a.elapsed_time(b) / 3 / 1e3)
        del m
    return out


def workload(name):
    import synth
    if name == "c1":
        return synth.c1()
    if name == "c4":
        return synth.c4()
    if name == "c2":
        return synth.c2()
    if name == "c3":
        return synth.c3()
    if name == "c5":
        return synth.c5()
    if name == "c2i":  # the c2 recipe on instantaneous measurements
        return synth.c2i()
    if name == "c2p":  # product kernel on instantaneous measurements (loglik only)
        return synth.c2p()
    if name == "c4h":  # 512 series of the c4 recipe (profiling captures)
        return synth.c4(n_series=512)
    if name == "c4s":  # small variant for quick checks
        return synth.c4(n_series=64, scale=0.25)
    raise ValueError(name)


class ClockSampler:
    """nvidia-smi samples every 50 ms, started before the warm-up (its own
    start-up takes a while); ``stop`` keeps the samples whose timestamps fall
    inside the timed window marked by ``mark``."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None
        self.window = None

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        # nvidia-smi takes a while to start: wait (bounded) for its first sample
        # so that a short timed region still has samples around it
        self._wait_lines(1, 10.0)

    def _n_lines(self):
        try:
            with open(self.path) as f:
                return sum(1 for _ in f)
        except Exception:
            return 0

    def _wait_lines(self, n, limit_s):
        t_end = time.time() + limit_s
        while self.proc is not None and self._n_lines() < n and time.time() < t_end:
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        # one more sample after the timed window closed (bounded wait)
        self._wait_lines(self._n_lines() + 2, 3.0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        try:
            import datetime
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    rows.append((ts, float(parts[2]), float(parts[3]),
                                 {nm for nm, v in zip(names, parts[6:10])
                                  if v.lower() == "active"}))
                except ValueError:
                    continue
            os.unlink(self.path)
        except Exception:
            pass
        if not rows:
            return None
        sel = rows
        where = "all samples"
        if self.window is not None:
            t0, t1 = self.window
            inside = [r for r in rows if t0 - 0.02 <= r[0] <= t1 + 0.02]
            if inside:
                sel, where = inside, "timed window"
            else:
                # window shorter than the sampling period: the samples next to it
                sel = sorted(rows, key=lambda r: min(abs(r[0] - t0), abs(r[0] - t1)))[:2]
                where = "nearest to the timed window"
        reasons = set().union(*[r[3] for r in sel])
        return {"sm_mhz": float(np.median([r[1] for r in sel])), "sm_max_mhz": sel[-1][2],
                "reasons": sorted(reasons), "samples": len(sel), "samples_from": where}


def oracle_sample_rate(wl, budget_s, n_proc, prefix_meas, grad=True, closed_form=True):
    """The FP64 oracle (log-likelihood, with ``grad`` also its complex-step
    gradient) on host cores.  ``closed_form``: its timing mode, closed forms for
    the discretisation (Appendix B's for underdamped SHO terms, the defining
    integrals worked out for critically damped ones; Van Loan for overdamped
    and product terms); else the Van Loan discretisation the parity tests use.

    Sample: the first ``prefix_meas`` measurements of consecutive series (or,
    for one series shared by parameter sets, of the series under consecutive
    sets), one job per process, repeated until ``budget_s`` of wall time has
    passed.  A single series with one set runs on one core.
    Returns (measurements/s, cores, description)."""
    import multiprocessing as mp

    import oracle
    oracle.build()
    jobs = []
    rows = wl.n_series if wl.theta_per_series else wl.theta.shape[0]
    if rows == 1:
        n_proc = 1
    for i in range(rows):
        s = i if wl.theta_per_series else 0
        ts, te, y, ye, inst = wl.series(s)
        k = min(prefix_meas, len(ts))
        jobs.append((wl.terms, wl.layout, (ts[:k], te[:k], y[:k], ye[:k],
                                           None if inst is None else inst[:k]), wl.theta[i],
                     grad, closed_form))
    done = 0
    with mp.get_context("spawn").Pool(n_proc) as pool:
        # start-up (process spawn, imports, the library load) outside the timing
        pool.map(oracle._series_job, [jobs[q % len(jobs)] for q in range(n_proc)])
        t0 = time.perf_counter()
        j = 0
        # batches of consecutive jobs, wrapping around the rows, until the
        # budget is spent
        while time.perf_counter() - t0 < budget_s:
            batch = [jobs[(j + q) % len(jobs)] for q in range(min(n_proc, len(jobs)))]
            pool.map(oracle._series_job, batch)
            done += sum(len(b[2][0]) for b in batch)
            j += len(batch)
    el = time.perf_counter() - t0
    what = "loglik + complex-step gradient" if grad else "loglik"
    unit = "series" if wl.theta_per_series else "parameter sets of the one series"
    plain = all(t in (1, 2) for t in wl.terms)
    disc = ("closed forms (Appendix B; Van Loan for any overdamped row)" if closed_form and plain
            else "Van Loan" + (" (product terms have no closed forms here)" if closed_form else ""))
    return done / el, n_proc, (f"oracle {what}, FP64 ({disc}), first {prefix_meas} "
                               f"measurements of {min(j, rows)} {unit}"
                               f"{' (cycled: ' + str(j) + ' jobs)' if j > rows else ''}, "
                               f"{n_proc} processes, {el:.1f} s")


def run_reference(args):
    """Reference arm: the oracle on host cores, same metric and config."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args.workload)
    grad = WORKLOADS[args.workload]
    n_proc = max(1, min(os.cpu_count() or 1, 16))
    prefix = 200 if wl.n_series > 1 else 2000
    budget = max(2.0, min(8.0, 150.0 / max(args.steps + args.warmup, 1)))
    for _ in range(args.warmup):
        oracle_sample_rate(wl, 0.5, n_proc, 64, grad=grad)
    rates = []
    desc = ""
    cores = n_proc
    for _ in range(args.steps):
        r, cores, desc = oracle_sample_rate(wl, budget, n_proc, prefix, grad=grad)
        rates.append(r)
    v = float(np.mean(rates))
    n_proc = cores
    units = wl.n_meas * (1 if wl.theta_per_series else wl.theta.shape[0])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            # one whole step of the workload at the sampled rate
            "ms_per_step": units / v * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "work": "loglik+grad" if grad else "loglik",
                       "n_series": wl.n_series, "n_meas": wl.n_meas,
                       "ms_per_step": "extrapolated from the bounded sample's rate"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": n_proc, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def loglik_errors(l32, l64, counts):
    """FP32 log-likelihood against FP64 on the same rows: the plain relative
    error max |dL|/|L| and how many rows exceed 1e-4 of it, the error over
    max(|L|, 0.1 N) (the parity tests' tolerance measure: relative where
    |L| >= 0.1 N, else per measurement) and the error per measurement."""
    l32, l64, n = np.asarray(l32, float), np.asarray(l64, float), np.asarray(counts, float)
    d = np.abs(l32 - l64)
    rel = d / np.abs(l64)
    return {"max_rel_err": float(rel.max()), "n_rows": int(len(rel)),
            "n_rows_rel_above_1e-4": int((rel > 1e-4).sum()),
            "max_err_over_max_L_0p1N": float(np.max(d / np.maximum(np.abs(l64), 0.1 * n))),
            "max_abs_err_per_meas": float(np.max(d / np.maximum(n, 1))),
            "max_abs_err": float(d.max())}


def timed(fn, reps, stream):
    """Mean milliseconds per call of fn over reps calls (CUDA events on the
    launching stream, after one warm-up call)."""
    import torch
    fn()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def run_ours(args):
    import torch

    import paper_2601_02527_gb300 as gp
    from paper_2601_02527_gb300 import build as gbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0 or world == 1:
        gbuild.build()
    if world > 1:
        torch.distributed.barrier()
    name = args.workload
    want_grad = WORKLOADS[name]
    wl_full = workload(name)
    per_series = bool(wl_full.theta_per_series)
    n_sets = int(wl_full.theta.shape[0])
    counts = np.diff(wl_full.offsets)
    # units of the metric: measurements, times the parameter sets applied to
    # every series when the sets are shared
    units_full = int(wl_full.n_meas) * (1 if per_series else n_sets)
    from paper_2601_02527_gb300 import shard
    # one series with one parameter set is split in time (contiguous chunk
    # ranges, one all-gather of span elements); otherwise series or shared
    # parameter sets are split across ranks with no exchange
    time_split = world > 1 and wl_full.n_series == 1 and per_series
    if time_split:
        wl = wl_full
    elif world > 1 and per_series:
        wl = wl_full.subset(shard.lpt_shards(counts, world)[rank])
    elif world > 1:
        # one series shared by the sets: the sets are split across ranks
        mine = np.array_split(np.arange(n_sets), world)[rank]
        wl = wl_full.with_theta(wl_full.theta[mine])
    else:
        wl = wl_full
    # CPU baseline first: its process pool is spawned before the first GPU call
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        ncore = max(1, min(os.cpu_count() or 1, 16))
        prefix = 200 if wl.n_series > 1 else 2000
        rate, cores, desc = oracle_sample_rate(wl, args.cpu_budget, ncore, prefix,
                                               grad=want_grad)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
        if want_grad:
            # the same oracle without the gradient: the log-likelihood alone
            r2, c2, d2 = oracle_sample_rate(wl, max(2.0, args.cpu_budget / 3), ncore, prefix,
                                            grad=False)
            cpu["loglik_only"] = {"value": r2, "unit": UNIT, "cores": c2, "sample": d2}
        if all(t in (1, 2) for t in wl.terms):
            # the Van Loan discretisation (the parity reference), timed apart
            r3, c3, d3 = oracle_sample_rate(wl, max(2.0, args.cpu_budget / 3), ncore, prefix,
                                            grad=want_grad, closed_form=False)
            cpu["van_loan"] = {"value": r3, "unit": UNIT, "cores": c3, "sample": d3}
    fp32_peak, n_sms = gp.measure_fp32_peak()
    t0 = time.perf_counter()
    model = gp.Model.from_workload(wl, chunk_len=args.chunk_len, ckpt_interval=args.ckpt_interval,
                                   combine_precision=args.combine_precision)
    build_s = time.perf_counter() - t0
    theta = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    # the autotuner picks schedule, chunk length (threads per series) and the
    # gradient's segment length on this workload (before the timed region)
    tuned = None
    if time_split and want_grad:
        raise SystemExit("a series split in time is timed for its log-likelihood only")
    if not args.no_autotune and name not in ("c1", "c2p") and not time_split:
        t0 = time.perf_counter()
        tuned = model.autotune(theta, per_series=per_series, grad=want_grad, reps=3)
        tuned["tune_s"] = time.perf_counter() - t0
    n_out = model.n_out(theta, per_series)
    ll = torch.empty(n_out, dtype=torch.float64, device="cuda")
    g = torch.empty(n_out, model.n_params, dtype=torch.float32, device="cuda")

    def step():
        if time_split:
            ll.copy_(shard.time_sharded_loglik(model, theta))
        elif want_grad:
            model.loglik_grad(theta, per_series=per_series, out=ll, grad=g)
        else:
            model.loglik(theta, per_series=per_series, out=ll)

    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    model.set_timing(True)
    model.get_timing()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n_launch0 = gp.launch_count()
    w0 = time.time()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    n_launches = gp.launch_count() - n_launch0
    torch.cuda.synchronize()
    clocks.mark(w0, time.time())
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    phases = model.get_timing()
    model.set_timing(False)
    clk = clocks.stop()
    n_events_all = int(model.info["n_events"])
    if world > 1 and not time_split:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        ne = torch.tensor([n_events_all], dtype=torch.int64, device="cuda")
        torch.distributed.all_reduce(ne)
        n_events_all = int(ne.item())
    ok = bool(torch.isfinite(ll).all().item()) and model.last_error()[0] < 0
    value = units_full / (ms / 1e3)
    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return
    # dominant kernel
    dom = max(phases, key=lambda k: phases[k][0])
    dom_ms, dom_n = phases[dom]
    dom_avg = dom_ms / max(dom_n, 1)
    peaks, src = load_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_nominal = n_sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s
    n_events = int(model.info["n_events"])
    n_vrows = 1 if per_series else int(wl.theta.shape[0])
    # the gradient phase is k_grad alone; its per-launch time from the
    # phase events recorded on the launching stream inside the timed region
    fpe = ALG_FLOPS_PER_EVENT.get(name)
    achieved = (fpe * n_events * n_vrows / (dom_avg / 1e3) / 1e12
                if fpe and dom == "grad" else None)
    ck_used = (tuned or {}).get("ckpt_interval", args.ckpt_interval or 32)
    L_used = (tuned or {}).get("chunk_len", args.chunk_len or 256)
    tr = TRAFFIC_PER_EVENT.get(name)
    traffic = (tr[0] * n_events * n_vrows
               if tr and (L_used, ck_used) == (tr[1], tr[2]) and dom == "grad" else None)
    step_bytes = (alg_bytes_per_meas(ck_used) if want_grad else 22.0) * units_full
    roofline = {"bound": "alu", "kernel": "k_grad" if dom == "grad" else dom,
                "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak if achieved else None, "traffic": traffic,
                "peak_source": f"measured: FP32 FMA-chain kernel on this GPU ({n_sms} SMs); "
                               f"nominal {n_sms} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                               f"{sm_mhz:.0f} MHz = {alu_nominal:.1f} TFLOP/s",
                "frac_of_nominal": achieved / alu_nominal if achieved else None,
                "kernel_ms_per_launch": dom_avg,
                "hbm_view": {"whole_step_gbs": step_bytes / (ms / 1e3) / 1e9,
                             "bytes_per_meas": alg_bytes_per_meas(ck_used) if want_grad else 22.0,
                             "peak_gbs": peaks.get("hbm_gbs"),
                             "frac": step_bytes / (ms / 1e3) / 1e9 / peaks.get("hbm_gbs", 6800.0),
                             "k_grad_dram_gbs": traffic / (dom_avg / 1e3) / 1e9 if traffic else None,
                             "peak_source": src},
                "phase_ms_per_step": {k: v[0] / max(args.steps, 1) for k, v in phases.items()
                                      if v[1]}}
    # end to end through the host-buffer C-ABI call: event stream + theta up, results down
    e2e = None
    if not args.no_e2e and want_grad:
        th_host = wl.theta.astype(np.float32)
        for _ in range(3):
            model.loglik_grad_host(th_host, per_series=per_series, reupload_events=True)
        k2 = max(2, min(args.steps, 20))
        t1 = time.perf_counter()
        for _ in range(k2):
            model.loglik_grad_host(th_host, per_series=per_series, reupload_events=True)
        el = (time.perf_counter() - t1) / k2
        # gaps (4 B) and tags (1 B) per event, (y, r0, w) per measurement, theta
        h2d = model.info["n_events"] * 5 + wl.n_meas * 12 + th_host.nbytes
        d2h = n_out * 8 + n_out * model.n_params * 4
        e2e = {"value": units_full / el, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": el * 1e3}
    # the plain FP64 per-series filter and the FP32 path's error against it
    extra = {"fp32_peak_tflops_measured": fp32_peak, "n_sms": n_sms,
             "combine_precision": args.combine_precision or 32}
    if not args.no_fp64:
        m64 = gp.Model.from_workload(wl, precision=64)
        # shared sets on one long series: four sets (one FP64 thread each)
        idx64 = (np.arange(n_out) if per_series
                 else np.linspace(0, n_out - 1, min(4, n_out)).astype(int))
        th64 = theta if per_series else theta[torch.as_tensor(idx64, device="cuda")]
        out64 = torch.empty(len(idx64), dtype=torch.float64, device="cuda")
        ms64 = timed(lambda: m64.loglik(th64, per_series=per_series, out=out64), 1, stream)
        units64 = wl.n_meas * (1 if per_series else len(idx64))
        extra["plain_fp64_filter"] = {"value": units64 / (ms64 / 1e3), "unit": UNIT,
                                      "ms_per_call": ms64, "work": "loglik only",
                                      "rows": int(len(idx64))}
        l32 = ll.cpu().numpy()[idx64]
        nrow = counts if per_series else np.full(len(idx64), wl.n_meas)
        extra["fp32_vs_fp64_loglik"] = loglik_errors(l32, out64.cpu().numpy(), nrow)
        extra["speedup_vs_plain_fp64"] = value / extra["plain_fp64_filter"]["value"]
        del m64
    if want_grad:
        ms_ll = timed(lambda: model.loglik(theta, per_series=per_series, out=ll), 3, stream)
        extra["fp32_loglik_only"] = {"value": units_full / (ms_ll / 1e3), "unit": UNIT}
        # conditioned mean and variance of every measurement (integrated RTS
        # smoother through the gradient walk), with the log-likelihood
        if per_series:
            ms_c = timed(lambda: model.condition(theta), 3, stream)
            extra["fp32_condition"] = {"value": units_full / (ms_c / 1e3), "unit": UNIT,
                                       "work": "loglik + conditioned mean/variance per "
                                               "measurement"}
    if not args.no_product and name == "c4":
        extra["product_kernel_loglik"] = product_extra(gp, stream)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if time_split else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": name, "work": "loglik+grad" if want_grad else "loglik",
                       "n_series": int(wl_full.n_series), "n_sets": n_sets,
                       "n_meas": int(wl_full.n_meas), "units_per_step": units_full,
                       "n_events": n_events_all,
                       "state_dim": model.info["state_dim"], "n_params": model.n_params,
                       "chunk_len": (tuned or {}).get("chunk_len", args.chunk_len),
                       "n_chunks": model.info["n_chunks"], "autotuned": tuned,
                       "l2": ("inputs larger than L2" if n_events_all * 13 > 129e6 else
                              "inputs smaller than L2 (reused from L2 between steps)"),
                       "parallelism": ("time-split series (span elements all-gathered)"
                                       if time_split else
                                       f"{'series' if per_series else 'parameter-set'}-sharded")
                                      + f" x{world}", "build_s": build_s},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": n_launches, "clocks": clk, "ok": ok, "extra": extra}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def run_accuracy(args):
    """FP32 error against FP64 for every workload configuration (one JSON line
    each, for the FP32 and the FP64 combination of chunk elements): the
    log-likelihood of the FP32 path (autotuned) against the plain FP64 GPU
    filter on every output row (c1: the FP64 path against the oracle; c5: four
    of the 256 sets), and the FP32 gradient against the oracle's complex-step
    gradient on sampled c4 series and on a 20000-measurement prefix of c5.
    Slow: the FP64 filter runs one thread per series."""
    import torch

    import oracle
    import paper_2601_02527_gb300 as gp
    import synth
    from paper_2601_02527_gb300 import build as gbuild
    gbuild.build()
    oracle.build()
    torch.cuda.set_device(0)
    names = args.accuracy_workloads.split(",")
    for name in names:
        wl = workload(name)
        wl.theta = wl.theta.astype(np.float32).astype(np.float64)
        per = bool(wl.theta_per_series)
        grad = WORKLOADS[name]
        th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
        counts = np.diff(wl.offsets)
        m64 = gp.Model.from_workload(wl, precision=64)
        rows64 = (np.arange(wl.n_series) if per else
                  np.linspace(0, wl.theta.shape[0] - 1, 4).astype(int))
        th64 = th if per else th[torch.as_tensor(rows64, device="cuda")]
        t0 = time.perf_counter()
        l64 = m64.loglik(th64, per_series=per).cpu().numpy()
        t64 = time.perf_counter() - t0
        if name == "c1":
            ref = oracle.loglik_workload(wl)
            print(json.dumps({"workload": name, "fp64_vs_oracle_max_rel":
                              float(np.max(np.abs(l64 - ref) / np.abs(ref)))}), flush=True)
            continue
        nrow = counts if per else np.full(len(rows64), wl.n_meas)
        for cp in (32, 64):
            out = {"workload": name, "combine_precision": cp, "n_series": int(wl.n_series),
                   "n_meas": int(wl.n_meas), "n_sets": int(wl.theta.shape[0]),
                   "fp64_filter_s": t64}
            m = gp.Model.from_workload(wl, combine_precision=cp)
            if name != "c2p":  # the product path has one schedule
                tuned = m.autotune(th, per_series=per, grad=grad, reps=1)
                out["autotuned"] = {k: tuned[k] for k in ("schedule", "chunk_len",
                                                          "chunk_combine", "ckpt_interval", "ms")}
            l32 = (m.loglik_grad(th, per_series=per)[0] if grad else
                   m.loglik(th, per_series=per)).cpu().numpy()
            out["loglik"] = loglik_errors(l32[rows64], l64, nrow)
            if name == "c4":
                idx = np.unique(np.argsort(counts)[np.linspace(0, len(counts) - 1, 8).astype(int)])
                _, g = m.loglik_grad(th)
                g = g.cpu().numpy()[idx]
                if cp == 32:
                    _, rg_c4 = oracle.loglik_workload(wl, series_idx=idx, grad=True, processes=8)
                out["grad_vs_oracle_max_rel_of_max"] = float(
                    np.max(np.abs(g - rg_c4) / np.abs(rg_c4).max(axis=1, keepdims=True)))
                out["grad_vs_oracle_max_componentwise_rel"] = float(
                    np.max(np.abs(g - rg_c4) / np.abs(rg_c4)))
                out["grad_sampled_series"] = [int(i) for i in idx]
            if name == "c5":
                n = 20000
                ts, te, y, ye, inst = wl.series(0)
                sets = [0, 85, 170, 255]
                pre = synth.Workload("c5p", wl.terms, wl.layout, np.array([0, n]), ts[:n], te[:n],
                                     y[:n], ye[:n], inst[:n], wl.theta[sets], False)
                mp = gp.Model.from_workload(pre, combine_precision=cp)
                _, gpre = mp.loglik_grad(torch.tensor(pre.theta, dtype=torch.float32,
                                                      device="cuda"), per_series=False)
                gpre = gpre.cpu().numpy()
                if cp == 32:
                    rg_c5 = []
                    for k in range(len(sets)):
                        one = synth.Workload("c5p", pre.terms, pre.layout, pre.offsets,
                                             pre.t_start, pre.t_end, pre.y, pre.yerr,
                                             pre.instrument, pre.theta[[k]], True)
                        rg_c5.append(oracle.loglik_workload(one, grad=True)[1][0])
                    rg_c5 = np.array(rg_c5)
                out["grad_prefix20000_vs_oracle_max_rel_of_max"] = float(
                    np.max(np.abs(gpre - rg_c5) / np.abs(rg_c5).max(axis=1, keepdims=True)))
                out["grad_prefix20000_vs_oracle_max_componentwise_rel"] = float(
                    np.max(np.abs(gpre - rg_c5) / np.abs(rg_c5)))
            print(json.dumps(out), flush=True)
            del m


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c4")
    ap.add_argument("--chunk-len", type=int, default=0)
    ap.add_argument("--ckpt-interval", type=int, default=0)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-product", action="store_true")
    ap.add_argument("--accuracy", action="store_true",
                    help="print FP32-vs-FP64 errors per workload instead of timing")
    ap.add_argument("--accuracy-workloads", default="c1,c2,c3,c4,c5,c2i,c2p")
    ap.add_argument("--combine-precision", type=int, default=0, choices=[0, 32, 64],
                    help="arithmetic of the cross-chunk combination (0: the library default)")
    args = ap.parse_args()
    if args.accuracy:
        run_accuracy(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
