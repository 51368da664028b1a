#!/usr/bin/env python
"""Benchmark: log-likelihood + gradient throughput of exact state-space GP
inference (time steps per second), FP64, one Matern-5/2 series (b = 3) of
N = 2^22 steps with dt ~ Exp(0.01), l = 0.5, s_f = 2, s_n = 0.05.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl spingp|reference]

Prints one JSON line (rank 0).  The device-timed value brackets each step's
spingp_grad call with CUDA events on its stream, after an untimed 256 MiB
write that flushes L2; with N GPUs (torchrun) the one series is split across
the ranks (one all-gather of the ranges' elements and one all-reduce per
step, strong scaling), the time is the max over ranks and the value counts
the series' steps once.  Extra keys: the roofline of the
dominant kernel (live stage timing), the HBM roofline of the whole step, the
median of CUDA-graph replays of the same call, the
end-to-end figure through the public API with host buffers, the "plain GPU
form" comparator (the forward kernel run 2P+1 times for central differences),
the oracle timed on host cores, and SM clocks sampled during the timed region.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "loglik+grad time steps/s (FP64, N=2^22,b=3) vs plain GPU form; % HBM roofline"
WORKLOAD = "matern52_n4m"

# FP64 work per time step of each stage of the gradient call for b = 3, counted
# with ncu at the benchmark's chunk length 108 (N = 2^21, one kernel and one
# launch per capture, `--only matern52_n4m --n 2097152 --chunk 108`): flops = 2 x DFMA + DADD + DMUL
# thread instructions; FP64 instructions = everything the FP64 pipe executed
# (the pipe issues one warp instruction per 16 cycles per SM whatever its kind).
FLOPS_PER_STEP = {"elimination": 171.5, "chunk_pass": 231.2}
FP64_INST_PER_STEP = {"elimination": 107.1, "chunk_pass": 141.6}
# DRAM bytes per step moved by the chunk pass (ncu dram__bytes_read + write,
# same capture); None once the kernel has changed since the counters were taken
DRAM_BYTES_PER_STEP = {"chunk_pass": 213.8}
# algorithmic HBM bytes per step of the whole call: t and y in (16 B); the
# gradient and log-likelihood outputs are O(1) per series
ALGO_BYTES_PER_STEP = 16.0
# Algorithmic FP64 work per step of one log-likelihood + gradient evaluation:
# the sequential method written as dense b x b algebra in the paper's
# coordinates (covariance Kalman filter, inversion-free adjoint, gradient
# contractions; the discretisation not counted), from the counted
# restatement in oracle/flops.py, 12 b^3 + (21 + 2 P_A) b^2 + 11 b + 11 with
# P_A the parameters the transition depends on.  Per workload: b = 3 (P_A = 1),
# b = 2 (P_A = 1), b = 16 (P_A = 3), b = 12 (P_A = 2).
ALGO_FLOPS_PER_STEP = {"matern52_n4m": 575.0, "batched_4096": 575.0, "matern32_n64m": 221.0,
                       "sum_qp_n1m": 56251.0, "m32_eq10_n1m": 24479.0}
# y of every synthetic series but the N = 1000 plain-method one (whose y is
# drawn from the state-space model)
Y_KIND = "two sinusoids + Gaussian noise (the paper's simulated data, Sec. 4.2)"
FP64_NOMINAL_TFLOPS = 152 * 2.07e9 * 4 / 1e12   # SMs x max SM clock x FP64 flop/clk/SM


def _algorithmic(key, steps_per_s, fp64_tflops):
    """The whole call against the FP64 peak, in units of the dense
    sequential method's arithmetic (ALGO_FLOPS_PER_STEP): above 1 where the
    GPU's formulation (Jordan coordinates, block structure, the variance
    scaling identity) needs fewer operations than the dense form."""
    fl = ALGO_FLOPS_PER_STEP[key]
    ach = fl * steps_per_s / 1e12
    return {"algorithmic_flops_per_step": fl, "algorithmic_achieved": ach,
            "algorithmic_frac": ach / fp64_tflops if fp64_tflops else None,
            "algorithmic_scope": "whole call; flops of the dense sequential method (oracle/flops.py)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="spingp", choices=["spingp", "reference"])
    ap.add_argument("--n", type=int, default=0, help="override the series length (profiling runs only)")
    ap.add_argument("--chunk", type=int, default=-1,
                    help="chunk length; -1 = autotune (with --only: the library default), 0 = library default")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparator", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the secondary workloads (b = 16 sum, 4096-series batch, N = 2^26)")
    ap.add_argument("--split", action="store_true",
                    help="the split-series path even on one GPU (under torchrun; N > 1 always uses it)")
    ap.add_argument("--only", default="",
                    help="profiling: time only this workload's gradient call (matern52_n4m, sum_qp_n1m, "
                         "m32_eq10_n1m, matern32_n64m or batched_4096), --n steps (--n series for the batch), "
                         "and print one short line")
    ap.add_argument("--call", default="grad", choices=["grad", "grad_posterior"],
                    help="with --only on a single series: the call to time (grad_posterior: the fused "
                         "gradient + posterior mean and variance)")
    ap.add_argument("--no-next", action="store_true",
                    help="skip the rows built beyond the hot path (prediction, literal mode, BTD solver, "
                         "EQ oracle rate, batched SCG)")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks during the timed region

class ClockSampler:
    """nvidia-smi samples every 25 ms, each with its timestamp; stop(t0, t1)
    keeps the samples taken inside the timed region [t0, t1] (wall clock),
    so the idle lead-in and tail do not enter the median."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 25

    def __init__(self, gpu_index, enabled=True):
        self.p = None
        if not enabled:
            return
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                       "-lms", str(self.PERIOD_MS), "-i", str(gpu_index)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    @staticmethod
    def _when(stamp):
        import datetime
        try:
            return datetime.datetime.strptime(stamp, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self, t0=None, t1=None):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        rows = []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                sm, smax, pw = float(f[2]), float(f[3]), float(f[4])
            except ValueError:
                continue
            rs = {name for name, val in zip(names, f[6:10]) if val.lower().startswith("active")}
            rows.append((self._when(f[0]), sm, smax, pw, rs))
        if not rows:
            return None
        inside = rows
        if t0 is not None and t1 is not None:
            inside = [r for r in rows if r[0] is not None and t0 <= r[0] <= t1]
        window = bool(inside) and t0 is not None
        if not inside:   # a region shorter than the period: the samples nearest to it
            mid = 0.5 * (t0 + t1) if t0 is not None else 0.0
            inside = sorted(rows, key=lambda r: abs((r[0] or 0.0) - mid))[:2]
        reasons = set().union(*(r[4] for r in inside))
        return {"sm_mhz": float(np.median([r[1] for r in inside])), "sm_max_mhz": max(r[2] for r in rows),
                "power_w_max": max(r[3] for r in inside), "reasons": sorted(reasons), "samples": len(inside),
                "in_timed_region": window, "period_ms": self.PERIOD_MS}


# ---------------------------------------------------------------- the oracle (CPU baseline / reference arm)

def oracle_rate(s, sample_n, reps=1):
    """Steps/s of the sequential FP64 oracle (Kalman filter + two-filter
    adjoint, one host thread) on the first sample_n steps of the workload."""
    from oracle import seq
    t, y = s.t[:sample_n], s.y[:sample_n]
    seq.grad(s.spec, s.theta, t[:1000], y[:1000])        # builds/loads the oracle library
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        seq.grad(s.spec, s.theta, t, y)
        times.append(time.perf_counter() - t0)
    return sample_n / float(np.median(times)), times


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1610_08035_gb300 import synth
    s = synth.single(WORKLOAD, n=args.n or None, seed=1)
    sample = len(s.t)                     # the whole series every step (~9 s on one core)
    for _ in range(args.warmup):
        oracle_rate(s, min(sample, 1 << 14))
    rates = []
    for _ in range(args.steps):
        r, _ = oracle_rate(s, sample)
        rates.append(r)
    value = float(np.median(rates))
    desc = "the whole %d-step series per step, sequential C oracle (Kalman filter + two-filter adjoint)" % sample
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sample / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": len(s.t), "b": 3, "model": "matern52",
                   "theta": [float(v) for v in s.theta], "parallelism": "single", "y": Y_KIND},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------- secondary workloads

def _time_calls(fn, K, flush, torch):
    """Mean device time of fn over K calls, L2 flushed (untimed) before each."""
    ms = 0.0
    for k in range(K):
        flush.fill_(k & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    return ms / K


# FP64 work per step executed by the per-step kernels of each secondary
# workload (discretisation, elimination, chunk pass; ncu: flops = 2 DFMA +
# DADD + DMUL thread instructions, and every FP64-pipe instruction), captured
# one kernel and one launch at a time with `--only <workload>` at 2^18 steps
# (b = 16, b = 12; chunk length 432), 2^22 (b = 2; 108) and 512 series of the
# batch.  The reduction levels (work per chunk, not per step) are left out of
# the flops and kept in the time.
WORKLOAD_EXEC_PER_STEP = {"sum_qp_n1m": (12310.5, 8059.1), "m32_eq10_n1m": (21120.6, 13421.2),
                          "matern32_n64m": (215.1, 144.1), "batched_4096": (397.6, 246.9)}
# The same for the fused gradient + posterior call (spingp_grad_posterior):
# the elimination as above, the chunk pass captured with `--only <workload>
# --call grad_posterior` (b = 16 at 2^18 steps, b = 2 at 2^22).
GRAD_POSTERIOR_EXEC_PER_STEP = {"sum_qp_n1m": (12398.8, 8251.7), "matern32_n64m": (222.1, 149.1)}


def extra_workloads(args, dev, flush, world, rank=0, fp64_tflops=None):
    """loglik + gradient throughput of the other configurations: the b = 16
    sum (Matern-3/2 + quasi-periodic), the paper's own b = 12 timing model
    (Matern-3/2 + the order-10 EQ approximation), the batch of 4096 independent series of
    uneven length, and the N = 2^26 Matern-3/2 series; each with its own
    launch count and, for the batch, the plain GPU form (forward kernel run
    2P+1 times per series, one launch sequence per series).  With several
    ranks the single series run as replicas (weak scaling) and the batch is
    sharded across ranks by series (strong scaling: the same 4096 series in
    total, no exchange on the data path)."""
    import torch
    import torch.distributed as dist

    from paper_1610_08035_gb300 import autotune, shard, spingp, synth

    def max_ms(v):
        if world == 1:
            return v
        x = torch.tensor([v], dtype=torch.float64, device=dev)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        return float(x.item())

    K = max(3, min(args.steps, 5))
    res = {}
    # oracle samples for the cpu baselines (about 5-10 s of host work each)
    oracle_sample = {"sum_qp_n1m": 1 << 15, "m32_eq10_n1m": 1 << 12, "matern32_n64m": 1 << 20}
    for name in ("sum_qp_n1m", "m32_eq10_n1m", "matern32_n64m"):
        s = synth.single(name)
        n = len(s.t)
        T, Y, TH = (torch.tensor(a, device=dev) for a in (s.t, s.y, s.theta))
        m = spingp.Model(s.spec)
        autotune.tune(m, T, Y, TH, spingp.WS_GRAD)
        P = m.num_params
        ll = torch.empty(1, dtype=torch.float64, device=dev)
        g = torch.empty(P, dtype=torch.float64, device=dev)
        for _ in range(3):
            m.grad(T, Y, TH, out=(ll, g))
        ms = max_ms(_time_calls(lambda: m.grad(T, Y, TH, sync=False, out=(ll, g)), K, flush, torch))
        st = spingp.spingp_ws_status(m.workspace(n, spingp.WS_GRAD, dev))
        entry = {"value": world * n / (ms * 1e-3), "unit": "steps/s", "ms_per_step": ms, "n": n,
                 "b": m.state_dim, "params": P, "chunk_len": m.chunk_len(n), "status": st, "y": Y_KIND,
                 "gpu_launches_per_step": spingp.spingp_launch_count(m.h, n, spingp.WS_GRAD)}
        roof = {"bound": "alu", "kernel": "whole call", "peak": fp64_tflops, "unit": "TFLOP/s",
                "peak_kind": "measured FP64 FMA probe (spingp_probe_fp64)"}
        roof.update(_algorithmic(name, n / (ms * 1e-3), fp64_tflops))
        ex = WORKLOAD_EXEC_PER_STEP.get(name)
        if ex is not None:
            fl, inst = ex
            roof.update({"achieved": fl * n / (ms * 1e-3) / 1e12, "frac": fl * n / (ms * 1e-3) / 1e12 / fp64_tflops,
                         "pipe_frac": inst * n / (ms * 1e-3) / (fp64_tflops * 1e12 / 2.0),
                         "flops_per_step": fl, "fp64_inst_per_step": inst})
        entry["roofline"] = roof
        if name in ("matern32_n64m", "sum_qp_n1m"):
            # the step these workloads are stated with: log-likelihood +
            # gradient + posterior (the long series' mean; the structured
            # model's variances through the selected inverse), captured once
            # in a CUDA graph and replayed: the fused call (one forward pass,
            # one reverse sweep) and, beside it, spingp_grad then
            # spingp_posterior in one graph
            mean = torch.empty(n, dtype=torch.float64, device=dev)
            var = torch.empty(n, dtype=torch.float64, device=dev)
            fused_out = (ll, g, mean, var, None)
            m.grad_posterior(T, Y, TH, out=fused_out)
            m.posterior(T, Y, TH, with_loglik=False, out=(mean, var, None))

            def capture(fn):
                gst = torch.cuda.Stream(device=dev)
                gst.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(gst):
                    gr = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(gr, stream=gst):
                        fn()
                torch.cuda.current_stream().wait_stream(gst)
                torch.cuda.synchronize()
                return gr

            def two_calls():
                m.grad(T, Y, TH, sync=False, out=(ll, g))
                m.posterior(T, Y, TH, sync=False, with_loglik=False, out=(mean, var, None))

            graph = capture(lambda: m.grad_posterior(T, Y, TH, sync=False, out=fused_out))
            gms = max_ms(_time_calls(graph.replay, K, flush, torch))
            st2 = spingp.spingp_ws_status(m.workspace(n, spingp.WS_GRAD, dev))
            graph2 = capture(two_calls)
            sms_ = max_ms(_time_calls(graph2.replay, K, flush, torch))
            fl, inst = GRAD_POSTERIOR_EXEC_PER_STEP[name]
            rate = n / (gms * 1e-3)
            entry["graph_grad_posterior"] = {
                "value": world * rate, "unit": "steps/s", "ms_per_step": gms, "captured_graph": True,
                "roofline": {"bound": "alu", "kernel": "whole call", "unit": "TFLOP/s", "peak": fp64_tflops,
                             "achieved": fl * rate / 1e12, "frac": fl * rate / 1e12 / fp64_tflops,
                             "pipe_frac": inst * rate / (fp64_tflops * 1e12 / 2.0), "flops_per_step": fl,
                             "fp64_inst_per_step": inst,
                             "peak_kind": "measured FP64 FMA probe (spingp_probe_fp64)"},
                "status": st2, "what": "spingp_grad_posterior (ll, gradient, mean and variance), one graph",
                "gpu_launches_per_step": spingp.spingp_launch_count(m.h, n, spingp.WS_GRAD),
                "separate_calls": {"ms_per_step": sms_, "what": "spingp_grad then spingp_posterior, one graph",
                                   "gpu_launches_per_step": spingp.spingp_launch_count(m.h, n, spingp.WS_GRAD)
                                   + spingp.spingp_launch_count(m.h, n, spingp.WS_POSTERIOR)}}
            del graph, graph2, mean, var
        if not args.no_cpu_baseline and world == 1:
            smp = oracle_sample[name]
            rate, _ = oracle_rate(s, smp)
            entry["cpu_baseline"] = {"value": rate, "unit": "steps/s", "cores": 1, "kind": "oracle",
                                     "sample": "first %d of %d steps, sequential C oracle, 1 host thread" % (smp, n)}
        res[name] = entry
        del T, Y, TH, m
        torch.cuda.empty_cache()
    # the batch (this rank's shard of whole series)
    s = synth.batched()
    n_all = len(s.t)
    if world > 1:
        mine = shard.lpt_shard(np.diff(s.extra["offsets"]), world)[rank]
        loc, tt, yy, thl = shard.local_batch(s.extra["offsets"], s.t, s.y, s.extra["thetas"], mine)
        s.t, s.y, s.theta = tt, yy, thl.reshape(-1).copy()
        s.extra = dict(offsets=loc, thetas=thl)
    off = torch.tensor(s.extra["offsets"], dtype=torch.int64, device=dev)
    T, Y = torch.tensor(s.t, device=dev), torch.tensor(s.y, device=dev)
    TH = torch.tensor(s.theta, device=dev)
    m = spingp.Model("matern52")
    bt = spingp.Batch(m, off, T, Y)
    B = bt.n_series
    ll = torch.empty(B, dtype=torch.float64, device=dev)
    g = torch.empty(3 * B, dtype=torch.float64, device=dev)
    autotune.tune_batch(bt, TH, spingp.WS_GRAD)
    for _ in range(3):
        bt.grad(TH, out=(ll, g))
    # the same call issued eagerly (the binding's host work and the launches
    # on the stream every call) ...
    ems = max_ms(_time_calls(lambda: bt.grad(TH, sync=False, out=(ll, g)), K, flush, torch))
    # ... and captured once into a CUDA graph and replayed (no host work per call)
    stream = torch.cuda.Stream(device=dev)
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            bt.grad(TH, sync=False, out=(ll, g))
    torch.cuda.current_stream().wait_stream(stream)
    ms = max_ms(_time_calls(graph.replay, K, flush, torch))
    n_total = len(s.t)
    nl = spingp.spingp_launch_count_batched(m.h, B, n_total, spingp.WS_GRAD)
    entry = {"value": n_all / (ms * 1e-3), "unit": "steps/s", "ms_per_step": ms, "n_series": 4096,
             "n_total": n_all, "b": 3, "captured_graph": True, "scaling": "strong", "y": Y_KIND,
             "chunk_len": m.chunk_len(n_total), "chunk_len_autotuned": True,
             "gpu_launches_per_step": nl,
             "eager": {"ms_per_step": ems, "value": n_all / (ems * 1e-3), "unit": "steps/s",
                       "graph_saving_ms": ems - ms, "graph_saving_frac": (ems - ms) / ems, "launches": nl}}
    roof = {"bound": "alu", "kernel": "whole call", "peak": fp64_tflops, "unit": "TFLOP/s",
            "peak_kind": "measured FP64 FMA probe (spingp_probe_fp64)"}
    roof.update(_algorithmic("batched_4096", n_all / (ms * 1e-3), fp64_tflops))
    ex = WORKLOAD_EXEC_PER_STEP.get("batched_4096")
    if ex is not None:
        fl, inst = ex
        roof.update({"achieved": fl * n_all / (ms * 1e-3) / 1e12, "frac": fl * n_all / (ms * 1e-3) / 1e12 / fp64_tflops,
                     "pipe_frac": inst * n_all / (ms * 1e-3) / (fp64_tflops * 1e12 / 2.0),
                     "flops_per_step": fl, "fp64_inst_per_step": inst})
    entry["roofline"] = roof
    if not args.no_comparator:
        # plain GPU form: per series, the forward kernel at theta and theta +- h e_p
        h = 1e-5
        offs = s.extra["offsets"]
        fwd = spingp.Model("matern52")
        thetas = torch.tensor(s.extra["thetas"], device=dev)
        pert = [thetas.clone()]
        for p in range(3):
            for sgn in (1.0, -1.0):
                v = thetas.clone()
                v[:, p] *= 1.0 + sgn * h
                pert.append(v)
        outs = torch.empty(len(pert), B, dtype=torch.float64, device=dev)
        views = [(T[offs[i]:offs[i + 1]], Y[offs[i]:offs[i + 1]]) for i in range(B)]
        pth = [[v[i].contiguous() for i in range(B)] for v in pert]

        def fd_step():
            for q in range(len(pert)):
                for i in range(B):
                    fwd.loglik(views[i][0], views[i][1], pth[q][i], sync=False, out=outs[q, i:i + 1])

        # workspaces sized once per length before timing
        for i in sorted(range(B), key=lambda i: -(offs[i + 1] - offs[i]))[:1]:
            fwd.loglik(views[i][0], views[i][1], pth[0][i])
        cms = max_ms(_time_calls(fd_step, 1, flush, torch))
        entry["comparator"] = {"kind": "forward kernel x 7 per series, one launch sequence per series",
                               "value": n_all / (cms * 1e-3), "unit": "steps/s", "ms_per_step": cms,
                               "speedup_of_batched_adjoint": cms / ms}
    if not args.no_cpu_baseline and world == 1:
        entry["cpu_baseline"] = batched_oracle_rate(s)
    res["batched_4096"] = entry
    return res


def batched_oracle_rate(s, n_series=1024):
    """The oracle over the batch's first n_series series, one series per task,
    on every host core (the C oracle runs with the interpreter lock released,
    so threads run in parallel): steps/s over the wall time."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import seq
    offs, th = s.extra["offsets"], s.extra["thetas"]
    k = min(n_series, len(offs) - 1)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    seq.grad("matern52", th[0], s.t[offs[0]:offs[0] + 100], s.y[offs[0]:offs[0] + 100])

    def one(i):
        seq.grad("matern52", th[i], s.t[offs[i]:offs[i + 1]], s.y[offs[i]:offs[i + 1]])

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(one, range(k)))
    sec = time.perf_counter() - t0
    steps = int(offs[k] - offs[0])
    return {"value": steps / sec, "unit": "steps/s", "cores": cores, "kind": "oracle",
            "sample": "first %d of %d series (%d steps), sequential C oracle per series, %d threads" % (
                k, len(offs) - 1, steps, cores)}


# Whole-call FP64 work per unit of the rows built beyond the hot path (ncu
# captures of each row's kernels; the b = 12 EQ and lag-one rows from their
# per-step kernels only): flops = 2 DFMA + DADD + DMUL thread
# instructions; instructions = everything the FP64 pipe executed.  Units:
# steps, or nodes for the BTD solver; the batched SCG's gradient evaluations
# use the chain kernels' counts above.
NEXT_FLOPS_PER_UNIT = {"prediction_n4m": 344.2, "literal_n1m": 2157.0, "btd_solve_n1m": 821.6,
                       "eq_b12_n1m": 21120.6, "scg_batch_4096": 171.5 + 231.2,
                       "posterior_lag1_n4m": 171.5 + 224.1}
NEXT_FP64_INST_PER_UNIT = {"prediction_n4m": 226.0, "literal_n1m": 1485.5, "btd_solve_n1m": 520.0,
                           "eq_b12_n1m": 13421.2, "scg_batch_4096": 107.1 + 141.6,
                           "posterior_lag1_n4m": 107.1 + 143.5}


def _next_roofline(key, units_per_s, fp64_tflops):
    """FP64 roofline of a whole call: achieved TFLOP/s against the measured
    FMA probe, and the FP64-pipe instruction fraction (None where the counts
    were not taken for the current kernels)."""
    fl, inst = NEXT_FLOPS_PER_UNIT[key], NEXT_FP64_INST_PER_UNIT[key]
    if fl is None or inst is None:
        return None
    ach = fl * units_per_s / 1e12
    return {"bound": "alu", "kernel": "whole call", "achieved": ach, "peak": fp64_tflops, "unit": "TFLOP/s",
            "frac": ach / fp64_tflops, "pipe_frac": inst * units_per_s / (fp64_tflops * 1e12 / 2.0),
            "flops_per_unit": fl, "fp64_inst_per_unit": inst, "traffic": None,
            "peak_kind": "measured FP64 FMA probe (spingp_probe_fp64)"}


def _oracle_seconds(fn, reps=1):
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        times.append(time.perf_counter() - t0)
    return float(np.median(times))


def next_rows(args, dev, flush, fp64_tflops):
    """The rows built beyond the hot path, each timed on the GPU (device time,
    L2 flushed before each call) with the oracle timed beside it on a bounded
    sample on one host thread:
      prediction_n4m  posterior of the N = 2^22, b = 3 series with 10 % of its
                      observations missing (test points, Eqs. mean4-mean6)
      posterior_lag1_n4m  the posterior of the same series with the first
                      off-diagonal of the selected inverse (Sec. 3.1)
      literal_n1m     the method as written: Theorem-1 assembly, block cyclic
                      reduction with selected inverse, Eq. dd1 gradient; b = 3,
                      N = 2^20 well-separated times (oracle: its Kalman form)
      btd_solve_n1m   the general BTD solver with selected inverse, b = 3,
                      2^20 nodes (oracle: the sequential block algorithm)
      eq_b12_n1m      the oracle rate for the b = 12 EQ model (its GPU rate is
                      in workloads)
      scg_batch_4096  5 SCG iterations on the 4096-series batch (2 gradient
                      evaluations per iteration plus 2)"""
    import torch

    from oracle import btd, scg, seq
    from paper_1610_08035_gb300 import spingp, synth

    K = 3
    res = {}
    # ---- prediction: the headline series with 10 % missing observations
    s = synth.single(WORKLOAD)
    n = len(s.t)
    rng = np.random.default_rng(11)
    y = s.y.copy()
    y[rng.random(n) < 0.1] = np.nan
    T, Y, TH = (torch.tensor(a, device=dev) for a in (s.t, y, s.theta))
    m = spingp.Model(s.spec)
    m.posterior(T, Y, TH, missing=True)
    ms = _time_calls(lambda: m.posterior(T, Y, TH, sync=False, missing=True), K, flush, torch)
    smp = 1 << 18
    osec = _oracle_seconds(lambda: seq.smoother(s.spec, s.theta, s.t[:smp], y[:smp]))
    res["prediction_n4m"] = {"value": n / (ms * 1e-3), "unit": "steps/s", "ms_per_step": ms, "n": n,
                             "chunk_len": m.chunk_len(n),
                             "roofline": _next_roofline("prediction_n4m", n / (ms * 1e-3), fp64_tflops),
                             "missing_fraction": 0.1, "gpu_launches_per_step":
                                 spingp.spingp_launch_count(m.h, n, spingp.WS_POSTERIOR),
                             "oracle": {"value": smp / osec, "unit": "steps/s", "cores": 1,
                                        "sample": "first %d steps, sequential C smoother" % smp}}
    # the same prediction through spingp_predict: the observed 90 % of the
    # steps and the other 10 % as test times handed over in random order
    # (sorted, merged and gathered on the device around the posterior pass)
    obs = ~np.isnan(y)
    ts = s.t[~obs][rng.permutation(int((~obs).sum()))]
    TO, YO, TS = (torch.tensor(a, device=dev) for a in (s.t[obs], s.y[obs], ts))
    m.predict(TO, YO, TH, TS)
    pms = _time_calls(lambda: m.predict(TO, YO, TH, TS, sync=False), K, flush, torch)
    res["prediction_n4m"]["predict_call"] = {
        "value": n / (pms * 1e-3), "unit": "steps/s (observed + test)", "ms_per_call": pms,
        "n_observed": int(obs.sum()), "n_test": len(ts), "test_order": "random",
        "what": "spingp_predict: device merge sort of the test times, merge, posterior, gather"}
    del T, Y, TH, m, TO, YO, TS
    torch.cuda.empty_cache()
    # ---- the posterior with the first off-diagonal of the selected inverse
    s = synth.single(WORKLOAD)
    n = len(s.t)
    T, Y, TH = (torch.tensor(a, device=dev) for a in (s.t, s.y, s.theta))
    m = spingp.Model(s.spec)
    m.posterior_lag1(T, Y, TH)
    ms = _time_calls(lambda: m.posterior_lag1(T, Y, TH, sync=False), K, flush, torch)
    smp = 1 << 18
    osec = _oracle_seconds(lambda: seq.smoother(s.spec, s.theta, s.t[:smp], s.y[:smp], blocks=True))
    res["posterior_lag1_n4m"] = {"value": n / (ms * 1e-3), "unit": "steps/s", "ms_per_step": ms, "n": n,
                                 "chunk_len": m.chunk_len(n),
                                 "roofline": _next_roofline("posterior_lag1_n4m", n / (ms * 1e-3), fp64_tflops),
                                 "gpu_launches_per_step": spingp.spingp_launch_count(m.h, n, spingp.WS_POSTERIOR),
                                 "oracle": {"value": smp / osec, "unit": "steps/s", "cores": 1,
                                            "sample": "first %d steps, sequential C RTS smoother with its "
                                                      "lag-one blocks" % smp}}
    del T, Y, TH, m
    torch.cuda.empty_cache()
    # ---- the method as written
    n = 1 << 20
    rng = np.random.default_rng(12)
    t = synth.separated_times(n, 0.5, rng)
    y = synth.two_sinusoids(t, 0.5, 2.0, 0.05, rng)
    th = np.array([0.5, 2.0, 0.05])
    T, Y, TH = (torch.tensor(a, device=dev) for a in (t, y, th))
    m = spingp.Model("matern52")
    m.literal(T, Y, TH, what=spingp.WS_GRAD)
    ms = _time_calls(lambda: m.literal(T, Y, TH, what=spingp.WS_GRAD, sync=False), K, flush, torch)
    smp = 1 << 18
    osec = _oracle_seconds(lambda: seq.grad("matern52", th, t[:smp], y[:smp]))
    res["literal_n1m"] = {"value": n / (ms * 1e-3), "unit": "steps/s", "ms_per_step": ms, "n": n, "b": 3,
                          "roofline": _next_roofline("literal_n1m", n / (ms * 1e-3), fp64_tflops),
                          "gpu_launches_per_step": spingp.spingp_literal_launch_count(n),
                          "oracle": {"value": smp / osec, "unit": "steps/s", "cores": 1,
                                     "sample": "first %d steps, sequential C oracle (Kalman form of the same "
                                               "log-likelihood and gradient)" % smp}}
    del T, Y, TH, m
    # ---- the general BTD solver
    D, O, r = synth.random_spd_btd(n, 3, seed=13)
    Dt, Ot, rt = (torch.tensor(a, device=dev) for a in (D, O, r))
    spingp.btd_solve(Dt, Ot, rt)
    ms = _time_calls(lambda: spingp.btd_solve(Dt, Ot, rt, sync=False), K, flush, torch)
    smp = 1 << 14
    osec = _oracle_seconds(lambda: btd.thomas(D[:smp], O[:smp - 1], r[:smp]))
    res["btd_solve_n1m"] = {"value": n / (ms * 1e-3), "unit": "nodes/s", "ms_per_step": ms, "n": n, "b": 3,
                            "roofline": _next_roofline("btd_solve_n1m", n / (ms * 1e-3), fp64_tflops),
                            "gpu_launches_per_step": spingp.spingp_btd_launch_count(n),
                            "oracle": {"value": smp / osec, "unit": "nodes/s", "cores": 1,
                                       "sample": "first %d nodes, sequential block LDL^T and selected inverse "
                                                 "(NumPy, one block per step)" % smp}}
    del Dt, Ot, rt
    torch.cuda.empty_cache()
    # ---- the b = 12 EQ model: oracle rate
    s = synth.single("m32_eq10_n1m")
    smp = 1 << 11
    osec = _oracle_seconds(lambda: seq.grad(s.spec, s.theta, s.t[:smp], s.y[:smp]))
    res["eq_b12_n1m"] = {"oracle": {"value": smp / osec, "unit": "steps/s", "cores": 1,
                                    "sample": "first %d steps, sequential C oracle" % smp}}
    # ---- batched SCG
    s = synth.batched()
    off = torch.tensor(s.extra["offsets"], dtype=torch.int64, device=dev)
    T, Y = torch.tensor(s.t, device=dev), torch.tensor(s.y, device=dev)
    bt = spingp.Batch(spingp.Model("matern52"), off, T, Y)
    S = bt.n_series
    th0 = torch.tensor(np.tile([1.0, 1.0, 0.2], (S, 1)), device=dev)
    iters = 5
    bt.optimize(th0, iterations=1)
    ms = _time_calls(lambda: bt.optimize(th0, iterations=iters, sync=False), 1, flush, torch)
    evals = 2 * iters + 2
    offs = s.extra["offsets"]
    nser = 8
    nst = int(offs[nser])
    osec = _oracle_seconds(lambda: [scg.scg(scg.gp_objective("matern52", s.t[offs[i]:offs[i + 1]],
                                                             s.y[offs[i]:offs[i + 1]], seq.grad),
                                            np.log([1.0, 1.0, 0.2]), iters) for i in range(nser)])
    res["scg_batch_4096"] = {"value": evals * len(s.t) / (ms * 1e-3), "unit": "steps/s (gradient evaluations)",
                             "ms_per_call": ms, "iterations": iters, "n_series": S, "n_total": len(s.t),
                             "series_iterations_per_s": S * iters / (ms * 1e-3),
                             "roofline": _next_roofline("scg_batch_4096", evals * len(s.t) / (ms * 1e-3),
                                                        fp64_tflops),
                             "oracle": {"value": evals * nst / osec, "unit": "steps/s (gradient evaluations)",
                                        "cores": 1, "sample": "the first %d series (%d steps), oracle SCG on the "
                                                              "sequential C oracle" % (nser, nst)}}
    return res


# ---------------------------------------------------------------- one workload alone (profiling)

def run_only(args):
    """The gradient call of one workload (with --call grad_posterior, the
    fused gradient + posterior call), --warmup untimed and --steps timed
    calls (L2 flushed before each), at the workload's size or --n steps
    (--n series for the batch): a command for ncu to capture."""
    import torch

    from paper_1610_08035_gb300 import spingp, synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    if args.only == "batched_4096":
        s = synth.batched(n_series=args.n or 4096)
        off = torch.tensor(s.extra["offsets"], dtype=torch.int64, device=dev)
        m = spingp.Model("matern52")
        bt = spingp.Batch(m, off, torch.tensor(s.t, device=dev), torch.tensor(s.y, device=dev))
        TH = torch.tensor(s.theta, device=dev)
        ll = torch.empty(bt.n_series, dtype=torch.float64, device=dev)
        g = torch.empty(3 * bt.n_series, dtype=torch.float64, device=dev)
        call = lambda: bt.grad(TH, sync=False, out=(ll, g))   # noqa: E731
        units, what = len(s.t), "steps (%d series)" % bt.n_series
    else:
        s = synth.single(args.only, n=args.n or None, seed=1 if args.only == WORKLOAD else None)
        T, Y, TH = (torch.tensor(a, device=dev) for a in (s.t, s.y, s.theta))
        m = spingp.Model(s.spec)
        ll = torch.empty(1, dtype=torch.float64, device=dev)
        g = torch.empty(m.num_params, dtype=torch.float64, device=dev)
        if args.call == "grad_posterior":
            mean = torch.empty(len(s.t), dtype=torch.float64, device=dev)
            var = torch.empty(len(s.t), dtype=torch.float64, device=dev)
            call = lambda: m.grad_posterior(T, Y, TH, sync=False, out=(ll, g, mean, var, None))   # noqa: E731
        else:
            call = lambda: m.grad(T, Y, TH, sync=False, out=(ll, g))   # noqa: E731
        units, what = len(s.t), "steps"
    if args.chunk > 0:
        m.set_chunk_len(args.chunk)
    for _ in range(max(args.warmup, 0)):
        call()
    torch.cuda.synchronize()
    ms = _time_calls(call, max(args.steps, 1), flush, torch)
    print(json.dumps({"only": args.only, "call": args.call, "units": units, "what": what, "ms_per_call": ms,
                      "value": units / (ms * 1e-3), "unit": "steps/s"}), flush=True)


# ---------------------------------------------------------------- the CUDA path

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.only:
        run_only(args)
        return
    import torch
    import torch.distributed as dist

    from paper_1610_08035_gb300 import autotune, spingp, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1 or args.split:
        dist.init_process_group("nccl", device_id=dev)
        main_split(args, world, rank, local, dev)
        dist.destroy_process_group()
        return

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    s = synth.single(WORKLOAD, n=args.n or None, seed=1)
    n = len(s.t)
    T = torch.tensor(s.t, device=dev)
    Y = torch.tensor(s.y, device=dev)
    TH = torch.tensor(s.theta, device=dev)
    model = spingp.Model(s.spec)
    if args.chunk >= 0:
        model.set_chunk_len(args.chunk)
    else:
        autotune.tune(model, T, Y, TH, spingp.WS_GRAD)
    L = model.chunk_len(n)
    ll = torch.empty(1, dtype=torch.float64, device=dev)
    g = torch.empty(3, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    for _ in range(max(args.warmup, 0)):
        model.grad(T, Y, TH, sync=True, out=(ll, g))
    fp64_tflops = spingp.spingp_probe_fp64(dev)
    # context for the design choice: the FP64 tensor-core instruction's rate on this device
    fp64_mma_tflops = spingp.spingp_probe_fp64_tensor(dev)

    # ---- device-timed region
    K = args.steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    spingp.spingp_profile_enable(model.h, True)
    spingp.spingp_profile_read(model.h)
    barrier()
    clocks = ClockSampler(local, enabled=not args.no_clocks)
    time.sleep(0.3 if not args.no_clocks else 0.0)
    w0 = time.time()
    for k in range(K):
        flush.fill_(k & 0xFF)                        # 256 MiB write: L2 (~126 MiB) flushed, untimed
        evs[k][0].record()
        model.grad(T, Y, TH, sync=False, out=(ll, g))
        evs[k][1].record()
    barrier()
    w1 = time.time()
    clk = clocks.stop(w0, w1)
    stages, calls = spingp.spingp_profile_read(model.h)
    spingp.spingp_profile_enable(model.h, False)
    st = spingp.spingp_ws_status(model.workspace(n, spingp.WS_GRAD, dev))
    if st != spingp.OK:
        raise spingp.SpinGPError(st, "benchmark step")
    ms_steps = [a.elapsed_time(b) for a, b in evs]
    total_ms = float(np.sum(ms_steps))
    if world > 1:
        tt = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    ms_per_step = total_ms / K
    value = world * n / (ms_per_step * 1e-3)

    # ---- roofline of the dominant stage (live stage times over the timed region)
    stage_ms = {k: v / max(calls, 1) for k, v in stages.items()}
    dom = max(stage_ms, key=stage_ms.get)
    flops = FLOPS_PER_STEP.get(dom)
    achieved = flops * n / (stage_ms[dom] * 1e-3) / 1e12 if flops else None
    traffic = DRAM_BYTES_PER_STEP.get(dom)
    inst = FP64_INST_PER_STEP.get(dom)
    roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fp64_tflops, "unit": "TFLOP/s",
            "frac": achieved / fp64_tflops if achieved else None,
            "traffic": traffic * n if traffic else None,
            "peak_kind": "measured FP64 FMA probe (spingp_probe_fp64); nominal %.3f" % FP64_NOMINAL_TFLOPS,
            "ms_per_launch": stage_ms[dom],
            # the FP64 pipe's instruction rate: every FP64 instruction (not only
            # FMAs) takes a pipe slot; peak = probe FMA rate = TFLOP/s / 2
            "fp64_inst_per_s": inst * n / (stage_ms[dom] * 1e-3) if inst else None,
            "pipe_frac": inst * n / (stage_ms[dom] * 1e-3) / (fp64_tflops * 1e12 / 2.0) if inst else None,
            "fp64_tensor_tflops": fp64_mma_tflops}
    roof.update(_algorithmic(WORKLOAD, n / (ms_per_step * 1e-3), fp64_tflops))
    hbm = {"algorithmic_bytes_per_step": ALGO_BYTES_PER_STEP,
           "achieved_gbs": ALGO_BYTES_PER_STEP * n / (ms_per_step * 1e-3) / 1e9}
    if traffic:
        # the dominant kernel's measured DRAM bytes (ncu, per step x N) over its
        # live launch time: the bandwidth it actually draws, beside the
        # algorithmic figure
        hbm["dominant_kernel_dram_gbs"] = traffic * n / (stage_ms[dom] * 1e-3) / 1e9
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        with open(peaks_path) as f:
            hbm_peak = json.load(f).get("hbm_gbs")
        hbm["peak_gbs"] = hbm_peak
        hbm["frac"] = hbm["achieved_gbs"] / hbm_peak if hbm_peak else None
        if traffic and hbm_peak:
            hbm["dominant_kernel_dram_frac"] = hbm["dominant_kernel_dram_gbs"] / hbm_peak
        hbm["peak_kind"] = "measured (MEASURED_PEAKS.json)"
    else:
        hbm["peak_gbs"] = 6800.0
        hbm["frac"] = hbm["achieved_gbs"] / 6800.0
        hbm["peak_kind"] = "fallback"

    out = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
           "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": n, "b": 3, "model": "matern52",
                      "theta": [float(v) for v in s.theta], "parallelism": "single", "y": Y_KIND,
                      "l2": "flushed between timed iterations (256 MiB write, untimed)"},
           "launch": {"chunk_len": L},
           "roofline": roof, "hbm_roofline": hbm, "stages_ms_per_call": stage_ms,
           "gpu_launches": spingp.spingp_launch_count(model.h, n, spingp.WS_GRAD) * K,
           "clocks": clk}

    # ---- the same call captured once in a CUDA graph: the median of at least
    # 20 replays, each timed alone with L2 flushed (untimed) before it
    gstream = torch.cuda.Stream(device=dev)
    gstream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(gstream):
        model.grad(T, Y, TH, sync=False, out=(ll, g))
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gstream):
            model.grad(T, Y, TH, sync=False, out=(ll, g))
    torch.cuda.current_stream().wait_stream(gstream)
    torch.cuda.synchronize()
    reps = max(K, 20)
    gms = []
    for k in range(reps):
        flush.fill_(k & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        torch.cuda.synchronize()
        gms.append(e0.elapsed_time(e1))
    st = spingp.spingp_ws_status(model.workspace(n, spingp.WS_GRAD, dev))
    if st != spingp.OK:
        raise spingp.SpinGPError(st, "graph replay")
    gmed = float(np.median(gms))
    out["graph_replay"] = {"value": world * n / (gmed * 1e-3), "unit": "steps/s", "ms_median": gmed,
                           "replays": reps, "gpu_launches_per_replay": spingp.spingp_launch_count(
                               model.h, n, spingp.WS_GRAD)}
    del graph

    # ---- end to end through the public API: pinned host buffers in (the
    # library overlaps their copy with the elimination), results to the host,
    # every step
    if not args.no_e2e:
        th = torch.from_numpy(s.t).pin_memory()
        yh = torch.from_numpy(s.y).pin_memory()
        thh = torch.from_numpy(s.theta).pin_memory()
        ll_h = torch.empty(1, dtype=torch.float64).pin_memory()
        g_h = torch.empty(3, dtype=torch.float64).pin_memory()
        model.grad_host(th, yh, thh, out=(ll_h, g_h))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record()
        for _ in range(K):
            model.grad_host(th, yh, thh, sync=False, out=(ll_h, g_h))
        e1.record()
        barrier()
        e2e_ms = e0.elapsed_time(e1) / K
        if world > 1:
            tt = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e2e_ms = float(tt.item())
        out["e2e"] = {"value": world * n / (e2e_ms * 1e-3), "unit": "steps/s", "h2d_bytes_per_step": 16 * n + 24,
                      "d2h_bytes_per_step": 32, "ms_per_step": e2e_ms, "api": "spingp_grad_host"}

    # ---- the plain GPU form: forward kernel (2P+1) times, central differences
    if not args.no_comparator:
        P = 3
        h = 1e-5
        thetas = [TH.clone()]
        for p in range(P):
            for sgn in (1.0, -1.0):
                v = TH.clone()
                v[p] = v[p] * (1.0 + sgn * h)
                thetas.append(v)
        lls = torch.empty(len(thetas), dtype=torch.float64, device=dev)
        fwd = spingp.Model(s.spec, chunk_len=L)
        for v in thetas:
            fwd.loglik(T, Y, v, sync=True)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        comp_ms = 0.0
        for k in range(K):
            flush.fill_(k & 0xFF)
            c0.record()
            for i, v in enumerate(thetas):
                fwd.loglik(T, Y, v, sync=False, out=lls[i:i + 1])
            c1.record()
            torch.cuda.synchronize()
            comp_ms += c0.elapsed_time(c1)
        comp_ms /= K
        lv = lls.cpu().numpy()
        fd = np.array([(lv[1 + 2 * p] - lv[2 + 2 * p]) / (2 * h * s.theta[p]) for p in range(P)])
        gad = g.cpu().numpy()
        out["comparator"] = {"kind": "forward kernel x %d (central differences, one launch sequence each)" % len(thetas),
                             "value": world * n / (comp_ms * 1e-3), "unit": "steps/s", "ms_per_step": comp_ms,
                             "speedup_of_adjoint": comp_ms / ms_per_step,
                             "fd_grad_rel_err": float(np.max(np.abs(fd - gad) / np.abs(gad)))}

    # ---- secondary workloads: the other configurations of the same path
    if not args.no_extra and not args.n:
        out["workloads"] = extra_workloads(args, dev, flush, world, rank, fp64_tflops)

    # ---- the rows built beyond the hot path, each with the oracle beside it
    if not args.no_next and not args.n and world == 1:
        out["next"] = next_rows(args, dev, flush, fp64_tflops)
        if "m32_eq10_n1m" in out.get("workloads", {}):
            w = out["workloads"]["m32_eq10_n1m"]
            out["next"]["eq_b12_n1m"].update({"value": w["value"], "unit": "steps/s", "ms_per_step": w["ms_per_step"],
                                               "roofline": _next_roofline("eq_b12_n1m", w["value"], fp64_tflops)})

    # ---- the oracle on the host cores (rank 0, single GPU only)
    if not args.no_cpu_baseline and world == 1:
        sample = min(n, 1 << 20)
        rate, _ = oracle_rate(s, sample)
        out["cpu_baseline"] = {"value": rate, "unit": "steps/s", "cores": 1, "kind": "oracle",
                               "sample": "first %d of %d steps, sequential C oracle (Kalman filter + two-filter "
                                         "adjoint), 1 host thread" % (sample, n)}
        # context: the dense oracle (Cholesky of the N x N covariance) on the
        # N = 1000 Matern-3/2 workload
        from oracle import dense
        s1 = synth.single("matern32_n1000")
        dsec = _oracle_seconds(lambda: dense.grad(s1.spec, s1.theta, s1.t, s1.y), reps=3)
        out["cpu_baseline"]["dense_oracle_n1000"] = {"value": len(s1.t) / dsec, "unit": "steps/s",
                                                     "seconds": dsec, "workload": "matern32_n1000"}

    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main_split(args, world, rank, local, dev):
    """N > 1 GPUs: the one series of the headline workload split across the
    ranks (strong scaling).  Rank r holds the r-th contiguous range; a step is
    the range's reduction to one element, one all-gather of the G elements,
    the range's finish from them and one all-reduce of (ll, gradient)
    (shard.grad_split_series).  The value counts the series' steps once."""
    import torch
    import torch.distributed as dist

    from paper_1610_08035_gb300 import autotune, shard, spingp, synth

    def barrier():
        dist.barrier()
        torch.cuda.synchronize()

    s = synth.single(WORKLOAD, n=args.n or None, seed=1)     # the same series on every rank
    n = len(s.t)
    a, b = shard.range_split(n, world)[rank]
    t_prev = None if rank == 0 else float(s.t[a - 1])
    T = torch.tensor(s.t[a:b], device=dev)
    Y = torch.tensor(s.y[a:b], device=dev)
    TH = torch.tensor(s.theta, device=dev)
    model = spingp.Model(s.spec)
    if args.chunk >= 0:
        model.set_chunk_len(args.chunk)
    else:
        autotune.tune(model, T, Y, TH, spingp.WS_GRAD)
    L = model.chunk_len(b - a)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(max(args.warmup, 0)):
        ll, g = shard.grad_split_series(model, T, Y, TH, t_prev)
    fp64_tflops = spingp.spingp_probe_fp64(dev)
    torch.cuda.synchronize()

    K = args.steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    barrier()
    clocks = ClockSampler(local, enabled=not args.no_clocks)
    time.sleep(0.3 if not args.no_clocks else 0.0)
    w0 = time.time()
    for k in range(K):
        flush.fill_(k & 0xFF)                        # 256 MiB write: L2 flushed, untimed
        evs[k][0].record()
        ll, g = shard.grad_split_series(model, T, Y, TH, t_prev, sync=False)
        evs[k][1].record()
    barrier()
    w1 = time.time()
    clk = clocks.stop(w0, w1)
    st = spingp.spingp_ws_status(model.workspace(b - a, spingp.WS_GRAD, dev, purpose="segment"))
    if st != spingp.OK:
        raise spingp.SpinGPError(st, "benchmark step")
    tt = torch.tensor([float(np.sum([e0.elapsed_time(e1) for e0, e1 in evs]))], dtype=torch.float64, device=dev)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ms_per_step = float(tt.item()) / K
    value = n / (ms_per_step * 1e-3)

    # per GPU: the whole step's FP64 work over its range
    flops = sum(FLOPS_PER_STEP.values()) * (b - a)
    inst = sum(FP64_INST_PER_STEP.values()) * (b - a)
    achieved = flops / (ms_per_step * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": "whole step per GPU (split series)", "achieved": achieved, "peak": fp64_tflops,
            "unit": "TFLOP/s", "frac": achieved / fp64_tflops, "traffic": None,
            "peak_kind": "measured FP64 FMA probe (spingp_probe_fp64)",
            "pipe_frac": inst / (ms_per_step * 1e-3) / (fp64_tflops * 1e12 / 2.0)}
    out = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
           "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": n, "b": 3, "model": "matern52",
                      "theta": [float(v) for v in s.theta], "parallelism": "series split over %d ranks" % world,
                      "y": Y_KIND, "l2": "flushed between timed iterations (256 MiB write, untimed)"},
           "launch": {"chunk_len": L},
           "roofline": roof,
           "hbm_roofline": {"algorithmic_bytes_per_step": ALGO_BYTES_PER_STEP,
                            "achieved_gbs": ALGO_BYTES_PER_STEP * n / (ms_per_step * 1e-3) / 1e9},
           "gpu_launches": spingp.spingp_segment_launch_count(model.h, b - a) * K,
           "clocks": clk}

    # end to end: the range's inputs from pinned host memory every step, the
    # result read back to the host
    if not args.no_e2e:
        th_h = torch.from_numpy(s.t[a:b].copy()).pin_memory()
        yh_h = torch.from_numpy(s.y[a:b].copy()).pin_memory()
        ll_h = torch.empty(1, dtype=torch.float64).pin_memory()
        g_h = torch.empty(3, dtype=torch.float64).pin_memory()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record()
        for _ in range(K):
            T.copy_(th_h, non_blocking=True)
            Y.copy_(yh_h, non_blocking=True)
            ll, g = shard.grad_split_series(model, T, Y, TH, t_prev, sync=False)
            ll_h.copy_(ll, non_blocking=True)
            g_h.copy_(g, non_blocking=True)
        e1.record()
        barrier()
        tt = torch.tensor([e0.elapsed_time(e1) / K], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_ms = float(tt.item())
        # bytes of the whole job (every rank copies its own range in, its share out)
        out["e2e"] = {"value": n / (e2e_ms * 1e-3), "unit": "steps/s", "h2d_bytes_per_step": 16 * n,
                      "d2h_bytes_per_step": 32 * world, "ms_per_step": e2e_ms,
                      "api": "spingp_segment_reduce + spingp_segment_grad per rank, NCCL all-gather and all-reduce"}
    # the other configurations: the batch sharded by series, the single series as replicas
    if not args.no_extra and not args.n:
        out["workloads"] = extra_workloads(args, dev, flush, world, rank, fp64_tflops)
    if rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
