"""Benchmark: Hawkes log-likelihood + location-gradient evaluations per second.

Workload: the N = 100,000, D = 2 synthetic data set shaped like the paper's
large gunfire-style workload (50 km square, 5 years, offspring mean 0.6,
decay 0.2/day, offspring sd 50 m, 100 m coarsening).  One step is one full
evaluation of ell (Eq. (1)) and d ell / d X (Appendix A) through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the
host cores instead (a bounded sample of the same workload, extrapolated to
N = 100,000 by the N^2 pair count).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "loglik+location-gradient evals/s and pairs/s at N=1e5, mixed vs FP64 GPU"
UNIT = "evals/s"
MAX_SM_MHZ_NOMINAL = 2070.0  # GB300 maximum SM clock
CPU_SAMPLE_N = 20_000        # events of the bounded CPU-oracle sample

# DRAM bytes (read + write) per launch of each pair kernel at N=1e5, D=2, from
# one ncu capture of the kernel sources whose SHA-256 (of the files in order)
# is recorded with it; reported as null once the sources have changed.
PAIR_KERNEL_SOURCES = [os.path.join(ROOT, "paper_2010_02994_gb300", "csrc", f)
                       for f in ("hk_pairs_mixed.cuh", "hk_pair_item.inc", "hk_sched.cuh")]
MEASURED_TRAFFIC = {"source_sha256": "f3711c7cd1870c43068b4ec4f38c3723e4abd943a22593de770f15267e701950",
                    "pass1_rates": 3670784, "pass2_gradient": 21906944}


def measured_traffic(kernel: str):
    import hashlib

    try:
        sha = hashlib.sha256(b"".join(open(f, "rb").read() for f in PAIR_KERNEL_SOURCES)).hexdigest()
    except OSError:
        return None
    return MEASURED_TRAFFIC.get(kernel) if sha == MEASURED_TRAFFIC["source_sha256"] else None


def pass_bound_cycles(d: int, which: str, fma_rate: float, ex2_rate: float) -> float:
    """SM cycles per unordered pair: max(FP32 ops / FMA rate, ex2 / MUFU rate),
    with the algorithmic counts of each pass (2D+9 and 4D+10 FP32 ops, two
    ex2 each; no hi/lo overhead) and the measured per-SM rates."""
    f1, f2, e1, e2 = 2 * d + 9, 4 * d + 10, 2, 2
    if which == "pass1":
        return max(f1 / fma_rate, e1 / ex2_rate)
    if which == "pass2":
        return max(f2 / fma_rate, e2 / ex2_rate)
    return max((f1 + f2) / fma_rate, (e1 + e2) / ex2_rate)


def eval_roofline(achieved_per_s: float, work_cycles: float, sms: int, clock_mhz: float, unit: str,
                  basis: str) -> dict:
    """Roofline of a whole call (trajectory, batch) against the FP32/MUFU
    bound: work_cycles is the sum over its evaluations of unordered pairs x
    SM-cycles per pair (pass_bound_cycles / bmds_bound_cycles); everything
    else the call does (sorting, finalizing, leapfrog updates) counts as
    time, not work."""
    peak = sms * clock_mhz * 1e6 / work_cycles
    return {"bound": "alu", "unit": unit, "achieved": achieved_per_s, "peak": peak, "frac": achieved_per_s / peak,
            "basis": basis}


def bmds_bound_cycles(d: int, fma_rate: float, ex2_rate: float) -> float:
    """SM cycles per unordered pair of the BMDS pair term (Eq. (4)) with its
    location and variance gradients: 4D+40 FP32 ops (difference, square,
    row and column gradient per dimension; distance, the normal tail as a
    degree-(4,5) rational, Phi, phi/Phi, log Phi, the value and sigma2
    terms) and four MUFU ops (rsqrt, ex2, rcp, lg2), no hi/lo overhead."""
    return max((4 * d + 40) / fma_rate, 4 / ex2_rate)


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines: list[str] = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)
        mhz, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(mhz)}


def dist_setup():
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, value: float, device=None) -> float:
    """The largest of every rank's value (the slowest rank's time)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    dev = device if (device is not None and dist.get_backend() == "nccl") else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_sample(n_sample: int, repeats: int = 1) -> dict:
    """Time the FP64 oracle (all host cores) on the first n_sample events of
    the workload: one full ell + grad per repeat."""
    import oracle
    import synth

    w = synth.scaled_down(synth.make_c5(), n_sample)
    cores = oracle.max_threads()
    times = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        oracle.loglik_and_grad(w.t, w.X, w.params, nthreads=cores)
        times.append(time.perf_counter() - t0)
    sec = statistics.median(times)
    pairs_per_s = float(n_sample) ** 2 / sec
    return {"sec_per_eval": sec, "pairs_per_s": pairs_per_s, "evals_per_s_at_1e5": pairs_per_s / 1e10,
            "cores": cores, "n_sample": n_sample}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, as it stands, on the host cores."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n_s = args.cpu_sample
    for _ in range(max(0, args.warmup_ref)):
        cpu_oracle_sample(n_s, 1)
    t0 = time.perf_counter()
    res = [cpu_oracle_sample(n_s, 1) for _ in range(args.steps_ref)]
    wall = time.perf_counter() - t0
    sec = statistics.median(r["sec_per_eval"] for r in res)
    value = float(n_s) ** 2 / sec / 1e10
    sample = (f"first {n_s} events (time order) of the N=1e5 D=2 workload; one full FP64 ell + grad_X per step; "
              f"evals/s at N=1e5 = measured pairs/s / 1e10")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps_ref, "warmup": args.warmup_ref, "ms_per_step": 1e3 * sec, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "c5_large_n100000_d2", "n": 100000, "d": 2, "sample_n": n_s,
                   "precision": "fp64 (CPU oracle)"},
        "pairs_per_s": float(n_s) ** 2 / sec,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": res[0]["cores"], "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line))
    return 0


def flush_l2(buf):
    buf.zero_()


def timed_calls(fn, stream, l2, reps: int = 10, warm: int = 2) -> float:
    """Median CUDA-event time (ms) of fn() on `stream`, L2 flushed before each call."""
    import torch

    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        flush_l2(l2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def bmds_workload(dev, stream, l2, fma_rate: float, ex2_rate: float, clock_mhz: float, sms: int) -> dict:
    """BMDS likelihood and gradients (Eq. (4)) on the influenza-shaped input:
    N = 4,733 cases, D = 6, block-structured Y (synth.make_bmds)."""
    import torch

    import synth
    from paper_2010_02994_gb300 import HawkesContext, hawkes_bmds_loglik_grad

    w = synth.make_bmds()
    n, d = w.X.shape
    ctx = HawkesContext(device=dev.index or 0, max_n=n, max_d=d)
    Y64 = torch.tensor(w.Y, device=dev)
    Y32 = Y64.float()
    X = torch.tensor(w.X, device=dev)
    out_t = (torch.empty((), dtype=torch.float64, device=dev), torch.empty((n, d), dtype=torch.float64, device=dev),
             torch.empty((), dtype=torch.float64, device=dev))
    res = {"workload": w.name, "n": n, "d": d}
    pairs = n * (n - 1) / 2
    bound_s = pairs * bmds_bound_cycles(d, fma_rate, ex2_rate) / (sms * clock_mhz * 1e6)
    for key, Y, prec, reps in (("mixed_y_f32", Y32, "mixed", 20), ("mixed_y_f64", Y64, "mixed", 20),
                               ("fp64", Y64, "fp64", 3)):
        m = timed_calls(lambda: hawkes_bmds_loglik_grad(ctx, Y, X, w.sigma2, prec, check=False, out=out_t),
                        stream, l2, reps=reps, warm=2)
        res[key] = {"ms_per_eval": m, "evals_per_s": 1e3 / m, "unordered_pairs_per_s": pairs / (m * 1e-3),
                    "y_bytes_per_eval": int(pairs * Y.element_size())}
        if prec == "mixed":
            res[key]["roofline"] = {"bound": "alu", "unit": "evals/s", "achieved": 1e3 / m,
                                    "peak": 1.0 / bound_s, "frac": bound_s / (m * 1e-3),
                                    "basis": (f"(4D+40)/{fma_rate:.1f} FP32 and 4/{ex2_rate:.1f} MUFU SM-cycles per "
                                              f"unordered pair at {clock_mhz:.0f} MHz, {sms} SMs (measured rates)")}
    ctx.sync_status()
    ctx.close()
    return res


def mwg_workload(dev, stream, l2) -> dict:
    """Metropolis-within-Gibbs over the locations of the gunfire-like
    workload (c2: N = 10,000, D = 2, 100 m boxes): per iteration a truncated
    normal proposal for a block of B events and the device-side MH step,
    30 iterations captured in one CUDA graph, timed with CUDA events."""
    import torch

    import synth
    from paper_2010_02994_gb300 import HawkesMwG, hawkes_loglik, HawkesContext

    w = synth.make_c2()
    t = torch.tensor(w.t, device=dev)
    X = torch.tensor(w.X, device=dev)
    lo = torch.tensor(w.box_lo, device=dev)
    hi = torch.tensor(w.box_hi, device=dev)
    iters = 30
    gen = torch.Generator(device=dev).manual_seed(12)
    res = {"workload": "c2_gunfire_like_n10000_d2", "n": w.n, "d": w.d, "iterations_per_graph": iters}
    for nb, prec in ((1, "fp64"), (32, "fp64"), (1, "mixed"), (32, "mixed")):
        s = HawkesMwG(t, X, w.params, max_block=nb, precision=prec)
        idx = torch.stack([torch.randperm(w.n, generator=gen, device=dev)[:nb] for _ in range(iters)])
        u = torch.rand((iters, nb, w.d), generator=gen, device=dev, dtype=torch.float64)
        log_u = torch.log(torch.rand(iters, generator=gen, device=dev, dtype=torch.float64))
        props = [(torch.empty((nb, w.d), dtype=torch.float64, device=dev),
                  torch.empty((), dtype=torch.float64, device=dev)) for _ in range(iters)]
        outs = [(torch.empty((), dtype=torch.float64, device=dev), torch.empty((), dtype=torch.int32, device=dev))
                for _ in range(iters)]

        def run():
            for k in range(iters):
                s.propose_box(idx[k], lo, hi, 0.02, u[k], out=props[k], check=False)
                s.step(idx[k], props[k][0], log_u[k], props[k][1], out=outs[k], check=False)

        run()
        torch.cuda.synchronize()
        s.sync_status()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                run()
        torch.cuda.synchronize()
        m = timed_calls(g.replay, stream, l2, reps=10, warm=2)
        s.sync_status()
        acc = int(sum(o[1].item() for o in outs))
        per = m / iters
        res[f"block_{nb}" + ("" if prec == "fp64" else "_mixed")] = {
                              "ms_per_iteration": per, "iterations_per_s": 1e3 / per,
                              "location_updates_per_s": nb * 1e3 / per,
                              "pair_terms_per_iteration": 3 * nb * w.n, "pair_term_precision": prec,
                              "accepted_last_replay": acc}
        s.close()
    # wildfire-like (c3: N = 5,000, circle priors of Eq. (3)): lens proposals of Eq. (6), 4 tries
    wc = synth.make_c3()
    centers_np, radii_np = synth.circle_priors(wc)
    tc, Xc = torch.tensor(wc.t, device=dev), torch.tensor(wc.X, device=dev)
    centers, radii = torch.tensor(centers_np, device=dev), torch.tensor(radii_np, device=dev)
    for nb, prec in ((1, "fp64"), (32, "fp64"), (1, "mixed"), (32, "mixed")):
        s = HawkesMwG(tc, Xc, wc.params, max_block=nb, precision=prec)
        idx = torch.stack([torch.randperm(wc.n, generator=gen, device=dev)[:nb] for _ in range(iters)])
        u = torch.rand((iters, nb, 4, 2), generator=gen, device=dev, dtype=torch.float64)
        log_u = torch.log(torch.rand(iters, generator=gen, device=dev, dtype=torch.float64))
        props = [(torch.empty((nb, 2), dtype=torch.float64, device=dev),
                  torch.empty((), dtype=torch.float64, device=dev)) for _ in range(iters)]
        outs = [(torch.empty((), dtype=torch.float64, device=dev), torch.empty((), dtype=torch.int32, device=dev))
                for _ in range(iters)]

        def run_c():
            for k in range(iters):
                s.propose_circle(idx[k], centers, radii, 0.5, 4, u[k], out=props[k], check=False)
                s.step(idx[k], props[k][0], log_u[k], props[k][1], out=outs[k], check=False)

        run_c()
        torch.cuda.synchronize()
        s.sync_status()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                run_c()
        torch.cuda.synchronize()
        m = timed_calls(g.replay, stream, l2, reps=10, warm=2)
        s.sync_status()
        per = m / iters
        res[f"circle_block_{nb}" + ("" if prec == "fp64" else "_mixed")] = {
            "workload": "c3_wildfire_like_n5000_d2_circles", "ms_per_iteration": per,
            "iterations_per_s": 1e3 / per, "location_updates_per_s": nb * 1e3 / per, "pair_term_precision": prec,
            "accepted_last_replay": int(sum(o[1].item() for o in outs))}
        s.close()
    # the same proposal evaluated by a full log-likelihood instead (what the increments avoid)
    ctx = HawkesContext(device=dev.index or 0, max_n=w.n, max_d=w.d)
    full = timed_calls(lambda: hawkes_loglik(ctx, t, X, w.params, "fp64", check=False), stream, l2, reps=5, warm=1)
    res["full_fp64_loglik_ms"] = full
    ctx.close()
    return res


def bmds_hawkes_hmc_workload(dev, stream, l2, fma_rate: float, ex2_rate: float, clock_mhz: float, sms: int,
                             steps: int = 20) -> dict:
    """HMC over the latent locations of the BMDS-Hawkes model (the influenza
    application): N = 4,733, D = 6, potential -ell - ell_B, `steps` leapfrog
    steps per trajectory (one CUDA graph), mixed precision with FP32 Y.  The
    paper reports 80 M states in about 10 days on a Titan V (about 93 per
    second) without stating the number of leapfrog steps; that figure is
    context, not a like-for-like comparison."""
    import numpy as np
    import torch

    import synth
    from paper_2010_02994_gb300 import HawkesContext, hawkes_bmds_hmc_trajectory

    w, b = synth.make_bmds_hawkes()
    ctx = HawkesContext(device=dev.index or 0, max_n=w.n, max_d=w.d)
    t = torch.tensor(w.t, device=dev)
    X = torch.tensor(w.X, device=dev)
    Y = torch.tensor(b.Y, device=dev).float()
    p0 = torch.tensor(np.random.default_rng(3).standard_normal(size=w.X.shape), device=dev)
    log_u = torch.tensor(-1e30, dtype=torch.float64, device=dev)
    eps = 5e-4
    run = lambda: hawkes_bmds_hmc_trajectory(ctx, t, X, p0, w.params, Y, b.sigma2, eps, steps, log_u, "mixed",
                                             check=False)
    m = timed_calls(run, stream, l2, reps=10, warm=2)  # the default form at this size
    ctx.set_option("bmds_fused", 1)
    m_fused = timed_calls(run, stream, l2, reps=10, warm=2)  # the BMDS term inside the gradient pass
    ctx.set_option("bmds_fused", 0)
    m_two = timed_calls(run, stream, l2, reps=10, warm=2)  # BMDS kernels on a second stream
    ctx.set_option("bmds_fused", 0)
    ctx.sync_status()
    ctx.close()
    pairs = w.n * (w.n - 1) / 2
    work = (steps + 1) * pairs * (pass_bound_cycles(w.d, "eval", fma_rate, ex2_rate)
                                  + bmds_bound_cycles(w.d, fma_rate, ex2_rate))
    return {"workload": w.name, "n": w.n, "d": w.d, "leapfrog_steps": steps, "precision": "mixed, FP32 Y",
            "ms_per_trajectory": m, "trajectories_per_s": 1e3 / m, "gradient_evals_per_s": (steps + 1) * 1e3 / m,
            "gradient": "BMDS kernels (gradient alone between the ends) beside the Hawkes passes",
            "fused_ms_per_trajectory": m_fused, "two_stream_ms_per_trajectory": m_two,
            "roofline": eval_roofline(1e3 / m, work, sms, clock_mhz, "trajectories/s",
                                      f"{steps + 1} Hawkes (6D+19 FP32, 4 ex2) and BMDS (4D+40 FP32, 4 MUFU) "
                                      f"evaluations per trajectory, measured per-SM rates, {clock_mhz:.0f} MHz"),
            "paper_context": "80 M states / ~10 days = ~93 states/s on a Titan V, leapfrog steps not stated"}


def other_workloads(dev, stream, l2, fma_rate: float, ex2_rate: float, clock_mhz: float, sms: int) -> dict:
    """Batched 64-set latent-space workload (one call, mixed path), one
    20-step HMC trajectory at N=1e4 (mixed path, CUDA graph) and the BMDS
    likelihood at the influenza size, timed with CUDA events; L2 flushed
    before each timed call."""
    import numpy as np
    import torch

    import synth
    from paper_2010_02994_gb300 import (HawkesContext, hawkes_batch_hmc_trajectory, hawkes_batch_loglik_grad,
                                        hmc_leapfrog_trajectory)

    out = {"bmds_influenza_like": bmds_workload(dev, stream, l2, fma_rate, ex2_rate, clock_mhz, sms),
           "mwg_gunfire_like": mwg_workload(dev, stream, l2),
           "bmds_hawkes_hmc_influenza_like": bmds_hawkes_hmc_workload(dev, stream, l2, fma_rate, ex2_rate, clock_mhz,
                                                                      sms)}
    sets = synth.make_c4()
    sizes = [w.n for w in sets]
    dims = [w.d for w in sets]
    ctx = HawkesContext(device=dev.index or 0, max_n=sum(sizes), max_d=8)
    t = torch.tensor(np.concatenate([w.t for w in sets]), device=dev)
    X = torch.tensor(np.concatenate([w.X.reshape(-1) for w in sets]), device=dev)
    params = [w.params for w in sets]
    for _ in range(2):
        hawkes_batch_loglik_grad(ctx, sizes, dims, t, X, params, check=False)
    torch.cuda.synchronize()
    ms = []
    for _ in range(10):
        flush_l2(l2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        hawkes_batch_loglik_grad(ctx, sizes, dims, t, X, params, check=False)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    ctx.sync_status()
    pairs = float(sum(n * n for n in sizes))
    m = statistics.median(ms)
    # the same batch with every dimension in one persistent launch per pass
    ctx.set_option("one_launch", 1)
    m_one = timed_calls(lambda: hawkes_batch_loglik_grad(ctx, sizes, dims, t, X, params, check=False), stream, l2,
                        reps=10, warm=2)
    ctx.sync_status()
    ctx.set_option("one_launch", 0)
    # the same batch in FP64 (every operation in double), as the accuracy reference
    hawkes_batch_loglik_grad(ctx, sizes, dims, t, X, params, precision="fp64", check=False)
    torch.cuda.synchronize()
    ms64 = []
    for _ in range(2):
        flush_l2(l2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        hawkes_batch_loglik_grad(ctx, sizes, dims, t, X, params, precision="fp64", check=False)
        b.record(stream)
        torch.cuda.synchronize()
        ms64.append(a.elapsed_time(b))
    ctx.sync_status()
    m64 = statistics.median(ms64)
    # the bound of a call: each set's unordered pairs at its dimension's per-pair bound
    c4_work = sum(n * (n - 1) / 2 * pass_bound_cycles(d, "eval", fma_rate, ex2_rate) for n, d in zip(sizes, dims))
    out["batched_c4"] = {"sets": len(sets), "events": sum(sizes), "dims": sorted(set(dims)), "ms_per_call": m,
                         "calls_per_s": 1e3 / m, "pairs_per_s": pairs / (m * 1e-3),
                         "roofline": eval_roofline(1e3 / m, c4_work, sms, clock_mhz, "calls/s",
                                                   "sum over the 64 sets of N(N-1)/2 x (6D+19)/FMA-rate SM-cycles "
                                                   f"(the FP32 bound at D = 2, 4, 8), {clock_mhz:.0f} MHz"),
                         "one_launch_ms_per_call": m_one,
                         "fp64_ms_per_call": m64, "fp64_pairs_per_s": pairs / (m64 * 1e-3)}
    ctx.close()

    w = synth.make_c2()
    ctx = HawkesContext(device=dev.index or 0, max_n=w.n, max_d=w.d)
    t = torch.tensor(w.t, device=dev)
    X = torch.tensor(w.X, device=dev)
    lo = torch.tensor(w.box_lo, device=dev)
    hi = torch.tensor(w.box_hi, device=dev)
    rng = np.random.default_rng(11)
    p0 = torch.tensor(rng.standard_normal(size=w.X.shape), device=dev)
    steps = w.meta.get("hmc_steps", 20)
    eps = 2e-3
    for _ in range(2):
        hmc_leapfrog_trajectory(ctx, t, X, p0, w.params, eps, steps, 0.0, lo, hi, check=False)
    torch.cuda.synchronize()
    ms = []
    for _ in range(10):
        flush_l2(l2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        hmc_leapfrog_trajectory(ctx, t, X, p0, w.params, eps, steps, 0.0, lo, hi, check=False)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    ctx.sync_status()
    m = statistics.median(ms)
    c2_work = (steps + 1) * w.n * (w.n - 1) / 2 * pass_bound_cycles(w.d, "eval", fma_rate, ex2_rate)
    out["hmc_c2"] = {"n": w.n, "d": w.d, "leapfrog_steps": steps, "ms_per_trajectory": m,
                     "trajectories_per_s": 1e3 / m, "grad_evals_per_s": (steps + 1) * 1e3 / m,
                     "roofline": eval_roofline(1e3 / m, c2_work, sms, clock_mhz, "trajectories/s",
                                               f"{steps + 1} evaluations x N(N-1)/2 pairs x (6D+19)/FMA-rate "
                                               f"SM-cycles, {clock_mhz:.0f} MHz")}
    ctx.close()
    # one HMC proposal per set over the 64 sets of c4 (unconstrained, 20 steps, one graph)
    ctx = HawkesContext(device=dev.index or 0, max_n=sum(sizes), max_d=8)
    t = torch.tensor(np.concatenate([w.t for w in sets]), device=dev)
    X = torch.tensor(np.concatenate([w.X.reshape(-1) for w in sets]), device=dev)
    p0 = torch.tensor(rng.standard_normal(size=X.shape[0]), device=dev)
    eps = [1e-3] * len(sets)
    log_u = torch.full((len(sets),), -1e300, dtype=torch.float64, device=dev)
    for _ in range(2):
        hawkes_batch_hmc_trajectory(ctx, sizes, dims, t, X, p0, params, eps, 20, log_u, check=False)
    torch.cuda.synchronize()
    ms = []
    for _ in range(5):
        flush_l2(l2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        hawkes_batch_hmc_trajectory(ctx, sizes, dims, t, X, p0, params, eps, 20, log_u, check=False)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    ctx.sync_status()
    m = statistics.median(ms)
    ctx.set_option("one_launch", 1)
    m_one = timed_calls(lambda: hawkes_batch_hmc_trajectory(ctx, sizes, dims, t, X, p0, params, eps, 20, log_u,
                                                            check=False), stream, l2, reps=5, warm=2)
    ctx.sync_status()
    ctx.set_option("one_launch", 0)
    out["batched_hmc_c4"] = {"sets": len(sets), "events": sum(sizes), "leapfrog_steps": 20, "ms_per_call": m,
                             "one_launch_ms_per_call": m_one,
                             "set_trajectories_per_s": len(sets) * 1e3 / m,
                             "roofline": eval_roofline(1e3 / m, 21 * c4_work, sms, clock_mhz, "calls/s",
                                                       "21 evaluations of every set per call, bound as batched_c4")}
    ctx.close()
    return out


def run_workload_calls(name: str, calls: int) -> int:
    """`calls` untimed calls of one of the other workloads (same inputs as their
    bench lines), for profiler captures of their kernels."""
    import numpy as np
    import torch

    import synth
    from paper_2010_02994_gb300 import (HawkesContext, HawkesMwG, hawkes_batch_loglik_grad,
                                        hawkes_bmds_hmc_trajectory, hawkes_bmds_loglik_grad,
                                        hawkes_loglik_grad_locations, hmc_leapfrog_trajectory)

    dev = torch.device("cuda", 0)
    if name in ("bmds", "bmds_f64y"):
        b = synth.make_bmds()
        ctx = HawkesContext(device=0, max_n=b.X.shape[0], max_d=b.X.shape[1])
        Y = torch.tensor(b.Y, device=dev)
        Y = Y if name == "bmds_f64y" else Y.float()
        X = torch.tensor(b.X, device=dev)
        for _ in range(calls):
            hawkes_bmds_loglik_grad(ctx, Y, X, b.sigma2, "mixed", check=False)
        ctx.sync_status()
        ctx.close()
    elif name in ("mwg1", "mwg32", "mwg32_mixed"):
        nb = 1 if name == "mwg1" else 32
        w = synth.make_c2()
        s = HawkesMwG(torch.tensor(w.t, device=dev), torch.tensor(w.X, device=dev), w.params, max_block=nb,
                      precision="mixed" if name.endswith("_mixed") else "fp64")
        lo, hi = torch.tensor(w.box_lo, device=dev), torch.tensor(w.box_hi, device=dev)
        gen = torch.Generator(device=dev).manual_seed(12)
        for _ in range(calls):
            idx = torch.randperm(w.n, generator=gen, device=dev)[:nb]
            u = torch.rand((nb, w.d), generator=gen, device=dev, dtype=torch.float64)
            Xn, lq = s.propose_box(idx, lo, hi, 0.02, u, check=False)
            s.step(idx, Xn, float(np.log(0.5)), lq, check=False)
        s.sync_status()
        s.close()
    elif name == "bmds_hmc":
        w, b = synth.make_bmds_hawkes()
        ctx = HawkesContext(device=0, max_n=w.n, max_d=w.d)
        t, X = torch.tensor(w.t, device=dev), torch.tensor(w.X, device=dev)
        Y = torch.tensor(b.Y, device=dev).float()
        p0 = torch.tensor(np.random.default_rng(3).standard_normal(size=w.X.shape), device=dev)
        for _ in range(calls):
            hawkes_bmds_hmc_trajectory(ctx, t, X, p0, w.params, Y, b.sigma2, 5e-4, 4, -1e30, "mixed", check=False)
        ctx.sync_status()
        ctx.close()
    elif name == "bmds_hmc_fused_n10000":
        # one-step BMDS-Hawkes trajectories at N = 10,000, D = 6, with the
        # BMDS term inside the gradient pass
        w, b = synth.make_bmds_hawkes(n=10_000)
        ctx = HawkesContext(device=0, max_n=w.n, max_d=w.d)
        ctx.set_option("bmds_fused", 1)
        t, X = torch.tensor(w.t, device=dev), torch.tensor(w.X, device=dev)
        Y = torch.tensor(b.Y, device=dev).float()
        p0 = torch.tensor(np.random.default_rng(3).standard_normal(size=w.X.shape), device=dev)
        for _ in range(calls):
            hawkes_bmds_hmc_trajectory(ctx, t, X, p0, w.params, Y, b.sigma2, 5e-4, 1, -1e30, "mixed", check=False)
        ctx.sync_status()
        ctx.close()
    elif name == "hmc_c2":
        w = synth.make_c2()
        ctx = HawkesContext(device=0, max_n=w.n, max_d=w.d)
        t, X = torch.tensor(w.t, device=dev), torch.tensor(w.X, device=dev)
        lo, hi = torch.tensor(w.box_lo, device=dev), torch.tensor(w.box_hi, device=dev)
        p0 = torch.tensor(np.random.default_rng(11).standard_normal(size=w.X.shape), device=dev)
        for _ in range(calls):
            hmc_leapfrog_trajectory(ctx, t, X, p0, w.params, 2e-3, 4, 0.0, lo, hi, check=False)
        ctx.sync_status()
        ctx.close()
    elif name == "fp64_c2":
        # the FP64 path (location gradient) on the gunfire-like events, N = 10,000, D = 2
        w = synth.make_c2()
        ctx = HawkesContext(device=0, max_n=w.n, max_d=w.d)
        t, X = torch.tensor(w.t, device=dev), torch.tensor(w.X, device=dev)
        for _ in range(calls):
            hawkes_loglik_grad_locations(ctx, t, X, w.params, precision="fp64", check=False)
        ctx.sync_status()
        ctx.close()
    else:
        sets = synth.make_c4()
        sizes, dims = [w.n for w in sets], [w.d for w in sets]
        ctx = HawkesContext(device=0, max_n=sum(sizes), max_d=8)
        t = torch.tensor(np.concatenate([w.t for w in sets]), device=dev)
        X = torch.tensor(np.concatenate([w.X.reshape(-1) for w in sets]), device=dev)
        for _ in range(calls):
            hawkes_batch_loglik_grad(ctx, sizes, dims, t, X, [w.params for w in sets], check=False)
        ctx.sync_status()
        ctx.close()
    torch.cuda.synchronize()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--cpu-sample", type=int, default=CPU_SAMPLE_N)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched and HMC workloads")
    ap.add_argument("--n", type=int, default=100_000)
    ap.add_argument("--kernels-only", action="store_true",
                    help="only run warmup + steps evaluations (for profiler captures); prints no JSON")
    ap.add_argument("--workload", default=None,
                    choices=["bmds", "bmds_f64y", "mwg1", "mwg32", "mwg32_mixed", "bmds_hmc", "hmc_c2",
                             "batched_c4", "fp64_c2", "bmds_hmc_fused_n10000"],
                    help="with --kernels-only: run warmup + steps calls of that other workload instead "
                         "(for profiler captures); prints no JSON")
    args = ap.parse_args()
    args.steps_ref = max(1, min(args.steps, 10))
    args.warmup_ref = min(args.warmup, 1)
    if args.impl == "reference":
        return run_reference(args)
    if args.kernels_only and args.workload:
        return run_workload_calls(args.workload, args.warmup + args.steps)

    import numpy as np
    import torch

    import synth
    from paper_2010_02994_gb300 import (HawkesContext, hawkes_loglik_grad_locations, hawkes_self_excitation_prob,
                                        probe_dfma_rate, probe_pipe_rates)

    world, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = synth.make_c5() if args.n == 100_000 else synth.scaled_down(synth.make_c5(), args.n)
    n, d = w.n, w.d
    ctx = HawkesContext(device=local, max_n=n, max_d=d)
    t = torch.tensor(w.t, device=dev)
    X = torch.tensor(w.X, device=dev)
    ell = torch.empty((), dtype=torch.float64, device=dev)
    g = torch.empty((n, d), dtype=torch.float64, device=dev)
    if args.kernels_only:
        for _ in range(args.warmup + args.steps):
            hawkes_loglik_grad_locations(ctx, t, X, w.params, precision="mixed", check=False, out=(ell, g, None))
        ctx.sync_status()
        torch.cuda.synchronize()
        ctx.close()
        return 0
    l2 = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def step(prec):
        hawkes_loglik_grad_locations(ctx, t, X, w.params, precision=prec, check=False, out=(ell, g, None))

    rates = probe_pipe_rates(local)
    fma_rate = 128.0 if not rates["fma_per_sm_clk"] > 0 else rates["fma_per_sm_clk"]
    ex2_rate = 16.0 if not rates["ex2_per_sm_clk"] > 0 else rates["ex2_per_sm_clk"]

    # --- device-resident timing (mixed path) ---------------------------------
    for _ in range(args.warmup):
        step("mixed")
    ctx.sync_status()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                          if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local)
    ctx.reset_stats()
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)  # the sampler's first line lands inside the timed region
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush_l2(l2)
        starts[k].record(stream)
        step("mixed")
        ends[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(world)
    clk = clocks.stop()
    launches = ctx.launch_count()
    ctx.sync_status()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms_mixed = max_over_ranks(world, sum(step_ms) / len(step_ms), dev)
    value = world * 1e3 / ms_mixed

    # --- per-kernel timing (events around each pair pass, same stream) -------
    ctx.set_option("profile", 1)
    ctx.reset_stats()
    prof_steps = min(20, args.steps)
    for _ in range(prof_steps):
        flush_l2(l2)
        step("mixed")
    torch.cuda.synchronize()
    k1, k2 = ctx.kernel_stats(0), ctx.kernel_stats(1)
    stages = {name: ctx.kernel_stats(i)["ms"] / prof_steps
              for i, name in enumerate(("pass1_rates", "pass2_gradient", "prep_sort_pack", "finalize_rates",
                                        "finalize_gradient"))}
    ctx.set_option("profile", 0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    pairs = 0.5 * n * (n - 1)

    which_name = {"pass1": "pass1_rates", "pass2": "pass2_gradient"}

    def roof(stat, which):
        achieved = stat["pairs"] / (stat["ms"] * 1e-3) / 1e9
        peak = sms * MAX_SM_MHZ_NOMINAL * 1e6 / pass_bound_cycles(d, which, fma_rate, ex2_rate) / 1e9
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair/s", "frac": achieved / peak,
                "traffic": measured_traffic(which_name[which]), "traffic_unit": "bytes per launch",
                "ms_per_launch": stat["ms"] / max(1, stat["launches"]),
                "peak_basis": (f"{sms} SMs x {MAX_SM_MHZ_NOMINAL:.0f} MHz / max(FP32 ops/{fma_rate:.1f}, "
                               f"ex2/{ex2_rate:.1f}) cycles per unordered pair (measured per-SM rates)")}

    r1, r2 = roof(k1, "pass1"), roof(k2, "pass2")
    dominant = ("pass2_gradient", r2) if k2["ms"] >= k1["ms"] else ("pass1_rates", r1)
    eval_peak = sms * MAX_SM_MHZ_NOMINAL * 1e6 / pass_bound_cycles(d, "both", fma_rate, ex2_rate) / pairs

    # --- far-block skipping (exact; reported apart from the dense headline) ---
    ell_dense, g_dense = ell.clone(), g.clone()
    ctx.set_option("skip_far_blocks", 1)
    for _ in range(3):
        step("mixed")
    torch.cuda.synchronize()
    sk = []
    for _ in range(min(50, args.steps)):
        flush_l2(l2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step("mixed")
        b.record(stream)
        torch.cuda.synchronize()
        sk.append(a.elapsed_time(b))
    ctx.sync_status()
    identical = bool(torch.equal(ell, ell_dense) and torch.equal(g, g_dense))
    ctx.set_option("skip_far_blocks", 0)
    ms_skip = sum(sk) / len(sk)
    skip_far = {"evals_per_s": 1e3 / ms_skip, "ms_per_step": ms_skip, "identical_to_dense": identical,
                "note": "pair blocks whose closest pair underflows FP32 are skipped; not the dense headline"}

    # --- FP64 GPU path on the same inputs ------------------------------------
    fp64 = None
    if args.fp64_steps > 0:
        step("fp64")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(args.fp64_steps):
            flush_l2(l2)
            e0.record(stream)
            step("fp64")
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        ctx.sync_status()
        ms64 = tot / args.fp64_steps
        # the ordered layout (every ordered pair, CUDA's exp) on the same inputs
        ctx.set_option("fp64_ordered", 1)
        step("fp64")
        torch.cuda.synchronize()
        flush_l2(l2)
        e0.record(stream)
        step("fp64")
        e1.record(stream)
        torch.cuda.synchronize()
        ms_ord = e0.elapsed_time(e1)
        ctx.set_option("fp64_ordered", 0)
        ctx.sync_status()
        dfma = probe_dfma_rate(local)
        # FP64 operations per unordered pair in the symmetric kernels when
        # every exponential is needed: rate pass 2D + 23, gradient pass 4D + 23
        # (two 7-operation exponentials each); exponentials that round to zero
        # for a whole warp are skipped, so spread-out data needs fewer
        ops = 6 * d + 46
        dense_ms = 0.5 * n * (n - 1) * ops / (dfma * sms * MAX_SM_MHZ_NOMINAL * 1e6) * 1e3
        fp64 = {"evals_per_s": 1e3 / ms64, "ms_per_step": ms64, "pairs_per_s": n * n / (ms64 * 1e-3),
                "steps": args.fp64_steps, "layout": "symmetric (each unordered pair once)",
                "ordered_layout_ms_per_step": ms_ord, "dfma_per_sm_clk": dfma,
                "fp64_ops_per_unordered_pair_dense": ops, "dense_fp64_issue_bound_ms_at_max_clock": dense_ms,
                "note": "the dense bound assumes every exponential is evaluated; terms that round to zero "
                        "in FP64 are skipped exactly, so spread-out data runs below it",
                "fp64_tflops_at_max_clock": 2.0 * dfma * sms * MAX_SM_MHZ_NOMINAL * 1e6 / 1e12}

    # --- end to end: host buffers, H2D + evaluation + D2H inside the timing --
    t_h = torch.tensor(w.t).pin_memory()
    X_h = torch.tensor(w.X).pin_memory()
    g_h = torch.empty((n, d), dtype=torch.float64).pin_memory()
    ell_h = torch.empty((), dtype=torch.float64).pin_memory()
    t_d = torch.empty_like(t)
    X_d = torch.empty_like(X)

    def e2e_step():
        t_d.copy_(t_h, non_blocking=True)
        X_d.copy_(X_h, non_blocking=True)
        hawkes_loglik_grad_locations(ctx, t_d, X_d, w.params, precision="mixed", check=False, out=(ell, g, None))
        g_h.copy_(g, non_blocking=True)
        ell_h.copy_(ell, non_blocking=True)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    es = [torch.cuda.Event(enable_timing=True) for _ in range(args.e2e_steps)]
    ee = [torch.cuda.Event(enable_timing=True) for _ in range(args.e2e_steps)]
    for k in range(args.e2e_steps):
        flush_l2(l2)
        es[k].record(stream)
        e2e_step()
        ee[k].record(stream)
    torch.cuda.synchronize()
    ctx.sync_status()
    ms_e2e = max_over_ranks(world, sum(a.elapsed_time(b) for a, b in zip(es, ee)) / args.e2e_steps, dev)
    h2d = t_h.numel() * 8 + X_h.numel() * 8
    d2h = g_h.numel() * 8 + 8

    # --- the other paper-shaped workloads (reported beside the headline) -----
    extra = {}
    if not args.no_extra:
        # the same inputs with the Theta gradient, and the self-excitation probabilities
        gp = torch.empty(6, dtype=torch.float64, device=dev)
        m_theta = timed_calls(lambda: hawkes_loglik_grad_locations(ctx, t, X, w.params, precision="mixed",
                                                                   grad_params=True, check=False, out=(ell, g, gp)),
                              stream, l2, reps=10, warm=2)
        m_sep = timed_calls(lambda: hawkes_self_excitation_prob(ctx, t, X, w.params, precision="mixed", check=False),
                            stream, l2, reps=10, warm=2)
        ctx.sync_status()
        extra["c5_same_inputs"] = {"loglik_grad_X_and_theta_ms": m_theta, "evals_per_s_with_theta": 1e3 / m_theta,
                                   "self_excitation_prob_ms": m_sep}
        extra.update(other_workloads(dev, stream, l2, fma_rate, ex2_rate, MAX_SM_MHZ_NOMINAL, sms))

    # --- CPU baseline: the oracle on the host cores ---------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_oracle_sample(args.cpu_sample, 1)
        cpu = {"value": cb["evals_per_s_at_1e5"], "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
               "sample": (f"first {cb['n_sample']} events (time order) of the N=1e5 D=2 workload, one full FP64 "
                          f"ell + grad_X in {cb['sec_per_eval']:.2f} s; evals/s at N=1e5 = pairs/s / 1e10"),
               "pairs_per_s": cb["pairs_per_s"]}

    per_step_launches = launches["own"] / max(1, args.steps)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "c5_large_n100000_d2" if n == 100_000 else f"c5_first{n}", "n": n, "d": d,
                   "precision": "mixed: f32 pair values and squared distances, f64 reductions",
                   "parallelism": "replicas only" if world > 1 else "single GPU",
                   "l2": "flushed between steps (512 MB write, untimed)"},
        "pairs_per_s": world * n * n / (ms_mixed * 1e-3),
        "unordered_pairs_per_s": world * pairs / (ms_mixed * 1e-3),
        "roofline": dict(dominant[1], kernel=dominant[0]),
        "roofline_kernels": {"pass1_rates": r1, "pass2_gradient": r2},
        "roofline_eval": {"achieved_evals_per_s": 1e3 / ms_mixed, "peak_evals_per_s": eval_peak,
                          "frac": (1e3 / ms_mixed) / eval_peak},
        "fp64_gpu": fp64,
        "skip_far_blocks": skip_far,
        "e2e": {"value": world * 1e3 / ms_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": ms_e2e},
        "cpu_baseline": cpu,
        "stages_ms_per_eval": stages,
        "other_workloads": extra,
        "clocks": clk,
        "gpu_launches": int(launches["own"]),
        "gpu_launches_per_step": per_step_launches,
        "library_sort_launches": int(launches["library"]),
        "sm_count": sms,
        "pipe_rates": rates,
        "wall_s": wall,
    }
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
