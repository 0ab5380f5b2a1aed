#!/usr/bin/env python
"""Benchmark: Coulomb pair interactions per second at N = 100 000 (one adaptive-cycle step).

One step is one pass of the whole hot path over one batch of synthetic input:
  1. float64 local energies e_i of all N charges (Sec. II C step 1: N(N-1)
     ordered pair interactions),
  2. 256 subdomains (m ~ U{200..5000}, the m nearest charges to a centre)
     relaxed together against all N for 200 mixed-precision projected
     Barzilai-Borwein steps (Sec. II C step 4, Sec. II E: m(N-1) pair
     interactions per subdomain per step),
  3. sequential float64 pairwise accept/reject of the relaxed subdomains.
The value is the ordered pair interactions of 1 and 2 divided by the whole
step's time (the accept passes of 3 are timed but not counted).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run; every rank relaxes its own
independently seeded configuration (weak scaling, no collective on the data path).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N = 100_000
N_SUB = 256
M_LO, M_HI = 200, 5000
RELAX_STEPS = 200
LOCAL_PREC = "fp64"  # the total energy needs 12+ digits: float64
# DRAM bytes of one relaxation-pass launch of this workload: dram__bytes_read.sum +
# dram__bytes_write.sum of k_pass_mixed launches 6..8 in one ncu capture of
# `python bench.py --steps 1 --warmup 1 --no-cpu-baseline --no-instances --config 3`; the capture
# must be retaken, or this set to None, whenever that kernel changes.
RELAX_PASS_DRAM_BYTES = 36.3e6
METRIC = "Coulomb pair-interactions/s (E+grad) at N=1e5, mixed vs FP64; relax time"
UNIT = "pair-interactions/s"
WORKLOAD = ("adaptive-cycle step at N=1e5: fp64 local energies of all charges + 256 subdomains "
            "(m~U[200,5000], nearest charges to a centre) x 200 mixed BB steps against all N + fp64 "
            "sequential accept; triangular-lattice background mapped to the arcsine density, 0.5% jitter, "
            "charges stored in Hilbert-curve order")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-instances", action="store_true", help="skip the batched-instances (C5) section")
    # a single small kernel case (used for profiler captures): no JSON bench line
    ap.add_argument("--case", choices=["allpairs", "relax", "full-relax", "cycle", "instances", "delta"], default=None)
    ap.add_argument("--batch", type=int, default=64, help="cycle case: subdomains per batch")
    ap.add_argument("--zone-steps", type=int, default=100, help="cycle case: relaxation steps per zone")
    ap.add_argument("--cycle-opt", choices=["bb", "lbfgsb_tu"], default="lbfgsb_tu", help="cycle case: zone optimiser")
    ap.add_argument("--single", action="store_true", help="cycle case: only N = --n (no N/8, N/4, N/2 runs)")
    ap.add_argument("--fixed-batches", action="store_true",
                    help="cycle case: fixed batches (overlapping zones skipped) instead of disjoint prefixes")
    ap.add_argument("--prec", choices=["mixed", "fp64", "fp64x"], default="mixed")
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--nsub", type=int, default=16)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--config", type=int, default=None, help="mixed pass launch shape (tc_set_pass_config)")
    return ap.parse_args()


def run_case(args):
    """One small workload of one kernel family, timed with CUDA events (for profiler runs)."""
    import torch

    import synth
    import paper_2609_24722_b300 as tc

    dev = torch.device("cuda", 0)
    if args.case == "full-relax":
        # the C4 workload with longer budgets than the bench line's entry: mixed steps past the 1e-4
        # tolerance, then float64-grade (fp64x) and float64 polishes
        print(json.dumps(run_full_relax(dev, n=args.n, max_polish=1000, polish_chunk=100)), flush=True)
        print(json.dumps(run_full_relax(dev, n=args.n, extra_mixed=20000, max_polish=2000,
                                        polish_precision="fp64x")), flush=True)
        return
    if args.case == "instances":
        # config C5 alone: 512 instances, mixed L-BFGS with a float64 polish, graph on and off
        print(json.dumps(run_instances(dev, rounds=2)), flush=True)
        return
    if args.case == "cycle":
        # cycle time against N at a fixed number of subdomain optimisations (Sec. II E)
        for n in ([args.n] if args.single else [args.n // 8, args.n // 4, args.n // 2, args.n]):
            print(json.dumps(run_cycle(dev, n=n, n_sub=args.nsub, batch=args.batch, steps=args.zone_steps,
                                       optimizer=args.cycle_opt, disjoint=not args.fixed_batches)))
        return
    if args.config is not None:
        from paper_2609_24722_b300 import _lib

        _lib.check(_lib.lib().tc_set_pass_config(_lib.TC_MIXED, args.config), "tc_set_pass_config")
    if args.case == "allpairs":
        pa = synth.arcsine_disk(args.n, 0)
        p = torch.tensor(pa[synth.zorder(pa)], device=dev)
        work = lambda: tc.grad(p, args.prec, with_energy=True)  # noqa: E731
        pairs = args.n * (args.n - 1)
    elif args.case == "delta":
        # the float64 pairwise energy change of the accept (k_pass<DELTA>): subdomains moved by ~1e-4
        import numpy as np

        pos = synth.lattice_disk(args.n, 0)
        pos = np.ascontiguousarray(pos[synth.zorder(pos)])
        subs = synth.subdomains(pos, args.nsub, 200, 2000, 2)
        idx, off = synth.to_csr(subs)
        new = pos[idx] + np.random.default_rng(3).normal(0.0, 1e-4, (idx.size, 2))
        new *= np.minimum(1.0, 1.0 / np.linalg.norm(new, axis=1))[:, None]
        p, it, of, nw = (torch.tensor(a, device=dev) for a in (pos, idx, off, new))
        if args.prec == "mixed":
            work = lambda: tc.subdomain_delta_energy_mixed(p, it, of, nw)  # noqa: E731
        else:
            work = lambda: tc.subdomain_delta_energy(p, it, of, nw)  # noqa: E731
        pairs = sum(len(s) for s in subs) * (args.n - 1)
    else:
        pos = synth.lattice_disk(args.n, 0)
        pos = pos[synth.zorder(pos)]
        subs = synth.subdomains(pos, args.nsub, 200, 2000, 2)
        idx, off = synth.to_csr(subs)
        p0 = torch.tensor(pos, device=dev)
        p = p0.clone()
        it, of = torch.tensor(idx, device=dev), torch.tensor(off, device=dev)
        eta = 1e-4 / args.n

        def work():
            p.copy_(p0)
            return tc.relax_subdomains(p, it, of, precision=args.prec, optimizer="bb", n_steps=10, step0=eta,
                                       alpha_min=0.0, alpha_max=10 * eta, accept=False)
        pairs = 10 * sum(len(s) for s in subs) * (args.n - 1)
    work()
    ts = []
    for _ in range(args.reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        work()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    tc.sync_status()
    ms = min(ts)
    print(json.dumps({"case": args.case, "prec": args.prec, "n": args.n, "ms": ms, "pairs_per_s": pairs / (ms / 1e3)}))


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(ms_local: float, units_local: float, world: int, device=None) -> tuple[float, float]:
    """Whole-job timing across ranks: (max step time over ranks in ms, aggregate units/s).

    Every rank does the same amount of work (weak scaling), so the job rate is
    world * units_local / max time.  Collective: one max all-reduce (any backend).
    """
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_local = float(t.item())
    return ms_local, world * units_local / (ms_local / 1e3)


def make_inputs(seed: int):
    import synth

    pos = synth.lattice_disk(N, seed)
    # charges are identical: store the configuration along a Hilbert curve so
    # nearby charges have nearby indices (compact row blocks and source tiles)
    pos = pos[synth.zorder(pos)]
    subs = synth.subdomains(pos, N_SUB, M_LO, M_HI, seed + 2)
    idx, off = synth.to_csr(subs)
    return pos, idx, off


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(pos, idx, off, seconds: float = 12.0) -> dict:
    """The CPU oracle, as it stands, on a bounded sample: subdomain rows against all N."""
    import numpy as np
    import oracle

    rows_all = idx[: off[min(N_SUB, len(off) - 1)]]
    # size the sample from a short calibration run
    t0 = time.perf_counter()
    oracle.rows_grad(pos, rows_all[:50])
    per_row = (time.perf_counter() - t0) / 50
    n_rows = int(max(50, min(len(rows_all), seconds / max(per_row, 1e-9))))
    rows = np.ascontiguousarray(rows_all[:n_rows])
    t0 = time.perf_counter()
    oracle.rows_grad(pos, rows)
    dt = time.perf_counter() - t0
    pairs = n_rows * (N - 1)
    out = {"value": pairs / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"float64 gradient + energy rows of the first {n_rows} subdomain charges against all "
                     f"{N} charges (tco_rows_grad, single thread, Neumaier sums), {dt:.1f} s"}
    # the same oracle source built with OpenMP: rows split over every host thread
    threads = oracle.threads(openmp=True)
    n_omp = int(min(len(rows_all), max(n_rows, n_rows * threads * 0.5)))
    rows = np.ascontiguousarray(rows_all[:n_omp])
    t0 = time.perf_counter()
    oracle.rows_grad(pos, rows, openmp=True)
    dt = time.perf_counter() - t0
    out["all_cores"] = {"value": n_omp * (N - 1) / dt, "unit": UNIT, "cores": threads, "kind": "oracle-openmp",
                        "sample": f"the first {n_omp} subdomain rows against all {N} charges "
                                  f"(tco_rows_grad built with -fopenmp, bit-identical rows), {dt:.1f} s"}
    # one full float64 E + gradient of the single-thread oracle at small N (N = 1e5 would take ~1 min)
    import synth

    full = {}
    for nn in (1000, 20000):
        pp = synth.arcsine_disk(nn, 0)
        t0 = time.perf_counter()
        oracle.grad(pp)
        oracle.energy(pp)
        full[str(nn)] = time.perf_counter() - t0
    out["full_energy_grad_s"] = full
    out["host"] = {"nproc": os.cpu_count(), "cpu_model": _cpu_model()}
    return out


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_c3_disjoint(pos_np, relax_kw: dict, flush, stream, reps: int = 2, seed: int = 0) -> dict:
    """One adaptive-cycle step (float64 local energies + 200 mixed BB steps + float64 accept) on 256
    pairwise disjoint subdomains holding 0.9 N charges (synth.disjoint_subdomains), timed like the
    headline step."""
    import numpy as np
    import torch

    import synth
    import paper_2609_24722_b300 as tc

    dev = flush.device
    subs = synth.disjoint_subdomains(pos_np, N_SUB, M_LO, M_HI, seed + 2)
    idx_np, off_np = synth.to_csr(subs)
    idx, off = torch.tensor(idx_np, device=dev), torch.tensor(off_np, device=dev)
    pos0 = torch.tensor(pos_np, device=dev)
    p = pos0.clone()
    ms, prof, acc = [], None, 0
    for k in range(reps + 1):
        p.copy_(pos0)
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tc.local_energy(p, LOCAL_PREC)
        r = tc.relax_subdomains(p, idx, off, **relax_kw)
        b.record(stream)
        torch.cuda.synchronize()
        if k > 0:
            ms.append(a.elapsed_time(b))
            prof = tc.relax_last_profile()
            acc = int((r.status == 1).sum().item())
    tc.sync_status()
    pairs = N * (N - 1) + RELAX_STEPS * prof["pass_pairs"]
    pass_ms = prof["pass_ms"] / max(prof["n_pass"], 1)
    return {"workload": f"{N_SUB} disjoint subdomains holding {int(off_np[-1])} charges (m ~ U[{M_LO},{M_HI}] "
                        f"scaled by 0.9 N / sum m, nearest charges not yet taken), {RELAX_STEPS} mixed BB steps, "
                        f"fp64 local energies and sequential accept",
            "ms_per_step": statistics.mean(ms), "pairs_per_s": pairs / (statistics.mean(ms) / 1e3),
            "relax_pass_ms": pass_ms, "relax_pass_pairs_per_s": prof["pass_pairs"] / (pass_ms / 1e3),
            "accepted_subdomains": acc, "skipped_overlap": int((r.status == 2).sum().item())}


def run_graph_effect(dev, n: int = 1000, steps: int = 500, reps: int = 3) -> dict:
    """The step loop as a CUDA graph against direct launches where launches dominate: one N = 1000
    instance (config C1's size), 500 mixed L-BFGS steps, each step a few microseconds of kernel time.
    The direct form is the profiled loop (an event between launches), the graph form replays the
    cached 64-step graph."""
    import numpy as np
    import torch

    import synth
    import paper_2609_24722_b300 as tc

    pos = torch.tensor(synth.arcsine_disk(n, 0), device=dev)
    world = torch.tensor(np.array([[0, n]], dtype=np.int64), device=dev)
    kw = dict(world=world, precision="mixed", optimizer="lbfgs", n_steps=steps, memory=8, step0=1e-4, maxstep=0.01,
              accept=False)
    out = {}
    for name, prof in (("graph", False), ("direct", True)):
        ts = []
        for _ in range(reps + 1):
            p = pos.clone()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            tc.relax_subdomains(p, profile=prof, **kw)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        out[f"{name}_ms"] = statistics.median(ts[1:])
    tc.sync_status()
    return {"workload": f"one instance of N={n}, {steps} mixed L-BFGS(8) steps", **out,
            "us_per_step_graph": 1e3 * out["graph_ms"] / steps, "us_per_step_direct": 1e3 * out["direct_ms"] / steps}


def run_instances(dev, seed: int = 3, n_inst: int = 512, rounds: int = 4, steps: int = 500,
                  polish: int = 20, fp64_steps: int = 10, polish_precision: str = "fp64"):
    """Config C5: 512 independent instances (N_k ~ U{100..5000}, arcsine init each), relaxed in one
    batched call per round (mixed L-BFGS, memory 8, then a float64 polish; polish_precision="fp64x"
    runs it as float64-grade double-float on the float32 pipes), 3 perturbation restarts
    (Gaussian kicks of 0.05 x the instance's lattice spacing) keeping each instance's best energy;
    then the same instances with float64 pair terms for a few steps (throughput side by side)."""
    import numpy as np
    import torch

    import oracle
    import synth
    import paper_2609_24722_b300 as tc

    pos_np, off = synth.instances(n_inst, 100, 5000, seed)
    sizes = np.diff(off)
    # each instance's charges stored along a Hilbert curve (a relabelling: compact row blocks and tiles)
    for k in range(n_inst):
        q = pos_np[off[k]:off[k + 1]]
        pos_np[off[k]:off[k + 1]] = q[synth.zorder(q)]
    world = torch.tensor(np.stack([off[:-1], off[1:]], 1), device=dev)
    h = np.sqrt(2 * math.pi / (math.sqrt(3.0) * sizes))
    sig = np.repeat(0.05 * h, sizes)
    best = pos_np.copy()
    best_e = np.full(n_inst, np.inf)
    kw = dict(precision="mixed", optimizer="lbfgs", n_steps=steps, memory=8, step0=1e-5,
              maxstep=0.1 * float(h.min()), polish_steps=polish, polish_gtol=0.0, accept=False,
              polish_precision=polish_precision,
              want_energy=True)
    ms_total, pairs_total, launches = 0.0, 0, 0
    ms_rounds = []
    for r in range(rounds):
        start = pos_np if r == 0 else synth.jitter_inside(best, sig, seed + 100 + r)
        p = torch.tensor(start, device=dev)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        res = tc.relax_subdomains(p, world=world, **kw)
        b.record()
        torch.cuda.synchronize()
        tc.sync_status()
        ms_total += a.elapsed_time(b)
        ms_rounds.append(a.elapsed_time(b))
        pairs_total += int((sizes * (sizes - 1)).sum()) * (steps + polish)
        e = res.energy.cpu().numpy()
        x = p.cpu().numpy()
        better = e < best_e
        for k in np.flatnonzero(better):
            best[off[k]:off[k + 1]] = x[off[k]:off[k + 1]]
        best_e = np.where(better, e, best_e)
    # the float64-polished energies against the oracle's evaluation of the same configurations
    check = [0, int(np.argmax(sizes)), n_inst - 1]
    parity = max(abs(best_e[k] - oracle.energy(best[off[k]:off[k + 1]])) / best_e[k] for k in check)
    # the first round again with the step loop launched directly instead of as a CUDA graph
    p = torch.tensor(pos_np, device=dev)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    tc.relax_subdomains(p, world=world, **{**kw, "profile": True})
    b.record()
    torch.cuda.synchronize()
    ms_nograph = a.elapsed_time(b)
    prof0 = tc.relax_last_profile()
    # float64 pair terms, same instances, a few steps
    p = torch.tensor(pos_np, device=dev)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    tc.relax_subdomains(p, world=world, **{**kw, "precision": "fp64", "n_steps": fp64_steps, "polish_steps": 0})
    b.record()
    torch.cuda.synchronize()
    ms64 = a.elapsed_time(b)
    pairs64 = int((sizes * (sizes - 1)).sum()) * fp64_steps
    return {"workload": f"{n_inst} instances, N_k~U[100,5000] (sum {int(sizes.sum())}), arcsine init in Hilbert order, "
                        f"{rounds - 1} kick restarts, mixed L-BFGS(8) {steps} steps + {polish_precision} polish {polish}",
            "relax_time_s": ms_total / 1e3, "pairs_per_s_mixed_with_polish": pairs_total / (ms_total / 1e3),
            "round0_s_graph": ms_rounds[0] / 1e3, "round0_s_no_graph": ms_nograph / 1e3,
            "round0_breakdown_ms": {k: prof0[k] for k in ("pass_ms", "update_ms", "relax_ms", "n_pass")},
            "pairs_per_s_fp64": pairs64 / (ms64 / 1e3), "fp64_steps": fp64_steps,
            "best_energy_sum": float(best_e.sum()),
            "fp64_energy_vs_oracle_max_rel": parity}


def run_full_relax(dev, n: int = N, seed: int = 0, max_mixed: int = 20000, max_polish: int = 100,
                   polish_precision: str = "fp64", line_search: int = 0, extra_mixed: int = 0,
                   oracle_check: bool = True, polish_chunk: int = 0) -> dict:
    """Config C4: one configuration of N charges (arcsine init, Hilbert order) relaxed by mixed-precision
    L-BFGS(8) on the wall map until the RMS of dE/dz falls below 1e-4 x the initial mean force F_ref
    (then `extra_mixed` more mixed steps), then float64 L-BFGS (or the float64-grade fp64x pass) towards
    1e-8 F_ref, stopping there or at max_polish steps.  The returned configuration's float64 energy,
    computed by the library in the polish call, is compared with the oracle's evaluation of the same
    configuration (one half of the sum of its rows' 1/r sums, rows split over every host thread).
    polish_chunk > 0 runs the polish as calls of that many steps (each restarts L-BFGS) and records
    the RMS and float64 energy after each in `polish_trace`."""
    import numpy as np
    import torch

    import oracle
    import synth
    import paper_2609_24722_b300 as tc

    pos = synth.arcsine_disk(n, seed)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    p = torch.tensor(pos, device=dev)
    g0 = tc.grad(p, "fp64")
    f_ref = float(torch.linalg.norm(g0, dim=1).mean().item())
    e0 = tc.energy(p, "fp64").item()
    world = torch.tensor([[0, n]], dtype=torch.int64, device=dev)
    h = math.sqrt(2 * math.pi / (math.sqrt(3.0) * n))
    kw = dict(world=world, optimizer="lbfgs", memory=8, step0=1e-6, maxstep=0.1 * h, accept=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r1 = tc.relax_subdomains(p, precision="mixed", n_steps=max_mixed, gtol=1e-4 * f_ref, line_search=line_search,
                             **kw)
    steps1 = int(r1.steps[0])
    if extra_mixed > 0:
        rx = tc.relax_subdomains(p, precision="mixed", n_steps=extra_mixed, line_search=line_search, **kw)
        steps1 += int(rx.steps[0])
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    e_mid = tc.energy(p, "fp64").item()
    torch.cuda.synchronize()
    t1b = time.perf_counter()
    trace = []
    if polish_chunk > 0:
        done = 0
        while done < max_polish:
            r2 = tc.relax_subdomains(p, precision=polish_precision, n_steps=min(polish_chunk, max_polish - done),
                                     gtol=1e-8 * f_ref, want_energy=True, **kw)
            done += int(r2.steps[0])
            trace.append([done, r2.rms[0].item(), r2.energy[0].item()])
            if r2.rms[0].item() < 1e-8 * f_ref or int(r2.steps[0]) == 0:
                break
        r2_steps = done
    else:
        r2 = tc.relax_subdomains(p, precision=polish_precision, n_steps=max_polish, gtol=1e-8 * f_ref,
                                 want_energy=True, **kw)
        r2_steps = int(r2.steps[0])
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    tc.sync_status()
    e = r2.energy[0].item()
    out = {"workload": f"N={n} arcsine init, mixed L-BFGS(8) to RMS dE/dz < 1e-4 F_ref (+{extra_mixed} steps), "
                       f"{polish_precision} polish towards 1e-8 F_ref (caps {max_mixed} / {max_polish} steps), "
                       f"F_ref = initial mean |F|, Armijo halvings per mixed step: {line_search}",
           "polish_stopped_by": "tolerance" if r2.rms[0].item() < 1e-8 * f_ref else "step cap",
           "mixed_steps": steps1, "mixed_rms": r1.rms[0].item(), "mixed_time_s": t1 - t0,
           "energy_after_mixed": e_mid,
           "polish_steps": r2_steps, "polish_rms": r2.rms[0].item(), "polish_time_s": t2 - t1b,
           "polish_ms_per_step": 1e3 * (t2 - t1b) / max(r2_steps, 1),
           "relax_time_s": (t1 - t0) + (t2 - t1b), "mean_force_initial": f_ref, "tolerance_polish": 1e-8 * f_ref,
           "energy_initial": e0, "energy_final": e, "E_over_N2": e / n ** 2, "pi_over_4": math.pi / 4}
    if trace:
        out["polish_trace"] = trace  # [steps so far, RMS dE/dz, float64 energy] after each call
    if oracle_check:
        x = p.cpu().numpy()
        t3 = time.perf_counter()
        _, rows = oracle.rows_grad(x, np.arange(n, dtype=np.int32), openmp=True)
        e_or = 0.5 * math.fsum(rows.tolist())
        out["oracle_energy"] = e_or
        out["energy_vs_oracle_rel"] = abs(e - e_or) / e_or
        out["oracle_s"] = time.perf_counter() - t3
    return out


def run_cycle(dev, n: int = N, n_sub: int = 256, batch: int = 64, steps: int = 100, m_min: int = 200,
              m_max: int = 4000, period: int = 64, seed: int = 0, local_precision: str = "mixed",
              optimizer: str = "lbfgsb_tu", disjoint: bool = True) -> dict:
    """The adaptive optimisation cycle (Sec. II C) on the GPU, after the border-interior split of
    Sec. II B (N_b of Eq. Nb pinned boundary charges, interior radius ramped from Eq. sigma to 1):
    per batch, local energies of all N charges, defect threshold e_i > mu - sigma_e, centres (80 % at
    defects, 20 % uniform in the disk), zones of the m nearest charges (m a triangle wave between
    m_min and m_max), `steps` mixed steps per zone against all N (projected BB, or the paper's
    L-BFGS-B on (t, u) with optimizer="lbfgsb_tu"), sequential float64 accept.  disjoint=True: a
    batch is the longest prefix of pairwise disjoint zones among the next `batch` subdomains, so no
    relaxed zone is discarded; disjoint=False: fixed batches, where overlapping zones are skipped."""
    import numpy as np
    import torch

    import synth
    import paper_2609_24722_b300 as tc

    pos = synth.lattice_disk(n, seed)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    p = torch.tensor(pos, device=dev)
    # border-interior split (Sec. II B): N_b of Eq. Nb pinned to the circle, the rest inside Eq. sigma
    flags = tc.border_split(p)
    u = torch.tensor(np.random.default_rng(seed + 7).random((n_sub, 3)), device=dev)
    eta = 1e-4 / n
    kw = dict(batch=batch, m_min=m_min, m_max=m_max, period=period, local_precision=local_precision,
              precision="mixed", optimizer=optimizer, n_steps=steps, step0=eta, alpha_min=0.0, alpha_max=10 * eta,
              sigma0=0.0, sigma1=1.0, disjoint=disjoint)
    if optimizer != "bb":
        # quasi-Newton: the first step is eta-scaled, later ones scale themselves; each charge moves
        # at most 1e-3 in (t, u) per step (a sixth of the local spacing at N = 1e5)
        kw.update(memory=8, maxstep=1e-3)
    sizes = np.diff(tc.zone_offsets(n, n_sub, m_min=m_min, m_max=m_max, period=period))
    # warm-up on a copy (graph capture, workspace growth)
    tc.cycle(p.clone(), u[: min(batch, n_sub)], flags, **kw)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    r, trace = tc.cycle(p, u, flags, **kw)
    b.record()
    torch.cuda.synchronize()
    tc.sync_status()
    ms = a.elapsed_time(b)
    tr = trace.cpu().numpy()
    n_batches = len(tr) - 1
    st = r.status.cpu().numpy()
    relaxed = st != 2
    # ordered pairs: every relaxed zone's rows against all N for steps + 1 passes, one local-energy
    # pass per batch
    pairs = int(sizes[relaxed].sum()) * (n - 1) * (steps + 1) + n_batches * n * (n - 1)
    # structure analysis of the cycle's end configuration (Sec. III C-D)
    tc.voronoi_order(p)
    torch.cuda.synchronize()
    a.record()
    _, _, summ, _ = tc.voronoi_order(p)
    b.record()
    torch.cuda.synchronize()
    tc.sync_status()
    structure = {"ms": a.elapsed_time(b), "P_z6": float(summ["P_z"][6]), "mean_abs_psi6": summ["mean_abs_psi6"],
                 "abs_mean_psi6": summ["abs_mean_psi6"]}
    form = (f"batches of the longest disjoint prefix of up to {batch} zones" if disjoint
            else f"fixed batches of {batch}")
    return {"workload": f"N={n} lattice background split into N_b={tc.boundary_count(n)} pinned boundary charges "
                        f"(Eq. Nb) and an interior disk whose radius ramps from Eq. sigma to 1; {n_sub} "
                        f"subdomains in {form}, zones of {m_min}..{m_max} nearest charges (triangle "
                        f"wave, period {period}), {steps} mixed {'BB' if optimizer == 'bb' else optimizer} steps each, "
                        f"{local_precision} local energies per batch, fp64 sequential accept",
            "cycle_time_s": ms / 1e3, "ms_per_subdomain": ms / n_sub, "pairs_per_s": pairs / (ms / 1e3),
            "batches": n_batches, "zones_relaxed": int(relaxed.sum()), "accepted": int((st == 1).sum()),
            "skipped_overlap": int((st == 2).sum()), "accepted_per_s": float((st == 1).sum()) / (ms / 1e3),
            "energy_start": float(tr[0]), "energy_end": float(tr[-1]), "energy_drop": float(tr[0] - tr[-1]),
            "structure": structure}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    import oracle

    pos, idx, off = make_inputs(0)
    per_step_rows = 3000
    times = []
    for k in range(args.warmup + args.steps):
        rows = np.ascontiguousarray(idx[(k * per_step_rows) % (len(idx) - per_step_rows):][:per_step_rows])
        t0 = time.perf_counter()
        oracle.rows_grad(pos, rows)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    ms = 1e3 * statistics.mean(times)
    value = per_step_rows * (N - 1) / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "n_sub": N_SUB, "relax_steps": RELAX_STEPS},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{per_step_rows} subdomain rows x {N} charges per step (tco_rows_grad)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.case:
        return run_case(args)
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2609_24722_b300 as tc
    from paper_2609_24722_b300 import build as tc_build

    world, rank, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    tc_build.build()

    # pick the launch shape of the mixed pass on this GPU (timed, results identical across shapes);
    # --config fixes it instead (profiler runs)
    from paper_2609_24722_b300 import autotune

    if args.config is not None:
        from paper_2609_24722_b300 import _lib

        _lib.check(_lib.lib().tc_set_pass_config(_lib.TC_MIXED, args.config), "tc_set_pass_config")
        tuned = {"best": args.config, "shapes": []}
    else:
        # on the timed workload's own shape: N charges, N_SUB subdomains of m ~ U{200..5000}
        # over the timed workload's RELAX_STEPS passes per shape: the shapes' pass times differ by
        # well under 1 %, and their order changes as the zones spread over the steps
        tuned = autotune.tune(n=N, nsub=N_SUB, reps=RELAX_STEPS - 1, seed=rank, cache=None)

    pos_np, idx_np, off_np = make_inputs(rank)
    pos0 = torch.tensor(pos_np, device=dev)
    pos = pos0.clone()
    idx = torch.tensor(idx_np, device=dev)
    off = torch.tensor(off_np, device=dev)
    eta = 1e-4 / N
    relax_kw = dict(precision="mixed", optimizer="bb", n_steps=RELAX_STEPS, step0=eta, alpha_min=0.0,
                    alpha_max=10 * eta, accept=True, profile=True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 126 MB L2
    stream = torch.cuda.current_stream()

    def step(p):
        e, loc = tc.local_energy(p, LOCAL_PREC)
        r = tc.relax_subdomains(p, idx, off, **relax_kw)
        return e, r

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        pos.copy_(pos0)
        step(pos)
    tc.sync_status()

    clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                          if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local)
    ms, profs, accepted = [], [], []
    clocks.start()
    for _ in range(args.steps):
        pos.copy_(pos0)
        flush.zero_()
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        e, r = step(pos)
        t1.record(stream)
        barrier()
        ms.append(t0.elapsed_time(t1))
        profs.append(tc.relax_last_profile())
        accepted.append(int((r.status == 1).sum().item()))
    clk = clocks.stop()
    tc.sync_status()
    prof = profs[-1]
    pairs_step = N * (N - 1) + RELAX_STEPS * prof["pass_pairs"]
    ms_step, value = aggregate(statistics.mean(ms), pairs_step, world, dev)

    # end to end through the public API: pinned host buffers in, results out, every step
    pos_h = torch.tensor(pos_np).pin_memory()
    idx_h = torch.tensor(idx_np).pin_memory()
    off_h = torch.tensor(off_np).pin_memory()
    out_h = torch.empty_like(pos_h).pin_memory()
    res_h = torch.empty((N_SUB, 4), dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(args.steps):
        flush.zero_()
        barrier()
        t0 = time.perf_counter()
        p_d = pos_h.to(dev, non_blocking=True)
        i_d = idx_h.to(dev, non_blocking=True)
        o_d = off_h.to(dev, non_blocking=True)
        e_d, _ = tc.local_energy(p_d, LOCAL_PREC)
        r = tc.relax_subdomains(p_d, i_d, o_d, **{**relax_kw, "profile": False})
        out_h.copy_(p_d, non_blocking=True)
        res_h[:, 0].copy_(r.delta_e, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_step, e2e_value = aggregate(statistics.mean(e2e_ms), pairs_step, world, dev)
    h2d = pos_h.numel() * 8 + idx_h.numel() * 4 + off_h.numel() * 8
    d2h = out_h.numel() * 8 + N_SUB * 8

    # side by side: one full E+grad at N = 1e5, mixed and float64 (all-pairs kernel)
    def time_allpairs(prec, reps):
        p = pos0.clone()
        tc.grad(p, prec, with_energy=True)
        ts = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tc.grad(p, prec, with_energy=True)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.mean(ts)

    # the C3 relaxation pass in each precision (two profiled steps each, no accept)
    c3_pass = {}
    for prec_name in ("fp64", "fp64x"):
        pc = pos0.clone()
        tc.relax_subdomains(pc, idx, off, **{**relax_kw, "precision": prec_name, "n_steps": 2, "accept": False})
        pr = tc.relax_last_profile()
        ms_p = pr["pass_ms"] / max(pr["n_pass"], 1)
        c3_pass[prec_name] = {"ms_per_pass": ms_p, "pairs_per_s": pr["pass_pairs"] / (ms_p / 1e3)}
    c3_pass["mixed"] = {"ms_per_pass": prof["pass_ms"] / max(prof["n_pass"], 1),
                        "pairs_per_s": prof["pass_pairs"] / (prof["pass_ms"] / max(prof["n_pass"], 1) / 1e3)}
    # the other reading of the subdomain workload (256 subdomains of m ~ U{200..5000} cannot be disjoint
    # in N = 1e5): 256 truly disjoint subdomains with m scaled by 0.9 N / sum(m), every one relaxed and
    # accepted on its own merit (no overlap skips)
    c3_disjoint = run_c3_disjoint(pos_np, relax_kw, flush, stream, reps=2, seed=rank)
    ms_mixed = time_allpairs("mixed", 5)
    ms_f64 = time_allpairs("fp64", 3)
    ms_f64x = time_allpairs("fp64x", 3)
    c5 = run_instances(dev) if not args.no_instances else None
    graph_effect = run_graph_effect(dev) if not args.no_instances else None
    # config C4: the full relaxation of one N = 1e5 configuration, float64 polish, oracle energy check
    c4 = run_full_relax(dev) if not args.no_instances else None
    if c5 is not None:
        c5x = run_instances(dev, polish=50, polish_precision="fp64x")
        c5["fp64x_polish_variant"] = {k: c5x[k] for k in ("workload", "relax_time_s", "pairs_per_s_mixed_with_polish",
                                                            "best_energy_sum", "fp64_energy_vs_oracle_max_rel")}
    # the cycle with the paper's optimiser per zone (L-BFGS-B on (t, u)), and with projected BB
    # (batches of disjoint zones), then the fixed batches whose overlapping zones are skipped
    cyc = run_cycle(dev, optimizer="lbfgsb_tu") if not args.no_instances else None
    if cyc is not None:
        keys = ("workload", "cycle_time_s", "ms_per_subdomain", "batches", "zones_relaxed", "accepted",
                "skipped_overlap", "accepted_per_s", "energy_start", "energy_end", "energy_drop")
        cb = run_cycle(dev, optimizer="bb")
        cyc["bb_variant"] = {k: cb[k] for k in keys}
        cf = run_cycle(dev, optimizer="lbfgsb_tu", disjoint=False)
        cyc["fixed_batches_variant"] = {k: cf[k] for k in keys}
    pipes = tc.probe_pipes()
    tc.sync_status()

    # roofline of the dominant kernel: the mixed relaxation pass (gradient only).
    # Algorithmic work per ordered pair: 8 float32 FMA-pipe operations
    # (dx, dy, r^2 as mul + fma, r^-3 as two muls, two gradient fmas) and 1 MUFU.RSQ.
    pass_ms = prof["pass_ms"] / max(prof["n_pass"], 1)
    achieved = prof["pass_pairs"] / (pass_ms / 1e3)
    peak = min(pipes["ffma_per_s"] / 8.0, pipes["mufu_per_s"])
    roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair/s",
                "frac": achieved / peak, "traffic": RELAX_PASS_DRAM_BYTES,
                "traffic_unit": "bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)",
                "kernel": "k_pass<mixed, grad> (relaxation pair pass)",
                "peak_source": "measured: tc_probe_pipes FFMA lane-ops/s / 8 and MUFU.RSQ/s, this run",
                "frac_of_pairmix_ceiling": achieved / pipes["pairmix_per_s"],
                "pipe_peaks": pipes}
    # the plain float64 form beside it: the all-pairs E + grad at N = 1e5 against the float64 pipe.
    # The pass takes each unordered pair once, except inside the two diagonal tiles of every row block
    # (512 rows), which take every ordered pair. Float64-pipe operations: per ordered pair of a
    # diagonal tile dx, dy; r^2 as a mul and an fma; 1/r from a float32 seed by one series step (mul,
    # fma, fma, mul, fma); r^-3 as two muls; two gradient fmas; one energy add: 14. Per unordered pair
    # elsewhere the same plus the source's two gradient fmas and energy add: 17.
    rb_rows = [min(512, N - b) for b in range(0, N, 512)]
    diag_ordered = sum(m * (m - 1) for m in rb_rows)
    fp64_ops = 14 * diag_ordered + 17 * (N * (N - 1) - diag_ordered) // 2
    fp64_ops_per_pair = fp64_ops / (N * (N - 1))
    fp64_achieved = N * (N - 1) / (ms_f64 / 1e3)
    fp64_peak = pipes["dfma_per_s"] / fp64_ops_per_pair
    roofline_fp64 = {"bound": "fp64", "achieved": fp64_achieved / 1e9, "peak": fp64_peak / 1e9, "unit": "Gpair/s",
                     "frac": fp64_achieved / fp64_peak, "kernel": "k_pass<F64, E+grad, symmetric> (all pairs, N=1e5)",
                     "ops_per_ordered_pair": fp64_ops_per_pair,
                     "peak_source": "measured: tc_probe_pipes DFMA ops/s / float64 ops per ordered pair, this run"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None if args.no_cpu_baseline else cpu_baseline(pos_np, idx_np, off_np)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 pair terms, f64 accumulation (mixed); f64 energies/accept",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "n_sub": N_SUB, "m_range": [M_LO, M_HI],
                   "relax_steps": RELAX_STEPS, "optimizer": "projected BB, step0 1e-4/N, alpha_max 1e-3/N",
                   "accept": "fp64 pairwise, sequential", "pairs_per_step": pairs_step,
                   "pairs_per_step_by_kind": {"energy_only_local_energies": N * (N - 1),
                                              "gradient_only_relaxation": RELAX_STEPS * prof["pass_pairs"],
                                              "energy_and_gradient": 0},
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replica x{world}",
                   "pass_shape": tuned["best"]},
        "pass_shape_ms": {str(r["config"]): round(r["relax_pass_ms"], 4) for r in tuned["shapes"]},
        "relax_time_s": ms_step / 1e3,
        "breakdown_ms": {"relax_pass": prof["pass_ms"], "relax_update": prof["update_ms"],
                         "relax_loop": prof["relax_ms"], "accept": prof["accept_ms"], "setup": prof["setup_ms"]},
        "accepted_subdomains": accepted[-1],
        "allpairs_n1e5": {"mixed_pairs_per_s": N * (N - 1) / (ms_mixed / 1e3), "mixed_ms": ms_mixed,
                          "fp64_pairs_per_s": N * (N - 1) / (ms_f64 / 1e3), "fp64_ms": ms_f64,
                          "fp64x_pairs_per_s": N * (N - 1) / (ms_f64x / 1e3), "fp64x_ms": ms_f64x},
        "c3_relax_pass_by_precision": c3_pass,
        "c3_disjoint_subdomains": c3_disjoint,
        "instances_c5": c5,
        "step_graph_vs_direct": graph_effect,
        "full_relax_c4": c4,
        "adaptive_cycle": cyc,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_step},
        "gpu_launches": args.steps * (prof["launches"] + 3),
        "roofline": roofline,
        "roofline_fp64": roofline_fp64,
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
