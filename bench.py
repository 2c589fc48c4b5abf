#!/usr/bin/env python
"""Benchmark of the B300 boundary-row D&C tridiagonal eigensolver.

Metric: FP64 tridiagonal eigenvalues per second at n = 65536.  One step solves the
four single-matrix families of the n = 65536 workload back to back on one stream:
(a) d, e iid Uniform(-1, 1) (seed 0), (b) Toeplitz d = 2, e = -1, (c) Wilkinson W+,
(d) W+_21 blocks glued by 1e-8.  value = 4 n / step time (inputs resident in HBM).

Printed as one JSON line (rank 0).  Besides the base keys it carries:
  roofline      dominant kernel's algorithmic FP64 rate (per-kernel CUDA events
                inside the timed region, work from the device counters, FP64
                operations per pair with an FMA or a reciprocal counted once)
                against the FP64 FMA rate measured in the same run; the nominal
                rate of the part is reported beside it
  cpu_baseline  the CPU oracle (Sturm bisection) on a bounded sample, host cores
  e2e           the same metric through the public API with pinned host inputs,
                host->device copies and the device->host read of the eigenvalues
                inside the timed region
  clocks        nvidia-smi samples taken during the timed region

``--impl reference`` times the oracle (the only reference this method has) on the
host cores instead.  Under torchrun (N > 1) every rank solves its own copy of the
workload (weak scaling, no data-path collective) and the slowest rank's time is
used; the reference arm runs on rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2605_26599_b300 import inputs  # noqa: E402

METRIC = "FP64 tridiag eigvals/s (n=64K)"
UNIT = "eigvals/s"
FAMILIES = ("a_uniform11", "b_toeplitz", "c_wilkinson", "d_glued_wilkinson")

# Algorithmic work in FP64 operations, an add, multiply, fused multiply-add,
# reciprocal or division each counted once.  Per (pole, root) pair summed or
# multiplied term by term: secular sweep 1 reciprocal + 4 (Delta, z^2 t, the psi and
# psi' sums); Lowner 1 division + 2; boundary rows 1 reciprocal + 6 (Delta, zhat t,
# t^2, low row, high row, norm).  Far blocks taken through their series (block
# expansion of large merges) are counted on the device, per evaluation, as the FP64
# operations they take: the FP64 Horner head of each series (its length set by the
# block's separation tier) plus the block's distance, reciprocal, argument and
# accumulation; the float tails of the series are not counted.
OPS = {  # stage: (ops per exact pair, pair counter, series operations counter)
    "secular": (5, "secular_pairs", "secular_series_ops"),
    "lowner": (3, "lowner_pairs", "lowner_series_ops"),
    "rows": (7, "rows_pairs", "rows_series_ops"),
}
OPS_PER_UNIT = {k: {"per_pair": v[0], "series": "FP64 operations counted on the device"}
                for k, v in OPS.items()}
# nominal FP64 rate of the part (1.25 TFLOP/s, an FMA counting two), in operations per
# second with an FMA counting one: 148 SMs x 2.032 GHz x about 2.08 FMA per SM clock
NOMINAL_FP64_OPS = 0.625e12


def stage_ops(stage: str, work: dict) -> int:
    """Algorithmic FP64 operations of one stage from the device work counters."""
    pp, pc, sc = OPS[stage]
    return pp * work[pc] + work[sc]


def family_inputs(n: int):
    return {
        "a_uniform11": inputs.uniform11(n, seed=0),
        "b_toeplitz": inputs.toeplitz(n, 2.0, -1.0),
        "c_wilkinson": inputs.wilkinson_plus(n),
        "d_glued_wilkinson": inputs.glued_wilkinson(n),
    }


def source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2605_26599_b300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        sms, maxs, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxs.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sms)), "sm_max_mhz": float(max(maxs)),
                "reasons": sorted(reasons), "samples": len(sms)}


def slowest_rank_ms(ms: float, dist, device="cpu") -> float:
    """Max over ranks of a per-rank step time (identity on one rank)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ms: float, world: int, eigvals_per_rank: int) -> float:
    """Whole-job eigenvalues per second: every rank solves its own copy (weak scaling)."""
    return world * eigvals_per_rank / (ms * 1e-3)


# ---------------------------------------------------------------------------
_LAST_SAMPLE = {}  # family -> (indices, oracle eigenvalues) of the last oracle_sample


def oracle_sample(n: int, per_family: int, fams) -> tuple[float, int]:
    """Time the bisection oracle on `per_family` evenly spaced eigenvalue indices of
    each family; returns (seconds, threads used)."""
    import oracle

    ks = np.linspace(0, n - 1, per_family).astype(np.int64)
    t0 = time.perf_counter()
    for name in FAMILIES:
        d, e = fams[name]
        _LAST_SAMPLE[name] = (ks, oracle.eigvals_select(d, e, ks))
    return time.perf_counter() - t0, oracle.last_threads


def cpu_baseline(n: int, fams, target_s: float = 12.0) -> dict:
    # grow the probe until it is long enough to extrapolate from (at least one index
    # per thread, about a second), then size the sample for target_s of oracle work
    per = 64
    t, _ = oracle_sample(n, per, fams)
    while t < 1.0 and per < n:
        per = min(n, per * 4)
        t, _ = oracle_sample(n, per, fams)
    # the probe's rate is pessimistic (thread start-up weighs on short runs): resize
    # once more from the sized run if it came out well short of the target
    for _ in range(2):
        per = int(min(n, max(per, per * target_s / max(t, 1e-3))))
        t, threads = oracle_sample(n, per, fams)
        if t >= 0.6 * target_s or per >= n:
            break
    nf = len(FAMILIES)
    return {"value": nf * per / t, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"Sturm bisection of {per} evenly spaced eigenvalue indices of each of the "
                      f"{nf} families at n={n} ({nf * per} eigenvalues, {t:.1f} s)"}


def accuracy_report(n: int, fams, lam: dict) -> dict:
    """Observed error of the timed solves, per family, from the oracle leg: the
    bisection sample the CPU baseline just computed (max |error| and the paper's
    normalised e_fwd / e_bwd, Sec. 5.1) and a certification of every eigenvalue by
    Sturm counts at the gate 8 n eps ||T||_1 and at gate / 16, / 256, / 4096 (the
    smallest radius at which all n pass bounds the error of the whole spectrum)."""
    import oracle

    eps = np.finfo(np.float64).eps
    out = {}
    for name in FAMILIES:
        d, e = fams[name]
        e = e[: n - 1]
        got = lam[name]
        tn = oracle.norm1(d, e)
        gate = 8 * n * eps * tn
        r = {"gate": gate, "norm1": tn}
        if name in _LAST_SAMPLE:
            ks, ref = _LAST_SAMPLE[name]
            err = float(np.max(np.abs(got[ks] - ref)))
            r.update({"sampled_indices": int(len(ks)), "max_err_sampled": err,
                      "max_err_sampled_over_gate": err / gate,
                      "max_err_sampled_over_eps_norm1": err / (eps * tn),
                      "e_fwd_sampled": oracle.e_fwd(got[ks], ref),
                      "e_bwd_sampled": oracle.e_bwd(got[ks], ref, d, e)})
        t0 = time.perf_counter()
        radius, nfail = oracle.certified_error(d, e, got, gate, levels=(1, 16, 256, 4096))
        r.update({"certified_all_n": nfail == 0, "not_certified": nfail,
                  "certified_radius": radius, "certified_radius_over_gate": radius / gate,
                  "certify_s": time.perf_counter() - t0})
        out[name] = r
    return out


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    n = args.size
    fams = family_inputs(n)
    import oracle

    oracle.build()
    per = args.ref_sample
    for _ in range(args.warmup):
        oracle_sample(n, per, fams)
    times = []
    threads = 0
    for _ in range(args.steps):
        t, threads = oracle_sample(n, per, fams)
        times.append(t)
    step = float(np.mean(times))
    value = len(FAMILIES) * per / step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"single tridiagonals n={n}, families a-d (uniform(-1,1) seed 0, "
                               "Toeplitz 2/-1, Wilkinson W+, glued W+_21)", "n": n,
                   "families": list(FAMILIES),
                   "step": f"oracle bisection of {per} eigenvalue indices per family"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{per} evenly spaced eigenvalue indices per family, n={n}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_ours(args, rank: int, world: int, dist) -> None:
    import torch

    import paper_2605_26599_b300 as tde

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.size
    fams = family_inputs(n)
    host = {}
    devt = {}
    outs = {}
    wss = {}
    for name in FAMILIES:
        d, e = fams[name]
        hd = torch.from_numpy(d).pin_memory()
        he = torch.from_numpy(e).pin_memory()
        host[name] = (hd, he)
        devt[name] = (hd.to(dev), he.to(dev))
        outs[name] = torch.empty(n, dtype=torch.float64, device=dev)
        wss[name] = tde.Workspace(tde.workspace_bytes(n, args.leaf), dev)
    host_out = {name: torch.empty(n, dtype=torch.float64).pin_memory() for name in FAMILIES}
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 126 MB L2

    def one_step():
        launches = 0
        for name in FAMILIES:
            d, e = devt[name]
            tde.eigvals(d, e, leaf=args.leaf, out=outs[name], ws=wss[name], check=False)
            launches += tde.last_launch_count()
        return launches

    def barrier():
        if dist is not None:
            dist.barrier()

    # correctness of the status words once, before timing
    one_step()
    for name in FAMILIES:
        info = tde.get_info(wss[name])
        if info != 0:
            raise RuntimeError(f"device status {info} on family {name}")
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    # stage pass, outside the timed region: an event pair around every kernel of
    # every stage, for the per-stage times and the choice of the dominant stage
    tde.profile_select(None)
    tde.profile_enable(True)
    for _ in range(args.steps):
        flush.zero_()
        one_step()
    torch.cuda.synchronize()
    tde.profile_enable(False)
    kprof_all = tde.profile_collect()
    ktimes = {k: v[0] / args.steps for k, v in kprof_all.items()}
    dominant = max(ktimes, key=ktimes.get)

    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    # timed region: events around the dominant stage's kernels only, so the
    # other stages run without event records between their launches
    tde.profile_select([dominant])
    tde.profile_enable(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    fam_ev = {name: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                     for _ in range(args.steps)] for name in FAMILIES}
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    launches = 0
    for i in range(args.steps):
        flush.zero_()  # L2 flush between steps, outside the event-timed region
        starts[i].record(stream)
        for name in FAMILIES:
            d, e = devt[name]
            fam_ev[name][i][0].record(stream)
            tde.eigvals(d, e, leaf=args.leaf, out=outs[name], ws=wss[name], check=False)
            fam_ev[name][i][1].record(stream)
            launches += tde.last_launch_count()
        ends[i].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    tde.profile_enable(False)
    kprof = tde.profile_collect()
    tde.profile_select(None)
    clocks = sampler.stop() if sampler else None
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    fam_ms = {name: float(np.mean([a.elapsed_time(b) for a, b in fam_ev[name]])) for name in FAMILIES}
    ms = slowest_rank_ms(float(np.mean(step_ms)), dist, dev)
    value = job_value(ms, world, len(FAMILIES) * n)

    # device work of one step (identical every step)
    work = {k: 0 for k in ("secular_pairs", "secular32_pairs", "lowner_pairs", "rows_pairs", "secular_sweeps",
                           "secular32_sweeps", "roots", "deflated", "rotations", "leaf_rotations",
                           "secular_far_blocks", "lowner_far_blocks", "rows_far_series",
                           "secular_series_ops", "lowner_series_ops", "rows_series_ops")}
    per_family_work = {}
    for name in FAMILIES:
        w = tde.read_work(wss[name])
        per_family_work[name] = w
        for k in work:
            work[k] += w[k]

    # end to end through the public API, pinned host buffers
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for name in FAMILIES:
            hd, he = host[name]
            d, e = devt[name]
            d.copy_(hd, non_blocking=True)
            e.copy_(he, non_blocking=True)
            tde.eigvals(d, e, leaf=args.leaf, out=outs[name], ws=wss[name], check=False)
            host_out[name].copy_(outs[name], non_blocking=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(ev0.elapsed_time(ev1))
    e2e_step = slowest_rank_ms(float(np.mean(e2e_ms)), dist, dev)
    h2d = sum(host[nm][0].numel() * 8 + host[nm][1].numel() * 8 for nm in FAMILIES)
    d2h = len(FAMILIES) * n * 8

    if rank != 0:
        return
    # roofline of the dominant kernel
    fma_per_s = tde.measure_fp64_peak()
    peak_tops = fma_per_s / 1e12  # FP64 operations per second, one per FMA
    dom_ms = kprof[dominant][0] / args.steps  # live, from the timed region
    klaunch = {k: v[1] / args.steps for k, v in kprof_all.items()}
    roof = {"bound": "alu", "kernel": dominant, "unit": "T FP64 ops/s (FMA counted once)",
            "peak": peak_tops,
            "peak_source": "FP64 FMA-chain microbenchmark run in this process; "
                           "MEASURED_PEAKS.json carries no FP64 figure",
            "peak_nominal": NOMINAL_FP64_OPS / 1e12,
            "ops_per_unit": OPS_PER_UNIT}
    if dominant in OPS:
        ops = stage_ops(dominant, work)
        achieved = ops / (dom_ms * 1e-3) / 1e12
        roof.update({"achieved": achieved, "frac": achieved / peak_tops,
                     "frac_nominal": achieved / (NOMINAL_FP64_OPS / 1e12),
                     "algorithmic_ops_per_step": ops,
                     "units_per_step": {"exact_pairs": work[OPS[dominant][1]],
                                        "series_ops": work[OPS[dominant][2]]},
                     "ms_per_step": dom_ms, "timing": "CUDA events around the stage's kernels "
                                                      "inside the timed region",
                     "launches_per_step": klaunch[dominant],
                     "avg_launch_ms": dom_ms / max(klaunch[dominant], 1)})
    else:
        roof.update({"achieved": None, "frac": None,
                     "note": f"dominant kernel {dominant} is not an FP64 pair kernel"})
    roof["traffic"] = load_traffic(dominant)
    executed = load_executed_rate(dominant)
    if executed is not None:
        # instruction-level reading of "% FP64 peak": FMA counted twice, against the
        # measured FMA rate times two
        executed["frac_of_measured"] = executed["executed_tflops"] / (2.0 * peak_tops)
        roof["executed_fp64_ncu"] = executed
    roof["numerator_note"] = (
        "algorithmic FP64 operations of the work actually done: exact (pole, root) pairs "
        "at 5/3/7 operations plus the FP64 heads of the block-expansion series of distant "
        "pole blocks (counted on the device); not the paper's all-pairs K^2 sweeps, which "
        "this solver evaluates only for nearby blocks")
    kernel_rates = {}
    for k in OPS:
        if ktimes.get(k, 0) > 0:
            ops = stage_ops(k, work)
            kernel_rates[k] = {"ms_per_step": ktimes[k], "tops": ops / (ktimes[k] * 1e-3) / 1e12,
                               "frac_of_peak": ops / (ktimes[k] * 1e-3) / 1e12 / peak_tops}
            ex = load_executed_rate(k)
            if ex is not None:  # instruction-level rate of the stage's top launch (ncu)
                ex["frac_of_measured"] = ex["executed_tflops"] / (2.0 * peak_tops)
                kernel_rates[k]["executed_fp64_ncu"] = ex

    cpu = cpu_baseline(n, fams) if (world == 1 and not args.no_cpu_baseline) else None
    accuracy = None
    if cpu is not None:
        accuracy = accuracy_report(n, fams, {name: outs[name].cpu().numpy() for name in FAMILIES})
    extras = {}
    which = set() if args.no_extras else set(x for x in args.extras.split(",") if x)
    if "batched" in which:
        extras["batched"] = batched_section(args, dev)
    if "backward" in which:
        extras["backward"] = backward_section(args, dev)
    if "rows" in which:
        extras["eigvec_rows"] = rows_section(args, dev, fma_per_s)
    if "dense" in which:
        extras["dense"] = dense_section(args, dev, fma_per_s)
    if "context" in which:
        extras["paper_context"] = context_section(args, dev)
    if "configs" in which:
        extras["other_configs"] = configs_section(args, dev)
    if "sweep" in which:
        extras["paper_family_sweep"] = sweep_section(args, dev)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"single tridiagonals n={n}, families a-d (uniform(-1,1) seed 0, "
                               "Toeplitz 2/-1, Wilkinson W+, glued W+_21)",
                   "n": n, "families": list(FAMILIES), "leaf": args.leaf,
                   "l2": "flushed between steps (256 MB write outside the event-timed region); "
                         "inputs are smaller than L2",
                   "per_family_ms": fam_ms, "step_ms_min": float(min(step_ms)),
                   "kernel_ms_per_step": ktimes,
                   "kernel_ms_source": "stage pass before the timed region (events around "
                                       "every kernel); inside the timed region only the "
                                       f"{dominant} stage carries events",
                   "wall_s_timed_region": wall, "work_per_step": work},
        "gpu_launches": launches,
        "roofline": roof,
        "kernel_fp64_rates": kernel_rates,
        "cpu_baseline": cpu,
        "accuracy": accuracy,
        "e2e": {"value": job_value(e2e_step, world, len(FAMILIES) * n), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_step},
        "clocks": clocks,
        "source_hash": source_hash(),
    }
    line.update(extras)
    print(json.dumps(line), flush=True)


def batched_section(args, dev) -> dict:
    """Config 3: 4096 Lanczos-style tridiagonals (orders log-uniform in [64, 4096]) solved
    by one CUDA-graph replay of the forest solver (launch shape autotuned on a 512-matrix
    sample), against the plain per-matrix loop on one stream."""
    import torch

    import oracle
    import paper_2605_26599_b300 as tde
    from paper_2605_26599_b300.batched import BatchedSolver, autotune

    d, e, off = inputs.batched_lanczos()
    B = len(off) - 1
    dt, et = torch.from_numpy(d).to(dev), torch.from_numpy(e).to(dev)
    best = autotune(off, dt, et, leaves=(4, 8, 16), warp_min_ks=(256, 512, 1024), reps=2,
                    sample=512)
    solver = BatchedSolver(off, leaf=best["leaf"], device=dev)
    solver(dt, et)
    for _ in range(args.warmup):
        solver.run()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    reps = max(args.steps, 3)
    ev[0].record()
    for _ in range(reps):
        solver.run()
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / reps
    lam = solver.run().cpu().numpy()
    # accuracy on 48 sampled matrices, 12 sampled eigenvalues each
    rng = np.random.default_rng(0)
    worst = 0.0
    for k in rng.choice(B, 48, replace=False):
        a, b = int(off[k]), int(off[k + 1])
        ks = np.unique(np.linspace(0, b - a - 1, 12).astype(np.int64))
        ref = oracle.eigvals_select(d[a:b], e[a:b - 1], ks)
        gate = 8 * (b - a) * np.finfo(np.float64).eps * oracle.norm1(d[a:b], e[a:b - 1])
        worst = max(worst, float(np.max(np.abs(lam[a:b][ks] - ref)) / gate))
    # the plain per-matrix loop (single-matrix entry point, one stream)
    ws = tde.Workspace(tde.workspace_bytes(4096, best["leaf"]), dev)
    out = torch.empty_like(dt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(B):
        a, b = int(off[k]), int(off[k + 1])
        tde.eigvals(dt[a:b], et[a:b], leaf=best["leaf"], out=out[a:b], ws=ws, check=False)
    torch.cuda.synchronize()
    loop_s = time.perf_counter() - t0
    tde.set_tuning()
    return {"workload": f"{B} Lanczos-style tridiagonals, n_k log-uniform [64, 4096], "
                        f"{int(off[-1])} rows (seed 0)",
            "solves_per_s": B / (ms * 1e-3), "ms_per_batch": ms, "graph": True,
            "tuned": {"leaf": best["leaf"], "warp_min_k": best["warp_min_k"],
                      "trials": len(best.get("trials", []))},
            "per_matrix_loop_solves_per_s": B / loop_s, "per_matrix_loop_ms": loop_s * 1e3,
            "speedup_vs_loop": (B / (ms * 1e-3)) / (B / loop_s),
            "max_err_over_gate_sampled": worst}


def rows_section(args, dev, fma_per_s: float) -> dict:
    """Requested eigenvector rows (Algorithm 1 with a general row list): 16 rows spread
    over the n = --size matrix, Toeplitz (weak deflation: the costly case) and
    uniform(-1, 1).  Time against the eigenvalues alone, the FP64 pipe use of the
    requested-row update (7 FP64 instructions per (pole, root) sweep shared by up to
    four rows, plus one fused multiply-add per row), and the identities
    Q_s Q_s^T = I, Q_s diag(lambda) Q_s^T = T[s][:, s] at full size."""
    import torch

    import oracle
    import paper_2605_26599_b300 as tde

    n, leaf, nsel = args.size, args.leaf, 16
    rows = np.linspace(0, n - 1, nsel).astype(np.int64)
    fams = family_inputs(n)
    res = {"rows_requested": nsel, "n": n, "leaf": leaf}
    for name in ("b_toeplitz", "a_uniform11"):
        d, e = fams[name]
        dt, et = torch.from_numpy(d).to(dev), torch.from_numpy(e).to(dev)
        rt = torch.from_numpy(rows).to(dev)
        ws = tde.Workspace(tde.eigvecs_rows_workspace_bytes(n, nsel, leaf), dev)
        lam = torch.empty(n, dtype=torch.float64, device=dev)
        q = torch.empty((nsel, n), dtype=torch.float64, device=dev)
        ews = tde.Workspace(tde.workspace_bytes(n, leaf), dev)
        tde.eigvecs_rows(dt, et, rt, leaf=leaf, out=lam, qrows=q, ws=ws)
        tde.eigvals(dt, et, leaf=leaf, out=lam, ws=ews)
        torch.cuda.synchronize()
        reps = 2
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        for _ in range(reps):
            tde.eigvals(dt, et, leaf=leaf, out=lam, ws=ews, check=False)
        ev[1].record()
        tde.profile_enable(True)
        for _ in range(reps):
            tde.eigvecs_rows(dt, et, rt, leaf=leaf, out=lam, qrows=q, ws=ws, check=False)
        ev[2].record()
        torch.cuda.synchronize()
        tde.profile_enable(False)
        kp = tde.profile_collect()
        w = tde.read_work(ws)
        info = tde.get_info(ws)
        vals_ms = ev[0].elapsed_time(ev[1]) / reps
        rows_ms = ev[1].elapsed_time(ev[2]) / reps
        upd_ms = kp["sel_rows"][0] / reps
        instr = 7 * w["sel_sweep_pairs"] + w["sel_row_pairs"]
        qn, ln = q.cpu().numpy(), lam.cpu().numpy()
        blk = oracle.principal_block(d, e[: n - 1], rows)
        res[name] = {
            "eigvals_ms": vals_ms, "eigvecs_rows_ms": rows_ms, "extra_ms_per_row": (rows_ms - vals_ms) / nsel,
            "row_update_ms": upd_ms, "row_bookkeeping_ms": kp["sel"][0] / reps,
            "row_pairs": w["sel_row_pairs"], "sweep_pairs": w["sel_sweep_pairs"],
            "row_update_fp64_pipe_frac": instr / (upd_ms * 1e-3) / fma_per_s if upd_ms > 0 else None,
            "orthonormality_err": float(np.abs(qn @ qn.T - np.eye(nsel)).max()),
            "block_identity_err": float(np.abs((qn * ln) @ qn.T - blk).max()),
            "device_status": info}
    return res


def dense_section(args, dev, fma_per_s: float) -> dict:
    """Dense front end (Householder reduction to tridiagonal form, then the
    boundary-row solver): a dense symmetric (G + G^T)/2 of order 8192, time and FP64
    rate of the reduction ((2/3) n^3 FMAs), trace / Frobenius invariants of the
    spectrum; the oracle (LAPACK on the host cores) timed beside it at n = 2048."""
    import time

    import torch

    import oracle
    import paper_2605_26599_b300 as tde

    res = {}
    for n in (int(x) for x in args.dense_sizes.split(",") if x):
        a = inputs.dense_goe(n, seed=1)
        at = torch.from_numpy(a).to(dev)
        ws = tde.Workspace(tde.dense_eigvals_workspace_bytes(n, args.leaf), dev)
        lam = tde.dense_eigvals(at, leaf=args.leaf, ws=ws)
        torch.cuda.synchronize()
        tde.profile_enable(True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        lam = tde.dense_eigvals(at, leaf=args.leaf, ws=ws, check=False)
        ev[1].record()
        torch.cuda.synchronize()
        tde.profile_enable(False)
        tri_ms = sum(v[0] for v in tde.profile_collect().values())
        ms = ev[0].elapsed_time(ev[1])
        fmas = sum(2 * m * (m + 1) for m in range(1, n))
        ln = lam.cpu().numpy()
        nrm = float(np.linalg.norm(a))
        r = {"ms": ms, "tridiagonal_solve_ms": tri_ms, "reduction_ms": ms - tri_ms,
             "reduction_fp64_fma_frac": fmas / ((ms - tri_ms) * 1e-3) / fma_per_s,
             "trace_err_rel": abs(ln.sum() - np.trace(a)) / nrm,
             "frobenius_err_rel": abs((ln ** 2).sum() - nrm ** 2) / nrm ** 2,
             "device_status": tde.get_info(ws)}
        if n == 2048:
            t0 = time.perf_counter()
            ref = oracle.dense_eigvals(a)
            r["oracle_cpu_ms"] = (time.perf_counter() - t0) * 1e3
            r["max_err_vs_oracle_over_gate"] = float(np.abs(ln - ref).max() / (8 * n * np.finfo(float).eps * nrm))
        res[f"n{n}"] = r
    res["workload"] = "dense symmetric (G + G^T)/2, G iid N(0,1), seed 1"
    return res


# The paper's GPU table (Sec. 5, H100 PCIe, values-only D&C, N = 49152): its families
# and milliseconds, for context only (different matrices: its generator is not
# reproducible; different GPU).
PAPER_H100_MS = {"paper_normal": 78.73, "paper_uniform": 85.75, "toeplitz025": 480.81,
                 "paper_clustered": 697.22}


def context_section(args, dev) -> dict:
    """The paper's four GPU families at N = 49152 with its protocol (2 warm-up, 5 timed
    runs, mean), beside its H100 milliseconds; max error against sampled oracle
    eigenvalues in units of the 8 N eps ||T||_1 gate."""
    import torch

    import oracle
    import paper_2605_26599_b300 as tde

    n = 49152
    res = {"n": n, "leaf": args.leaf, "protocol": "2 warm-up + 5 timed runs, mean, CUDA events"}
    for fam, h100 in PAPER_H100_MS.items():
        d, e = inputs.family(fam, n, seed=0)
        e = e[: n - 1]
        dt = torch.from_numpy(d).to(dev)
        et = torch.from_numpy(np.concatenate([e, [0.0]])).to(dev)
        ws = tde.Workspace(tde.workspace_bytes(n, args.leaf), dev)
        lam = torch.empty(n, dtype=torch.float64, device=dev)
        for _ in range(2):
            tde.eigvals(dt, et, leaf=args.leaf, out=lam, ws=ws)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(5):
            tde.eigvals(dt, et, leaf=args.leaf, out=lam, ws=ws, check=False)
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / 5
        ks = np.unique(np.concatenate([np.linspace(0, n - 1, 64).astype(np.int64), [0, 1, n - 2, n - 1]]))
        ref = oracle.eigvals_select(d, e, ks)
        err = float(np.abs(np.sort(lam.cpu().numpy())[ks] - ref).max())
        res[fam] = {"ms": ms, "paper_h100_ms": h100, "h100_over_b300": h100 / ms,
                    "max_err_over_gate_sampled": err / (8 * n * np.finfo(float).eps * oracle.norm1(d, e)),
                    "device_status": tde.get_info(ws)}
    return res


def _time_solve(tde, dt, et, leaf, reps, warm=3):
    """Mean event-timed ms of `reps` solves after `warm` untimed ones (L2 flushed
    before every timed solve, outside its events); returns (ms, eigenvalues, status,
    workspace bytes)."""
    import torch

    n = dt.shape[0]
    ws = tde.Workspace(tde.workspace_bytes(n, leaf), dt.device)
    lam = torch.empty(n, dtype=torch.float64, device=dt.device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dt.device)
    for _ in range(warm):
        tde.eigvals(dt, et, leaf=leaf, out=lam, ws=ws, check=False)
    total = 0.0
    for _ in range(reps):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        tde.eigvals(dt, et, leaf=leaf, out=lam, ws=ws, check=False)
        ev[1].record()
        torch.cuda.synchronize()
        total += ev[0].elapsed_time(ev[1])
    return total / reps, lam.cpu().numpy(), tde.get_info(ws), ws.nbytes


def configs_section(args, dev) -> dict:
    """The other single-matrix configurations, timed like the headline step (3 warm-up,
    L2 flushed before each timed solve): n = 2048 uniform(-1, 1) seed 0 at leaf 32 (every
    eigenvalue against the bisection oracle), and the large orders n = 131072, 262144
    with d ~ N(0,1), e ~ |N(0,1)| (seed 0) and the graded matrix, with the workspace
    bytes (O(n): asserted <= 256 n in the tests) and the error against 64 sampled oracle
    eigenvalues."""
    import torch

    import oracle
    import paper_2605_26599_b300 as tde

    eps = np.finfo(np.float64).eps
    res = {}
    d, e = inputs.uniform11(2048, seed=0)
    ms, lam, info, wsb = _time_solve(tde, torch.from_numpy(d).to(dev), torch.from_numpy(e).to(dev),
                                     32, reps=max(args.steps, 5))
    ref = oracle.eigvals_bisect(d, e[:2047])
    gate = 8 * 2048 * eps * oracle.norm1(d, e[:2047])
    res["n2048_uniform11_leaf32"] = {
        "ms": ms, "eigvals_per_s": 2048 / (ms * 1e-3), "leaf": 32, "workspace_bytes": wsb,
        "max_err_all": float(np.abs(lam - ref).max()),
        "max_err_all_over_gate": float(np.abs(lam - ref).max()) / gate, "device_status": info}
    # the same matrix with the default leaf order (the leaf QR is a chain of dependent
    # FP64 operations, so shorter leaves and more merge levels win on this part)
    ms8, lam8, info8, wsb8 = _time_solve(tde, torch.from_numpy(d).to(dev), torch.from_numpy(e).to(dev),
                                         args.leaf, reps=max(args.steps, 5))
    res["n2048_uniform11_default_leaf"] = {
        "ms": ms8, "eigvals_per_s": 2048 / (ms8 * 1e-3), "leaf": args.leaf,
        "max_err_all_over_gate": float(np.abs(lam8 - ref).max()) / gate, "device_status": info8}
    for n in (131072, 262144):
        for fam in ("normal", "graded"):
            d, e = inputs.family(fam, n, seed=0)
            ms, lam, info, wsb = _time_solve(tde, torch.from_numpy(d).to(dev),
                                             torch.from_numpy(e).to(dev), args.leaf,
                                             reps=max(args.steps, 3))
            ks = np.unique(np.concatenate([np.linspace(0, n - 1, 60).astype(np.int64),
                                           [0, 1, n - 2, n - 1]]))
            ref = oracle.eigvals_select(d, e[: n - 1], ks)
            gate = 8 * n * eps * oracle.norm1(d, e[: n - 1])
            err = float(np.abs(lam[ks] - ref).max())
            res[f"n{n}_{fam}"] = {"ms": ms, "eigvals_per_s": n / (ms * 1e-3), "leaf": args.leaf,
                                  "workspace_bytes": wsb, "workspace_bytes_per_row": wsb / n,
                                  "max_err_sampled": err, "max_err_sampled_over_gate": err / gate,
                                  "device_status": info}
    return res


SWEEP_FAMILIES = ("paper_uniform", "paper_normal", "toeplitz025", "paper_clustered")
SWEEP_N = (4096, 8192, 16384, 32768, 49152, 65536)


def sweep_section(args, dev) -> dict:
    """The paper's four families (Sec. 5.1: uniform and normal diagonals with
    off-diagonals U(0.1, 0.3), Toeplitz 2 / 0.25, clustered) at N = 4096 ... 65536:
    ms per solve (3 warm-up, 5 timed, L2 flushed), eigvals/s, and the exponent p of a
    least-squares fit ms ~ c N^p over the sweep, the shape the paper's scaling
    statements describe (near-linear for the random families, close to quadratic for
    Toeplitz and clustered)."""
    import torch

    import paper_2605_26599_b300 as tde

    res = {"n": list(SWEEP_N), "leaf": args.leaf}
    for fam in SWEEP_FAMILIES:
        ms_all = []
        for n in SWEEP_N:
            d, e = inputs.family(fam, n, seed=0)
            ms, _, info, _ = _time_solve(tde, torch.from_numpy(d).to(dev),
                                         torch.from_numpy(e).to(dev), args.leaf, reps=5)
            if info != 0:
                raise RuntimeError(f"device status {info} in the sweep ({fam}, n={n})")
            ms_all.append(ms)
        x, y = np.log(np.asarray(SWEEP_N, dtype=float)), np.log(np.asarray(ms_all))
        p = float(np.polyfit(x, y, 1)[0])
        p_top = float(np.polyfit(x[-3:], y[-3:], 1)[0])
        res[fam] = {"ms": ms_all, "eigvals_per_s": [n / (m * 1e-3) for n, m in zip(SWEEP_N, ms_all)],
                    "fitted_exponent": p, "fitted_exponent_top3": p_top}
    return res


def backward_section(args, dev) -> dict:
    """Config 4: 256 tridiagonals of order 8192 (d ~ N(0,1), e ~ |N(0,0.5)|), loss
    L = sum_i w_i lambda_i^2: forward (batched) and the hand-written adjoint, timed
    separately, in the default O(n) workspace (4 checkpoint slots, levels recomputed)
    and in the every-level layout; gradient error against the dense-eigh gradient on
    n = 256 copies."""
    import torch

    import oracle
    import paper_2605_26599_b300 as tde

    d, e, off, w = inputs.grad_batch()
    dt, et = torch.from_numpy(d).to(dev), torch.from_numpy(e).to(dev)
    wt = torch.from_numpy(w).to(dev)
    leaf = 8
    fws = tde.Workspace(tde.batched_workspace_bytes(off, leaf), dev)
    offd = torch.from_numpy(off).to(dev)
    lam = torch.empty_like(dt)
    gl = torch.empty_like(dt)

    def fwd():
        tde.eigvals_batched(dt, et, off, leaf=leaf, out=lam, ws=fws, check=False, offsets_dev=offd)

    res = {"workload": "256 tridiagonals n=8192, d~N(0,1), e~|N(0,0.5)|, L=sum w lambda^2",
           "rows": int(off[-1]), "leaf": leaf, "forward_workspace_bytes": fws.nbytes}
    reps = max(args.steps, 3)
    grads = {}
    for name, slots in (("o_n", None), ("levels", 0)):
        bws = tde.Workspace(tde.backward_workspace_bytes(off, leaf, slots), dev)

        def bwd():
            torch.mul(wt, lam, out=gl)
            gl.mul_(2.0)
            return tde.eigvals_backward(dt, et, gl, offsets=off, leaf=leaf, ws=bws, check=False,
                                        offsets_dev=offd, slots=slots)

        for _ in range(2):
            fwd()
            bwd()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        for _ in range(reps):
            fwd()
        ev[1].record()
        for _ in range(reps):
            out = bwd()
        ev[2].record()
        torch.cuda.synchronize()
        fms = ev[0].elapsed_time(ev[1]) / reps
        bms = ev[1].elapsed_time(ev[2]) / reps
        grads[name] = out[1].cpu().numpy()
        res[name] = {"forward_ms": fms, "backward_ms": bms, "bwd_over_fwd": bms / fms,
                     "backward_workspace_bytes": bws.nbytes,
                     "backward_workspace_bytes_per_row": bws.nbytes / int(off[-1]),
                     "device_status": tde.get_info(bws)}
    res["layouts_bitwise_equal"] = bool(np.array_equal(grads["o_n"], grads["levels"]))
    # accuracy on n = 256 copies of the family against the dense-eigh gradient
    worst = 0.0
    for seed in range(4):
        dd, ee = inputs.normal_absnormal(256, seed=100 + seed, e_scale=0.5)
        ww = np.random.default_rng(200 + seed).uniform(0, 1, 256)
        ddt = torch.from_numpy(dd).to(dev)
        eet = torch.from_numpy(np.concatenate([ee, [0.0]])).to(dev)
        lm = tde.eigvals(ddt, eet, leaf=leaf)
        _, gd, ge = tde.eigvals_backward(ddt, eet, 2.0 * torch.from_numpy(ww).to(dev) * lm, leaf=leaf)
        rd, re_ = oracle.grad_dense(dd, ee, ww)
        worst = max(worst, float(np.max(np.abs(gd.cpu().numpy() - rd)) / np.max(np.abs(rd))),
                    float(np.max(np.abs(ge.cpu().numpy()[:255] - re_)) / np.max(np.abs(re_))))
    res["grad_rel_err_vs_dense_eigh_n256"] = worst
    # headline figures: the default O(n) layout
    res.update({"forward_ms": res["o_n"]["forward_ms"], "backward_ms": res["o_n"]["backward_ms"],
                "bwd_over_fwd": res["o_n"]["bwd_over_fwd"],
                "backward_workspace_bytes": res["o_n"]["backward_workspace_bytes"]})
    return res


def load_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from a committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    entry = rec.get(kernel)
    if not entry or entry.get("source_hash") != source_hash():
        return None
    return entry.get("dram_bytes_per_launch")


def load_executed_rate(kernel: str):
    """ncu's executed FP64 rate of `kernel`'s top launches ((dadd + dmul + 2 dfma) per
    second over the launch) from a committed summary, if it was taken on the current
    kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    entry = rec.get(kernel)
    if not entry or entry.get("source_hash") != source_hash() or "executed_tflops" not in entry:
        return None
    return {"executed_tflops": entry["executed_tflops"], "launches": entry.get("launches"),
            "what": entry.get("executed_what")}


def main():
    global FAMILIES
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=65536, help="matrix order n")
    ap.add_argument("--leaf", type=int, default=8,
                    help="largest leaf order of the split tree (8: fastest measured on B300)")
    ap.add_argument("--families", default=",".join(FAMILIES),
                    help="comma-separated subset of the four families (profiling runs)")
    ap.add_argument("--ref-sample", type=int, default=96,
                    help="eigenvalue indices per family per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip every extra measurement (see --extras)")
    ap.add_argument("--dense-sizes", default="2048,8192",
                    help="orders of the dense front end's section (comma list)")
    ap.add_argument("--extras", default="configs,batched,backward,sweep,rows,dense,context",
                    help="which extra measurements to run (comma list of configs, batched, "
                         "backward, sweep, rows, dense, context)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    fams = tuple(f for f in args.families.split(",") if f)
    if not fams or any(f not in FAMILIES for f in fams):
        ap.error(f"--families must be a subset of {','.join(FAMILIES)}")
    FAMILIES = fams

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist

        backend = "nccl" if torch.cuda.is_available() and args.impl == "ours" else "gloo"
        tdist.init_process_group(backend=backend)
        dist = tdist
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
