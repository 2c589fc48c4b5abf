"""Repeated batched solves under a CUDA graph, and the launch-shape autotuner.

``BatchedSolver`` fixes a packing (matrix orders), captures one call of
``tde_eigvals_batched`` -- every level of every tree in shared launches -- into a
CUDA graph and replays it.  The host work of a call (planning the forest, about
ten launches per tree level) is paid once at capture; a replay is a single
graph launch.

``autotune`` picks the leaf order of the split trees and the warp-per-root
threshold (``tde_set_tuning``) for a packing by timing graph replays on the
caller's data, and caches the choice under a signature of the packing (batch
size, rows, histogram of log2 orders)."""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import _host_offsets, batched_workspace_bytes, eigvals_batched, get_tuning, set_tuning
from . import Workspace

DEFAULT_LEAVES = (4, 8, 16, 32)
DEFAULT_WARP_MIN_K = (128, 256, 512, 1024)


class BatchedSolver:
    """Eigenvalues of a fixed packing, one CUDA-graph replay per call.

    ``solver(d, e)`` copies d and e (CUDA float64, packed like ``offsets``) into the
    captured input buffers, replays the graph and returns the output buffer (which
    the next call overwrites).  The launch tuning active at construction is the one
    captured."""

    def __init__(self, offsets, leaf: int = 8, device="cuda", graph: bool = True):
        import torch

        self.offsets = _host_offsets(offsets)
        self.total = int(self.offsets[-1])
        self.leaf = int(leaf)
        self.device = torch.device(device)
        self.offsets_dev = torch.from_numpy(self.offsets).to(self.device)
        self.d = torch.zeros(max(self.total, 1), dtype=torch.float64, device=self.device)
        self.e = torch.zeros(max(self.total, 1), dtype=torch.float64, device=self.device)
        self.out = torch.empty(max(self.total, 1), dtype=torch.float64, device=self.device)
        self.ws = Workspace(batched_workspace_bytes(self.offsets, self.leaf), self.device)
        self.tuning = get_tuning()
        self.graph = None
        if graph and self.total > 0:
            side = torch.cuda.Stream(device=self.device)
            side.wait_stream(torch.cuda.current_stream(self.device))
            with torch.cuda.stream(side):  # warm-up outside the capture (module loading)
                self._launch(side)
            torch.cuda.current_stream(self.device).wait_stream(side)
            torch.cuda.synchronize(self.device)
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._launch(torch.cuda.current_stream(self.device))

    def _launch(self, stream):
        eigvals_batched(self.d, self.e, self.offsets, leaf=self.leaf, out=self.out, ws=self.ws,
                        stream=stream, check=False, offsets_dev=self.offsets_dev)

    def run(self):
        """Replay on the current stream (inputs already in self.d / self.e)."""
        if self.graph is not None:
            self.graph.replay()
        elif self.total > 0:
            import torch

            self._launch(torch.cuda.current_stream(self.device))
        return self.out[: self.total]

    def __call__(self, d=None, e=None):
        if d is not None:
            self.d[: self.total].copy_(d[: self.total], non_blocking=True)
        if e is not None:
            self.e[: self.total].copy_(e[: self.total], non_blocking=True)
        return self.run()


def signature(offsets) -> str:
    off = _host_offsets(offsets)
    sizes = np.diff(off)
    hist = np.bincount(np.ceil(np.log2(np.maximum(sizes, 1))).astype(np.int64), minlength=32)
    return f"B{len(sizes)}-N{int(off[-1])}-H" + ".".join(str(int(x)) for x in hist)


def _time_solver(solver, d, e, reps: int) -> float:
    import torch

    solver(d, e)
    solver.run()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(reps):
        solver.run()
    ev1.record()
    ev1.synchronize()
    return ev0.elapsed_time(ev1) / reps


def autotune(offsets, d, e, leaves=DEFAULT_LEAVES, warp_min_ks=DEFAULT_WARP_MIN_K, reps: int = 2,
             cache_path: str | None = None, sample: int | None = None, seed: int = 0) -> dict:
    """Coordinate search over the leaf order, then the warp-per-root threshold, by
    timing graph replays.  ``sample`` tunes on that many randomly chosen matrices of
    the packing (same size distribution, less time).  Returns
    {"leaf", "warp_min_k", "ms", "trials", "signature"} and leaves the thread's tuning
    set to the winner."""
    off = _host_offsets(offsets)
    key = signature(off)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        best = cache[key]
        set_tuning(best["warp_min_k"])
        return dict(best, cached=True)
    if sample is not None and sample < len(off) - 1:
        import torch

        idx = np.sort(np.random.default_rng(seed).choice(len(off) - 1, sample, replace=False))
        sizes = np.diff(off)[idx]
        sub = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        pos = np.concatenate([np.arange(off[k], off[k + 1]) for k in idx])
        pos_t = torch.from_numpy(pos).to(d.device)
        d, e, off = d[pos_t], e[pos_t], sub
    trials = []

    def trial(leaf, wmk):
        set_tuning(wmk)
        solver = BatchedSolver(off, leaf=leaf, device=d.device)
        ms = _time_solver(solver, d, e, reps)
        trials.append({"leaf": leaf, "warp_min_k": wmk, "ms": ms})
        return ms

    default_wmk = 256  # the library's default
    best_leaf = min(leaves, key=lambda lf: trial(lf, default_wmk))
    best_wmk = min(warp_min_ks, key=lambda w: trial(best_leaf, w) if w != default_wmk else
                   next(t["ms"] for t in trials if t["leaf"] == best_leaf and t["warp_min_k"] == w))
    best = {"leaf": int(best_leaf), "warp_min_k": int(best_wmk),
            "ms": min(t["ms"] for t in trials if t["leaf"] == best_leaf and t["warp_min_k"] == best_wmk),
            "signature": key, "trials": trials, "sampled_matrices": sample}
    set_tuning(best_wmk)
    if cache_path:
        cache[key] = best
        try:
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return best


def log2_ceil(n: int) -> int:
    return int(math.ceil(math.log2(max(n, 1))))


def _main(argv=None) -> None:
    """Time graph replays of the batched forest on the synthetic packing of 4096
    Lanczos-style tridiagonals (orders log-uniform in [64, 4096]) and print one JSON
    line: ``python -m paper_2605_26599_b300.batched [--leaf 16] [--warp-min-k 512]
    [--reps 3]``."""
    import argparse

    import torch

    from . import inputs, last_launch_count

    ap = argparse.ArgumentParser(description=_main.__doc__.split("\n")[0])
    ap.add_argument("--leaf", type=int, default=16)
    ap.add_argument("--warp-min-k", type=int, default=512)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args(argv)
    d, e, off = inputs.batched_lanczos()
    dt, et = torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()
    set_tuning(args.warp_min_k)
    solver = BatchedSolver(off, leaf=args.leaf)
    launches = last_launch_count()
    ms = _time_solver(solver, dt, et, args.reps)
    set_tuning()
    print(json.dumps({"matrices": len(off) - 1, "rows": int(off[-1]), "leaf": args.leaf,
                      "warp_min_k": args.warp_min_k, "replay_ms": ms,
                      "launches_per_replay": launches}))


if __name__ == "__main__":
    _main()
