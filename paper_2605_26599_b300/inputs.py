"""Seeded synthetic tridiagonal inputs (shared by the solver's tests, the oracle's
tests and the benchmark).  This module holds none of the solver's arithmetic: it
only draws (d, e) arrays.

Random draws use ``numpy.random.default_rng(seed)`` (PCG64) in float64, drawing
``d`` first and then ``e``.  The paper's own matrices come from an unspecified
xorshift generator (Sec. 5.1) and cannot be reproduced; these families follow its
distributions and the workload shapes the solver is benchmarked on.

Every generator returns ``(d, e)`` with ``len(d) == n`` and ``len(e) == n - 1``.
"""
from __future__ import annotations

import math

import numpy as np


def uniform11(n: int, seed: int = 0):
    """d, e iid Uniform(-1, 1)."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(-1.0, 1.0, n)
    e = rng.uniform(-1.0, 1.0, max(n - 1, 0))
    return d, e


def toeplitz(n: int, a: float = 2.0, b: float = -1.0):
    """Constant tridiag(b, a, b); spectrum a + 2 b cos(k pi / (n + 1))."""
    return np.full(n, float(a)), np.full(max(n - 1, 0), float(b))


def wilkinson_plus(n: int):
    """Wilkinson W+_n: d_i = |i - (n - 1) / 2| (i = 0..n-1), e = 1.  For even n the
    diagonal holds half-integers."""
    i = np.arange(n, dtype=np.float64)
    return np.abs(i - (n - 1) / 2.0), np.ones(max(n - 1, 0))


def glued_wilkinson(n: int, block: int = 21, glue: float = 1e-8):
    """W+_block blocks (d_i = |i - (block - 1) / 2|, e = 1 inside a block) tiled
    along the diagonal to length n (the last block truncated) and joined by
    off-diagonal entries equal to ``glue``."""
    i = np.arange(n)
    j = (i % block).astype(np.float64)
    d = np.abs(j - (block - 1) / 2.0)
    e = np.ones(max(n - 1, 0))
    if n > 1:
        e[(np.arange(n - 1) % block) == block - 1] = glue
    return d, e


def normal_absnormal(n: int, seed: int = 0, e_scale: float = 1.0):
    """d ~ N(0, 1), e ~ |N(0, e_scale)| (e_scale is the standard deviation)."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal(n)
    e = np.abs(rng.standard_normal(max(n - 1, 0))) * e_scale
    return d, e


def graded(n: int):
    """d_i = 10^(-12 i / n), e_i = 10^(-6 i / n)."""
    i = np.arange(n, dtype=np.float64)
    d = 10.0 ** (-12.0 * i / n)
    e = 10.0 ** (-6.0 * np.arange(max(n - 1, 0), dtype=np.float64) / n)
    return d, e


def lanczos_like(n: int, rng):
    """d ~ Uniform(-1, 1), e ~ sqrt(Uniform(0.1, 1)) from an existing generator."""
    d = rng.uniform(-1.0, 1.0, n)
    e = np.sqrt(rng.uniform(0.1, 1.0, max(n - 1, 0)))
    return d, e


def batched_sizes(batch: int = 4096, lo: int = 64, hi: int = 4096, seed: int = 0):
    """Matrix orders drawn log-uniform in [lo, hi]: n_k = floor(exp(U(ln lo, ln(hi+1))))."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi + 1), batch)
    return np.minimum(np.floor(np.exp(u)).astype(np.int64), hi)


def batched_lanczos(batch: int = 4096, lo: int = 64, hi: int = 4096, seed: int = 0):
    """A packed batch of Lanczos-style Jacobi matrices of log-uniform orders.

    Returns (d, e, offsets): matrix k occupies rows offsets[k]..offsets[k+1]-1 of the
    packed d and e; e has the same length as d and its entry at the last row of each
    matrix is unused (set to 0)."""
    sizes = batched_sizes(batch, lo, hi, seed)
    rng = np.random.default_rng(seed + 1)
    offsets = np.zeros(batch + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    total = int(offsets[-1])
    d = np.empty(total)
    e = np.zeros(total)
    for k in range(batch):
        a, b = int(offsets[k]), int(offsets[k + 1])
        dk, ek = lanczos_like(b - a, rng)
        d[a:b] = dk
        e[a:b - 1] = ek
    return d, e, offsets


def grad_batch(batch: int = 256, n: int = 8192, seed: int = 0, e_scale: float = 0.5):
    """Differentiation workload: ``batch`` matrices of order n with d ~ N(0, 1),
    e ~ |N(0, e_scale)| and loss weights w ~ Uniform(0, 1); packed like
    ``batched_lanczos``.  Returns (d, e, offsets, w)."""
    rng = np.random.default_rng(seed)
    total = batch * n
    offsets = np.arange(batch + 1, dtype=np.int64) * n
    d = np.empty(total)
    e = np.zeros(total)
    for k in range(batch):
        d[k * n:(k + 1) * n] = rng.standard_normal(n)
        e[k * n:(k + 1) * n - 1] = np.abs(rng.standard_normal(n - 1)) * e_scale
    w = rng.uniform(0.0, 1.0, total)
    return d, e, offsets, w


# Context families with the distributions of the paper's experiments (Sec. 5.1).
def paper_uniform(n: int, seed: int = 0):
    """d ~ U[-1, 1], e ~ U[0.10, 0.30]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, n), rng.uniform(0.10, 0.30, max(n - 1, 0))


def paper_normal(n: int, seed: int = 0):
    """d ~ N(0, 1), e ~ U[0.10, 0.30]."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n), rng.uniform(0.10, 0.30, max(n - 1, 0))


def paper_clustered(n: int):
    """d_i = 1 + 1e-12 (i - (n + 1) / 2), e_i = 1e-4 (1 + 0.1 cos(0.33 i)), i 1-based."""
    i = np.arange(1, n + 1, dtype=np.float64)
    d = 1.0 + 1e-12 * (i - (n + 1) / 2.0)
    j = np.arange(1, n, dtype=np.float64)
    return d, 1e-4 * (1.0 + 0.1 * np.cos(0.33 * j))


def dense_goe(n: int, seed: int = 0):
    """Dense symmetric (G + G^T) / 2 with G iid N(0, 1), float64, C order."""
    g = np.random.default_rng(seed).standard_normal((n, n))
    return 0.5 * (g + g.T)


def dense_planted(n: int, seed: int = 0, reflectors: int = 4):
    """(A, lam): A = H_k ... H_1 diag(lam) H_1 ... H_k with lam iid U(-1, 1) (sorted)
    and k random Householder reflectors H = I - 2 u u^T / u^T u, so A is dense with a
    spectrum known up to the rounding of forming it."""
    rng = np.random.default_rng(seed)
    lam = np.sort(rng.uniform(-1.0, 1.0, n))
    a = np.diag(lam)
    for _ in range(reflectors):
        u = rng.standard_normal(n)
        u /= np.linalg.norm(u)
        au = a @ u
        # H a H = a - 2 u (a u)^T - 2 (a u) u^T + 4 (u^T a u) u u^T
        a = a - 2.0 * np.outer(u, au) - 2.0 * np.outer(au, u) + 4.0 * float(u @ au) * np.outer(u, u)
    a = 0.5 * (a + a.T)
    return a, lam


FAMILIES = {
    "uniform11": uniform11,
    "toeplitz": lambda n, seed=0: toeplitz(n, 2.0, -1.0),
    "toeplitz025": lambda n, seed=0: toeplitz(n, 2.0, 0.25),
    "wilkinson": lambda n, seed=0: wilkinson_plus(n),
    "glued_wilkinson": lambda n, seed=0: glued_wilkinson(n),
    "normal": normal_absnormal,
    "graded": lambda n, seed=0: graded(n),
    "paper_uniform": paper_uniform,
    "paper_normal": paper_normal,
    "paper_clustered": lambda n, seed=0: paper_clustered(n),
}


def family(name: str, n: int, seed: int = 0):
    """(d, e) of the named family at order n."""
    return FAMILIES[name](n, seed)
