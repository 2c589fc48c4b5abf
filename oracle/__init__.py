"""CPU oracle for the eigenvalue-only tridiagonal eigensolver -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may import this package.  The CUDA solver in ``paper_2605_26599_b300``
never imports it, and the two share no code; the only common module is the seeded
input generator ``paper_2605_26599_b300.inputs`` which holds none of the method's
arithmetic.

Contents (each function cites the passage of the paper it follows):

* ``eigvals_bisect`` / ``eigvals_select`` -- Sturm-count bisection in plain C
  (``sturm.c``), the definition of the quantity the boundary-row D&C returns
  (Sec. 3.1, Eq. dc-split / merge-problem: the spectrum of T; Theorem
  "BR computes the same eigenvalues as conventional D&C").
* ``sturm_counts`` / ``certify`` / ``certified_error`` -- the same Sturm count at
  many points, which certifies every eigenvalue of a computed spectrum within a
  radius from 2n counts (lambda_k >= x iff count(x) <= k).
* ``jacobi_eigh`` -- dense cyclic Jacobi in plain C for n <= 64, an independent
  second route to the spectrum and to the eigenvector rows.
* ``gate`` / ``e_fwd`` / ``e_bwd`` -- the acceptance bound 8 n eps ||T||_1 and the
  paper's normalised accuracy metrics (Sec. 5.1, e_fwd and e_bwd).
* ``secular_eigvals_dense`` -- the eigenvalues of diag(D) + rho z z^T (Eq.
  merge-problem) via a dense LAPACK symmetric eigensolver; a library primitive
  serving as one step.
* ``boundary_rows_dense`` -- the first and last rows of the eigenvector matrix of a
  tridiagonal (the boundary-row state B_v of Eq. boundary-state) via dense eigh.
* ``torn_subproblem`` -- the Cuppen tearing of Eq. (1) / Eq. dc-split.
* ``grad_dense`` -- dL/dd, dL/de for L = sum_i w_i lambda_i^2 from the dense
  eigenvectors: d lambda_i / d d_j = q_ji^2, d lambda_i / d e_j = 2 q_ji q_(j+1)i.
* ``grad_dense_spectral`` -- the same for a spectral loss sum_i F(lambda_i), given
  F' (defined across multiple eigenvalues).
* ``paper_workspace_bytes`` -- the paper's workspace formulas (Sec. 4.2, Sec. 5.3).

Parity pins for every function live in ``tests/test_oracle.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "sturm.c")
_lock = threading.Lock()
_lib = None

EPS = float(np.finfo(np.float64).eps)  # DBL_EPSILON = 2^-52 (the gate's eps)


def build(force: bool = False) -> str:
    """Compile ``sturm.c`` into ``liboracle.so`` (gcc, OpenMP, IEEE double, no fast-math)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _SO, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            dp = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_tridiag_norm1.restype = ctypes.c_double
            lib.oracle_tridiag_norm1.argtypes = [ctypes.c_int64, dp, dp]
            lib.oracle_sturm_count.restype = ctypes.c_int64
            lib.oracle_sturm_count.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double]
            lib.oracle_eigvals_bisect.restype = ctypes.c_int
            lib.oracle_eigvals_bisect.argtypes = [ctypes.c_int64, dp, dp, dp]
            lib.oracle_eigvals_bisect_select.restype = ctypes.c_int
            lib.oracle_eigvals_bisect_select.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_int64,
                                                         i64p, dp]
            lib.oracle_sturm_counts.restype = ctypes.c_int
            lib.oracle_sturm_counts.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_int64, dp, i64p]
            lib.oracle_jacobi_eigh.restype = ctypes.c_int
            lib.oracle_jacobi_eigh.argtypes = [ctypes.c_int, dp, dp, dp]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _prep(d, e):
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = d.shape[0]
    e = np.ascontiguousarray(e, dtype=np.float64)[: max(n - 1, 0)]
    if n > 1 and e.shape[0] != n - 1:
        raise ValueError("e must hold n-1 off-diagonal entries")
    if e.shape[0] == 0:
        e = np.zeros(1)
    return d, e, n


last_threads = 0  # OpenMP threads the last bisection call used


def norm1(d, e) -> float:
    """||T||_1 = max_j (|e_{j-1}| + |d_j| + |e_j|)."""
    d, e, n = _prep(d, e)
    if n == 0:
        return 0.0
    return float(_load().oracle_tridiag_norm1(n, _dp(d), _dp(e)))


def sturm_count(d, e, x: float) -> int:
    """Number of eigenvalues of tridiag(e, d, e) strictly below x."""
    d, e, n = _prep(d, e)
    return int(_load().oracle_sturm_count(n, _dp(d), _dp(e), float(x)))


def sturm_counts(d, e, xs) -> np.ndarray:
    """For every query point x: the number of eigenvalues of tridiag(e, d, e) strictly
    below x (negative LDL^T pivots of T - xI, Sylvester's law of inertia)."""
    global last_threads
    d, e, n = _prep(d, e)
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    out = np.zeros(xs.shape[0], dtype=np.int64)
    if xs.shape[0]:
        last_threads = _load().oracle_sturm_counts(
            n, _dp(d), _dp(e), xs.shape[0], _dp(xs), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return out


def certify(d, e, lam_hat, radius):
    """Certify a computed spectrum eigenvalue by eigenvalue without bisecting it.

    ``lam_hat`` is ascending; ``radius`` is a scalar or one value per index.  The
    k-th smallest eigenvalue (0-based) lambda_k of T satisfies
    lambda_k >= lam_hat[k] - r  iff  count(lam_hat[k] - r) <= k, and
    lambda_k <  lam_hat[k] + r  iff  count(lam_hat[k] + r) >= k + 1,
    so ``|lam_hat[k] - lambda_k| <= r`` holds exactly where both conditions hold
    (the definition of the spectrum, Sec. 3.1; 2n Sturm counts in all).  Returns the
    boolean array of certified indices."""
    lam_hat = np.asarray(lam_hat, dtype=np.float64)
    n = lam_hat.shape[0]
    if n != len(d):
        raise ValueError("lam_hat must hold one value per row of T")
    r = np.broadcast_to(np.asarray(radius, dtype=np.float64), (n,))
    c = sturm_counts(d, e, np.concatenate([lam_hat - r, lam_hat + r]))
    k = np.arange(n)
    return (c[:n] <= k) & (c[n:] >= k + 1)


def certified_error(d, e, lam_hat, gate_value, levels=(1, 8, 64, 512)):
    """Smallest radius gate_value / L, L in ``levels`` (ascending), at which every
    eigenvalue of ``lam_hat`` is certified by :func:`certify`; returns
    (radius, number of indices not certified at the gate itself).  The radius is
    an upper bound on max_k |lam_hat[k] - lambda_k| (up to the Sturm count's own
    rounding, a few eps ||T||_1) and ``inf`` when the gate itself fails."""
    ok = certify(d, e, lam_hat, gate_value)
    nfail = int(np.count_nonzero(~ok))
    if nfail:
        return float("inf"), nfail
    best = float(gate_value)
    for lv in levels[1:]:
        if not np.all(certify(d, e, lam_hat, gate_value / lv)):
            break
        best = float(gate_value) / lv
    return best, 0


def eigvals_bisect(d, e) -> np.ndarray:
    """All eigenvalues of tridiag(e, d, e), ascending, by Sturm bisection (Sec. 3.1)."""
    global last_threads
    d, e, n = _prep(d, e)
    out = np.empty(n)
    if n:
        last_threads = _load().oracle_eigvals_bisect(n, _dp(d), _dp(e), _dp(out))
    return out


def eigvals_select(d, e, ks) -> np.ndarray:
    """Eigenvalues with the given 0-based ascending indices, by Sturm bisection."""
    global last_threads
    d, e, n = _prep(d, e)
    ks = np.ascontiguousarray(ks, dtype=np.int64)
    out = np.empty(ks.shape[0])
    if ks.shape[0]:
        if ks.min() < 0 or ks.max() >= n:
            raise ValueError("eigenvalue index out of range")
        last_threads = _load().oracle_eigvals_bisect_select(
            n, _dp(d), _dp(e), ks.shape[0], ks.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            _dp(out))
    return out


def jacobi_eigh(a):
    """Dense cyclic Jacobi (n <= 64): returns (w ascending, V with matching columns)."""
    a = np.array(a, dtype=np.float64, copy=True, order="C")
    n = a.shape[0]
    if n > 64:
        raise ValueError("jacobi_eigh is for n <= 64")
    w = np.empty(n)
    v = np.empty((n, n))
    sweeps = _load().oracle_jacobi_eigh(n, _dp(a), _dp(w), _dp(v))
    if sweeps < 0:
        raise RuntimeError("Jacobi did not converge")
    order = np.argsort(w, kind="stable")
    return w[order], v[:, order]


def dense(d, e) -> np.ndarray:
    """The dense symmetric matrix tridiag(e, d, e)."""
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    t = np.diag(d)
    if n > 1:
        e = np.asarray(e, dtype=np.float64)[: n - 1]
        t += np.diag(e, 1) + np.diag(e, -1)
    return t


def gate(d, e) -> float:
    """Acceptance bound on max |lambda_hat - lambda|: 8 n eps ||T||_1."""
    n = len(d)
    return 8.0 * n * EPS * norm1(d, e)


def e_fwd(lam_hat, lam_ref) -> float:
    """Normalised forward error of Sec. 5.1: ||l_hat - l_ref||_inf / max(1, ||l_ref||_inf)."""
    lam_ref = np.asarray(lam_ref)
    if lam_ref.size == 0:
        return 0.0
    return float(np.max(np.abs(np.asarray(lam_hat) - lam_ref)) / max(1.0, np.max(np.abs(lam_ref))))


def e_bwd(lam_hat, lam_ref, d, e) -> float:
    """Normalised backward error of Sec. 5.1: ||l_hat - l_ref||_inf / max(1, ||T||_inf)."""
    lam_ref = np.asarray(lam_ref)
    if lam_ref.size == 0:
        return 0.0
    return float(np.max(np.abs(np.asarray(lam_hat) - lam_ref)) / max(1.0, norm1(d, e)))


def secular_eigvals_dense(D, z, rho) -> np.ndarray:
    """Eigenvalues of A(P) = diag(D) + rho z z^T (Appendix A.1 secular problem; Eq.
    merge-problem) by a dense LAPACK symmetric eigensolver (library primitive)."""
    D = np.asarray(D, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    a = np.diag(D) + rho * np.outer(z, z)
    return np.linalg.eigvalsh(a)


def eigh_dense(d, e):
    """Dense eigen-decomposition of tridiag(e, d, e): (lambda ascending, Q)."""
    return np.linalg.eigh(dense(d, e))


def boundary_rows_dense(d, e):
    """(lambda, blo, bhi): eigenvalues ascending and the first / last rows of the
    eigenvector matrix (the boundary-row state B_v = (blo(Q_v), bhi(Q_v)) of Eq.
    boundary-state).  Columns carry an arbitrary sign each."""
    lam, q = eigh_dense(d, e)
    return lam, q[0, :].copy(), q[-1, :].copy()


def eigvec_rows(d, e, rows):
    """(lambda, Q[rows, :]): eigenvalues ascending and the requested rows of the
    eigenvector matrix (Algorithm 1's selected rows (Q_v)_sigma at the root node,
    sigma any row list), from the dense eigen-decomposition.  Columns carry an
    arbitrary sign each."""
    lam, q = eigh_dense(d, e)
    return lam, q[np.asarray(rows, dtype=np.int64), :].copy()


def dense_eigvals(a) -> np.ndarray:
    """Eigenvalues (ascending) of a dense symmetric matrix (the problem the dense
    pipeline of Sec. 2 solves), by LAPACK's symmetric eigensolver on the full matrix."""
    a = np.asarray(a, dtype=np.float64)
    return np.linalg.eigvalsh(0.5 * (a + a.T))


def principal_block(d, e, rows) -> np.ndarray:
    """T[rows][:, rows] of tridiag(e, d, e), entry by entry from the definition of T
    (d on the diagonal, e_i between rows i and i+1, zero elsewhere)."""
    d = np.asarray(d, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    r = np.asarray(rows, dtype=np.int64)
    out = np.zeros((len(r), len(r)))
    for a, i in enumerate(r):
        for b, j in enumerate(r):
            if i == j:
                out[a, b] = d[i]
            elif abs(int(i) - int(j)) == 1:
                out[a, b] = e[min(i, j)]
    return out


def torn_subproblem(d, e, cut):
    """Cuppen tearing at position ``cut`` (Eq. 1 / Eq. dc-split): returns
    (d_left, e_left, d_right, e_right, rho, s) with T = diag(T_L, T_R) + rho u u^T,
    u = e_{cut-1} + s e_cut, rho = |beta|, s = sign(beta), beta = e[cut-1]."""
    d = np.array(d, dtype=np.float64)
    e = np.array(e, dtype=np.float64)
    beta = e[cut - 1]
    rho = abs(beta)
    s = 1.0 if beta >= 0 else -1.0
    dl = d[:cut].copy()
    dr = d[cut:].copy()
    dl[-1] -= rho
    dr[0] -= rho
    return dl, e[: cut - 1].copy(), dr, e[cut:].copy(), rho, s


def merge_problem(d, e, cut):
    """The merge problem of Eq. merge-problem for one cut, from dense child
    eigen-decompositions: returns (D, z, rho', RLO, RHI) unsorted, with
    D = Lambda_L (+) Lambda_R, z = concat(bhi(Q_L), s blo(Q_R)) / sqrt(2),
    rho' = 2 rho, and the rows RLO = [blo(Q_L), 0], RHI = [0, bhi(Q_R)] of
    diag(Q_L, Q_R) that the parent's boundary rows are formed from."""
    dl, el, dr, er, rho, s = torn_subproblem(d, e, cut)
    lam_l, ql = eigh_dense(dl, el)
    lam_r, qr = eigh_dense(dr, er)
    D = np.concatenate([lam_l, lam_r])
    z = np.concatenate([ql[-1, :], s * qr[0, :]]) / np.sqrt(2.0)
    rlo = np.concatenate([ql[0, :], np.zeros(len(lam_r))])
    rhi = np.concatenate([np.zeros(len(lam_l)), qr[-1, :]])
    return D, z, 2.0 * rho, rlo, rhi


def grad_dense(d, e, w):
    """Gradient of L = sum_i w_i lambda_i^2 with respect to d and e, from the dense
    eigenvectors q_i of T: dL/dd_j = sum_i 2 w_i lambda_i q_ji^2 and
    dL/de_j = sum_i 4 w_i lambda_i q_ji q_(j+1)i (first-order perturbation of a
    simple eigenvalue: d lambda_i = q_i^T dT q_i)."""
    lam, q = eigh_dense(d, e)
    coef = 2.0 * np.asarray(w, dtype=np.float64) * lam
    gd = (q * q) @ coef
    ge = 2.0 * ((q[:-1, :] * q[1:, :]) @ coef)
    return gd, ge


def grad_dense_spectral(d, e, fprime):
    """Gradient of the spectral function L = sum_i F(lambda_i) = trace F(T) with
    respect to d and e, from the dense eigen-decomposition: dL/dd_j = sum_i
    F'(lambda_i) q_ji^2 and dL/de_j = 2 sum_i F'(lambda_i) q_ji q_(j+1)i (the first-order
    perturbation of each eigenvalue; summed over an eigenspace of equal
    eigenvalues it involves only that eigenspace's projector, so it is defined for
    multiple eigenvalues too).  ``fprime`` maps the eigenvalues to F'(lambda)."""
    lam, q = eigh_dense(d, e)
    coef = np.asarray(fprime(lam), dtype=np.float64)
    gd = (q * q) @ coef
    ge = 2.0 * ((q[:-1, :] * q[1:, :]) @ coef)
    return gd, ge


def loss(d, e, w) -> float:
    """L = sum_i w_i lambda_i^2 with lambda from the bisection oracle."""
    lam = eigvals_bisect(d, e)
    return float(np.dot(np.asarray(w, dtype=np.float64), lam * lam))


def paper_workspace_bytes(n: int) -> dict:
    """Workspace formulas of Sec. 4.2: BR queries 16N doubles + 7N 32-bit ints; the
    internal values-only D&C needs 1 + 3N + 2N ceil(log2 N) + 3N^2 reals and
    6 + 6N + 5N ceil(log2 N) ints.  Sec. 5.3 adds D/E (2N doubles) for ~172N bytes."""
    import math
    lg = math.ceil(math.log2(n)) if n > 1 else 0
    br = 16 * n * 8 + 7 * n * 4
    internal = (1 + 3 * n + 2 * n * lg + 3 * n * n) * 8 + (6 + 6 * n + 5 * n * lg) * 4
    return {"br": br, "br_with_de": br + 2 * n * 8, "internal_real": (1 + 3 * n + 2 * n * lg
                                                                        + 3 * n * n) * 8,
            "internal": internal}
