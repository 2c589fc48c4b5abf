"""GPU parity of the secular solver's block expansion.

In FP64 sweeps of large merges, distant blocks of 128 poles are summed through a
series of their moments (10 to 35 terms by separation), and only the blocks near the current point term
by term.  The tests lower the threshold so that every merge with 256 or more
active poles goes through the expansion in the warp-per-root kernel.  They compare
every eigenvalue with the Sturm bisection oracle, and the error with that of the
same solve summing all poles exactly.  The matrices give evenly spread poles
(Toeplitz, uniform), tight clusters with neighbouring clusters at several distances
(glued Wilkinson with several glue strengths and block orders), graded magnitudes
and poles pressed into one narrow band (the paper's clustered family)."""
import numpy as np
import pytest

import oracle
from paper_2605_26599_b300 import inputs

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def tde():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_26599_b300 as tde_mod

    return tde_mod


def solve(tde, d, e, mp_min_k, warp_min_k=256):
    import torch

    saved = tde.get_tuning()
    prev = tde.set_multipole(mp_min_k)
    try:
        tde.set_tuning(warp_min_k=warp_min_k, small_list_min=1)
        return tde.eigvals(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(),
                           leaf=8).cpu().numpy()
    finally:
        tde.set_tuning(**saved)
        tde.set_multipole(prev)


def glued(n, block, glue):
    d, e = inputs.glued_wilkinson(n, block=block, glue=glue)
    return d, e[: n - 1]


def fam(name, n):
    d, e = inputs.family(name, n, seed=4)
    return d, e[: n - 1]


CASES = [
    ("toeplitz", lambda: fam("toeplitz", 4096)),
    ("uniform", lambda: fam("uniform11", 4000)),
    ("normal", lambda: fam("normal", 3500)),
    ("graded", lambda: fam("graded", 3000)),
    ("paper_clustered", lambda: fam("paper_clustered", 4096)),
    ("glued 21 1e-8", lambda: glued(4200, 21, 1e-8)),
    ("glued 21 1e-5", lambda: glued(3000, 21, 1e-5)),
    ("glued 21 1e-11", lambda: glued(3000, 21, 1e-11)),
    ("glued 11 1e-8", lambda: glued(2500, 11, 1e-8)),
    ("glued 7 1e-6", lambda: glued(2000, 7, 1e-6)),
    ("glued 31 1e-9", lambda: glued(3100, 31, 1e-9)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_block_expansion_every_eigenvalue(tde, name, make):
    d, e = make()
    n = len(d)
    ref = oracle.eigvals_bisect(d, e)
    nrm = oracle.norm1(d, e)
    lam = solve(tde, d, e, mp_min_k=256)
    err = np.abs(lam - ref).max()
    assert err <= 8 * n * EPS * nrm
    # no loss against the solve that sums every pole exactly
    err_exact = np.abs(solve(tde, d, e, mp_min_k=1 << 30) - ref).max()
    assert err <= max(2.0 * err_exact, 16 * EPS * nrm), (err, err_exact)


def test_expansion_counts_and_default(tde):
    # the expansion runs (series evaluations counted) and the default threshold
    # gives the same eigenvalues as the all-exact solve to within rounding
    import torch

    n = 8192
    d, e = fam("toeplitz", n)
    dt, et = torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()
    ws = tde.Workspace(tde.workspace_bytes(n, 8))
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    prev = tde.set_multipole(0)
    try:
        tde.eigvals(dt, et, leaf=8, out=out, ws=ws)
        work = tde.read_work(ws)
        lam = out.cpu().numpy()
        tde.set_multipole(1 << 30)
        tde.eigvals(dt, et, leaf=8, out=out, ws=ws)
        work_exact = tde.read_work(ws)
        lam_exact = out.cpu().numpy()
    finally:
        tde.set_multipole(prev)
    assert work["secular_far_blocks"] > 0 and work_exact["secular_far_blocks"] == 0
    assert work["secular_pairs"] < work_exact["secular_pairs"]
    # FP64 operations per far-block evaluation: the overhead plus the tier's heads
    # (secular 7 + 10 .. 35, Lowner 4 + 6 .. 21, rows 5 + chains + heads)
    fb, lb = work["secular_far_blocks"], work["lowner_far_blocks"]
    assert 17 * fb <= work["secular_series_ops"] <= 42 * fb
    assert lb > 0 and 10 * lb <= work["lowner_series_ops"] <= 25 * lb
    assert work["rows_series_ops"] > 0 and work_exact["rows_series_ops"] == 0
    assert work_exact["secular_series_ops"] == work_exact["lowner_series_ops"] == 0
    assert np.abs(lam - lam_exact).max() <= 16 * EPS * oracle.norm1(d, e)


def forced(tde):
    """Context: expansion from K = 256 on, warp-per-root kernel from K = 256 on."""
    import contextlib

    @contextlib.contextmanager
    def ctx():
        saved = tde.get_tuning()
        prev = tde.set_multipole(256)
        try:
            tde.set_tuning(warp_min_k=256, small_list_min=1)
            yield
        finally:
            tde.set_tuning(**saved)
            tde.set_multipole(prev)

    return ctx()


@pytest.mark.parametrize("name", ["toeplitz", "uniform11", "normal", "paper_clustered"])
@pytest.mark.parametrize("n", [1000, 2000])
def test_requested_rows_with_expansion(tde, name, n):
    # eigenvector rows from the boundary-row state of merges that use all three
    # expansions (secular sums, Löwner products, row sums): orthonormal, reproducing
    # T's principal block, and equal (per column, up to sign) to dense eigh
    import torch

    d, e = fam(name, n)
    rng = np.random.default_rng(n)
    rows = [0, n - 1, n // 2, n // 2 - 1] + list(rng.integers(0, n, size=4))
    r = torch.tensor(np.asarray(rows, dtype=np.int64)).cuda()
    with forced(tde):
        lam, q = tde.eigvecs_rows(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(), r, leaf=8)
    lam, q = lam.cpu().numpy(), q.cpu().numpy()
    nrm = max(1.0, oracle.norm1(d, e))
    tol = 64 * n * EPS
    same = (np.asarray(rows)[:, None] == np.asarray(rows)[None, :]).astype(np.float64)
    assert np.abs(q @ q.T - same).max() <= tol
    assert np.abs((q * lam) @ q.T - oracle.principal_block(d, e, rows)).max() <= tol * nrm
    lam_ref, qref = oracle.eigvec_rows(d, e, rows)
    assert np.abs(lam - lam_ref).max() <= 8 * n * EPS * nrm
    gaps = np.full(n, np.inf)
    dl = np.diff(lam_ref)
    gaps[:-1] = np.minimum(gaps[:-1], dl)
    gaps[1:] = np.minimum(gaps[1:], dl)
    sign = np.where(np.sum(q * qref, axis=0) >= 0, 1.0, -1.0)
    err = np.abs(q - qref * sign).max(axis=0)
    bound = 1e-13 + 64 * n * EPS * nrm / np.maximum(gaps, 1e-300)
    assert np.all(err <= bound)


@pytest.mark.parametrize("name", ["toeplitz", "uniform11", "normal"])
def test_gradient_with_expansion(tde, name):
    # the adjoint's forward and reverse passes use the expansions at every merge
    # (including root merges) from K = 256 on; the gradient of sum w lambda^2 matches
    # the dense-eigh oracle gradient
    import torch

    n = 1536
    d, e = fam(name, n)
    w = np.random.default_rng(7).uniform(0, 1, n)
    dt = torch.from_numpy(d).cuda()
    et = torch.from_numpy(np.concatenate([e, [0.0]])).cuda()
    with forced(tde):
        lam = tde.eigvals(dt, et, leaf=8)
        gl = 2.0 * torch.from_numpy(w).cuda() * lam
        _, gd, ge = tde.eigvals_backward(dt, et, gl, leaf=8)
    rd, re_ = oracle.grad_dense(d, e, w)
    gd, ge = gd.cpu().numpy(), ge.cpu().numpy()[: n - 1]
    assert np.max(np.abs(gd - rd)) <= 1e-8 * np.max(np.abs(rd))
    assert np.max(np.abs(ge - re_)) <= 1e-8 * np.max(np.abs(re_))


@pytest.mark.gpu
@pytest.mark.parametrize("offdiag", [-1.0, 0.25])
def test_superblocks_toeplitz_closed_form(tde, offdiag):
    """Toeplitz n = 65536: its top merges hold 16k-33k poles, so the secular sweeps
    go through superblocks of 32 blocks.  Every eigenvalue against the closed form
    d + 2 e cos(k pi / (n + 1))."""
    import torch

    n = 65536
    d, e = inputs.toeplitz(n, 2.0, offdiag)
    dt, et = torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()
    ws = tde.Workspace(tde.workspace_bytes(n, 8))
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    tde.eigvals(dt, et, leaf=8, out=out, ws=ws)
    lam = out.cpu().numpy()
    k = np.arange(1, n + 1)
    exact = np.sort(2.0 + 2.0 * offdiag * np.cos(k * np.pi / (n + 1)))
    norm = 2.0 + 2.0 * abs(offdiag)
    assert np.abs(lam - exact).max() <= 8 * EPS * norm
    work = tde.read_work(ws)
    assert work["secular_far_blocks"] > 0
