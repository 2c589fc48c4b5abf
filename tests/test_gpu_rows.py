"""GPU parity for requested eigenvector rows (Algorithm 1 with a general row list
sigma): tde_eigvecs_rows through the C ABI against the oracle's dense
eigen-decomposition (columns compared after one sign per column, with a
tolerance scaled by the column's eigenvalue gap) and, at any size, against the
identities Q_s Q_s^T = I and Q_s diag(lambda) Q_s^T = T[s][:, s]."""
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


def run(tde, d, e, rows, leaf=0):
    import torch

    dt = torch.from_numpy(np.ascontiguousarray(d)).cuda()
    et = torch.from_numpy(np.ascontiguousarray(e if len(e) else np.zeros(1))).cuda()
    r = torch.tensor(np.asarray(rows, dtype=np.int64)).cuda()
    lam, q = tde.eigvecs_rows(dt, et, r, leaf=leaf)
    return lam.cpu().numpy(), q.cpu().numpy()


def request(n, rng, k=6):
    # unordered, with a repeat, always including both ends and a middle pair
    base = [0, n - 1, n // 2, max(n // 2 - 1, 0)]
    extra = list(rng.integers(0, n, size=k))
    rows = base + extra + [extra[0]]
    rng.shuffle(rows)
    return rows


def check_identities(q, lam, d, e, rows, tol):
    rows = np.asarray(rows)
    same = (rows[:, None] == rows[None, :]).astype(np.float64)
    assert np.abs(q @ q.T - same).max() <= tol, "requested rows are not orthonormal"
    blk = oracle.principal_block(d, e, rows)
    nrm = max(1.0, oracle.norm1(d, e))
    assert np.abs((q * lam) @ q.T - blk).max() <= tol * nrm, "Q_s diag(lambda) Q_s^T != T[s][:, s]"


def check_columns(q, qref, lam_ref, nrm, n):
    # one sign per column, shared by all requested rows; error bound ~ eps ||T|| / gap
    gaps = np.full(n, np.inf)
    if n > 1:
        dl = np.diff(lam_ref)
        gaps[:-1] = np.minimum(gaps[:-1], dl)
        gaps[1:] = np.minimum(gaps[1:], dl)
    sign = np.where(np.sum(q * qref, axis=0) >= 0, 1.0, -1.0)
    err = np.abs(q - qref * sign).max(axis=0)
    bound = 1e-13 + 64 * n * EPS * nrm / np.maximum(gaps, 1e-300)
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, f"columns {bad[:5]} differ: err {err[bad[:5]]} bound {bound[bad[:5]]}"


FAMS = ["uniform11", "toeplitz", "normal", "paper_uniform", "graded", "toeplitz025"]


@pytest.mark.parametrize("fam", FAMS)
@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 33, 64, 100, 257, 1000])
@pytest.mark.parametrize("leaf", [4, 8, 32])
def test_rows_against_dense(tde, fam, n, leaf):
    d, e = inputs.family(fam, n, seed=n)
    e = e[: max(n - 1, 0)]
    rng = np.random.default_rng(n + leaf)
    rows = request(n, rng)
    lam, q = run(tde, d, e, rows, leaf)
    lam_ref, qref = oracle.eigvec_rows(d, e, rows)
    nrm = oracle.norm1(d, e)
    assert np.abs(lam - lam_ref).max() <= 8 * n * EPS * nrm + 1e-300
    check_columns(q, qref, lam_ref, nrm, n)
    check_identities(q, lam, d, e, rows, 1e-12)
    # repeated requests give identical rows
    for a in range(len(rows)):
        for b in range(a):
            if rows[a] == rows[b]:
                assert np.array_equal(q[a], q[b])


@pytest.mark.parametrize("fam", ["wilkinson", "glued_wilkinson", "paper_clustered"])
@pytest.mark.parametrize("n", [21, 64, 672, 2000])
def test_rows_identities_clustered(tde, fam, n):
    # near-degenerate spectra: single columns are ill-determined, the identities are not
    d, e = inputs.family(fam, n, seed=0)
    e = e[: n - 1]
    rows = request(n, np.random.default_rng(1), k=12)
    lam, q = run(tde, d, e, rows)
    check_identities(q, lam, d, e, rows, 1e-11)


@pytest.mark.parametrize("fam", ["uniform11", "toeplitz", "wilkinson", "glued_wilkinson"])
def test_rows_large_identities_and_eigenvalues(tde, fam):
    # n = 32768: the eigenvalues are those of tde_eigvals bit for bit (the same
    # roots and placement), and the requested rows satisfy the identities
    import torch

    n = 32768
    d, e = inputs.family(fam, n, seed=0)
    e = e[: n - 1]
    rows = request(n, np.random.default_rng(2), k=20)
    lam, q = run(tde, d, e, rows)
    lam0 = tde.eigvals(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()).cpu().numpy()
    assert np.array_equal(lam, lam0)
    check_identities(q, lam, d, e, rows, 1e-10)


def test_rows_many_requests_and_all_rows(tde):
    # every row of a 300 x 300 matrix: the full eigenvector matrix, orthogonal, T Q = Q Lambda
    n = 300
    d, e = inputs.family("uniform11", n, seed=3)
    e = e[: n - 1]
    rows = list(range(n))[::-1]
    lam, q = run(tde, d, e, rows, leaf=8)
    Q = q[::-1]
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-12
    T = oracle.dense(d, e)
    assert np.abs(T @ Q - Q * lam).max() < 1e-12 * oracle.norm1(d, e)


def test_rows_zero_requests_and_bad_row(tde):
    import torch

    n = 100
    d, e = inputs.family("uniform11", n, seed=4)
    dt, et = torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()
    lam, q = tde.eigvecs_rows(dt, et, torch.zeros(0, dtype=torch.int64, device="cuda"))
    assert q.shape == (0, n)
    assert np.array_equal(lam.cpu().numpy(), tde.eigvals(dt, et).cpu().numpy())
    with pytest.raises(tde.TdeError):
        tde.eigvecs_rows(dt, et, torch.tensor([3, n, 5], dtype=torch.int64, device="cuda"))
    lam, q = tde.eigvecs_rows(dt, et, torch.tensor([3, -1, 5], dtype=torch.int64, device="cuda"),
                              check=False)
    qn = q.cpu().numpy()
    assert np.all(qn[1] == 0.0) and np.abs(qn[0]).max() > 0 and np.abs(qn[2]).max() > 0
