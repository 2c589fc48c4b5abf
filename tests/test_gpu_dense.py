"""GPU parity for the dense front end (Householder reduction to tridiagonal form,
then the boundary-row solver): tde_dense_eigvals through the C ABI against the
oracle (LAPACK on the full matrix) and against planted spectra, within
8 n eps ||A||_F, plus trace / Frobenius invariants at larger sizes."""
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


def run(tde, a, leaf=0):
    import torch

    return tde.dense_eigvals(torch.from_numpy(np.ascontiguousarray(a)).cuda(), leaf=leaf).cpu().numpy()


def gate(a):
    n = a.shape[0]
    return 8 * n * EPS * np.linalg.norm(a) + 1e-300


@pytest.mark.parametrize("n", [1, 2, 3, 10, 63, 64, 65, 127, 128, 129, 300, 1000])
def test_goe_against_lapack(tde, n):
    a = inputs.dense_goe(n, seed=n)
    lam = run(tde, a)
    assert np.all(np.diff(lam) >= 0)
    err = np.abs(lam - oracle.dense_eigvals(a)).max()
    assert err <= gate(a), f"{err:.3e} > {gate(a):.3e}"


@pytest.mark.parametrize("n", [50, 777, 2500])
@pytest.mark.parametrize("leaf", [8, 32])
def test_planted_spectrum(tde, n, leaf):
    a, lam0 = inputs.dense_planted(n, seed=n + leaf)
    lam = run(tde, a, leaf)
    err = np.abs(lam - lam0).max()
    assert err <= gate(a), f"{err:.3e} > {gate(a):.3e}"


def test_structured_matrices(tde):
    # a tridiagonal input is already reduced; a diagonal one has its diagonal as spectrum;
    # a rank-one matrix has one nonzero eigenvalue
    n = 200
    d, e = inputs.toeplitz(n, 2.0, -1.0)
    lam = run(tde, oracle.dense(d, e))
    ref = 2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    assert np.abs(lam - ref).max() <= 8 * n * EPS * 4
    diag = np.random.default_rng(1).uniform(-3, 3, n)
    assert np.abs(run(tde, np.diag(diag)) - np.sort(diag)).max() <= 8 * n * EPS * 3
    u = np.random.default_rng(2).standard_normal(n)
    lam = run(tde, np.outer(u, u))
    assert abs(lam[-1] - u @ u) <= 8 * n * EPS * (u @ u) and np.abs(lam[:-1]).max() <= 8 * n * EPS * (u @ u)
    assert np.array_equal(run(tde, np.zeros((n, n))), np.zeros(n))


def test_only_one_triangle_is_read(tde):
    # the strictly lower triangle of the row-major array is never read (NaN there is harmless)
    n = 150
    a = inputs.dense_goe(n, seed=7)
    b = a.copy()
    b[np.tril_indices(n, -1)] = np.nan
    assert np.array_equal(run(tde, b), run(tde, a))


def test_leading_dimension_and_invariants_n4096(tde):
    import torch

    n = 4096
    a, lam0 = inputs.dense_planted(n, seed=11, reflectors=3)
    big = torch.zeros((n, n + 37), dtype=torch.float64, device="cuda")
    big[:, :n] = torch.from_numpy(a).cuda()
    lam = tde.dense_eigvals(big[:, :n]).cpu().numpy()
    assert np.abs(lam - lam0).max() <= gate(a)
    assert abs(lam.sum() - np.trace(a)) <= n * EPS * np.linalg.norm(a) * 8
    assert abs((lam ** 2).sum() - (a ** 2).sum()) <= n * EPS * np.linalg.norm(a) ** 2 * 8
