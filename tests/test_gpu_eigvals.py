"""GPU parity: the CUDA boundary-row D&C (through the C ABI) against the Sturm
bisection oracle, element by element after sorting, within 8 n eps ||T||_1."""
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


def run(tde, d, e, leaf=0):
    import torch

    dt = torch.from_numpy(np.ascontiguousarray(d)).cuda()
    et = torch.from_numpy(np.ascontiguousarray(e if len(e) else np.zeros(1))).cuda()
    return tde.eigvals(dt, et, leaf=leaf).cpu().numpy()


def assert_gate(lam, ref, d, e):
    n = len(d)
    err = np.max(np.abs(np.sort(lam) - ref)) if n else 0.0
    # 8 n eps ||T||_1, plus an absolute floor of a few DBL_MIN: the oracle's Sturm
    # count replaces a zero pivot by -pivmin (pivmin = DBL_MIN max(1, max e^2))
    gate = 8 * n * EPS * oracle.norm1(d, e) + 1e-300
    assert err <= gate, f"max |dlambda| = {err:.3e} > gate {gate:.3e}"
    return err


SMALL_FAMILIES = ["uniform11", "toeplitz", "wilkinson", "glued_wilkinson", "normal", "graded",
                  "paper_uniform", "paper_normal", "paper_clustered", "toeplitz025"]


@pytest.mark.parametrize("fam", SMALL_FAMILIES)
@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 32, 33, 64, 65, 100, 257, 1000])
def test_small_families(tde, fam, n):
    d, e = inputs.family(fam, n, seed=n)
    lam = run(tde, d, e)
    assert np.all(np.diff(lam) >= 0), "output must be ascending"
    assert_gate(lam, oracle.eigvals_bisect(d, e), d, e)


@pytest.mark.parametrize("leaf", [1, 2, 7, 16, 32, 64])
@pytest.mark.parametrize("fam", ["uniform11", "toeplitz", "wilkinson", "glued_wilkinson"])
def test_leaf_sizes_n2048(tde, fam, leaf):
    # Theorem (BR = conventional D&C): the eigenvalues do not depend on the tree
    d, e = inputs.family(fam, 2048, seed=0)
    lam = run(tde, d, e, leaf=leaf)
    assert_gate(lam, oracle.eigvals_bisect(d, e), d, e)


def test_config0_uniform_n2048_leaf32(tde):
    d, e = inputs.uniform11(2048, seed=0)
    lam = run(tde, d, e, leaf=32)
    ref = oracle.eigvals_bisect(d, e)
    assert_gate(lam, ref, d, e)
    assert abs(lam.sum() - d.sum()) <= 2048 * 8 * EPS * oracle.norm1(d, e)
