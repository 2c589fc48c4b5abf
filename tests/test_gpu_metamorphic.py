"""GPU metamorphic and edge-case tests of tde_eigvals: relations every spectrum
obeys (shift, scale, reversal, sign of the couplings, direct sums), the degenerate
inputs the method has (diagonal, zero, constant, tiny orders), extreme magnitudes
and non-finite inputs (reported through the device status, not by a fault)."""
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


def run(tde, d, e, leaf=8, check=True):
    import torch

    d = np.ascontiguousarray(d, dtype=np.float64)
    e = np.ascontiguousarray(e if len(e) else np.zeros(1), dtype=np.float64)
    return tde.eigvals(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(), leaf=leaf,
                       check=check).cpu().numpy()


def gate(d, e):
    return 8 * len(d) * EPS * oracle.norm1(d, e) + 1e-300


FAMS = ["uniform11", "toeplitz", "wilkinson", "glued_wilkinson", "normal", "paper_clustered"]


@pytest.mark.parametrize("fam", FAMS)
@pytest.mark.parametrize("n", [100, 4097])
def test_shift(tde, fam, n):
    d, e = inputs.family(fam, n, seed=3)
    e = e[: n - 1]
    sigma = 3.7
    lam = run(tde, d, e)
    lam_s = run(tde, d + sigma, e)
    assert np.abs(lam_s - (lam + sigma)).max() <= gate(d + sigma, e) + gate(d, e)


@pytest.mark.parametrize("fam", FAMS)
def test_power_of_two_scale_is_exact(tde, fam):
    # the solver scales T by a power of two itself, so 2^k T gives 2^k lambda bit for bit
    n = 3000
    d, e = inputs.family(fam, n, seed=5)
    e = e[: n - 1]
    lam = run(tde, d, e)
    for k in (-40, 7, 300):
        assert np.array_equal(run(tde, np.ldexp(d, k), np.ldexp(e, k)), np.ldexp(lam, k))


@pytest.mark.parametrize("fam", ["uniform11", "normal", "toeplitz025"])
def test_general_scale(tde, fam):
    n = 2000
    d, e = inputs.family(fam, n, seed=6)
    e = e[: n - 1]
    alpha = -3.7
    lam = run(tde, d, e)
    lam_a = run(tde, alpha * d, alpha * e)
    assert np.abs(lam_a - np.sort(alpha * lam)).max() <= gate(alpha * d, alpha * e) + abs(alpha) * gate(d, e)


@pytest.mark.parametrize("fam", FAMS)
def test_reversal_and_coupling_signs(tde, fam):
    # P T P (P the reversal) and D T D (D = diag(+-1)) are similar to T
    n = 2500
    d, e = inputs.family(fam, n, seed=7)
    e = e[: n - 1]
    lam = run(tde, d, e)
    signs = np.where(np.random.default_rng(8).random(n - 1) < 0.5, -1.0, 1.0)
    assert np.abs(run(tde, d[::-1], e[::-1]) - lam).max() <= 2 * gate(d, e)
    assert np.abs(run(tde, d, e * signs) - lam).max() <= 2 * gate(d, e)


def test_direct_sum_of_blocks(tde):
    # zero couplings split T into independent blocks: the spectrum is the union
    rng = np.random.default_rng(9)
    sizes = [1, 17, 300, 64, 2, 1000, 33]
    ds, es, ref = [], [], []
    for m in sizes:
        d = rng.uniform(-1, 1, m)
        e = rng.uniform(-1, 1, m - 1)
        ds.append(d)
        es.append(np.concatenate([e, [0.0]]))
        ref.append(oracle.eigvals_bisect(d, e))
    d = np.concatenate(ds)
    e = np.concatenate(es)[:-1]
    lam = run(tde, d, e)
    assert np.abs(lam - np.sort(np.concatenate(ref))).max() <= gate(d, e)


def test_degenerate_inputs(tde):
    rng = np.random.default_rng(10)
    # diagonal: the sorted diagonal, exactly
    d = rng.uniform(-5, 5, 5000)
    assert np.array_equal(run(tde, d, np.zeros(4999)), np.sort(d))
    # zero and constant matrices
    assert np.array_equal(run(tde, np.zeros(777), np.zeros(776)), np.zeros(777))
    assert np.array_equal(run(tde, np.full(513, 2.5), np.zeros(512)), np.full(513, 2.5))
    # orders 1 and 2 (closed form)
    assert np.array_equal(run(tde, np.array([-3.25]), np.zeros(0)), np.array([-3.25]))
    p, q, r = 0.5, 2.0, -1.5
    h = np.hypot((p - r) / 2, q)
    assert np.allclose(run(tde, np.array([p, r]), np.array([q])), [(p + r) / 2 - h, (p + r) / 2 + h],
                       rtol=0, atol=4 * EPS * 4)


@pytest.mark.parametrize("k", [-1000, 900])
def test_extreme_magnitudes(tde, k):
    # far from 1 in either direction: scaled by 2^k the result stays finite and exact
    n = 1500
    d, e = inputs.family("uniform11", n, seed=11)
    e = e[: n - 1]
    lam = run(tde, d, e)
    lam_k = run(tde, np.ldexp(d, k), np.ldexp(e, k))
    assert np.all(np.isfinite(lam_k))
    assert np.array_equal(lam_k, np.ldexp(lam, k))


@pytest.mark.parametrize("where", ["d", "e"])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_non_finite_input_is_reported(tde, where, bad):
    n = 1000
    d, e = inputs.family("uniform11", n, seed=12)
    d, e = d.copy(), e[: n - 1].copy()
    (d if where == "d" else e)[317] = bad
    with pytest.raises(tde.TdeError):
        run(tde, d, e)
    # the device stays usable: a clean solve right after is exact as before
    d2, e2 = inputs.family("uniform11", 300, seed=13)
    e2 = e2[:299]
    assert np.abs(run(tde, d2, e2) - oracle.eigvals_bisect(d2, e2)).max() <= gate(d2, e2)
