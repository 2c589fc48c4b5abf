"""GPU parity at the full single-matrix workload sizes (n = 32768 ... 262144).

Every eigenvalue is certified against the oracle's Sturm counts: the k-th
computed value lambda_hat_k passes when count(lambda_hat_k - g) <= k and
count(lambda_hat_k + g) >= k + 1, i.e. the k-th eigenvalue of T lies within the
gate g = 8 n eps ||T||_1 of it (2n counts per matrix, no bisection).  A sample of
indices is also bisected by the oracle to report the observed error, and the
trace and Frobenius invariants, the closed-form Toeplitz spectrum, ascending order
and the O(n) workspace bound are checked beside it."""
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


def solve(tde, d, e, leaf=0):
    import torch

    return tde.eigvals(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(), leaf=leaf).cpu().numpy()


def sample_indices(n, count=192):
    ks = np.linspace(0, n - 1, count).astype(np.int64)
    return np.unique(np.concatenate([ks, [0, 1, 2, n // 2, n - 3, n - 2, n - 1]]))


def check_full(d, e, lam, sample=192):
    n = len(d)
    tn = oracle.norm1(d, e)
    gate = 8 * n * EPS * tn
    assert np.all(np.diff(lam) >= 0)
    ok = oracle.certify(d, e, lam, gate)
    bad = np.nonzero(~ok)[0]
    assert bad.size == 0, f"{bad.size} eigenvalues outside the gate, first at index {bad[:8]}"
    ks = sample_indices(n, sample)
    ref = oracle.eigvals_select(d, e, ks)
    err = float(np.max(np.abs(lam[ks] - ref)))
    assert err <= gate, f"sampled max |dlambda| {err:.3e} > gate {gate:.3e}"
    # trace and Frobenius invariants (every eigenvalue within the gate)
    assert abs(lam.sum() - d.sum()) <= n * gate
    assert abs((lam * lam).sum() - (d * d).sum() - 2 * (e * e).sum()) <= 2 * n * tn * gate
    return err


@pytest.mark.parametrize("n", [32768, 49152, 65536])
@pytest.mark.parametrize("fam", ["uniform11", "toeplitz", "wilkinson", "glued_wilkinson"])
def test_single_matrix_families(tde, fam, n):
    d, e = inputs.family(fam, n, seed=0)
    lam = solve(tde, d, e)
    check_full(d, e, lam)
    if fam == "toeplitz":  # closed form, every eigenvalue
        k = np.arange(1, n + 1)
        ref = np.sort(2.0 - 2.0 * np.cos(k * np.pi / (n + 1)))
        assert np.max(np.abs(lam - ref)) <= 8 * n * EPS * 4.0


def test_glued_wilkinson_literal_32_blocks(tde):
    # the literal reading of "32 glued W+_21 blocks": n = 672
    d, e = inputs.glued_wilkinson(32 * 21)
    lam = solve(tde, d, e)
    ref = oracle.eigvals_bisect(d, e)
    assert np.max(np.abs(lam - ref)) <= 8 * len(d) * EPS * oracle.norm1(d, e)


@pytest.mark.parametrize("n", [131072, 262144])
@pytest.mark.parametrize("fam", ["normal", "graded"])
def test_large_o_n_workspace(tde, fam, n):
    d, e = inputs.family(fam, n, seed=0)
    assert tde.workspace_bytes(n) <= 256 * n
    lam = solve(tde, d, e)
    check_full(d, e, lam, sample=96)


def _certify_packed(d, e, off, lam):
    """Every eigenvalue of every matrix of a packing, certified at its own gate."""
    bad = []
    for k in range(len(off) - 1):
        a, b = int(off[k]), int(off[k + 1])
        if b == a:
            continue
        dk, ek = d[a:b], e[a:b - 1]
        gate = 8 * (b - a) * EPS * oracle.norm1(dk, ek) + 1e-300
        assert np.all(np.diff(lam[a:b]) >= 0)
        ok = oracle.certify(dk, ek, lam[a:b], gate)
        if not ok.all():
            bad.append((k, b - a, int(np.count_nonzero(~ok))))
    assert not bad, f"matrices with eigenvalues outside their gate: {bad[:8]}"


def test_batched_full_configuration_every_eigenvalue(tde):
    # the batched workload as specified: 4096 Lanczos-style tridiagonals, orders
    # log-uniform in [64, 4096] (3,911,691 rows), one forest solve; every eigenvalue
    # of every matrix certified by Sturm counts
    import torch

    d, e, off = inputs.batched_lanczos()
    lam = tde.eigvals_batched(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(), off,
                              leaf=16).cpu().numpy()
    _certify_packed(d, e, off, lam)


def test_gradient_configuration_forward_every_eigenvalue(tde):
    # the differentiation workload's forward pass: 256 tridiagonals of order 8192
    # (d ~ N(0,1), e ~ |N(0,0.5)|), every eigenvalue certified, through the batched
    # solver and through the adjoint's own forward pass (the eigenvalues it returns)
    import torch

    d, e, off, w = inputs.grad_batch()
    dt, et = torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()
    lam = tde.eigvals_batched(dt, et, off, leaf=8)
    _certify_packed(d, e, off, lam.cpu().numpy())
    gl = 2.0 * torch.from_numpy(w).cuda() * lam
    lam2, _, _ = tde.eigvals_backward(dt, et, gl, offsets=off, leaf=8)
    assert np.array_equal(lam2.cpu().numpy(), lam.cpu().numpy())
