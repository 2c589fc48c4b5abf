"""GPU checks of the hand-written adjoint (tde_eigvals_backward / TdeEigvals)
for L = sum_i w_i lambda_i^2 against the dense-eigh oracle gradient, central
finite differences and exact identities."""
import numpy as np
import pytest

import oracle
from paper_2605_26599_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tde():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_26599_b300 as tde_mod

    return tde_mod


def gpu_grad(tde, d, e, w, leaf=8, offsets=None):
    import torch

    dt = torch.from_numpy(d).cuda()
    et = torch.from_numpy(np.concatenate([e, np.zeros(len(d) - len(e))])).cuda()
    lam = (tde.eigvals(dt, et, leaf=leaf) if offsets is None
           else tde.eigvals_batched(dt, et, offsets, leaf=leaf))
    gl = 2.0 * torch.from_numpy(w).cuda() * lam
    lam2, gd, ge = tde.eigvals_backward(dt, et, gl, offsets=offsets, leaf=leaf)
    return lam2.cpu().numpy(), gd.cpu().numpy(), ge.cpu().numpy()


def rel_inf(g, ref):
    return np.max(np.abs(g - ref)) / max(np.max(np.abs(ref)), 1e-300)


@pytest.mark.parametrize("fam", ["normal_half", "uniform11", "paper_uniform", "toeplitz",
                                 "paper_normal"])
@pytest.mark.parametrize("n", [2, 7, 16, 100, 256])
@pytest.mark.parametrize("leaf", [4, 8])
def test_gradient_matches_dense_eigh(tde, fam, n, leaf):
    if fam == "normal_half":
        d, e = inputs.normal_absnormal(n, seed=n, e_scale=0.5)
    else:
        d, e = inputs.family(fam, n, seed=n)
    w = np.random.default_rng(n + 1).uniform(0, 1, n)
    lam, gd, ge = gpu_grad(tde, d, e, w, leaf)
    rd, re_ = oracle.grad_dense(d, e, w)
    assert rel_inf(gd, rd) <= 1e-8, (rel_inf(gd, rd))
    assert rel_inf(ge[: n - 1], re_) <= 1e-8, (rel_inf(ge[: n - 1], re_))


def test_gradient_batched_matches_single(tde):
    d, e, off = inputs.batched_lanczos(batch=12, lo=64, hi=600, seed=4)
    w = np.random.default_rng(2).uniform(0, 1, len(d))
    _, gd, ge = gpu_grad(tde, d, e[:-1], w, offsets=off)
    for k in range(len(off) - 1):
        a, b = int(off[k]), int(off[k + 1])
        rd, re_ = oracle.grad_dense(d[a:b], e[a:b - 1], w[a:b])
        assert rel_inf(gd[a:b], rd) <= 1e-8
        assert rel_inf(ge[a:b - 1], re_) <= 1e-8
        assert ge[b - 1] == 0.0


def test_gradient_identities_and_finite_differences_n8192(tde):
    import torch

    n = 8192
    d, e = inputs.normal_absnormal(n, seed=0, e_scale=0.5)
    w = np.random.default_rng(1).uniform(0, 1, n)
    lam, gd, ge = gpu_grad(tde, d, e, w)
    # rows of Q have unit norm: sum_j dL/dd_j = sum_i 2 w_i lambda_i
    s = np.sum(2 * w * lam)
    assert abs(gd.sum() - s) <= 1e-9 * np.sum(np.abs(2 * w * lam))
    # Euler: each eigenvalue is homogeneous of degree 1 in (d, e)
    lhs = d @ gd + e @ ge[: n - 1]
    rhs = np.sum(2 * w * lam * lam)
    assert abs(lhs - rhs) <= 1e-9 * np.sum(2 * w * lam * lam)

    def loss(dd, ee):
        lt = tde.eigvals(torch.from_numpy(dd).cuda(), torch.from_numpy(ee).cuda(), leaf=8)
        return float(np.dot(w, lt.cpu().numpy() ** 2))

    h = 1e-6
    rng = np.random.default_rng(3)
    for j in rng.choice(n - 1, 16, replace=False):
        dp, dm = d.copy(), d.copy()
        dp[j] += h
        dm[j] -= h
        fd = (loss(dp, e) - loss(dm, e)) / (2 * h)
        assert abs(fd - gd[j]) <= 1e-5 * max(1.0, abs(gd[j])), (j, fd, gd[j])
        ep, em = e.copy(), e.copy()
        ep[j] += h
        em[j] -= h
        fd = (loss(d, ep) - loss(d, em)) / (2 * h)
        assert abs(fd - ge[j]) <= 1e-5 * max(1.0, abs(ge[j])), (j, fd, ge[j])


def test_autograd_function(tde):
    import torch

    d, e = inputs.normal_absnormal(300, seed=5, e_scale=0.5)
    w = np.random.default_rng(6).uniform(0, 1, 300)
    dt = torch.from_numpy(d).cuda().requires_grad_(True)
    et = torch.from_numpy(e).cuda().requires_grad_(True)
    lam = tde.eigvals_autograd(dt, et)
    loss = (torch.from_numpy(w).cuda() * lam * lam).sum()
    loss.backward()
    rd, re_ = oracle.grad_dense(d, e, w)
    assert rel_inf(dt.grad.cpu().numpy(), rd) <= 1e-8
    assert rel_inf(et.grad.cpu().numpy(), re_) <= 1e-8
