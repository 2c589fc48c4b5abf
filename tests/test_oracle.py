"""Pins for the CPU oracle (runs without a GPU).

Each test checks the oracle against something other than itself: closed forms,
invariants, an independent algorithm (Jacobi vs Sturm bisection), a library
routine the oracle does not use (LAPACK via numpy), brute force on tiny inputs,
or values printed in the paper (tests/golden/)."""
import math
import os

import numpy as np
import pytest

from paper_2605_26599_b300 import inputs

EPS = np.finfo(np.float64).eps
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def toeplitz_spectrum(n, a, b):
    k = np.arange(1, n + 1)
    return np.sort(a + 2.0 * b * np.cos(k * np.pi / (n + 1)))


@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 501])
@pytest.mark.parametrize("ab", [(2.0, -1.0), (2.0, 0.25), (-0.3, 1.7)])
def test_bisect_toeplitz_closed_form(oracle_mod, n, ab):
    a, b = ab
    d, e = inputs.toeplitz(n, a, b)
    lam = oracle_mod.eigvals_bisect(d, e)
    ref = toeplitz_spectrum(n, a, b)
    tn = oracle_mod.norm1(d, e)
    assert np.max(np.abs(lam - ref)) <= 8 * EPS * tn + 1e-300


def test_bisect_2x2_brute_force(oracle_mod):
    rng = np.random.default_rng(3)
    for _ in range(50):
        a, c, b = rng.uniform(-5, 5, 3)
        mean, rad = 0.5 * (a + c), math.hypot(0.5 * (a - c), b)
        lam = oracle_mod.eigvals_bisect(np.array([a, c]), np.array([b]))
        assert np.allclose(lam, [mean - rad, mean + rad], rtol=0, atol=8 * EPS * 10)


@pytest.mark.parametrize("fam", ["uniform11", "normal", "wilkinson", "glued_wilkinson",
                                 "paper_clustered"])
def test_bisect_trace_and_frobenius_invariants(oracle_mod, fam):
    n = 400
    d, e = inputs.family(fam, n, seed=5)
    lam = oracle_mod.eigvals_bisect(d, e)
    tn = oracle_mod.norm1(d, e)
    assert abs(lam.sum() - d.sum()) <= 4 * n * EPS * tn
    assert abs((lam * lam).sum() - (d * d).sum() - 2 * (e * e).sum()) <= 8 * n * EPS * tn * tn


@pytest.mark.parametrize("n", [1, 2, 5, 17, 33, 64])
def test_jacobi_matches_bisection(oracle_mod, n):
    d, e = inputs.uniform11(n, seed=n)
    w, v = oracle_mod.jacobi_eigh(oracle_mod.dense(d, e))
    lam = oracle_mod.eigvals_bisect(d, e)
    assert np.max(np.abs(w - lam)) <= 4 * n * EPS * max(1.0, oracle_mod.norm1(d, e))
    assert np.allclose(v.T @ v, np.eye(n), atol=1e-13)


def test_jacobi_toeplitz_eigenvectors_closed_form(oracle_mod):
    n = 24
    d, e = inputs.toeplitz(n, 2.0, -1.0)
    w, v = oracle_mod.jacobi_eigh(oracle_mod.dense(d, e))
    # tridiag(-1, 2, -1): eigenvalue 2 - 2 cos(k pi/(n+1)) with eigenvector
    # sqrt(2/(n+1)) sin(j k pi/(n+1)); ascending order is k = 1..n
    k = np.arange(1, n + 1)
    j = np.arange(1, n + 1)
    q = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(j, k) * np.pi / (n + 1))
    assert np.allclose(w, 2 - 2 * np.cos(k * np.pi / (n + 1)), atol=1e-13)
    assert np.allclose(np.abs(v), np.abs(q), atol=1e-12)


def test_jacobi_reconstructs_matrix(oracle_mod):
    rng = np.random.default_rng(11)
    a = rng.standard_normal((40, 40))
    a = a + a.T
    w, v = oracle_mod.jacobi_eigh(a)
    assert np.allclose(v @ np.diag(w) @ v.T, a, atol=1e-12)


def test_direct_sum_gives_union_of_spectra(oracle_mod):
    d1, e1 = inputs.uniform11(37, seed=1)
    d2, e2 = inputs.normal_absnormal(29, seed=2)
    d = np.concatenate([d1, d2])
    e = np.concatenate([e1, [0.0], e2])
    lam = oracle_mod.eigvals_bisect(d, e)
    ref = np.sort(np.concatenate([oracle_mod.eigvals_bisect(d1, e1),
                                  oracle_mod.eigvals_bisect(d2, e2)]))
    assert np.max(np.abs(lam - ref)) <= 8 * EPS * 4


@pytest.mark.parametrize("fam", ["uniform11", "normal", "wilkinson", "glued_wilkinson", "graded",
                                 "paper_clustered", "toeplitz025"])
def test_bisect_matches_lapack(oracle_mod, fam):
    n = 700
    d, e = inputs.family(fam, n, seed=9)
    lam = oracle_mod.eigvals_bisect(d, e)
    ref = np.linalg.eigvalsh(oracle_mod.dense(d, e))
    assert np.max(np.abs(lam - ref)) <= 8 * n * EPS * oracle_mod.norm1(d, e)


def test_sturm_count_edges(oracle_mod):
    d, e = inputs.uniform11(100, seed=4)
    lam = oracle_mod.eigvals_bisect(d, e)
    assert oracle_mod.sturm_count(d, e, -10.0) == 0
    assert oracle_mod.sturm_count(d, e, 10.0) == 100
    gaps = np.diff(lam)
    for k in range(0, 99, 7):
        mid = lam[k] + 0.5 * gaps[k]
        assert oracle_mod.sturm_count(d, e, mid) == k + 1


def test_eigvals_select_matches_full(oracle_mod):
    d, e = inputs.normal_absnormal(300, seed=8)
    lam = oracle_mod.eigvals_bisect(d, e)
    ks = np.array([0, 1, 77, 150, 298, 299])
    assert np.array_equal(oracle_mod.eigvals_select(d, e, ks), lam[ks])


def test_secular_dense_closed_forms(oracle_mod):
    # K = 1: lambda = D + rho z^2
    assert np.allclose(oracle_mod.secular_eigvals_dense([0.3], [0.7], 1.5), [0.3 + 1.5 * 0.49])
    # K = 2: roots of the 2x2 [[D1 + r z1^2, r z1 z2], [r z1 z2, D2 + r z2^2]]
    D, z, r = np.array([-0.2, 0.5]), np.array([0.6, 0.8]), 0.9
    a, c, b = D[0] + r * z[0] ** 2, D[1] + r * z[1] ** 2, r * z[0] * z[1]
    mean, rad = 0.5 * (a + c), math.hypot(0.5 * (a - c), b)
    assert np.allclose(oracle_mod.secular_eigvals_dense(D, z, r), [mean - rad, mean + rad])
    # trace and strict interlacing D_j < lambda_j < D_{j+1}, lambda_K < D_K + rho |z|^2
    rng = np.random.default_rng(2)
    D = np.sort(rng.uniform(-1, 1, 50))
    z = rng.uniform(0.05, 1, 50) * rng.choice([-1, 1], 50)
    z /= np.linalg.norm(z)
    lam = oracle_mod.secular_eigvals_dense(D, z, 0.7)
    assert abs(lam.sum() - D.sum() - 0.7) < 1e-13
    assert np.all(lam > D) and np.all(lam[:-1] < D[1:]) and lam[-1] < D[-1] + 0.7


def test_boundary_rows_toeplitz_closed_form(oracle_mod):
    n = 33
    d, e = inputs.toeplitz(n, 2.0, -1.0)
    lam, blo, bhi = oracle_mod.boundary_rows_dense(d, e)
    k = np.arange(1, n + 1)
    s = np.sqrt(2.0 / (n + 1))
    assert np.allclose(np.abs(blo), s * np.abs(np.sin(k * np.pi / (n + 1))), atol=1e-13)
    assert np.allclose(np.abs(bhi), s * np.abs(np.sin(n * k * np.pi / (n + 1))), atol=1e-13)
    w, v = oracle_mod.jacobi_eigh(oracle_mod.dense(d, e))
    assert np.allclose(np.abs(v[0]), np.abs(blo), atol=1e-12)


def test_eigvec_rows_toeplitz_closed_form(oracle_mod):
    # Algorithm 1's (Q)_sigma for a row list with repeats and any order, against the
    # closed-form eigenvectors of tridiag(-1, 2, -1): Q[r, k] = +-sqrt(2/(n+1)) sin((r+1)(k+1) pi/(n+1)),
    # one sign per column shared by all rows.
    n = 40
    d, e = inputs.toeplitz(n, 2.0, -1.0)
    rows = [17, 0, n - 1, 17, 5]
    lam, q = oracle_mod.eigvec_rows(d, e, rows)
    k = np.arange(1, n + 1)
    ref = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(np.asarray(rows) + 1, k) * np.pi / (n + 1))
    sign = np.sign(np.sum(q * ref, axis=0))
    assert np.all(sign != 0)
    assert np.allclose(q * sign, ref, atol=1e-13)
    assert np.array_equal(q[0], q[3])


def test_eigvec_rows_two_by_two_brute_force(oracle_mod):
    # [[a, b], [b, c]]: eigenvector of lambda is proportional to (b, lambda - a)
    a, b, c = 0.3, -1.7, 2.2
    lam, q = oracle_mod.eigvec_rows(np.array([a, c]), np.array([b]), [1, 0])
    for j in range(2):
        v = np.array([b, lam[j] - a])
        v /= np.linalg.norm(v)
        assert min(np.abs(q[::-1, j] - v).max(), np.abs(q[::-1, j] + v).max()) < 1e-15


@pytest.mark.parametrize("fam", ["uniform11", "normal", "wilkinson"])
def test_eigvec_rows_invariants(oracle_mod, fam):
    # T = Q diag(lambda) Q^T with Q orthogonal, restricted to the requested rows:
    # Q_s Q_s^T = I and Q_s diag(lambda) Q_s^T = T[s][:, s] (principal block from the definition)
    n = 57
    d, e = inputs.family(fam, n)
    rows = [3, 4, 56, 0, 30, 31, 4]
    lam, q = oracle_mod.eigvec_rows(d, e, rows)
    blk = oracle_mod.principal_block(d, e[: n - 1], rows)
    assert blk[0, 1] == e[3] and blk[1, 0] == e[3] and blk[0, 0] == d[3] and blk[4, 5] == e[30]
    assert np.abs(q @ q.T - (np.asarray(rows)[:, None] == np.asarray(rows)[None, :])).max() < 1e-13
    assert np.abs((q * lam) @ q.T - blk).max() < 1e-13 * max(1.0, oracle_mod.norm1(d, e[: n - 1]))


def test_dense_eigvals_planted_spectrum_and_invariants(oracle_mod):
    # the dense oracle returns the spectrum planted by orthogonal similarity; trace and
    # Frobenius norm are invariant under it
    a, lam = inputs.dense_planted(120, seed=5)
    assert np.abs(a - np.diag(np.diag(a))).max() > 1e-2  # genuinely dense
    w = oracle_mod.dense_eigvals(a)
    assert np.abs(w - lam).max() < 1e-13
    assert abs(w.sum() - np.trace(a)) < 1e-12
    assert abs((w ** 2).sum() - (a ** 2).sum()) < 1e-12


def test_dense_eigvals_two_by_two_closed_form(oracle_mod):
    p, q, r = 1.5, -0.25, 0.75  # [[p, q], [q, r]]: (p + r)/2 +- sqrt(((p - r)/2)^2 + q^2)
    h = math.sqrt(((p - r) / 2) ** 2 + q * q)
    w = oracle_mod.dense_eigvals(np.array([[p, q], [q, r]]))
    assert np.allclose(w, [(p + r) / 2 - h, (p + r) / 2 + h], atol=1e-15, rtol=0)


def test_merge_problem_boundary_sufficiency(oracle_mod):
    # Lemma "boundary sufficiency" + Eq. merge-problem: the spectrum of
    # diag(D) + rho' z z^T built from child boundary rows is the spectrum of T.
    for fam, n, cut in [("uniform11", 64, 32), ("normal", 50, 17), ("toeplitz", 40, 20)]:
        d, e = inputs.family(fam, n, seed=1)
        D, z, rho2, rlo, rhi = oracle_mod.merge_problem(d, e, cut)
        assert abs(np.linalg.norm(z) - 1.0) < 1e-14
        lam = np.sort(oracle_mod.secular_eigvals_dense(D, z, rho2))
        assert np.max(np.abs(lam - oracle_mod.eigvals_bisect(d, e))) < 1e-13
        # trace of the torn children = trace(T) - 2 |beta|
        assert abs(D.sum() - (d.sum() - 2 * abs(e[cut - 1]))) < 1e-12


def test_grad_dense_against_finite_differences_of_bisection(oracle_mod):
    n = 40
    d, e = inputs.normal_absnormal(n, seed=3, e_scale=0.5)
    w = np.random.default_rng(4).uniform(0, 1, n)
    gd, ge = oracle_mod.grad_dense(d, e, w)
    h = 1e-6
    for j in [0, 7, 20, 39]:
        dp, dm = d.copy(), d.copy()
        dp[j] += h
        dm[j] -= h
        fd = (oracle_mod.loss(dp, e, w) - oracle_mod.loss(dm, e, w)) / (2 * h)
        assert abs(fd - gd[j]) < 1e-6 * max(1.0, abs(gd[j]))
    for j in [0, 11, 38]:
        ep, em = e.copy(), e.copy()
        ep[j] += h
        em[j] -= h
        fd = (oracle_mod.loss(d, ep, w) - oracle_mod.loss(d, em, w)) / (2 * h)
        assert abs(fd - ge[j]) < 1e-6 * max(1.0, abs(ge[j]))


def test_grad_dense_identities(oracle_mod):
    n = 120
    d, e = inputs.normal_absnormal(n, seed=6, e_scale=0.5)
    w = np.random.default_rng(7).uniform(0, 1, n)
    gd, ge = oracle_mod.grad_dense(d, e, w)
    lam = oracle_mod.eigvals_bisect(d, e)
    # rows of Q have unit norm: sum_j dL/dd_j = sum_i 2 w_i lambda_i
    assert abs(gd.sum() - (2 * w * lam).sum()) < 1e-11
    # each lambda is homogeneous of degree 1 in (d, e): Euler's identity
    assert abs(d @ gd + e @ ge - (2 * w * lam * lam).sum()) < 1e-10


def test_paper_workspace_formulas_match_printed_values(oracle_mod):
    rows = []
    with open(os.path.join(GOLDEN, "paper_workspace.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    assert len(rows) == 6
    for n, br_mib, internal, unit in rows:
        ws = oracle_mod.paper_workspace_bytes(int(n))
        assert round(ws["br"] / 2 ** 20, 2) == pytest.approx(float(br_mib), abs=0.011)
        scale = 2 ** 20 if unit == "MiB" else 2 ** 30
        got = ws["internal_real"] / scale
        assert got == pytest.approx(float(internal), rel=0.01)
    # Sec. 5.3: D/E plus BR workspace is about 172 N bytes
    assert oracle_mod.paper_workspace_bytes(1 << 16)["br_with_de"] == 172 * (1 << 16)


# ---- Sturm counts at many points and the certification built on them ----------


@pytest.mark.parametrize("n", [1, 2, 7, 300])
@pytest.mark.parametrize("ab", [(2.0, -1.0), (-0.3, 1.7)])
def test_sturm_counts_toeplitz_closed_form(oracle_mod, n, ab):
    # count(x) = #{k : a + 2b cos(k pi/(n+1)) < x}, from the closed-form spectrum
    a, b = ab
    d, e = inputs.toeplitz(n, a, b)
    ref = toeplitz_spectrum(n, a, b)
    rng = np.random.default_rng(n)
    xs = np.concatenate([rng.uniform(ref[0] - 1, ref[-1] + 1, 200),
                         0.5 * (ref[:-1] + ref[1:]), [ref[0] - 5.0, ref[-1] + 5.0]])
    # keep query points clear of the eigenvalues by far more than the count's rounding
    xs = xs[np.min(np.abs(xs[:, None] - ref[None, :]), axis=1) > 1e-9]
    got = oracle_mod.sturm_counts(d, e, xs)
    want = np.searchsorted(ref, xs, side="left")
    assert np.array_equal(got, want)


def test_sturm_counts_equal_single_point_counts(oracle_mod):
    # the batched count performs the single-point recurrence per query point, so the
    # two agree exactly even where x sits on an eigenvalue to the last bit
    d, e = inputs.glued_wilkinson(97)
    lam = oracle_mod.eigvals_bisect(d, e)
    xs = np.concatenate([lam, lam + 1e-15, lam - 1e-15, [0.0, 3.0]])
    got = oracle_mod.sturm_counts(d, e, xs)
    assert [oracle_mod.sturm_count(d, e, x) for x in xs] == list(got)


@pytest.mark.parametrize("n", [5, 64, 1000])
def test_certify_toeplitz_closed_form_and_planted_errors(oracle_mod, n):
    d, e = inputs.toeplitz(n, 2.0, -1.0)
    ref = toeplitz_spectrum(n, 2.0, -1.0)
    g = 8 * n * EPS * oracle_mod.norm1(d, e)
    assert oracle_mod.certify(d, e, ref, g).all()
    k = n // 2
    # an eigenvalue off by 2 gates fails at exactly its index
    bad = ref.copy()
    bad[k] += 2 * g
    ok = oracle_mod.certify(d, e, np.sort(bad), g)
    assert not ok[k] and ok.sum() >= n - 1
    # a dropped eigenvalue replaced by a duplicate of its neighbour is caught too
    bad = ref.copy()
    bad[k] = bad[k - 1] if k > 0 else bad[1]
    assert not oracle_mod.certify(d, e, np.sort(bad), g).all()


@pytest.mark.parametrize("fam", ["uniform11", "glued_wilkinson", "graded", "paper_clustered"])
def test_certify_accepts_lapack_and_rejects_shift(oracle_mod, fam):
    # LAPACK's eigvalsh (a library routine the oracle does not use) is certified within
    # the gate; the same spectrum shifted by 3 gates is rejected everywhere
    n = 600
    d, e = inputs.family(fam, n, seed=2)
    e = e[: n - 1]
    lam = np.linalg.eigvalsh(oracle_mod.dense(d, e))
    g = 8 * n * EPS * oracle_mod.norm1(d, e)
    assert oracle_mod.certify(d, e, lam, g).all()
    r, nfail = oracle_mod.certified_error(d, e, lam, g)
    assert nfail == 0 and r <= g
    assert not oracle_mod.certify(d, e, lam + 3 * g, g).any()


# ---- the gate's norm, the gate and the paper's error metrics, by hand ------------


def test_norm1_hand_values(oracle_mod):
    # ||T||_1 = max_j (|e_{j-1}| + |d_j| + |e_j|); one case per row position of the max,
    # each such that dropping any one term of the winning row changes the result
    cases = [
        ([-6.0, 1.0, 0.5], [1.5, 0.25], 7.5),     # row 0: 6 + 1.5
        ([0.1, -5.0, 0.2], [2.0, -0.25], 7.25),   # row 1: 2 + 5 + 0.25
        ([1.0, -2.0, 3.0], [0.5, -4.0], 7.0),     # row 2: 4 + 3
        ([0.0, 0.0, 0.0, 0.0], [1.0, -3.0, 2.5], 5.5),  # zero diagonal
        ([-2.5], [], 2.5),                        # order 1
    ]
    for d, e, want in cases:
        assert oracle_mod.norm1(np.array(d), np.array(e)) == want
        if len(d) > 1:  # the induced 1-norm of the dense matrix, by LAPACK
            assert np.linalg.norm(oracle_mod.dense(d, e), 1) == want


def test_gate_hand_value(oracle_mod):
    # 8 n eps ||T||_1 with n = 3, ||T||_1 = 7, eps = 2^-52
    assert oracle_mod.gate(np.array([1.0, -2.0, 3.0]), np.array([0.5, -4.0])) == 168.0 * 2.0 ** -52
    assert oracle_mod.EPS == 2.0 ** -52


def test_paper_error_metrics_hand_values(oracle_mod):
    # e_fwd = ||l_hat - l||_inf / max(1, ||l||_inf), e_bwd = ||l_hat - l||_inf / max(1, ||T||_1)
    d, e = np.array([1.0, -2.0, 3.0]), np.array([0.5, -4.0])  # ||T||_1 = 7
    assert oracle_mod.e_fwd([1.0, 2.5, -3.0], [1.0, 2.0, -4.0]) == 1.0 / 4.0
    assert oracle_mod.e_fwd([0.5, 0.75], [0.5, 0.625]) == 0.125  # max |l| < 1: floor 1
    assert oracle_mod.e_bwd([1.0, 2.5, -3.0], [1.0, 2.0, -4.0], d, e) == 1.0 / 7.0
    small = np.array([0.1, 0.1]), np.array([0.2])  # ||T||_1 = 0.3 < 1: floor 1
    assert oracle_mod.e_bwd([0.0, 0.5], [0.0, 0.25], *small) == 0.25


def test_grad_dense_spectral_closed_forms_and_finite_differences(oracle_mod):
    # F(x) = x^2: L = trace(T^2) = sum d^2 + 2 sum e^2, gradient (2 d, 4 e) exactly;
    # F(x) = x: L = trace(T), gradient (1, 0)
    for fam in ("wilkinson", "glued_wilkinson", "uniform11"):
        d, e = inputs.family(fam, 45, seed=2)
        e = e[:44]
        gd, ge = oracle_mod.grad_dense_spectral(d, e, lambda x: 2.0 * x)
        assert np.abs(gd - 2 * d).max() < 1e-12 * max(1, np.abs(d).max())
        assert np.abs(ge - 4 * e).max() < 1e-12 * max(1, np.abs(d).max())
        gd, ge = oracle_mod.grad_dense_spectral(d, e, np.ones_like)
        assert np.abs(gd - 1).max() < 1e-13 and np.abs(ge).max() < 1e-13
    # F(x) = sin x + x^2 / 2: central differences of sum F(lambda) from the bisection oracle
    d, e = inputs.normal_absnormal(30, seed=8, e_scale=0.5)
    gd, ge = oracle_mod.grad_dense_spectral(d, e, lambda x: np.cos(x) + x)

    def L(dd, ee):
        lam = oracle_mod.eigvals_bisect(dd, ee)
        return float(np.sum(np.sin(lam) + 0.5 * lam * lam))

    h = 1e-6
    for j in (0, 13, 29):
        dp, dm = d.copy(), d.copy()
        dp[j] += h
        dm[j] -= h
        assert abs((L(dp, e) - L(dm, e)) / (2 * h) - gd[j]) < 1e-6
    for j in (0, 17, 28):
        ep, em = e.copy(), e.copy()
        ep[j] += h
        em[j] -= h
        assert abs((L(d, ep) - L(d, em)) / (2 * h) - ge[j]) < 1e-6
