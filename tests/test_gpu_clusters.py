"""GPU parity of the secular solver's cluster evaluation.

Roots whose two bracketing poles sit in a cluster of poles too close together for
the single-precision stage are solved with exact sums over a near range of poles
plus Taylor sums of the poles outside it, in the warp-per-root kernel.  The tests
send every merge of glued matrices through that kernel (a low warp_min_k), so the
cluster path runs at every level, and compare every eigenvalue with the Sturm
bisection oracle.  The glue strengths and block orders give clusters of different
spans and neighbouring clusters at different distances.  That covers near ranges
that hold one cluster, near ranges widened to neighbouring clusters, and clusters
left to the full sums.  A second check compares the error with that of the same
solve without the warp kernel (no cluster evaluation)."""
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


def solve(tde, d, e, warp_min_k):
    import torch

    saved = tde.get_tuning()
    try:
        tde.set_tuning(warp_min_k=warp_min_k, small_list_min=1)
        return tde.eigvals(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(),
                           leaf=8).cpu().numpy()
    finally:
        tde.set_tuning(**saved)


CASES = [(21, 1e-8, 4200), (21, 1e-5, 3000), (21, 1e-11, 3000), (11, 1e-8, 2500),
         (31, 1e-9, 3100), (7, 1e-6, 2000)]


@pytest.mark.parametrize("block,glue,n", CASES)
def test_glued_clusters_every_eigenvalue(tde, block, glue, n):
    d, e = inputs.glued_wilkinson(n, block=block, glue=glue)
    e = e[: n - 1]
    ref = oracle.eigvals_bisect(d, e)
    nrm = oracle.norm1(d, e)
    lam = solve(tde, d, e, warp_min_k=16)
    err = np.abs(lam - ref).max()
    assert err <= 8 * n * EPS * nrm
    # no loss against the full-sum path (warp kernel off: every merge below 2^30)
    err_full = np.abs(solve(tde, d, e, warp_min_k=1 << 30) - ref).max()
    assert err <= max(2.0 * err_full, 16 * EPS * nrm), (err, err_full)


def test_glued_clusters_default_tuning_matches(tde):
    # the default launch shape (cluster evaluation at the large merges only) agrees
    # with the all-warp-kernel solve to within the rounding of either
    n = 6000
    d, e = inputs.glued_wilkinson(n)
    e = e[: n - 1]
    import torch

    lam_default = tde.eigvals(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(),
                              leaf=8).cpu().numpy()
    lam_warp = solve(tde, d, e, warp_min_k=16)
    nrm = oracle.norm1(d, e)
    assert np.abs(lam_default - lam_warp).max() <= 32 * EPS * nrm
