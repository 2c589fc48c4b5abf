"""GPU parity of the batched solver (a forest of uneven split trees processed
level by level in shared launches) against the oracle and against the
single-matrix entry point."""
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


def solve_batched(tde, d, e, offsets, leaf=0):
    import torch

    return tde.eigvals_batched(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(), offsets,
                               leaf=leaf).cpu().numpy()


def check_each(d, e, offsets, lam, sample=None):
    worst = 0.0
    for k in range(len(offsets) - 1):
        a, b = int(offsets[k]), int(offsets[k + 1])
        if b == a:
            continue
        dk, ek = d[a:b], e[a:b - 1]
        gate = 8 * (b - a) * EPS * oracle.norm1(dk, ek) + 1e-300
        lk = lam[a:b]
        assert np.all(np.diff(lk) >= 0)
        if sample is None or b - a <= sample:
            ref = oracle.eigvals_bisect(dk, ek)
            err = np.max(np.abs(lk - ref))
        else:
            ks = np.unique(np.linspace(0, b - a - 1, sample).astype(np.int64))
            err = np.max(np.abs(lk[ks] - oracle.eigvals_select(dk, ek, ks)))
        assert err <= gate, (k, b - a, err, gate)
        worst = max(worst, err / gate if gate > 0 else 0)
    return worst


@pytest.mark.parametrize("leaf", [4, 8, 32])
def test_batched_lanczos_small_batch(tde, leaf):
    d, e, off = inputs.batched_lanczos(batch=48, lo=64, hi=700, seed=3)
    lam = solve_batched(tde, d, e, off, leaf)
    check_each(d, e, off, lam)


def test_batched_equals_single_matrix_solves(tde):
    import torch

    d, e, off = inputs.batched_lanczos(batch=24, lo=64, hi=1500, seed=5)
    lam = solve_batched(tde, d, e, off, 8)
    for k in range(len(off) - 1):
        a, b = int(off[k]), int(off[k + 1])
        single = tde.eigvals(torch.from_numpy(d[a:b].copy()).cuda(), torch.from_numpy(e[a:b].copy()).cuda(),
                             leaf=8).cpu().numpy()
        gate = 8 * (b - a) * EPS * oracle.norm1(d[a:b], e[a:b - 1])
        assert np.max(np.abs(single - lam[a:b])) <= gate


def test_forest_roots_equal_single_solves(tde):
    """A forest sorts its small-K list by K; a single matrix keeps the deflation
    kernels' order.  Both take the list in tiles of one root per lane with four-lane
    sweeps, and a root's operations and sums do not depend on where it sits in the
    list or in its tile, so with every root on the small-K path (warp_min_k above
    every K, no hand-over of short lists) a matrix's eigenvalues must agree bit for
    bit between the two.  Matrices of one order below 1024 rows keep every other
    kernel the same: the per-merge deflation kernels depend only on the merge order,
    and the lanes per root only on the step's largest merge order."""
    import torch

    n = 1000
    mats = [inputs.uniform11(n, 7), inputs.wilkinson_plus(n), inputs.glued_wilkinson(n),
            inputs.toeplitz(n), inputs.paper_clustered(n), inputs.normal_absnormal(n, 3)]
    rng = np.random.default_rng(11)
    mats.append(inputs.lanczos_like(n, rng))
    d = np.concatenate([m[0] for m in mats])
    e = np.concatenate([np.append(m[1][: n - 1], 0.0) for m in mats])
    off = np.arange(len(mats) + 1, dtype=np.int64) * n
    tde.set_tuning(1 << 20, 1)
    try:
        forest = solve_batched(tde, d, e, off, 8)
        for k, (dk, ek) in enumerate(mats):
            single = tde.eigvals(torch.from_numpy(np.ascontiguousarray(dk)).cuda(),
                                 torch.from_numpy(np.ascontiguousarray(ek[: n - 1])).cuda(),
                                 leaf=8).cpu().numpy()
            assert np.array_equal(single.view(np.int64), forest[k * n:(k + 1) * n].view(np.int64)), k
    finally:
        tde.set_tuning()
    check_each(d, e, off, forest)


def test_forest_long_lists_tiles_equal_single_solves(tde):
    """320 matrices of order 1000 (six families): the forest's small-K lists are long
    enough for tiles of 16 and 32 roots per warp, whose rounds sweep the roots of
    several lanes per group in turn.  Every matrix's eigenvalues equal its single
    solve bit for bit, and one matrix of each family matches the oracle.  (Below
    1024 rows the forest and the single solves deflate with the same kernels; above,
    a single matrix's top merges take the cluster kernel, whose run sums round
    differently.)"""
    import torch

    n = 1000
    rng = np.random.default_rng(5)
    mats = []
    for k in range(320):
        f = k % 6
        if f == 0:
            mats.append(inputs.uniform11(n, 100 + k))
        elif f == 1:
            mats.append(inputs.normal_absnormal(n, 200 + k))
        elif f == 2:
            mats.append(inputs.lanczos_like(n, rng))
        elif f == 3:
            mats.append(inputs.toeplitz(n))
        elif f == 4:
            mats.append(inputs.wilkinson_plus(n))
        else:
            mats.append(inputs.glued_wilkinson(n))
    d = np.concatenate([m[0] for m in mats])
    e = np.concatenate([np.append(m[1][: n - 1], 0.0) for m in mats])
    off = np.arange(len(mats) + 1, dtype=np.int64) * n
    tde.set_tuning(1 << 20, 1)
    try:
        forest = solve_batched(tde, d, e, off, 8)
        for k, (dk, ek) in enumerate(mats):
            single = tde.eigvals(torch.from_numpy(np.ascontiguousarray(dk)).cuda(),
                                 torch.from_numpy(np.ascontiguousarray(ek[: n - 1])).cuda(),
                                 leaf=8).cpu().numpy()
            assert np.array_equal(single.view(np.int64), forest[k * n:(k + 1) * n].view(np.int64)), k
    finally:
        tde.set_tuning()
    pick = [0, 1, 2, 4, 5, 9]  # one matrix of each family
    sub_off = np.arange(len(pick) + 1, dtype=np.int64) * n
    sub_d = np.concatenate([mats[k][0] for k in pick])
    sub_e = np.concatenate([np.append(mats[k][1][: n - 1], 0.0) for k in pick])
    sub_lam = np.concatenate([forest[k * n:(k + 1) * n] for k in pick])
    check_each(sub_d, sub_e, sub_off, sub_lam, sample=256)


def test_forest_packing_order_changes_no_root(tde):
    """The forest's small-K list is sorted by K and taken in tiles, so permuting the
    matrices of a packing reorders the list and regroups the tiles; each matrix's
    eigenvalues must not change by a bit (orders below 1024 rows, so the deflation
    kernels do not depend on the packing either)."""
    rng = np.random.default_rng(21)
    mats = []
    for k in range(96):
        n = int(rng.integers(40, 1000))
        f = k % 4
        if f == 0:
            mats.append(inputs.uniform11(n, 300 + k))
        elif f == 1:
            mats.append(inputs.lanczos_like(n, rng))
        elif f == 2:
            mats.append(inputs.glued_wilkinson(n))
        else:
            mats.append(inputs.normal_absnormal(n, 400 + k))

    def pack(order):
        d = np.concatenate([mats[k][0] for k in order])
        e = np.concatenate([np.append(mats[k][1][: len(mats[k][0]) - 1], 0.0) for k in order])
        off = np.concatenate([[0], np.cumsum([len(mats[k][0]) for k in order])]).astype(np.int64)
        return d, e, off

    fwd = list(range(len(mats)))
    rev = fwd[::-1]
    da, ea, oa = pack(fwd)
    db, eb, ob = pack(rev)
    la = solve_batched(tde, da, ea, oa, 8)
    lb = solve_batched(tde, db, eb, ob, 8)
    for pos_b, k in enumerate(rev):
        a0, a1 = int(oa[k]), int(oa[k + 1])
        b0, b1 = int(ob[pos_b]), int(ob[pos_b + 1])
        assert np.array_equal(la[a0:a1].view(np.int64), lb[b0:b1].view(np.int64)), k
    check_each(da, ea, oa, la, sample=64)


def test_forest_one_large_matrix_among_many_small(tde):
    """A forest holding one matrix of order 40000 among 200 of orders 16 to 300: the
    large matrix's top merges take the warp kernel with the block expansion while the
    small merges of every level go through the K-sorted list and its tiles, in the
    same launches.  Every matrix against the oracle (sampled indices for the large
    one, all eigenvalues for the small ones)."""
    rng = np.random.default_rng(33)
    parts = [inputs.uniform11(40000, 7)]
    for k in range(200):
        n = int(rng.integers(16, 301))
        parts.append(inputs.lanczos_like(n, rng) if k % 2 else inputs.glued_wilkinson(n))
    sizes = [len(p[0]) for p in parts]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    d = np.concatenate([p[0] for p in parts])
    e = np.concatenate([np.append(p[1][: len(p[0]) - 1], 0.0) for p in parts])
    lam = solve_batched(tde, d, e, off, 8)
    check_each(d, e, off, lam, sample=128)


def test_batched_edge_packings(tde):
    # empty matrices, order 1 and 2, a leaf-sized one and a larger one, mixed families
    parts = [inputs.uniform11(0), inputs.uniform11(1, seed=1), inputs.toeplitz(2), inputs.uniform11(0),
             inputs.wilkinson_plus(8), inputs.glued_wilkinson(300), inputs.normal_absnormal(1025, seed=2),
             inputs.uniform11(1, seed=9)]
    sizes = [len(p[0]) for p in parts]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    d = np.concatenate([p[0] for p in parts])
    e = np.zeros(len(d))
    for (dk, ek), a in zip(parts, off[:-1]):
        e[a:a + len(ek)] = ek
    for leaf in (1, 8, 64):
        lam = solve_batched(tde, d, e, off, leaf)
        check_each(d, e, off, lam)


def test_batched_full_forest_sampled(tde):
    # the 4096-matrix Lanczos-style forest, every matrix checked on sampled indices
    d, e, off = inputs.batched_lanczos()
    lam = solve_batched(tde, d, e, off, 8)
    idx = np.random.default_rng(0).choice(len(off) - 1, 256, replace=False)
    for k in idx:
        a, b = int(off[k]), int(off[k + 1])
        sub = np.array([0, b - a], dtype=np.int64)
        check_each(d[a:b], e[a:b], sub, lam[a:b], sample=24)
    # trace invariant of every matrix at once
    for k in range(len(off) - 1):
        a, b = int(off[k]), int(off[k + 1])
        tn = oracle.norm1(d[a:b], e[a:b - 1])
        assert abs(lam[a:b].sum() - d[a:b].sum()) <= (b - a) * 8 * (b - a) * EPS * tn


def test_graph_replay_matches_direct_call_bitwise(tde):
    import torch

    from paper_2605_26599_b300.batched import BatchedSolver

    d, e, off = inputs.batched_lanczos(batch=64, lo=64, hi=2048, seed=7)
    dt, et = torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()
    direct = tde.eigvals_batched(dt, et, off, leaf=8).cpu().numpy()
    solver = BatchedSolver(off, leaf=8)
    first = solver(dt, et).cpu().numpy()
    second = solver(dt, et).cpu().numpy()
    assert np.array_equal(first, direct) and np.array_equal(second, direct)
    # new inputs through the same graph
    d2, e2, _ = inputs.batched_lanczos(batch=64, lo=64, hi=2048, seed=7)
    d2 = d2 * 3.0 + 1.0
    lam2 = solver(torch.from_numpy(d2).cuda(), et).cpu().numpy()
    check_each(d2, e, off, lam2, sample=16)


def test_autotune_picks_valid_shape_and_keeps_results(tde, tmp_path):
    import torch

    from paper_2605_26599_b300.batched import BatchedSolver, autotune

    d, e, off = inputs.batched_lanczos(batch=96, lo=64, hi=1024, seed=11)
    dt, et = torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()
    cache = str(tmp_path / "tune.json")
    best = autotune(off, dt, et, leaves=(8, 16), warp_min_ks=(256, 512), reps=1, cache_path=cache)
    assert best["leaf"] in (8, 16) and best["warp_min_k"] in (256, 512)
    again = autotune(off, dt, et, cache_path=cache)
    assert again["cached"] and again["leaf"] == best["leaf"]
    lam = BatchedSolver(off, leaf=best["leaf"])(dt, et).cpu().numpy()
    check_each(d, e, off, lam, sample=16)
    tde.set_tuning()
