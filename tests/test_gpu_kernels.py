"""GPU checks of individual device building blocks through the C ABI."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_26599_b300 import _lib

    return _lib.load()


def test_refined_reciprocal_matches_ieee_division(lib):
    import torch

    rng = np.random.default_rng(0)
    mant = rng.uniform(1.0, 2.0, 200000)
    expo = rng.integers(-100, 100, 200000)
    sign = rng.choice([-1.0, 1.0], 200000)
    x = sign * np.ldexp(mant, expo)
    x = np.concatenate([x, [1.0, -1.0, 3.0, 0.1, 1e-30, 7e29, 1.0 - 2 ** -52, 1.0 + 2 ** -52]])
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    rc = lib.tde_check_reciprocal(x.shape[0], ctypes.c_void_p(xt.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    got = out.cpu().numpy()
    ref = 1.0 / x
    rel = np.abs(got - ref) / np.abs(ref)
    # within one unit in the last place of IEEE 1/x
    assert rel.max() <= 2 * EPS, rel.max()


def test_refined_rsqrt_matches_cuda_and_ieee(lib):
    import torch

    rng = np.random.default_rng(1)
    mant = rng.uniform(1.0, 4.0, 200000)
    expo = rng.integers(-400, 400, 200000)
    x = np.ldexp(mant, expo)
    x = np.concatenate([x, [1.0, 2.0, 3.0, 0.25, 1e-300, 1e300, 1.0 - 2 ** -52, 1.0 + 2 ** -52]])
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    rc = lib.tde_check_rsqrt(x.shape[0], ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    got = out.cpu().numpy()
    ieee = 1.0 / np.sqrt(x)                  # correctly rounded sqrt, then division
    cuda = torch.rsqrt(xt).cpu().numpy()     # CUDA's own reciprocal square root
    assert (np.abs(got - ieee) / ieee).max() <= 2 * EPS
    assert (np.abs(got - cuda) / cuda).max() <= 2 * EPS
    assert lib.tde_check_rsqrt(-1, None, None, None) == -1


def test_profile_select_records_only_the_chosen_classes(lib):
    import torch

    import paper_2605_26599_b300 as tde

    n = 4096
    d = torch.full((n,), 2.0, dtype=torch.float64, device="cuda")
    e = torch.full((n - 1,), -1.0, dtype=torch.float64, device="cuda")
    tde.eigvals(d, e)
    torch.cuda.synchronize()
    try:
        tde.profile_select(None)
        tde.profile_enable(True)
        lam_all = tde.eigvals(d, e)
        tde.profile_enable(False)
        every = tde.profile_collect()
        tde.profile_select(["secular", "rows"])
        tde.profile_enable(True)
        lam_sel = tde.eigvals(d, e)
        tde.profile_enable(False)
        chosen = tde.profile_collect()
    finally:
        tde.profile_enable(False)
        tde.profile_select(None)
    assert every["secular"][1] > 0 and every["rows"][1] > 0 and every["deflate"][1] > 0
    for name, (ms, count) in chosen.items():
        if name in ("secular", "rows"):
            assert count == every[name][1] and ms > 0.0
        else:
            assert count == 0 and ms == 0.0
    # recording fewer events changes no result
    assert torch.equal(lam_all, lam_sel)
