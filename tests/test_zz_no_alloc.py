"""GPU tests of tde_eigvals_noalloc, the entry point for callers that cannot
allocate device memory: code handed device pointers by a framework that owns
every allocation (and may forbid new ones while it captures or replays work), or
code that must not add traffic to a memory pool it does not control.  Such a
caller can pass d, e and lambda but not the O(n) workspace tde_eigvals asks for,
so this entry point runs the solver on a 4 MiB array compiled into the library.

Collected last on purpose.  Every call goes through the C ABI.  The results are
compared with the oracle (every eigenvalue certified within 8 n eps ||T||_1 by
Sturm counts) and with tde_eigvals, the entry point that takes a caller
workspace, within the same gate, on two calls in a row with different inputs, so
stale contents of the shared array from the first call would show up in the
second.  The device status word is read back through tde_noalloc_get_info."""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_26599_b300 as tde
    from paper_2605_26599_b300 import _lib

    return torch, tde, _lib, _lib.load()


def _noalloc(env, d, e, leaf=0):
    """One tde_eigvals_noalloc call through the C ABI; returns (rc, lambda, info)."""
    torch, _, _lib, lib = env
    n = d.shape[0]
    lam = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.tde_eigvals_noalloc(n, ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(e.data_ptr()),
                                 ctypes.c_void_p(lam.data_ptr()), leaf, stream)
    info = ctypes.c_int32(-99)
    assert lib.tde_noalloc_get_info(stream, ctypes.byref(info)) == _lib.TDE_OK
    return rc, lam.cpu().numpy(), info.value


def _check(env, d_np, e_np, leaf=0):
    torch, tde, _lib, _ = env
    n = len(d_np)
    d = torch.from_numpy(d_np).cuda()
    e = torch.from_numpy(e_np).cuda()
    rc, got, info = _noalloc(env, d, e, leaf)
    assert rc == _lib.TDE_OK and info == 0
    gate = 8 * n * EPS * oracle.norm1(d_np, e_np[: n - 1])
    assert np.all(np.isfinite(got)) and np.all(np.diff(got) >= 0)
    ok = oracle.certify(d_np, e_np[: n - 1], got, gate)
    assert ok.all(), f"{np.count_nonzero(~ok)} eigenvalues outside the gate"
    ref = tde.eigvals(d, e, leaf=leaf).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= gate


def test_noalloc_matches_oracle_and_workspace_entry_point_two_calls(env):
    from paper_2605_26599_b300 import inputs

    # two calls in a row, different orders and spectra
    _check(env, *inputs.uniform11(5000, seed=3))
    _check(env, *inputs.wilkinson_plus(3001))


def test_noalloc_largest_order_smallest_leaf(env):
    # n = TDE_NOALLOC_MAX_N with leaf 1 needs the largest workspace of any accepted call
    from paper_2605_26599_b300 import inputs

    d, e = inputs.glued_wilkinson(16384)
    _check(env, d, e, leaf=1)


def test_noalloc_reports_nonfinite_input_and_recovers(env):
    torch, _, _lib, _ = env
    from paper_2605_26599_b300 import inputs

    d_np, e_np = inputs.uniform11(777, seed=5)
    d_bad = d_np.copy()
    d_bad[300] = np.nan
    rc, _, info = _noalloc(env, torch.from_numpy(d_bad).cuda(), torch.from_numpy(e_np).cuda())
    assert rc == _lib.TDE_OK and info == _lib.TDE_ENONFINITE
    # the next call resets the status word and solves normally
    _check(env, d_np, e_np)


def test_noalloc_rejects_orders_beyond_its_array(env):
    torch, _, _lib, lib = env
    n = 16385
    d = torch.zeros(n, dtype=torch.float64, device="cuda")
    e = torch.zeros(n, dtype=torch.float64, device="cuda")
    lam = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc = lib.tde_eigvals_noalloc(n, ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(e.data_ptr()),
                                 ctypes.c_void_p(lam.data_ptr()), 0,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _lib.TDE_EWORKSPACE
