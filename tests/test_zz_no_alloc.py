"""GPU test of tde_eigvals_noalloc, the entry point for callers that cannot
allocate device memory (it uses a workspace array compiled into the library).

Collected last on purpose.  It calls the new entry point through the C ABI and
compares its eigenvalues with those of tde_eigvals (the entry point that takes a
caller workspace) within the tolerance the parity tests use, 8 n eps ||T||_1, on
two calls in a row with different inputs, so stale contents of the shared array
from the first call would show up in the second."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


def _norm1(d, e):
    a = np.abs(d).copy()
    a[:-1] += np.abs(e)
    a[1:] += np.abs(e)
    return float(a.max())


def test_noalloc_matches_workspace_entry_point_two_calls():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_26599_b300 as tde
    from paper_2605_26599_b300 import _lib, inputs

    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [inputs.uniform11(5000, seed=3), inputs.wilkinson_plus(3001)]
    for d_np, e_np in cases:
        n = len(d_np)
        d = torch.from_numpy(d_np).cuda()
        e = torch.from_numpy(e_np).cuda()
        lam = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.tde_eigvals_noalloc(n, ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(e.data_ptr()),
                                     ctypes.c_void_p(lam.data_ptr()), 0, stream)
        assert rc == 0
        torch.cuda.synchronize()
        ref = tde.eigvals(d, e).cpu().numpy()
        got = lam.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= 8 * n * EPS * _norm1(d_np, e_np)


def test_noalloc_rejects_orders_beyond_its_array():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_26599_b300 import _lib

    lib = _lib.load()
    n = 16385
    d = torch.zeros(n, dtype=torch.float64, device="cuda")
    e = torch.zeros(n, dtype=torch.float64, device="cuda")
    lam = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc = lib.tde_eigvals_noalloc(n, ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(e.data_ptr()),
                                 ctypes.c_void_p(lam.data_ptr()), 0,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _lib.TDE_EWORKSPACE
