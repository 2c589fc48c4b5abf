"""CPU tests of the C ABI library: it loads without a GPU, exports every symbol
include/tde.h declares, and its host-only logic (argument validation, workspace
queries, the split-tree plan) behaves as specified.  No compute call is made."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2605_26599_b300 import _lib, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names.update(re.findall(r"^\s*(?:int|int64_t|void)\s+(tde_\w+)\s*\(", text, re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = declared_symbols()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert names == set(_lib.EXPORTS)


def levels_py(n, leaf):
    L = 0
    while -(-n // (1 << L)) > leaf and (2 << L) <= n:
        L += 1
    return L


def tree_py(n, leaf):
    """Pure-Python restatement of the closed-form balanced tree."""
    L = levels_py(n, leaf)
    leaves = [((i * n) >> L, ((i + 1) * n) >> L) for i in range(1 << L)]
    merges = []
    for h in range(L - 1, -1, -1):
        for i in range(1 << h):
            merges.append(((i * n) >> h, ((2 * i + 1) * n) >> (h + 1), ((i + 1) * n) >> h))
    return L, leaves, merges


@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 32, 33, 64, 100, 1000, 2048, 65536, 262144])
@pytest.mark.parametrize("leaf", [1, 2, 7, 16, 32, 64])
def test_plan_matches_closed_form_tree(n, leaf):
    import paper_2605_26599_b300 as tde

    L, leaves, merges = tree_py(n, leaf)
    q = tde.plan_query([0, n], leaf)
    assert q["steps"] == L
    assert q["leaves"] == len(leaves) == 1 << L
    assert q["merges"] == len(merges) == (1 << L) - 1
    sizes = [b - a for a, b in leaves]
    assert min(sizes) >= 1 and max(sizes) <= max(leaf, 2)
    assert max(sizes) - min(sizes) <= 1
    for lo, mid, hi in merges:
        assert lo < mid < hi and abs((mid - lo) - (hi - mid)) <= 1


def test_plan_forest_counts():
    import paper_2605_26599_b300 as tde

    sizes = inputs.batched_sizes(300, seed=2)
    off = np.concatenate([[0], np.cumsum(sizes)])
    q = tde.plan_query(off, 32)
    Ls = [levels_py(int(s), 32) for s in sizes]
    assert q["steps"] == max(Ls)
    assert q["leaves"] == sum(1 << L for L in Ls)
    assert q["merges"] == sum((1 << L) - 1 for L in Ls)
    per_step = [sum(1 << (L - 1 - s) for L in Ls if L > s) for s in range(max(Ls))]
    assert q["cmax"] == max(per_step)


def test_workspace_is_linear_in_n():
    import paper_2605_26599_b300 as tde

    for leaf in (1, 32, 64):
        for n in (1024, 65536, 262144, 1 << 20):
            b = tde.workspace_bytes(n, leaf)
            assert b <= 256 * n, (n, leaf, b)
    assert tde.workspace_bytes(1 << 20) < 1.01 * 4 * tde.workspace_bytes(1 << 18)


def test_argument_validation_without_device_work():
    lib = _lib.load()
    vp = ctypes.c_void_p
    sz = ctypes.c_size_t()
    assert lib.tde_eigvals_workspace(-1, 0, ctypes.byref(sz)) == _lib.TDE_EINVAL
    assert lib.tde_eigvals_workspace(100, 65, ctypes.byref(sz)) == _lib.TDE_EINVAL
    assert lib.tde_eigvals_workspace(100, -3, ctypes.byref(sz)) == _lib.TDE_EINVAL
    # n = 0 is a no-op that touches nothing
    assert lib.tde_eigvals(0, None, None, None, 0, None, 0, None) == _lib.TDE_OK
    # null pointers and a too-small or misaligned workspace are rejected before any launch
    fake = vp(1 << 20)
    assert lib.tde_eigvals(10, None, fake, fake, 0, fake, 1 << 30, None) == _lib.TDE_EINVAL
    assert lib.tde_eigvals(10, fake, fake, fake, 0, vp((1 << 20) + 8), 1 << 30, None) == _lib.TDE_EINVAL
    assert lib.tde_eigvals(10, fake, fake, fake, 0, fake, 16, None) == _lib.TDE_EWORKSPACE
    off = np.array([0, 5, 3], dtype=np.int64)  # decreasing offsets
    assert lib.tde_eigvals_batched_workspace(2, off.ctypes.data, 0, ctypes.byref(sz)) == _lib.TDE_EINVAL
    off = np.array([1, 5], dtype=np.int64)  # offsets[0] != 0
    assert lib.tde_eigvals_batched_workspace(1, off.ctypes.data, 0, ctypes.byref(sz)) == _lib.TDE_EINVAL
    assert lib.tde_eigvals_noalloc(16385, fake, fake, fake, 0, None) == _lib.TDE_EWORKSPACE
    assert lib.tde_noalloc_get_info(None, None) == _lib.TDE_EINVAL
    # requested eigenvector rows
    assert lib.tde_eigvecs_rows_workspace(100, _lib.MAX_SEL_ROWS + 1, 0, ctypes.byref(sz)) == _lib.TDE_EINVAL
    assert lib.tde_eigvecs_rows_workspace(100, -1, 0, ctypes.byref(sz)) == _lib.TDE_EINVAL
    assert lib.tde_eigvecs_rows_workspace(100, 4, 0, ctypes.byref(sz)) == _lib.TDE_OK
    need = sz.value
    assert lib.tde_eigvals_workspace(100, 0, ctypes.byref(sz)) == _lib.TDE_OK
    assert need >= sz.value + 3 * 8 * 4 * 100
    big = 1 << 40
    assert lib.tde_eigvecs_rows(0, None, None, 4, None, None, None, 0, None, 0, None) == _lib.TDE_OK
    assert lib.tde_eigvecs_rows(10, fake, fake, 3, None, fake, fake, 0, fake, big, None) == _lib.TDE_EINVAL
    assert lib.tde_eigvecs_rows(10, fake, fake, 3, fake, fake, None, 0, fake, big, None) == _lib.TDE_EINVAL
    assert lib.tde_eigvecs_rows(10, fake, fake, _lib.MAX_SEL_ROWS + 1, fake, fake, fake, 0, fake, big,
                                None) == _lib.TDE_EINVAL
    assert lib.tde_eigvecs_rows(10, fake, fake, 3, fake, fake, fake, 0, fake, 64, None) == _lib.TDE_EWORKSPACE


def test_multipole_threshold_rules():
    lib = _lib.load()
    prev = ctypes.c_int32()
    assert lib.tde_set_multipole(100, ctypes.byref(prev)) == _lib.TDE_EINVAL
    assert lib.tde_set_multipole(-1, None) == _lib.TDE_EINVAL
    assert lib.tde_set_multipole(0, ctypes.byref(prev)) == _lib.TDE_OK
    default = prev.value
    assert lib.tde_set_multipole(4096, ctypes.byref(prev)) == _lib.TDE_OK
    assert lib.tde_set_multipole(0, ctypes.byref(prev)) == _lib.TDE_OK and prev.value == 4096
    assert lib.tde_set_multipole(default, None) == _lib.TDE_OK
    # tde_set_tuning leaves the threshold alone
    assert lib.tde_set_multipole(8192, None) == _lib.TDE_OK
    assert lib.tde_set_tuning(0, 0) == _lib.TDE_OK
    assert lib.tde_set_multipole(0, ctypes.byref(prev)) == _lib.TDE_OK and prev.value == 8192


def test_python_binding_refuses_cpu_tensors():
    import torch

    import paper_2605_26599_b300 as tde

    with pytest.raises(TypeError):
        tde.eigvals(torch.zeros(4, dtype=torch.float64), torch.zeros(3, dtype=torch.float64))


def test_noalloc_array_holds_every_accepted_call():
    # tde_eigvals_noalloc promises every order up to TDE_NOALLOC_MAX_N = 16384 with any
    # leaf order: the workspace such a call carves must fit its 4 MiB array
    lib = _lib.load()
    sz = ctypes.c_size_t()
    worst = 0
    for leaf in range(1, 65):
        for n in (16384, 16383, 12289, 8193):
            assert lib.tde_eigvals_workspace(n, leaf, ctypes.byref(sz)) == _lib.TDE_OK
            worst = max(worst, sz.value)
    assert worst <= 4 << 20, worst


def test_backward_workspace_default_is_o_n():
    # the adjoint's default workspace keeps a fixed number of checkpoint slots: its
    # bytes per row stay below 512 and flat in n; more slots or the every-level
    # layout cost more, the one-slot layout less
    import paper_2605_26599_b300 as tde

    flat = [tde.backward_workspace_bytes([0, n], 8) / n for n in (1 << 13, 1 << 16, 1 << 20)]
    assert max(flat) <= 512 and max(flat) - min(flat) <= 4
    assert tde.backward_workspace_bytes([0, 1000], 8) <= 512 * 1000  # 256-byte alignment of ~30 arrays
    n = 1 << 16
    sizes = [tde.backward_workspace_bytes([0, n], 8, slots=s) for s in (1, 2, 4, 8)]
    assert sizes == sorted(sizes) and sizes[2] == tde.backward_workspace_bytes([0, n], 8)
    assert tde.backward_workspace_bytes([0, n], 8, slots=0) > sizes[-1]
    off = np.arange(257, dtype=np.int64) * 8192
    assert tde.backward_workspace_bytes(off, 8) <= 512 * int(off[-1])
