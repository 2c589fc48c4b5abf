"""paper_2605_26599_b300 -- a B300 (sm_103a) boundary-row divide-and-conquer solver
for all eigenvalues of real symmetric tridiagonal matrices, in FP64.

The computation lives in ``libtde.so`` (hand-written CUDA kernels behind the C ABI
declared in ``include/tde.h``).  This module only marshals arguments: PyTorch
supplies device memory and the current CUDA stream.  There is no CPU fallback --
a missing library or a CPU tensor raises.

    import torch, paper_2605_26599_b300 as tde
    lam = tde.eigvals(d, e)                    # one tridiagonal, d[n], e[n-1]
    lam = tde.eigvals_batched(d, e, offsets)   # packed forest
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import TdeError  # noqa: F401

__all__ = ["eigvals", "eigvals_batched", "eigvals_backward", "TdeEigvals", "eigvals_autograd", "workspace_bytes", "batched_workspace_bytes",
           "get_info", "measure_fp64_peak", "last_launch_count", "TdeError", "Workspace",
           "profile_enable", "profile_select", "profile_collect", "read_work"]


def _torch():
    import torch

    return torch


def workspace_bytes(n: int, leaf: int = 0) -> int:
    """Device workspace bytes for one tridiagonal of order n."""
    out = ctypes.c_size_t()
    _lib.check("tde_eigvals_workspace", _lib.load().tde_eigvals_workspace(int(n), int(leaf),
                                                                          ctypes.byref(out)))
    return int(out.value)


def _host_offsets(offsets) -> np.ndarray:
    if hasattr(offsets, "detach"):
        offsets = offsets.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))


def batched_workspace_bytes(offsets, leaf: int = 0) -> int:
    """Device workspace bytes for a packed batch (offsets: B+1 non-decreasing ints)."""
    off = _host_offsets(offsets)
    out = ctypes.c_size_t()
    _lib.check("tde_eigvals_batched_workspace",
               _lib.load().tde_eigvals_batched_workspace(off.shape[0] - 1, off.ctypes.data, int(leaf),
                                                         ctypes.byref(out)))
    return int(out.value)


class Workspace:
    """A reusable device workspace (a uint8 torch tensor, 256-byte aligned)."""

    def __init__(self, nbytes: int, device="cuda"):
        torch = _torch()
        self.nbytes = int(nbytes)
        self._buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        base = self._buf.data_ptr()
        self.ptr = (base + 255) & ~255

    def ensure(self, nbytes: int) -> "Workspace":
        return self if nbytes <= self.nbytes else Workspace(nbytes, self._buf.device)


def _check_tensor(t, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (the solver has no CPU path)")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def get_info(ws: Workspace, stream=None) -> int:
    """Device status word of the last call that used ``ws`` (synchronises)."""
    info = ctypes.c_int32()
    _lib.check("tde_get_info", _lib.load().tde_get_info(ctypes.c_void_p(ws.ptr), _stream_ptr(stream),
                                                        ctypes.byref(info)))
    return int(info.value)


def eigvals(d, e, leaf: int = 0, out=None, ws: Workspace | None = None, stream=None,
            check: bool = True):
    """All eigenvalues (ascending) of tridiag(e, d, e); d: [n], e: [n-1] (or [n], the
    last entry ignored), float64 CUDA tensors.  With check=True the device status is
    read back (one synchronisation) and a numerical failure raises TdeError."""
    torch = _torch()
    _check_tensor(d, "d")
    n = d.shape[0]
    if n > 1:
        _check_tensor(e, "e")
        if e.shape[0] < n - 1:
            raise ValueError("e must hold at least n-1 entries")
    lam = out if out is not None else torch.empty(n, dtype=torch.float64, device=d.device)
    if n == 0:
        return lam
    need = workspace_bytes(n, leaf)
    ws = Workspace(need, d.device) if ws is None else ws.ensure(need)
    rc = _lib.load().tde_eigvals(n, ctypes.c_void_p(d.data_ptr()),
                                 ctypes.c_void_p(e.data_ptr() if n > 1 else 0),
                                 ctypes.c_void_p(lam.data_ptr()), int(leaf), ctypes.c_void_p(ws.ptr),
                                 ws.nbytes, _stream_ptr(stream))
    _lib.check("tde_eigvals", rc)
    if check:
        info = get_info(ws, stream)
        if info != 0:
            raise TdeError("tde_eigvals (device status)", info)
    return lam


def eigvecs_rows_workspace_bytes(n: int, nsel: int, leaf: int = 0) -> int:
    """Bytes of workspace ``eigvecs_rows`` needs (tde_eigvecs_rows_workspace)."""
    b = ctypes.c_size_t()
    _lib.check("tde_eigvecs_rows_workspace",
               _lib.load().tde_eigvecs_rows_workspace(int(n), int(nsel), int(leaf), ctypes.byref(b)))
    return b.value


def eigvecs_rows(d, e, rows, leaf: int = 0, out=None, qrows=None, ws: Workspace | None = None,
                 stream=None, check: bool = True):
    """Eigenvalues (ascending) and the requested rows of the eigenvector matrix Q of
    tridiag(e, d, e): returns (lam, qrows) with qrows[q, j] = Q[rows[q], j], column j
    belonging to lam[j] (T = Q diag(lam) Q^T; column signs arbitrary but shared by
    all requested rows).  ``rows``: int64 CUDA tensor (or a sequence, copied to the
    device), any order, repeats allowed, at most MAX_SEL_ROWS entries."""
    torch = _torch()
    _check_tensor(d, "d")
    n = d.shape[0]
    if n > 1:
        _check_tensor(e, "e")
        if e.shape[0] < n - 1:
            raise ValueError("e must hold at least n-1 entries")
    if not (hasattr(rows, "is_cuda") and rows.is_cuda):
        rows = torch.as_tensor(np.asarray(rows, dtype=np.int64)).to(d.device)
    if rows.dtype != torch.int64 or rows.dim() != 1:
        raise ValueError("rows must be a 1-D int64 tensor")
    rows = rows.contiguous()
    nsel = rows.shape[0]
    if nsel > _lib.MAX_SEL_ROWS:
        raise ValueError(f"at most {_lib.MAX_SEL_ROWS} requested rows per call")
    lam = out if out is not None else torch.empty(n, dtype=torch.float64, device=d.device)
    q = qrows if qrows is not None else torch.empty((nsel, n), dtype=torch.float64, device=d.device)
    if n == 0:
        return lam, q
    need = eigvecs_rows_workspace_bytes(n, nsel, leaf)
    ws = Workspace(need, d.device) if ws is None else ws.ensure(need)
    rc = _lib.load().tde_eigvecs_rows(n, ctypes.c_void_p(d.data_ptr()),
                                      ctypes.c_void_p(e.data_ptr() if n > 1 else 0), nsel,
                                      ctypes.c_void_p(rows.data_ptr() if nsel else 0),
                                      ctypes.c_void_p(lam.data_ptr()),
                                      ctypes.c_void_p(q.data_ptr() if nsel else 0), int(leaf),
                                      ctypes.c_void_p(ws.ptr), ws.nbytes, _stream_ptr(stream))
    _lib.check("tde_eigvecs_rows", rc)
    if check:
        info = get_info(ws, stream)
        if info != 0:
            raise TdeError("tde_eigvecs_rows (device status)", info)
    return lam, q


def dense_eigvals_workspace_bytes(n: int, leaf: int = 0) -> int:
    """Bytes of workspace ``dense_eigvals`` needs (tde_dense_eigvals_workspace)."""
    b = ctypes.c_size_t()
    _lib.check("tde_dense_eigvals_workspace",
               _lib.load().tde_dense_eigvals_workspace(int(n), int(leaf), ctypes.byref(b)))
    return b.value


def dense_eigvals(A, leaf: int = 0, out=None, ws: Workspace | None = None, stream=None,
                  check: bool = True):
    """All eigenvalues (ascending) of a dense symmetric float64 CUDA matrix A (n x n):
    Householder reduction to tridiagonal form, then the boundary-row solver.  Only one
    triangle is read (the upper one of the row-major tensor)."""
    torch = _torch()
    if not isinstance(A, torch.Tensor) or not A.is_cuda:
        raise TypeError("A must be a CUDA tensor (the solver has no CPU path)")
    if A.dtype != torch.float64:
        raise TypeError("A must be float64")
    if A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be a square matrix")
    if A.stride(1) != 1 or A.stride(0) < A.shape[0]:
        raise ValueError("A must have unit stride along its second dimension and rows of at least n")
    n = A.shape[0]
    lam = out if out is not None else torch.empty(n, dtype=torch.float64, device=A.device)
    if n == 0:
        return lam
    need = dense_eigvals_workspace_bytes(n, leaf)
    ws = Workspace(need, A.device) if ws is None else ws.ensure(need)
    rc = _lib.load().tde_dense_eigvals(n, ctypes.c_void_p(A.data_ptr()), int(A.stride(0)),
                                       ctypes.c_void_p(lam.data_ptr()), int(leaf),
                                       ctypes.c_void_p(ws.ptr), ws.nbytes, _stream_ptr(stream))
    _lib.check("tde_dense_eigvals", rc)
    if check:
        info = get_info(ws, stream)
        if info != 0:
            raise TdeError("tde_dense_eigvals (device status)", info)
    return lam


def eigvals_batched(d, e, offsets, leaf: int = 0, out=None, ws: Workspace | None = None,
                    stream=None, check: bool = True, offsets_dev=None):
    """Eigenvalues of a packed batch: matrix k owns rows offsets[k]:offsets[k+1] of d,
    e and of the result (each matrix's eigenvalues ascending).  ``offsets`` is a host
    sequence (B+1); ``offsets_dev`` optionally the same values as a CUDA int64 tensor."""
    torch = _torch()
    off = _host_offsets(offsets)
    _check_tensor(d, "d")
    _check_tensor(e, "e")
    total = int(off[-1])
    if d.shape[0] < total or e.shape[0] < total - 1:
        raise ValueError("d / e shorter than offsets[-1]")
    lam = out if out is not None else torch.empty(total, dtype=torch.float64, device=d.device)
    if total == 0:
        return lam
    if offsets_dev is None:
        offsets_dev = torch.from_numpy(off).to(d.device)
    need = batched_workspace_bytes(off, leaf)
    ws = Workspace(need, d.device) if ws is None else ws.ensure(need)
    rc = _lib.load().tde_eigvals_batched(
        off.shape[0] - 1, off.ctypes.data, ctypes.c_void_p(offsets_dev.data_ptr()),
        ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
        int(leaf), ctypes.c_void_p(ws.ptr), ws.nbytes, _stream_ptr(stream))
    _lib.check("tde_eigvals_batched", rc)
    if check:
        info = get_info(ws, stream)
        if info != 0:
            raise TdeError("tde_eigvals_batched (device status)", info)
    return lam


def plan_query(offsets, leaf: int = 0) -> dict:
    """Host-only split-tree plan of a packing: steps, leaves, merges, max merges/step."""
    off = _host_offsets(offsets)
    out = (ctypes.c_int64 * 4)()
    _lib.check("tde_plan_query", _lib.load().tde_plan_query(off.shape[0] - 1, off.ctypes.data,
                                                            int(leaf), out))
    return {"steps": int(out[0]), "leaves": int(out[1]), "merges": int(out[2]), "cmax": int(out[3])}


def set_tuning(warp_min_k: int = 0, small_list_min: int = 0) -> None:
    """Launch-shape tuning of later calls on this thread (0 = default)."""
    _lib.check("tde_set_tuning", _lib.load().tde_set_tuning(int(warp_min_k), int(small_list_min)))


def set_multipole(min_k: int = 0) -> int:
    """Threshold K of the secular solver's block expansion for later calls on this
    thread (0 = default 1024; a value above every K turns it off).  Returns the
    previous threshold."""
    prev = ctypes.c_int32()
    _lib.check("tde_set_multipole", _lib.load().tde_set_multipole(int(min_k), ctypes.byref(prev)))
    return int(prev.value)


def get_tuning() -> dict:
    out = (ctypes.c_int32 * 2)()
    _lib.check("tde_get_tuning", _lib.load().tde_get_tuning(out))
    return {"warp_min_k": int(out[0]), "small_list_min": int(out[1])}


def backward_workspace_bytes(offsets, leaf: int = 8, slots: int | None = None) -> int:
    """Device workspace bytes for tde_eigvals_backward on a packing: the default O(n)
    layout (4 checkpoint slots) when ``slots`` is None, else the layout with that many
    slots (0: every level checkpointed, no recomputation)."""
    off = _host_offsets(offsets)
    out = ctypes.c_size_t()
    if slots is None:
        _lib.check("tde_eigvals_backward_workspace",
                   _lib.load().tde_eigvals_backward_workspace(off.shape[0] - 1, off.ctypes.data,
                                                              int(leaf), ctypes.byref(out)))
    else:
        _lib.check("tde_eigvals_backward_workspace_slots",
                   _lib.load().tde_eigvals_backward_workspace_slots(
                       off.shape[0] - 1, off.ctypes.data, int(leaf), int(slots), ctypes.byref(out)))
    return int(out.value)


def eigvals_backward(d, e, grad_lambda, offsets=None, leaf: int = 8, ws: Workspace | None = None,
                     stream=None, check: bool = True, offsets_dev=None, lam_out=None,
                     slots: int | None = None):
    """(lambda, dL/dd, dL/de) for dL/dlambda = grad_lambda, by the adjoint sweep of
    tde_eigvals_backward.  offsets=None means one matrix of order len(d); e is
    packed like d (the entry at each matrix's last row is ignored, its gradient 0).
    The workspace layout follows ``slots`` (see backward_workspace_bytes); a
    caller-provided ``ws`` larger than that picks the layout its size allows."""
    torch = _torch()
    _check_tensor(d, "d")
    _check_tensor(grad_lambda, "grad_lambda")
    n = d.shape[0]
    off = _host_offsets(offsets if offsets is not None else [0, n])
    total = int(off[-1])
    if e is None or e.shape[0] < total:
        e_full = torch.zeros(max(total, 1), dtype=torch.float64, device=d.device)
        if e is not None and e.shape[0] > 0:
            e_full[: e.shape[0]] = e
        e = e_full
    _check_tensor(e, "e")
    lam = lam_out if lam_out is not None else torch.empty(total, dtype=torch.float64, device=d.device)
    gd = torch.empty(total, dtype=torch.float64, device=d.device)
    ge = torch.empty(max(total, 1), dtype=torch.float64, device=d.device)
    if total == 0:
        return lam, gd, ge[:0]
    if offsets_dev is None:
        offsets_dev = torch.from_numpy(off).to(d.device)
    need = backward_workspace_bytes(off, leaf, slots)
    ws = Workspace(need, d.device) if ws is None else ws.ensure(need)
    rc = _lib.load().tde_eigvals_backward(
        off.shape[0] - 1, off.ctypes.data, ctypes.c_void_p(offsets_dev.data_ptr()),
        ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(e.data_ptr()),
        ctypes.c_void_p(grad_lambda.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
        ctypes.c_void_p(gd.data_ptr()), ctypes.c_void_p(ge.data_ptr()), int(leaf),
        ctypes.c_void_p(ws.ptr), ws.nbytes, _stream_ptr(stream))
    _lib.check("tde_eigvals_backward", rc)
    if check:
        info = get_info(ws, stream)
        if info != 0:
            raise TdeError("tde_eigvals_backward (device status)", info)
    return lam, gd, ge[:total]


def _make_autograd():
    torch = _torch()

    class TdeEigvals(torch.autograd.Function):
        """lambda = eigvals(tridiag(e, d, e)) with a hand-written adjoint (the reverse
        merge sweep of tde_eigvals_backward).  offsets (host) packs several matrices."""

        @staticmethod
        def forward(ctx, d, e, offsets=None, leaf=8):
            n = d.shape[0]
            off = _host_offsets(offsets if offsets is not None else [0, n])
            ctx.save_for_backward(d, e)
            ctx.off = off
            ctx.leaf = leaf
            if offsets is None:
                return eigvals(d, e, leaf=leaf)
            return eigvals_batched(d, e, off, leaf=leaf)

        @staticmethod
        def backward(ctx, grad_lambda):
            d, e = ctx.saved_tensors
            _, gd, ge = eigvals_backward(d, e, grad_lambda.contiguous(), offsets=ctx.off, leaf=ctx.leaf)
            return gd, ge[: e.shape[0]], None, None

    return TdeEigvals


class _Lazy:
    cls = None


def TdeEigvals():  # noqa: N802 - mirrors a class name
    if _Lazy.cls is None:
        _Lazy.cls = _make_autograd()
    return _Lazy.cls


def eigvals_autograd(d, e, offsets=None, leaf: int = 8):
    """Differentiable eigenvalues (see TdeEigvals)."""
    return TdeEigvals().apply(d, e, offsets, leaf)


def measure_fp64_peak() -> float:
    """Measured FP64 FMA instructions per second of the current device (all lanes)."""
    out = ctypes.c_double()
    _lib.check("tde_measure_fp64_peak", _lib.load().tde_measure_fp64_peak(ctypes.byref(out)))
    return float(out.value)


def last_launch_count() -> int:
    """Kernel launches the last compute call on this thread enqueued."""
    return int(_lib.load().tde_last_launch_count())


def profile_enable(on: bool = True) -> None:
    """Record a CUDA event pair around every kernel of subsequent calls on this thread."""
    _lib.check("tde_profile_enable", _lib.load().tde_profile_enable(1 if on else 0))


def profile_select(classes=None) -> None:
    """Restrict the profiler to the named kernel classes on this thread (None: all)."""
    mask = 0
    for name in classes or ():
        mask |= 1 << _lib.KERNEL_NAMES.index(name)
    _lib.check("tde_profile_select", _lib.load().tde_profile_select(mask))


def profile_collect() -> dict:
    """{kernel class: (milliseconds, launches)} since the last collect (synchronises)."""
    n = len(_lib.KERNEL_NAMES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    _lib.check("tde_profile_collect", _lib.load().tde_profile_collect(n, ms, cnt))
    return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(_lib.KERNEL_NAMES)}


def profile_collect_steps(nsteps: int) -> list:
    """Per-merge-step breakdown since the last collect: a list of nsteps dicts
    {kernel class: (milliseconds, launches)} (synchronises)."""
    n = len(_lib.KERNEL_NAMES)
    rows = nsteps + 1
    ms = (ctypes.c_double * (n * rows))()
    cnt = (ctypes.c_int64 * (n * rows))()
    _lib.check("tde_profile_collect_steps",
               _lib.load().tde_profile_collect_steps(n, nsteps, ms, cnt))
    return [{name: (float(ms[(s + 1) * n + i]), int(cnt[(s + 1) * n + i]))
             for i, name in enumerate(_lib.KERNEL_NAMES)} for s in range(nsteps)]


def read_work(ws: Workspace, stream=None) -> dict:
    """Device work counters of the last call that used ``ws`` (synchronises)."""
    n = len(_lib.WORK_NAMES)
    out = (ctypes.c_ulonglong * n)()
    _lib.check("tde_read_work", _lib.load().tde_read_work(ctypes.c_void_p(ws.ptr), _stream_ptr(stream),
                                                          out, n))
    return {name: int(out[i]) for i, name in enumerate(_lib.WORK_NAMES)}
