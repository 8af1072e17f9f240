"""GB300-native findpts / findpts_eval (arXiv 1811.04891, Sec. 2.1).

Thin ctypes binding over the C ABI in ``include/findpts_gb.h``: every function
here only marshals torch CUDA tensors into device pointers and calls the
library of the same name, whose CUDA kernels do all the work.  There is no CPU
fallback: importing the package fails loudly when the shared library cannot
be built or loaded.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import torch

from . import build as _build

FP_OK, FP_ERR_INVALID_ARG, FP_ERR_OOM, FP_ERR_CUDA, FP_ERR_TIMEOUT, FP_ERR_NOT_SETUP = range(6)
INSIDE, BORDER, NOT_FOUND, RETRY = 0, 1, 2, 3
PREC_FP64, PREC_MIXED = 0, 1


class FindptsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


class fp_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol_accept", ctypes.c_double),
                ("tol_border", ctypes.c_double), ("max_newton", ctypes.c_int),
                ("hash_cells_per_elem", ctypes.c_double), ("tie_band", ctypes.c_double),
                ("points_per_block", ctypes.c_int)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        path = _build.build()
    L = ctypes.CDLL(path)
    vp, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.fp_default_opts.argtypes = [ctypes.POINTER(fp_opts)]
    L.fp_default_opts.restype = None
    L.fp_setup.argtypes = [ctypes.POINTER(vp), vp, i64, ci, vp, vp, ctypes.POINTER(fp_opts), vp]
    L.fp_setup.restype = ci
    L.fp_reserve.argtypes = [vp, i64]
    L.fp_reserve.restype = ci
    L.fp_find.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    L.fp_find.restype = ci
    L.fp_find_static.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    L.fp_find_static.restype = ci
    L.fp_workspace_create.argtypes = [vp, i64, i64, ctypes.POINTER(vp)]
    L.fp_workspace_create.restype = ci
    L.fp_workspace_free.argtypes = [vp]
    L.fp_workspace_free.restype = None
    L.fp_find_ws.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    L.fp_find_ws.restype = ci
    L.fp_workspace_last_pairs.argtypes = [vp, ctypes.POINTER(i64)]
    L.fp_workspace_last_pairs.restype = ci
    L.fp_batch_create.argtypes = [ctypes.POINTER(vp), ci, ctypes.POINTER(vp), ctypes.POINTER(i64), ci,
                                  ctypes.POINTER(vp), ctypes.c_double]
    L.fp_batch_create.restype = ci
    L.fp_batch_run.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.fp_batch_run.restype = ci
    L.fp_batch_tune.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, ci, ctypes.POINTER(ctypes.c_double)]
    L.fp_batch_tune.restype = ci
    L.fp_batch_schedule.argtypes = [vp, ci, ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(ci)]
    L.fp_batch_schedule.restype = ci
    L.fp_batch_mode.argtypes = [vp, ctypes.POINTER(ci)]
    L.fp_batch_mode.restype = ci
    L.fp_batch_groups.argtypes = [vp, ctypes.POINTER(ci)]
    L.fp_batch_groups.restype = ci
    L.fp_batch_group_info.argtypes = [vp, ci, ctypes.POINTER(ci), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                      ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]
    L.fp_batch_group_info.restype = ci
    L.fp_batch_profile.argtypes = [vp, ci]
    L.fp_batch_profile.restype = ci
    L.fp_batch_band_hits.argtypes = [vp, ctypes.POINTER(i64)]
    L.fp_batch_band_hits.restype = ci
    L.fp_batch_capture.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    L.fp_batch_capture.restype = ci
    L.fp_batch_launch.argtypes = [vp, vp]
    L.fp_batch_launch.restype = ci
    L.fp_batch_last_error.argtypes = [vp]
    L.fp_batch_last_error.restype = ctypes.c_char_p
    L.fp_batch_free.argtypes = [vp]
    L.fp_batch_free.restype = None
    L.fp_fields_create.argtypes = [vp, ci, vp, ctypes.POINTER(vp), vp]
    L.fp_fields_create.restype = ci
    L.fp_fields_free.argtypes = [vp]
    L.fp_fields_free.restype = None
    L.fp_eval_df.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp]
    L.fp_eval_df.restype = ci
    L.fp_find_eval.argtypes = [vp, i64, vp, vp, ci, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.fp_find_eval.restype = ci
    L.fp_find_eval_host.argtypes = [vp, i64, vp, vp, ci, vp, vp, vp, vp, vp, vp, vp, vp, i64, i64, vp]
    L.fp_find_eval_host.restype = ci
    L.fp_points_create.argtypes = [vp, i64, ctypes.POINTER(vp)]
    L.fp_points_create.restype = ci
    L.fp_points_free.argtypes = [vp]
    L.fp_points_free.restype = None
    L.fp_points_set.argtypes = [vp, vp, vp, vp, vp, vp]
    L.fp_points_set.restype = ci
    L.fp_eval_points.argtypes = [vp, vp, vp, vp, vp]
    L.fp_eval_points.restype = ci
    L.fp_setup_2d.argtypes = list(L.fp_setup.argtypes)
    L.fp_setup_2d.restype = ci
    L.fp_find_warm.argtypes = [vp, i64, vp, vp, vp, vp, ci, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.fp_find_warm.restype = ci
    L.fp_update_coords.argtypes = [vp, vp, vp, ci, vp]
    L.fp_update_coords.restype = ci
    L.fp_find_eval_ws.argtypes = [vp, vp, i64, vp, vp, ci, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.fp_find_eval_ws.restype = ci
    L.fp_bfaces_create.argtypes = [vp, vp, ctypes.POINTER(vp), vp]
    L.fp_bfaces_create.restype = ci
    L.fp_bfaces_free.argtypes = [vp]
    L.fp_bfaces_free.restype = None
    L.fp_bfaces_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.fp_bfaces_info.restype = ci
    L.fp_bfaces_nodes.argtypes = [vp, vp, vp, vp, vp, vp]
    L.fp_bfaces_nodes.restype = ci
    L.fp_flux_correct.argtypes = [vp, vp, vp, vp, vp, vp]
    L.fp_flux_correct.restype = ci
    L.fp_flux_correct_iface.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.fp_flux_correct_iface.restype = ci
    L.fp_bfaces_iface.argtypes = [vp, ctypes.POINTER(i64), vp, vp]
    L.fp_bfaces_iface.restype = ci
    L.fp_bfaces_refresh.argtypes = [vp, vp]
    L.fp_bfaces_refresh.restype = ci
    L.fp_bfaces_sort_iface.argtypes = [vp, vp, vp]
    L.fp_bfaces_sort_iface.restype = ci
    L.fp_extrapolate.argtypes = [ci, i64, ctypes.POINTER(vp), vp, vp]
    L.fp_extrapolate.restype = ci
    L.fp_eval.argtypes = [vp, i64, vp, vp, vp, ci, vp, vp, vp]
    L.fp_eval.restype = ci
    L.fp_free.argtypes = [vp]
    L.fp_free.restype = None
    L.fp_error_string.argtypes = [ci]
    L.fp_error_string.restype = ctypes.c_char_p
    L.fp_last_error.argtypes = [vp]
    L.fp_last_error.restype = ctypes.c_char_p
    L.fp_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(ci), ctypes.POINTER(i64),
                          ctypes.POINTER(i64), ctypes.POINTER(ci)]
    L.fp_info.restype = ci
    L.fp_debug_boxes.argtypes = [vp, vp, vp, vp, vp, vp]
    L.fp_debug_boxes.restype = ci
    L.fp_profile.argtypes = [vp, ci]
    L.fp_profile.restype = ci
    L.fp_set_mixed_refine.argtypes = [vp, ci]
    L.fp_set_mixed_refine.restype = ci
    L.fp_set_eval_staging.argtypes = [vp, ci]
    L.fp_set_eval_staging.restype = ci
    L.fp_profile_read.argtypes = [vp, ci, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
    L.fp_profile_read.restype = ci
    L.fp_launch_count.argtypes = []
    L.fp_launch_count.restype = i64
    L.fp_last_find_stats.argtypes = [vp, ctypes.POINTER(i64)]
    L.fp_last_find_stats.restype = ci
    L.fp_newton_paths.argtypes = [vp, ctypes.POINTER(i64)]
    L.fp_newton_paths.restype = ci
    L.fp_workspace_bytes.argtypes = [vp, i64, i64, ctypes.POINTER(i64)]
    L.fp_workspace_bytes.restype = ci
    L.fp_memory.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.fp_memory.restype = ci
    L.fp_band_hits.argtypes = [vp, ctypes.POINTER(i64)]
    L.fp_band_hits.restype = ci
    L.fp_fma_probe.argtypes = [ci, i64, ci, vp, ctypes.POINTER(ctypes.c_double), vp]
    L.fp_fma_probe.restype = ci
    L.fp_probe_threads.argtypes = [ci]
    L.fp_probe_threads.restype = i64
    _lib = L
    return L


def lib():
    return _load()


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(st: int, h=None):
    if st != FP_OK:
        L = lib()
        msg = L.fp_last_error(h).decode() if h is not None else L.fp_last_error(None).decode()
        raise FindptsError(st, msg or L.fp_error_string(st).decode())


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    return t.contiguous()


def default_opts(**kw) -> fp_opts:
    o = fp_opts()
    lib().fp_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


@dataclass
class Handle:
    ptr: ctypes.c_void_p
    E: int
    N: int
    dim: int = 3

    def __del__(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            try:
                lib().fp_free(self.ptr)
            except Exception:
                pass
            self.ptr = ctypes.c_void_p(None)

    def info(self):
        E, N, nc, nnz, ns = (ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int())
        _check(lib().fp_info(self.ptr, ctypes.byref(E), ctypes.byref(N), ctypes.byref(nc),
                             ctypes.byref(nnz), ctypes.byref(ns)), self.ptr)
        return {"E": E.value, "N": N.value, "ncell": nc.value, "nnz": nnz.value, "nsub": ns.value}


def fp_setup(coords: torch.Tensor, N: int, sub: Optional[torch.Tensor] = None,
             dist: Optional[torch.Tensor] = None, opts: Optional[fp_opts] = None,
             stream=None) -> Handle:
    """Post a mesh: coords [3][E][(N+1)^3] float64 CUDA tensor, sub [E] int32,
    dist [E][(N+1)^3] float64 or None."""
    coords = _dev(coords, torch.float64, "coords")
    E = coords.shape[1]
    if coords.ndim != 3 or coords.shape[0] != 3 or coords.shape[2] != (N + 1) ** 3:
        raise ValueError("coords must be [3][E][(N+1)^3]")
    sub = None if sub is None else _dev(sub, torch.int32, "sub")
    dist = None if dist is None else _dev(dist, torch.float64, "dist")
    h = ctypes.c_void_p()
    st = lib().fp_setup(ctypes.byref(h), _ptr(coords), E, N, _ptr(sub), _ptr(dist),
                        None if opts is None else ctypes.byref(opts), _stream(stream))
    _check(st, None)
    return Handle(ptr=h, E=E, N=N)


def fp_setup_2d(coords: torch.Tensor, N: int, sub: Optional[torch.Tensor] = None,
                dist: Optional[torch.Tensor] = None, opts: Optional[fp_opts] = None,
                stream=None) -> Handle:
    """Post a 2D quadrilateral mesh: coords [2][E][(N+1)^2] float64 CUDA
    tensor, sub [E] int32, dist [E][(N+1)^2] float64 (required with more than
    one subdomain).  FP64 form only."""
    coords = _dev(coords, torch.float64, "coords")
    if coords.ndim != 3 or coords.shape[0] != 2 or coords.shape[2] != (N + 1) ** 2:
        raise ValueError("coords must be [2][E][(N+1)^2]")
    E = coords.shape[1]
    sub = None if sub is None else _dev(sub, torch.int32, "sub")
    dist = None if dist is None else _dev(dist, torch.float64, "dist")
    h = ctypes.c_void_p()
    st = lib().fp_setup_2d(ctypes.byref(h), _ptr(coords), E, N, _ptr(sub), _ptr(dist),
                           None if opts is None else ctypes.byref(opts), _stream(stream))
    _check(st, None)
    return Handle(ptr=h, E=E, N=N, dim=2)


def fp_reserve(h: Handle, P: int):
    _check(lib().fp_reserve(h.ptr, int(P)), h.ptr)


def fp_find(h: Handle, pts: torch.Tensor, qsess: Optional[torch.Tensor] = None, out=None, stream=None):
    """Locate points pts [d][P] float64 (d = the handle's dimension).
    Returns (code, sub, elem, rst [d][P], dist2)."""
    pts = _dev(pts, torch.float64, "pts")
    P = pts.shape[1]
    qsess = None if qsess is None else _dev(qsess, torch.int32, "qsess")
    dev = pts.device
    if out is None:
        out = _find_outs(P, dev, h.dim)
    code, sub, elem, rst, dist2 = out
    st = lib().fp_find(h.ptr, P, _ptr(pts), _ptr(qsess), _ptr(code), _ptr(sub), _ptr(elem), _ptr(rst),
                       _ptr(dist2), _stream(stream))
    _check(st, h.ptr)
    return code, sub, elem, rst, dist2


class Workspace:
    """Scratch for asynchronous finds (fp_workspace_create); one call at a time."""

    def __init__(self, h: Handle, max_points: int, max_pairs: int = 0):
        self.ptr = ctypes.c_void_p()
        self.handle = h
        self.max_points = int(max_points)
        _check(lib().fp_workspace_create(h.ptr, int(max_points), int(max_pairs), ctypes.byref(self.ptr)), h.ptr)

    def __del__(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            try:
                lib().fp_workspace_free(self.ptr)
            except Exception:
                pass
            self.ptr = ctypes.c_void_p(None)

    def last_pairs(self) -> int:
        n = ctypes.c_int64()
        _check(lib().fp_workspace_last_pairs(self.ptr, ctypes.byref(n)))
        return n.value


def fp_find_ws(h: Handle, ws: Workspace, pts: torch.Tensor, qsess: Optional[torch.Tensor] = None, out=None,
               stream=None):
    """Asynchronous find (no host wait, no allocation in the library call)."""
    pts = _dev(pts, torch.float64, "pts")
    P = pts.shape[1]
    qsess = None if qsess is None else _dev(qsess, torch.int32, "qsess")
    dev = pts.device
    if out is None:
        out = _find_outs(P, dev, h.dim)
    code, sub, elem, rst, dist2 = out
    st = lib().fp_find_ws(h.ptr, ws.ptr, P, _ptr(pts), _ptr(qsess), _ptr(code), _ptr(sub), _ptr(elem), _ptr(rst),
                          _ptr(dist2), _stream(stream))
    _check(st, h.ptr)
    return code, sub, elem, rst, dist2


class Batch:
    """Independent instances (handles) located and interpolated together
    (fp_batch_*).  Inputs/outputs are concatenated in instance order."""

    def __init__(self, handles, npts, fields=None, pairs_per_point: float = 2.0):
        L = lib()
        self.handles = list(handles)             # keep them alive
        self.npts = [int(x) for x in npts]
        self.P = sum(self.npts)
        self.fields = None if fields is None else [_dev(f, torch.float64, "fields") for f in fields]
        F = 0 if fields is None else int(self.fields[0].shape[0])
        self.F = F
        hp = (ctypes.c_void_p * len(self.handles))(*[h.ptr.value for h in self.handles])
        npa = (ctypes.c_int64 * len(self.npts))(*self.npts)
        fp_arr = None
        if fields is not None:
            fp_arr = (ctypes.c_void_p * len(self.fields))(*[f.data_ptr() for f in self.fields])
        self.ptr = ctypes.c_void_p()
        st = L.fp_batch_create(ctypes.byref(self.ptr), len(self.handles), hp, npa, F, fp_arr,
                               float(pairs_per_point))
        if st != FP_OK:
            raise FindptsError(st, "fp_batch_create failed")

    def __del__(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            try:
                lib().fp_batch_free(self.ptr)
            except Exception:
                pass
            self.ptr = ctypes.c_void_p(None)

    def _chk(self, st):
        if st != FP_OK:
            raise FindptsError(st, lib().fp_batch_last_error(self.ptr).decode())

    def outputs(self, device=None):
        dev = device or torch.device("cuda")
        P = self.P
        return (torch.empty(P, dtype=torch.int32, device=dev), torch.empty(P, dtype=torch.int32, device=dev),
                torch.empty(P, dtype=torch.int32, device=dev), torch.empty((3, P), dtype=torch.float64, device=dev),
                torch.empty(P, dtype=torch.float64, device=dev),
                torch.empty((max(self.F, 1), P), dtype=torch.float64, device=dev))

    def _args(self, pts, outs):
        code, sub, elem, rst, d2, val = outs
        return (_ptr(pts), _ptr(code), _ptr(sub), _ptr(elem), _ptr(rst), _ptr(d2),
                _ptr(val) if self.F > 0 else None)

    def run(self, pts, outs, stream=None):
        pts = _dev(pts, torch.float64, "pts")
        self._chk(lib().fp_batch_run(self.ptr, *self._args(pts, outs), _stream(stream)))
        return outs

    def tune(self, pts, outs, reps: int = 2, stream=None) -> float:
        pts = _dev(pts, torch.float64, "pts")
        ms = ctypes.c_double()
        self._chk(lib().fp_batch_tune(self.ptr, *self._args(pts, outs), _stream(stream), int(reps), ctypes.byref(ms)))
        return ms.value

    def schedule(self, group: int = 0, block: int = 0, blocks_per_sm: int = 0, tile: int = 0):
        """(threads per block, blocks per SM, pairs per work item) of one
        group's Newton stage; positive arguments set them."""
        b, s, t = ctypes.c_int(block), ctypes.c_int(blocks_per_sm), ctypes.c_int(tile)
        self._chk(lib().fp_batch_schedule(self.ptr, int(group), ctypes.byref(b), ctypes.byref(s), ctypes.byref(t)))
        return b.value, s.value, t.value

    def mode(self, sequential: int = -1) -> int:
        """1 when the groups' launches run one after another, 0 when
        concurrently; 0 or 1 sets the mode first."""
        m = ctypes.c_int(int(sequential))
        self._chk(lib().fp_batch_mode(self.ptr, ctypes.byref(m)))
        return m.value

    def groups(self) -> int:
        n = ctypes.c_int()
        self._chk(lib().fp_batch_groups(self.ptr, ctypes.byref(n)))
        return n.value

    def group_info(self, group: int) -> dict:
        N, E, P, pairs = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        tn, te = ctypes.c_double(), ctypes.c_double()
        self._chk(lib().fp_batch_group_info(self.ptr, int(group), ctypes.byref(N), ctypes.byref(E), ctypes.byref(P),
                                            ctypes.byref(pairs), ctypes.byref(tn), ctypes.byref(te)))
        return {"N": N.value, "E": E.value, "P": P.value, "pairs": pairs.value, "newton_ms": tn.value,
                "eval_ms": te.value}

    def profile(self, enable: bool = True):
        self._chk(lib().fp_batch_profile(self.ptr, 1 if enable else 0))

    def band_hits(self) -> dict:
        c = (ctypes.c_int64 * 3)()
        self._chk(lib().fp_batch_band_hits(self.ptr, c))
        return {k: int(c[i]) for i, k in enumerate(BAND_KINDS)}

    def capture(self, pts, outs):
        pts = _dev(pts, torch.float64, "pts")
        self._chk(lib().fp_batch_capture(self.ptr, *self._args(pts, outs)))

    def launch(self, stream=None):
        self._chk(lib().fp_batch_launch(self.ptr, _stream(stream)))


STATIC_MAX_POINTS = 16384
STATIC_MAX_PAIRS = 65536


def fp_find_static(h: Handle, pts: torch.Tensor, qsess: Optional[torch.Tensor] = None, out=None, stream=None):
    """fp_find without any device allocation in the call (scratch in a fixed
    device array; at most STATIC_MAX_POINTS points).  Pass preallocated
    `out` tensors to keep the whole call allocation-free."""
    pts = _dev(pts, torch.float64, "pts")
    P = pts.shape[1]
    qsess = None if qsess is None else _dev(qsess, torch.int32, "qsess")
    dev = pts.device
    if out is None:
        out = _find_outs(P, dev, h.dim)
    code, sub, elem, rst, dist2 = out
    st = lib().fp_find_static(h.ptr, P, _ptr(pts), _ptr(qsess), _ptr(code), _ptr(sub), _ptr(elem), _ptr(rst),
                              _ptr(dist2), _stream(stream))
    _check(st, h.ptr)
    return code, sub, elem, rst, dist2


def fp_eval(h: Handle, code: torch.Tensor, elem: torch.Tensor, rst: torch.Tensor, fields: torch.Tensor,
            out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Interpolate fields [F][E][(N+1)^3] (or [E][(N+1)^3]) at located points -> [F][P]."""
    fields = _dev(fields, torch.float64, "fields")
    if fields.ndim == 2:
        fields = fields.unsqueeze(0)
    F = fields.shape[0]
    P = code.shape[0]
    if out is None:
        out = torch.empty((F, P), dtype=torch.float64, device=fields.device)
    st = lib().fp_eval(h.ptr, P, _ptr(code), _ptr(elem), _ptr(rst), F, _ptr(fields), _ptr(out),
                       _stream(stream))
    _check(st, h.ptr)
    return out


class Fields:
    """Fields posted as double-float pairs for fp_eval_df (mixed form)."""

    def __init__(self, h: Handle, fields: torch.Tensor, stream=None):
        fields = _dev(fields, torch.float64, "fields")
        if fields.ndim == 2:
            fields = fields.unsqueeze(0)
        self.F = int(fields.shape[0])
        self.handle = h
        self.ptr = ctypes.c_void_p()
        _check(lib().fp_fields_create(h.ptr, self.F, _ptr(fields), ctypes.byref(self.ptr), _stream(stream)), h.ptr)

    def __del__(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            try:
                lib().fp_fields_free(self.ptr)
            except Exception:
                pass
            self.ptr = ctypes.c_void_p(None)


def fp_eval_df(h: Handle, f: Fields, code: torch.Tensor, elem: torch.Tensor, rst: torch.Tensor,
               out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Double-float interpolation of posted fields at located points -> [F][P]."""
    P = code.shape[0]
    if out is None:
        out = torch.empty((f.F, P), dtype=torch.float64, device=code.device)
    st = lib().fp_eval_df(h.ptr, f.ptr, P, _ptr(code), _ptr(elem), _ptr(rst), _ptr(out), _stream(stream))
    _check(st, h.ptr)
    return out


def _find_outs(P, dev, dim: int = 3):
    return (torch.empty(P, dtype=torch.int32, device=dev), torch.empty(P, dtype=torch.int32, device=dev),
            torch.empty(P, dtype=torch.int32, device=dev), torch.empty((dim, P), dtype=torch.float64, device=dev),
            torch.empty(P, dtype=torch.float64, device=dev))


def _eval_args(fields, posted):
    if posted is not None:
        return posted.F, None, posted.ptr
    fields = _dev(fields, torch.float64, "fields")
    if fields.ndim == 2:
        fields = fields.unsqueeze(0)
    return int(fields.shape[0]), fields, None


def fp_find_eval(h: Handle, pts: torch.Tensor, qsess: Optional[torch.Tensor] = None, fields=None,
                 posted: Optional["Fields"] = None, out=None, values: Optional[torch.Tensor] = None, stream=None):
    """Fused find + eval: returns (code, sub, elem, rst, dist2, values [F][P]).
    Uses posted double-float fields when given, else FP64 `fields`."""
    pts = _dev(pts, torch.float64, "pts")
    P = pts.shape[1]
    qsess = None if qsess is None else _dev(qsess, torch.int32, "qsess")
    F, f64, fptr = _eval_args(fields, posted)
    out = out or _find_outs(P, pts.device, h.dim)
    if values is None:
        values = torch.empty((F, P), dtype=torch.float64, device=pts.device)
    code, sub, elem, rst, dist2 = out
    st = lib().fp_find_eval(h.ptr, P, _ptr(pts), _ptr(qsess), F, _ptr(f64), fptr, _ptr(code), _ptr(sub), _ptr(elem),
                            _ptr(rst), _ptr(dist2), _ptr(values), _stream(stream))
    _check(st, h.ptr)
    return code, sub, elem, rst, dist2, values


def fp_find_eval_ws(h: Handle, ws: "Workspace", pts: torch.Tensor, qsess: Optional[torch.Tensor] = None, fields=None,
                    posted: Optional["Fields"] = None, out=None, values: Optional[torch.Tensor] = None, stream=None):
    """Asynchronous fused find + eval with the scratch in `ws`."""
    pts = _dev(pts, torch.float64, "pts")
    P = pts.shape[1]
    qsess = None if qsess is None else _dev(qsess, torch.int32, "qsess")
    F, f64, fptr = _eval_args(fields, posted)
    out = out or _find_outs(P, pts.device, h.dim)
    if values is None:
        values = torch.empty((F, P), dtype=torch.float64, device=pts.device)
    code, sub, elem, rst, dist2 = out
    st = lib().fp_find_eval_ws(h.ptr, ws.ptr, P, _ptr(pts), _ptr(qsess), F, _ptr(f64), fptr, _ptr(code), _ptr(sub),
                               _ptr(elem), _ptr(rst), _ptr(dist2), _ptr(values), _stream(stream))
    _check(st, h.ptr)
    return code, sub, elem, rst, dist2, values


def fp_find_eval_host(h: Handle, pts: torch.Tensor, qsess: Optional[torch.Tensor] = None, fields=None,
                      posted: Optional["Fields"] = None, out=None, values: Optional[torch.Tensor] = None,
                      chunk: int = 0, max_pairs: int = 0, stream=None):
    """find (+ eval when fields or posted are given) over points in HOST
    memory (CPU tensor [3][P] float64, pinned for speed), streamed through
    the device in chunks with the copies overlapping the search.  Returns
    CPU tensors (code, sub, elem, rst [3][P], dist2[, values [F][P]])."""
    if not isinstance(pts, torch.Tensor) or pts.is_cuda or pts.dtype != torch.float64 or not pts.is_contiguous():
        raise TypeError("pts: expected a contiguous float64 CPU tensor")
    if pts.ndim != 2 or pts.shape[0] != 3:
        raise ValueError("pts must be [3][P]")
    P = pts.shape[1]
    if qsess is not None and (qsess.is_cuda or qsess.dtype != torch.int32 or not qsess.is_contiguous()):
        raise TypeError("qsess: expected a contiguous int32 CPU tensor")
    F, f64, fptr = (0, None, None) if fields is None and posted is None else _eval_args(fields, posted)
    pin = pts.is_pinned()
    if out is None:
        out = (torch.empty(P, dtype=torch.int32, pin_memory=pin), torch.empty(P, dtype=torch.int32, pin_memory=pin),
               torch.empty(P, dtype=torch.int32, pin_memory=pin), torch.empty((3, P), dtype=torch.float64, pin_memory=pin),
               torch.empty(P, dtype=torch.float64, pin_memory=pin))
    if F and values is None:
        values = torch.empty((F, P), dtype=torch.float64, pin_memory=pin)
    code, sub, elem, rst, dist2 = out
    st = lib().fp_find_eval_host(h.ptr, P, _ptr(pts), _ptr(qsess), F, _ptr(f64), fptr, _ptr(code), _ptr(sub),
                                 _ptr(elem), _ptr(rst), _ptr(dist2), _ptr(values if F else None), int(chunk),
                                 int(max_pairs), _stream(stream))
    _check(st, h.ptr)
    return (code, sub, elem, rst, dist2, values) if F else (code, sub, elem, rst, dist2)


class Points:
    """Posted points (fp_points_*): split basis values of located points,
    kept for repeated evaluation of posted fields at the same (e, r)."""

    def __init__(self, h: Handle, P: int):
        self.handle = h
        self.P = int(P)
        self.ptr = ctypes.c_void_p()
        _check(lib().fp_points_create(h.ptr, self.P, ctypes.byref(self.ptr)), h.ptr)

    def __del__(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            try:
                lib().fp_points_free(self.ptr)
            except Exception:
                pass
            self.ptr = ctypes.c_void_p(None)

    def set(self, code: torch.Tensor, elem: torch.Tensor, rst: torch.Tensor, stream=None):
        code = _dev(code, torch.int32, "code")
        elem = _dev(elem, torch.int32, "elem")
        rst = _dev(rst, torch.float64, "rst")
        if code.numel() != self.P or elem.numel() != self.P or rst.shape != (3, self.P):
            raise ValueError("code, elem [P] and rst [3][P] must match the posted point count")
        _check(lib().fp_points_set(self.handle.ptr, self.ptr, _ptr(code), _ptr(elem), _ptr(rst), _stream(stream)),
               self.handle.ptr)

    def eval(self, posted: "Fields", out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((posted.F, self.P), dtype=torch.float64, device=torch.device("cuda"))
        _check(lib().fp_eval_points(self.handle.ptr, posted.ptr, self.ptr, _ptr(out), _stream(stream)),
               self.handle.ptr)
        return out


UPDATE_DEFAULT_DIST = 1


def fp_update_coords(h: Handle, coords: torch.Tensor, dist: Optional[torch.Tensor] = None,
                     default_dist: bool = False, stream=None):
    """Moving mesh: replace the node coordinates [3][E][(N+1)^3] of the
    handle's mesh and rebuild boxes, hash grid and FP32 geometry in place.
    `coords` may be a CUDA tensor or a CPU tensor (pinned for speed)."""
    if not isinstance(coords, torch.Tensor) or coords.dtype != torch.float64 or not coords.is_contiguous():
        raise TypeError("coords: expected a contiguous float64 tensor")
    if tuple(coords.shape) != (h.dim, h.E, (h.N + 1) ** h.dim):
        raise ValueError("coords must be [d][E][(N+1)^d] of the handle's mesh")
    dist = None if dist is None else _dev(dist, torch.float64, "dist")
    st = lib().fp_update_coords(h.ptr, _ptr(coords), _ptr(dist), UPDATE_DEFAULT_DIST if default_dist else 0,
                                _stream(stream))
    _check(st, h.ptr)


def fp_find_warm(h: Handle, pts: torch.Tensor, warm=None, qsess: Optional[torch.Tensor] = None, fields=None,
                 posted: Optional["Fields"] = None, out=None, values: Optional[torch.Tensor] = None, stream=None):
    """find (+ eval when fields or posted are given) with Newton warm-started
    from `warm` = (elem [P], rst [3][P]) of an earlier find; `out` may be the
    tuple that holds `warm` (in-place update).  Returns fp_find's tuple, plus
    the values [F][P] when evaluating."""
    pts = _dev(pts, torch.float64, "pts")
    P = pts.shape[1]
    qsess = None if qsess is None else _dev(qsess, torch.int32, "qsess")
    we, wr = (None, None) if warm is None else (_dev(warm[0], torch.int32, "warm elem"),
                                                _dev(warm[1], torch.float64, "warm rst"))
    F, f64, fptr = (0, None, None) if fields is None and posted is None else _eval_args(fields, posted)
    out = out or _find_outs(P, pts.device, h.dim)
    if F and values is None:
        values = torch.empty((F, P), dtype=torch.float64, device=pts.device)
    code, sub, elem, rst, dist2 = out
    st = lib().fp_find_warm(h.ptr, P, _ptr(pts), _ptr(qsess), _ptr(we), _ptr(wr), F, _ptr(f64), fptr, _ptr(code),
                            _ptr(sub), _ptr(elem), _ptr(rst), _ptr(dist2), _ptr(values if F else None),
                            _stream(stream))
    _check(st, h.ptr)
    return (code, sub, elem, rst, dist2, values) if F else (code, sub, elem, rst, dist2)


class BFaces:
    """Boundary-face quadrature of marked faces (fp_bfaces_*) for the
    mass-flux correction of interpolated interface data."""

    def __init__(self, h: Handle, kind: torch.Tensor, stream=None):
        if not isinstance(kind, torch.Tensor) or not kind.is_cuda or kind.dtype != torch.int8:
            raise TypeError("kind: expected an int8 CUDA tensor [E][6]")
        kind = kind.contiguous()
        self.handle = h
        self.ptr = ctypes.c_void_p()
        st = lib().fp_bfaces_create(h.ptr, _ptr(kind), ctypes.byref(self.ptr), _stream(stream))
        if st != FP_OK:
            raise FindptsError(st, "fp_bfaces_create failed")
        nf, M = ctypes.c_int64(), ctypes.c_int64()
        lib().fp_bfaces_info(self.ptr, ctypes.byref(nf), ctypes.byref(M))
        self.nfaces, self.M = nf.value, M.value
        mi = ctypes.c_int64()
        lib().fp_bfaces_iface(self.ptr, ctypes.byref(mi), None, None)
        self.Mi = mi.value

    def sort_iface(self, elem: torch.Tensor, stream=None):
        """Renumber the interface nodes by donor element (elem [Mi] int32,
        found at the current iface_points order)."""
        elem = _dev(elem, torch.int32, "elem")
        if elem.numel() != self.Mi:
            raise ValueError("elem must hold one element id per interface node")
        st = lib().fp_bfaces_sort_iface(self.ptr, _ptr(elem), _stream(stream))
        if st != FP_OK:
            raise FindptsError(st, "fp_bfaces_sort_iface failed")

    def refresh(self, stream=None):
        """Recompute node positions, normals and weights after fp_update_coords."""
        st = lib().fp_bfaces_refresh(self.ptr, _stream(stream))
        if st != FP_OK:
            raise FindptsError(st, "fp_bfaces_refresh failed")

    def iface_points(self, device=None, out: Optional[torch.Tensor] = None):
        """Positions [3][Mi] of the interface nodes (listing order)."""
        pts = out if out is not None else torch.empty((3, self.Mi), dtype=torch.float64,
                                                      device=device or torch.device("cuda"))
        st = lib().fp_bfaces_iface(self.ptr, None, _ptr(pts), _stream(None))
        if st != FP_OK:
            raise FindptsError(st, "fp_bfaces_iface failed")
        return pts

    def __del__(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            try:
                lib().fp_bfaces_free(self.ptr)
            except Exception:
                pass
            self.ptr = ctypes.c_void_p(None)

    def nodes(self, device=None):
        """(x [3][M], normal [3][M], dA [M], kind [M]) as device tensors."""
        dev = device or torch.device("cuda")
        M = self.M
        x = torch.empty((3, M), dtype=torch.float64, device=dev)
        nr = torch.empty((3, M), dtype=torch.float64, device=dev)
        dA = torch.empty(M, dtype=torch.float64, device=dev)
        kd = torch.empty(M, dtype=torch.int8, device=dev)
        st = lib().fp_bfaces_nodes(self.ptr, _ptr(x), _ptr(nr), _ptr(dA), _ptr(kd), _stream(None))
        if st != FP_OK:
            raise FindptsError(st, "fp_bfaces_nodes failed")
        return x, nr, dA, kd


def fp_flux_correct(bf: BFaces, u: torch.Tensor, u_out: Optional[torch.Tensor] = None, stream=None):
    """Eq. consv2 / corr: returns (u_out [3][M], gamma, flux) with gamma and
    flux as one-element device tensors."""
    u = _dev(u, torch.float64, "u")
    if u_out is None:
        u_out = torch.empty_like(u)
    g = torch.empty(1, dtype=torch.float64, device=u.device)
    fl = torch.empty(1, dtype=torch.float64, device=u.device)
    st = lib().fp_flux_correct(bf.ptr, _ptr(u), _ptr(u_out), _ptr(g), _ptr(fl), _stream(stream))
    if st != FP_OK:
        raise FindptsError(st, "fp_flux_correct failed")
    return u_out, g, fl


def fp_flux_correct_iface(bf: "BFaces", u_iface: torch.Tensor, u_pres: torch.Tensor, u_out=None, stream=None):
    """Flux correction with interpolated interface values u_iface [3][Mi] and
    prescribed values u_pres [3][M]; returns (u_out, gamma, flux)."""
    if u_out is None:
        u_out = torch.empty_like(u_pres)
    g = torch.empty(1, dtype=torch.float64, device=u_pres.device)
    fl = torch.empty(1, dtype=torch.float64, device=u_pres.device)
    st = lib().fp_flux_correct_iface(bf.ptr, _ptr(u_iface), _ptr(u_pres), _ptr(u_out), _ptr(g), _ptr(fl),
                                     _stream(stream))
    if st != FP_OK:
        raise FindptsError(st, "fp_flux_correct_iface failed")
    return u_out, g, fl


def fp_extrapolate(hist, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Order-len(hist) extrapolation in time (newest first), equal steps."""
    m = len(hist)
    h0 = hist[0]
    if out is None:
        out = torch.empty_like(h0)
    arr = (ctypes.c_void_p * m)(*[t.data_ptr() for t in hist])
    st = lib().fp_extrapolate(m, h0.numel(), arr, _ptr(out), _stream(stream))
    if st != FP_OK:
        raise FindptsError(st, "fp_extrapolate failed")
    return out


PROF_KINDS = {"screen": 0, "sort": 1, "newton": 2, "rank": 3, "eval": 4}


def fp_profile(h: Handle, enable: bool = True):
    _check(lib().fp_profile(h.ptr, int(bool(enable))), h.ptr)


def fp_set_eval_staging(h: Handle, enable: bool = True):
    """Fused eval of posted fields from shared memory (same results)."""
    _check(lib().fp_set_eval_staging(h.ptr, int(bool(enable))), h.ptr)


def fp_set_mixed_refine(h: Handle, max_residuals: int):
    """Mixed form: compensated residuals per pair before the full FP64
    Newton (0..8, default 3; 0 sends every pair to the full FP64 Newton)."""
    _check(lib().fp_set_mixed_refine(h.ptr, int(max_residuals)), h.ptr)


def fp_profile_read(h: Handle, kind: str):
    """(total device ms, launches) of one kernel class since the last read."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(lib().fp_profile_read(h.ptr, PROF_KINDS[kind], ctypes.byref(ms), ctypes.byref(n)), h.ptr)
    return ms.value, n.value


def fp_last_find_stats(h: Handle) -> int:
    """Candidate pairs of the handle's last fp_find."""
    n = ctypes.c_int64()
    _check(lib().fp_last_find_stats(h.ptr, ctypes.byref(n)), h.ptr)
    return n.value


def fp_newton_paths(h: Handle) -> dict:
    """Mixed-form Newton path counts since the last read (profiling on)."""
    c = (ctypes.c_int64 * 4)()
    _check(lib().fp_newton_paths(h.ptr, c), h.ptr)
    return {"rejected_fp32": c[0], "fp32_not_converged": c[1], "fp64_step_converged": c[2], "fallback": c[3]}


def fp_workspace_bytes(h: Handle, max_points: int, max_pairs: int = 0) -> int:
    """Device bytes a workspace of this size holds on the handle's mesh."""
    b = ctypes.c_int64()
    _check(lib().fp_workspace_bytes(h.ptr, int(max_points), int(max_pairs), ctypes.byref(b)), h.ptr)
    return b.value


def fp_memory(h: Handle) -> dict:
    """Device bytes of the handle: the resident mesh and search structures,
    and its own find workspace."""
    r, w = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().fp_memory(h.ptr, ctypes.byref(r), ctypes.byref(w)), h.ptr)
    return {"resident": r.value, "workspace": w.value}


BAND_KINDS = ("accept", "border", "owner")


def fp_band_hits(h: Handle) -> dict:
    """Near-tie counts of the handle's classifications since the last read
    (synchronises the device and resets them)."""
    c = (ctypes.c_int64 * 3)()
    _check(lib().fp_band_hits(h.ptr, c), h.ptr)
    return {k: int(c[i]) for i, k in enumerate(BAND_KINDS)}


PROBE_KINDS = {"f64": 0, "f32": 1, "df": 2, "f32x2": 3, "df2": 4}


def fp_probe_threads(blocks_per_sm: int = 4) -> int:
    return int(lib().fp_probe_threads(int(blocks_per_sm)))


def fp_fma_probe(kind: str, iters: int, sink: torch.Tensor, blocks_per_sm: int = 4, stream=None) -> float:
    """Enqueue one multiply-add chain probe launch (kind 'f64', 'f32' or 'df')
    writing one double per thread to `sink`; returns the launch's flops."""
    sink = _dev(sink, torch.float64, "sink")
    if sink.numel() < fp_probe_threads(blocks_per_sm):
        raise ValueError("sink smaller than fp_probe_threads(blocks_per_sm)")
    fl = ctypes.c_double(0.0)
    _check(lib().fp_fma_probe(PROBE_KINDS[kind], int(iters), int(blocks_per_sm), _ptr(sink), ctypes.byref(fl),
                              _stream(stream)))
    return fl.value


def fp_launch_count() -> int:
    return int(lib().fp_launch_count())


def fp_debug_boxes(h: Handle):
    """Per-element padded axis boxes and the hash grid (for tests)."""
    inf = h.info()
    dev = torch.device("cuda")
    aabb = torch.empty((h.E, 6), dtype=torch.float64, device=dev)
    grid = torch.empty(9, dtype=torch.float64, device=dev)
    cs = torch.empty(inf["ncell"] + 1, dtype=torch.int32, device=dev)
    ce = torch.empty(max(inf["nnz"], 1), dtype=torch.int32, device=dev)
    _check(lib().fp_debug_boxes(h.ptr, _ptr(aabb), _ptr(grid), _ptr(cs), _ptr(ce), _stream(None)), h.ptr)
    torch.cuda.synchronize()
    return aabb, grid, cs, ce


# ---------------------------------------------------------------------------
# The rest of the C ABI under its own names.  Objects the library creates come
# back as the classes above (which free them when collected); the *_free calls
# free them at once.  Argument marshalling only, as everywhere in this module.
# ---------------------------------------------------------------------------
def _release(obj, free_fn):
    if obj is not None and getattr(obj, "ptr", None) is not None and obj.ptr.value:
        free_fn(obj.ptr)
        obj.ptr = ctypes.c_void_p(None)


def fp_default_opts(**kw) -> fp_opts:
    """fp_default_opts, with keyword overrides (see default_opts)."""
    return default_opts(**kw)


def fp_error_string(status: int) -> str:
    return lib().fp_error_string(int(status)).decode()


def fp_last_error(h: Optional[Handle] = None) -> str:
    return lib().fp_last_error(None if h is None else h.ptr).decode()


def fp_info(h: Handle) -> dict:
    return h.info()


def fp_free(h: Handle):
    _release(h, lib().fp_free)


def fp_workspace_create(h: Handle, max_points: int, max_pairs: int = 0) -> Workspace:
    return Workspace(h, max_points, max_pairs)


def fp_workspace_free(ws: Workspace):
    _release(ws, lib().fp_workspace_free)


def fp_workspace_last_pairs(ws: Workspace) -> int:
    return ws.last_pairs()


def fp_fields_create(h: Handle, fields: torch.Tensor, stream=None) -> Fields:
    return Fields(h, fields, stream)


def fp_fields_free(f: Fields):
    _release(f, lib().fp_fields_free)


def fp_points_create(h: Handle, P: int) -> Points:
    return Points(h, P)


def fp_points_free(q: Points):
    _release(q, lib().fp_points_free)


def fp_points_set(h: Handle, q: Points, code: torch.Tensor, elem: torch.Tensor, rst: torch.Tensor, stream=None):
    if q.handle is not h:
        raise ValueError("posted points belong to another handle")
    q.set(code, elem, rst, stream)


def fp_eval_points(h: Handle, f: Fields, q: Points, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    if q.handle is not h:
        raise ValueError("posted points belong to another handle")
    return q.eval(f, out, stream)


def fp_batch_create(handles, npts, fields=None, pairs_per_point: float = 2.0) -> Batch:
    return Batch(handles, npts, fields, pairs_per_point)


def fp_batch_run(b: Batch, pts: torch.Tensor, outs, stream=None):
    return b.run(pts, outs, stream)


def fp_batch_tune(b: Batch, pts: torch.Tensor, outs, reps: int = 2, stream=None) -> float:
    return b.tune(pts, outs, reps, stream)


def fp_batch_schedule(b: Batch, group: int = 0, block: int = 0, blocks_per_sm: int = 0, tile: int = 0):
    return b.schedule(group, block, blocks_per_sm, tile)


def fp_batch_mode(b: Batch, sequential: int = -1) -> int:
    return b.mode(sequential)


def fp_batch_groups(b: Batch) -> int:
    return b.groups()


def fp_batch_group_info(b: Batch, group: int) -> dict:
    return b.group_info(group)


def fp_batch_profile(b: Batch, enable: bool = True):
    b.profile(enable)


def fp_batch_band_hits(b: Batch) -> dict:
    return b.band_hits()


def fp_batch_capture(b: Batch, pts: torch.Tensor, outs):
    b.capture(pts, outs)


def fp_batch_launch(b: Batch, stream=None):
    b.launch(stream)


def fp_batch_last_error(b: Batch) -> str:
    return lib().fp_batch_last_error(b.ptr).decode()


def fp_batch_free(b: Batch):
    _release(b, lib().fp_batch_free)


def fp_bfaces_create(h: Handle, kind: torch.Tensor, stream=None) -> BFaces:
    return BFaces(h, kind, stream)


def fp_bfaces_free(bf: BFaces):
    _release(bf, lib().fp_bfaces_free)


def fp_bfaces_info(bf: BFaces):
    """(number of listed faces, number of face nodes M)."""
    return bf.nfaces, bf.M


def fp_bfaces_nodes(bf: BFaces, device=None):
    return bf.nodes(device)


def fp_bfaces_refresh(bf: BFaces, stream=None):
    bf.refresh(stream)


def fp_bfaces_sort_iface(bf: BFaces, elem: torch.Tensor, stream=None):
    bf.sort_iface(elem, stream)


def fp_bfaces_iface(bf: BFaces, device=None, out: Optional[torch.Tensor] = None):
    """(Mi, interface node positions [3][Mi])."""
    return bf.Mi, bf.iface_points(device, out)
