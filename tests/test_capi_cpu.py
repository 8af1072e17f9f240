"""CPU-side checks of the boundary: the shared library builds, loads without a
GPU and exports every entry point that include/findpts_gb.h declares; the
Python binding rejects bad arguments before any device work."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "findpts_gb.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fp_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("fp_setup", "fp_find", "fp_eval", "fp_free", "fp_error_string", "fp_reserve"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_1811_04891_gb300 as fg
    L = fg.lib()
    for n in declared_functions():
        assert hasattr(L, n), n


def test_host_only_entry_points_without_gpu():
    import paper_1811_04891_gb300 as fg
    L = fg.lib()
    assert L.fp_error_string(fg.FP_ERR_INVALID_ARG) == b"invalid argument"
    o = fg.default_opts()
    assert o.tol_accept == 1e-12 and o.tol_border == 1e-6 and o.precision == fg.PREC_FP64
    assert L.fp_find(None, 1, None, None, None, None, None, None, None, None) == fg.FP_ERR_NOT_SETUP
    assert L.fp_eval(None, 1, None, None, None, 1, None, None, None) == fg.FP_ERR_NOT_SETUP


def test_binding_rejects_cpu_tensors():
    import torch

    import paper_1811_04891_gb300 as fg
    with pytest.raises(TypeError):
        fg.fp_setup(torch.zeros((3, 1, 8), dtype=torch.float64), 1)


def test_binding_has_every_entry_point_by_name():
    """The Python binding exposes each C entry point under its own name."""
    import paper_1811_04891_gb300 as fg
    missing = [n for n in declared_functions() if not callable(getattr(fg, n, None))]
    assert not missing, missing
    assert fg.fp_error_string(fg.FP_ERR_NOT_SETUP) == fg.lib().fp_error_string(fg.FP_ERR_NOT_SETUP).decode()
    assert fg.fp_default_opts(precision=fg.PREC_MIXED).precision == fg.PREC_MIXED


def test_argument_checks_before_any_device_work():
    """Bad arguments and missing handles are refused on the host, with the
    status the header documents, before the library touches a device."""
    import ctypes

    import paper_1811_04891_gb300 as fg
    L = fg.lib()
    o = fg.default_opts()
    h = ctypes.c_void_p()
    out = ctypes.c_void_p()
    INV, NOSET = fg.FP_ERR_INVALID_ARG, fg.FP_ERR_NOT_SETUP
    assert L.fp_setup(ctypes.byref(h), None, 8, 0, None, None, ctypes.byref(o), None) == INV      # N < 1
    assert L.fp_setup(ctypes.byref(h), None, 8, 16, None, None, ctypes.byref(o), None) == INV     # N > 15
    assert L.fp_setup(ctypes.byref(h), None, 0, 3, None, None, ctypes.byref(o), None) == INV      # E < 1
    assert L.fp_setup(ctypes.byref(h), None, 8, 3, None, None, ctypes.byref(o), None) == INV      # no coords
    assert L.fp_setup(None, None, 8, 3, None, None, ctypes.byref(o), None) == INV
    assert L.fp_last_error(None) == b"fp_setup: null handle pointer"
    assert L.fp_workspace_create(None, 10, 0, ctypes.byref(out)) == NOSET
    assert L.fp_points_create(None, 10, ctypes.byref(out)) == NOSET
    assert L.fp_bfaces_create(None, None, ctypes.byref(out), None) == NOSET
    assert L.fp_find_static(None, 1, None, None, None, None, None, None, None, None) == NOSET
    assert L.fp_update_coords(None, None, None, 0, None) == NOSET
    assert L.fp_find_eval_host(None, 1, None, None, 0, None, None, None, None, None, None, None, None, 0, 0,
                               None) == NOSET
    assert L.fp_extrapolate(0, 10, None, None, None) == INV                                       # m outside 1..3
    assert L.fp_batch_create(ctypes.byref(out), 0, None, None, 0, None, 2.0) == INV               # no instances
    assert L.fp_batch_schedule(None, 0, None, None, None) == INV
    assert L.fp_batch_groups(None, None) == INV
    assert L.fp_batch_mode(None, None) == INV
    assert L.fp_batch_profile(None, 1) == INV
    assert L.fp_bfaces_info(None, None, None) == INV
    cnt = (ctypes.c_int64 * 3)()
    assert L.fp_band_hits(None, cnt) == NOSET
    assert L.fp_set_mixed_refine(None, 3) == NOSET
    assert L.fp_set_eval_staging(None, 1) == NOSET
    assert L.fp_fma_probe(5, 10, 1, None, None, None) == INV                                      # kind outside 0..4
    assert L.fp_fma_probe(0, 0, 1, None, None, None) == INV                                       # iters < 1
