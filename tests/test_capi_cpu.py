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
