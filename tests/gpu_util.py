"""Helpers shared by the GPU parity tests: run the CUDA path through the
Python binding of the C ABI and compare it with the CPU oracle."""
import numpy as np
import torch

import oracle

TOL_RST = {0: 1e-12, 1: 1e-10}       # FP64 form / mixed form (|delta r| bound)
TOL_EVAL_REL = 1e-12                 # eval, relative to the field's max |nodal value|


def gpu_find(mesh, pts, qsess=None, prec=0, dist="mesh", fields=None, refine=None, paths=False, **opt):
    """refine: fp_set_mixed_refine before the find; paths: return the mixed
    form's Newton path counts (fp_newton_paths) under "paths"."""
    import paper_1811_04891_gb300 as fg
    dev = torch.device("cuda:0")
    d = mesh.dist if isinstance(dist, str) and dist == "mesh" else dist
    h = fg.fp_setup(torch.from_numpy(np.ascontiguousarray(mesh.coords)).to(dev), mesh.N,
                    torch.from_numpy(mesh.sub).to(dev),
                    None if d is None else torch.from_numpy(np.ascontiguousarray(d)).to(dev),
                    opts=fg.default_opts(precision=prec, **opt))
    if refine is not None:
        fg.fp_set_mixed_refine(h, refine)
    if paths:
        fg.fp_profile(h, True)
    qs = None if qsess is None else torch.from_numpy(np.ascontiguousarray(qsess, dtype=np.int32)).to(dev)
    code, sub, elem, rst, d2 = fg.fp_find(h, torch.from_numpy(np.ascontiguousarray(pts)).to(dev), qs)
    out = None
    if fields is not None:
        out = fg.fp_eval(h, code, elem, rst, torch.from_numpy(np.ascontiguousarray(fields)).to(dev))
    torch.cuda.synchronize()
    res = {"code": code.cpu().numpy(), "sub": sub.cpu().numpy(), "elem": elem.cpu().numpy(),
           "rst": rst.cpu().numpy(), "dist2": d2.cpu().numpy(), "handle": h, "band": fg.fp_band_hits(h)}
    if out is not None:
        res["eval"] = out.cpu().numpy()
    if paths:
        res["paths"] = fg.fp_newton_paths(h)
    return res


def oracle_find(mesh, pts, qsess=None, dist="mesh", fields=None, **kw):
    d = mesh.dist if isinstance(dist, str) and dist == "mesh" else dist
    ref = oracle.find(mesh.coords, mesh.N, mesh.sub, pts, qsess=qsess, dist=d, **kw)
    if fields is not None:
        ref["eval"] = oracle.evaluate(mesh.N, ref["code"], ref["elem"], ref["rst"], fields)
    return ref


NO_BAND = {"accept": 0, "border": 0, "owner": 0}


def assert_parity(g, r, prec=0, fields=None, he=None, band=None):
    """Element-by-element parity of a GPU result with the oracle's.  `band`,
    when given, is the expected near-tie count per kind (fp_band_hits)."""
    if band is not None:
        assert g["band"] == band, g["band"]
    np.testing.assert_array_equal(g["code"], r["code"])
    np.testing.assert_array_equal(g["elem"], r["elem"])
    np.testing.assert_array_equal(g["sub"], r["sub"])
    found = r["code"] != oracle.NOT_FOUND
    drst = np.abs(g["rst"][:, found] - r["rst"][:, found]).max() if found.any() else 0.0
    assert drst <= TOL_RST[prec], f"max |delta r| = {drst:.3e}"
    assert np.all(g["rst"][:, ~found] == 0.0)
    assert np.all(np.isinf(g["dist2"][~found]))
    border = r["code"] == oracle.BORDER
    if border.any():
        dd = np.abs(np.sqrt(g["dist2"][border]) - np.sqrt(r["dist2"][border]))
        assert dd.max() <= 1e-12, dd.max()
    if fields is not None:
        scale = np.abs(fields).reshape(fields.shape[0] if fields.ndim == 3 else 1, -1).max(axis=1)
        ge, re_ = g["eval"], r["eval"]
        assert np.array_equal(np.isnan(ge), np.isnan(re_))
        ok = ~np.isnan(re_)
        err = np.where(ok, np.abs(ge - re_), 0.0) / scale[:, None]
        assert err.max() <= TOL_EVAL_REL, f"eval rel err {err.max():.3e}"
    return drst
