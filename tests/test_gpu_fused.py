"""GPU tests of the fused find + eval (fp_find_eval, fp_find_eval_ws): the
values must equal a separate fp_find followed by fp_eval (FP64 fields) or
fp_eval_df (posted double-float fields), bit for bit, with NaN where a point
is not found."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_04891_gb300 as fg
    fg.lib()
    return fg


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("posted", [False, True])
def test_fused_equals_separate(fg, prec, posted):
    mesh, q = synth.deformed_cube(ne=6, P_uniform=25000, P_face=2500)
    dev = torch.device("cuda:0")
    h = fg.fp_setup(torch.from_numpy(mesh.coords).to(dev), mesh.N, torch.from_numpy(mesh.sub).to(dev),
                    opts=fg.default_opts(precision=prec))
    # include points outside the mesh
    pts = np.concatenate([q.pts, synth.uniform_points(3000, 5, lo=(-0.5,) * 3, hi=(1.5,) * 3)], axis=1)
    t = torch.from_numpy(pts).to(dev)
    fields = torch.from_numpy(q.fields).to(dev)
    pf = fg.Fields(h, fields) if posted else None
    r = fg.fp_find(h, t)
    sep = (fg.fp_eval_df(h, pf, r[0], r[2], r[3]) if posted else fg.fp_eval(h, r[0], r[2], r[3], fields))
    fused = fg.fp_find_eval(h, t, fields=fields, posted=pf)
    ws = fg.Workspace(h, t.shape[1])
    fused_ws = fg.fp_find_eval_ws(h, ws, t, fields=fields, posted=pf)
    torch.cuda.synchronize()
    for a, b, c in zip(r, fused[:5], fused_ws[:5]):
        assert torch.equal(a, b) and torch.equal(a, c)
    sv, fv, wv = sep.cpu().numpy(), fused[5].cpu().numpy(), fused_ws[5].cpu().numpy()
    np.testing.assert_array_equal(sv, fv)
    np.testing.assert_array_equal(sv, wv)
    nf = r[0].cpu().numpy() == fg.NOT_FOUND
    assert nf.any() and np.isnan(fv[:, nf]).all() and np.isfinite(fv[:, ~nf]).all()


@pytest.mark.parametrize("N", [3, 7])
def test_staged_eval_equals_unstaged(fg, N):
    """Posted fields evaluated from shared memory (fp_set_eval_staging) give
    the values of the unstaged fused eval and of fp_eval_df, bit for bit:
    odd and even n, tiles spanning several elements, losers and points
    outside the mesh inside tiles."""
    mesh, q = synth.deformed_cube(ne=5, N=N, P_uniform=20000, P_face=2000)
    dev = torch.device("cuda:0")
    h = fg.fp_setup(torch.from_numpy(mesh.coords).to(dev), mesh.N, torch.from_numpy(mesh.sub).to(dev),
                    opts=fg.default_opts(precision=fg.PREC_MIXED))
    pts = np.concatenate([q.pts, synth.uniform_points(2000, 6, lo=(-0.5,) * 3, hi=(1.5,) * 3)], axis=1)
    t = torch.from_numpy(pts).to(dev)
    pf = fg.Fields(h, torch.from_numpy(q.fields).to(dev))
    plain = fg.fp_find_eval(h, t, posted=pf)
    fg.fp_set_eval_staging(h, True)
    staged = fg.fp_find_eval(h, t, posted=pf)
    ws = fg.Workspace(h, t.shape[1])
    staged_ws = fg.fp_find_eval_ws(h, ws, t, posted=pf)
    sep = fg.fp_eval_df(h, pf, plain[0], plain[2], plain[3])
    torch.cuda.synchronize()
    for a, b in zip(plain[:5], staged[:5]):
        assert torch.equal(a, b)
    pv, sv, wv, ev = (x.cpu().numpy() for x in (plain[5], staged[5], staged_ws[5], sep))
    np.testing.assert_array_equal(pv, sv)
    np.testing.assert_array_equal(pv, wv)
    np.testing.assert_array_equal(pv, ev)
    assert np.isfinite(sv).any()
