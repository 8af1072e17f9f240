"""GPU tests of the asynchronous find (fp_find_ws): identical results to
fp_find, capacity overflow reported per point, replay from a captured CUDA
graph, and two workspaces running concurrently on two streams."""
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


def _setup(fg, mesh, prec):
    dev = torch.device("cuda:0")
    d = None if mesh.dist is None else torch.from_numpy(mesh.dist).to(dev)
    return fg.fp_setup(torch.from_numpy(mesh.coords).to(dev), mesh.N, torch.from_numpy(mesh.sub).to(dev), d,
                       opts=fg.default_opts(precision=prec))


def _np(t):
    return [x.cpu().numpy() for x in t]


@pytest.mark.parametrize("prec", [0, 1])
def test_ws_matches_fp_find(fg, prec):
    mesh, q = synth.deformed_cube(ne=8, P_uniform=40000, P_face=4000, with_fields=False)
    h = _setup(fg, mesh, prec)
    pts = torch.from_numpy(q.pts).cuda()
    ref = _np(fg.fp_find(h, pts))
    ws = fg.Workspace(h, q.P)
    got = _np(fg.fp_find_ws(h, ws, pts))
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)
    assert ws.last_pairs() == fg.fp_last_find_stats(h)


@pytest.mark.parametrize("prec", [0, 1])
def test_ws_multisubdomain(fg, prec):
    mesh, q = synth.box_annulus()
    h = _setup(fg, mesh, prec)
    pts = torch.from_numpy(q.pts).cuda()
    qs = torch.from_numpy(q.qsess).cuda()
    ref = _np(fg.fp_find(h, pts, qs))
    ws = fg.Workspace(h, q.P)
    got = _np(fg.fp_find_ws(h, ws, pts, qs))
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)


def test_ws_overflow_marks_retry(fg):
    mesh, q = synth.deformed_cube(ne=6, P_uniform=20000, P_face=0, with_fields=False)
    h = _setup(fg, mesh, 1)
    pts = torch.from_numpy(q.pts).cuda()
    ref = _np(fg.fp_find(h, pts))
    ws = fg.Workspace(h, q.P, max_pairs=q.P // 2)
    code, sub, elem, rst, d2 = _np(fg.fp_find_ws(h, ws, pts))
    retry = code == fg.RETRY
    assert retry.any() and (~retry).any()
    assert ws.last_pairs() > q.P // 2
    # every point that was searched is complete and identical
    for a, b in zip(ref, (code, sub, elem, rst, d2)):
        np.testing.assert_array_equal(a[..., ~retry], b[..., ~retry])
    assert np.all(elem[retry] == -1) and np.all(np.isinf(d2[retry]))
    # the retried points are a suffix of the point order
    first = np.argmax(retry)
    assert retry[first:].all()


def test_graph_capture_and_replay(fg):
    mesh, q = synth.deformed_cube(ne=6, P_uniform=30000, P_face=1000)
    h = _setup(fg, mesh, 1)
    dev = torch.device("cuda:0")
    P = q.P
    fields = torch.from_numpy(q.fields).to(dev)
    pts_static = torch.from_numpy(q.pts).to(dev)
    outs = (torch.empty(P, dtype=torch.int32, device=dev), torch.empty(P, dtype=torch.int32, device=dev),
            torch.empty(P, dtype=torch.int32, device=dev), torch.empty((3, P), dtype=torch.float64, device=dev),
            torch.empty(P, dtype=torch.float64, device=dev))
    val = torch.empty((fields.shape[0], P), dtype=torch.float64, device=dev)
    ws = fg.Workspace(h, P)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):                       # warm-up outside capture
        fg.fp_find_ws(h, ws, pts_static, out=outs)
        fg.fp_eval(h, outs[0], outs[2], outs[3], fields, out=val)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fg.fp_find_ws(h, ws, pts_static, out=outs)
        fg.fp_eval(h, outs[0], outs[2], outs[3], fields, out=val)
    for seed in (5, 6):
        new_pts = torch.from_numpy(synth.uniform_points(P, seed=seed)).to(dev)
        pts_static.copy_(new_pts)
        g.replay()
        torch.cuda.synchronize()
        ref = _np(fg.fp_find(h, new_pts))
        refv = fg.fp_eval(h, *[torch.from_numpy(x).to(dev) for x in (ref[0], ref[2], ref[3])], fields)
        for a, b in zip(ref, _np(outs)):
            np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(refv.cpu().numpy(), val.cpu().numpy())


def test_two_workspaces_two_streams(fg):
    mesh, q = synth.deformed_cube(ne=6, P_uniform=30000, P_face=2000, with_fields=False)
    h = _setup(fg, mesh, 1)
    dev = torch.device("cuda:0")
    a = torch.from_numpy(q.pts[:, :16000].copy()).to(dev)
    b = torch.from_numpy(q.pts[:, 16000:].copy()).to(dev)
    wa, wb = fg.Workspace(h, a.shape[1]), fg.Workspace(h, b.shape[1])
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(3):
        with torch.cuda.stream(sa):
            ra = fg.fp_find_ws(h, wa, a, stream=sa)
        with torch.cuda.stream(sb):
            rb = fg.fp_find_ws(h, wb, b, stream=sb)
    torch.cuda.synchronize()
    ref = _np(fg.fp_find(h, torch.from_numpy(q.pts).to(dev)))
    for r_all, x, y in zip(ref, _np(ra), _np(rb)):
        np.testing.assert_array_equal(r_all, np.concatenate([x, y], axis=-1))
