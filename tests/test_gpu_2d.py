"""GPU parity of the 2D (quadrilateral) variant against the CPU oracle:
deformed quads at several orders with points inside, outside and within
1e-9 of element edges; the 2D overset workload (box + annulus, session
tags, distance-to-boundary owner rule); three overlapping rectangles with
closed-form delta; the fused find + eval; moving meshes with warm starts;
and the calls that reject 2D handles."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_RST, assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_04891_gb300 as fg
    fg.lib()
    return fg


def _setup(fg, coords, N, sub=None, dist=None, **opt):
    dev = torch.device("cuda:0")
    return fg.fp_setup_2d(torch.from_numpy(np.ascontiguousarray(coords)).to(dev), N,
                          None if sub is None else torch.from_numpy(sub).to(dev),
                          None if dist is None else torch.from_numpy(np.ascontiguousarray(dist)).to(dev),
                          opts=fg.default_opts(**opt))


def _run(fg, h, pts, qsess=None, fields=None):
    dev = torch.device("cuda:0")
    qs = None if qsess is None else torch.from_numpy(np.ascontiguousarray(qsess, dtype=np.int32)).to(dev)
    code, sub, elem, rst, d2 = fg.fp_find(h, torch.from_numpy(np.ascontiguousarray(pts)).to(dev), qs)
    res = {"code": code.cpu().numpy(), "sub": sub.cpu().numpy(), "elem": elem.cpu().numpy(),
           "rst": rst.cpu().numpy(), "dist2": d2.cpu().numpy()}
    if fields is not None:
        res["eval"] = fg.fp_eval(h, code, elem, rst, torch.from_numpy(fields).to(dev)).cpu().numpy()
    return res


@pytest.mark.parametrize("N", [1, 3, 5, 7, 9])
def test_2d_parity_deformed(fg, N):
    coords = synth.quad_mesh((8, 6), N, amp_frac=0.1)
    E = coords.shape[1]
    sub = np.zeros(E, np.int32)
    pts = np.concatenate([synth.uniform_points_2d(6000, seed=N, lo=(-0.05, -0.05), hi=(1.05, 1.05)),
                          synth.edge_points_2d(coords, N, 1500, seed=10 + N),
                          np.array([[np.nan, 0.5], [0.5, np.inf], [1.0, 1.0], [0.0, 0.0]]).T], axis=1)
    fields = np.stack([synth.field_u_2d(coords), coords[0] * coords[1] ** 2])
    h = _setup(fg, coords, N, sub)
    g = _run(fg, h, pts, fields=fields)
    ref = oracle.find(coords, N, sub, pts)
    ref["eval"] = oracle.evaluate(N, ref["code"], ref["elem"], ref["rst"], fields)
    assert_parity(g, ref, 0, fields=fields)
    assert (ref["code"] == oracle.INSIDE).sum() > 6000
    assert (ref["code"] == oracle.NOT_FOUND).sum() > 100


def test_2d_overset_walsh(fg):
    mesh, q = synth.walsh_2d(N=7, n_box=16, ring=(16, 3))
    h = _setup(fg, mesh.coords, mesh.N, mesh.sub, mesh.dist)
    g = _run(fg, h, q.pts, q.qsess, fields=q.fields)
    ref = oracle.find(mesh.coords, mesh.N, mesh.sub, q.pts, qsess=q.qsess, dist=mesh.dist)
    ref["eval"] = oracle.evaluate(mesh.N, ref["code"], ref["elem"], ref["rst"], q.fields)
    assert_parity(g, ref, 0, fields=q.fields)
    assert (g["code"] == 0).all() and (g["sub"] != q.qsess).all()
    # untagged points in the overlap: the owner rule compares D^k; the box's
    # distance to its own boundary (>= pi - 1.4) exceeds the annulus's
    # (<= 0.4) everywhere in the annulus, so the box owns every point
    pts = synth.uniform_points_2d(4000, seed=3, lo=(1.5, 1.5), hi=(4.8, 4.8))
    g = _run(fg, h, pts)
    ref = oracle.find(mesh.coords, mesh.N, mesh.sub, pts, dist=mesh.dist)
    assert_parity(g, ref, 0)
    assert (g["sub"][g["code"] == 0] == 0).all()
    # with the roles reversed (D^box scaled below D^annulus) the annulus owns its region
    d2 = mesh.dist.copy()
    d2[mesh.sub == 0] *= 0.01
    h2 = _setup(fg, mesh.coords, mesh.N, mesh.sub, d2)
    g = _run(fg, h2, pts)
    ref = oracle.find(mesh.coords, mesh.N, mesh.sub, pts, dist=d2)
    assert_parity(g, ref, 0)
    assert len(np.unique(g["sub"][g["code"] == 0])) == 2


@pytest.mark.parametrize("N", [2, 4])
def test_2d_owner_closed_form(fg, N):
    mesh = synth.tiny_overlap_2d(N)
    h = _setup(fg, mesh.coords, N, mesh.sub, mesh.dist)
    pts = synth.uniform_points_2d(3000, seed=N, lo=(-0.1, -0.1), hi=(2.1, 1.1))
    for tag in (-1, 0, 1, 2):
        qs = np.full(pts.shape[1], tag, np.int32)
        g = _run(fg, h, pts, qs)
        ref = oracle.find(mesh.coords, N, mesh.sub, pts, qsess=qs, dist=mesh.dist)
        assert_parity(g, ref, 0)


def test_2d_fused_find_eval_and_edges(fg):
    coords = synth.quad_mesh((5, 5), 6, amp_frac=0.08)
    E = coords.shape[1]
    h = _setup(fg, coords, 6, np.zeros(E, np.int32))
    pts = torch.from_numpy(synth.uniform_points_2d(5000, seed=4, lo=(-0.1, -0.1), hi=(1.1, 1.1))).cuda()
    f = torch.from_numpy(np.stack([synth.field_u_2d(coords)])).cuda()
    fused = fg.fp_find_eval(h, pts, fields=f)
    plain = fg.fp_find(h, pts)
    for a in range(5):
        assert torch.equal(fused[a], plain[a])
    ev = fg.fp_eval(h, plain[0], plain[2], plain[3], f)
    assert torch.equal(torch.isnan(ev), torch.isnan(fused[5]))
    ok = ~torch.isnan(ev)
    assert torch.equal(ev[ok], fused[5][ok])
    empty = fg.fp_find(h, torch.zeros((2, 0), dtype=torch.float64, device="cuda"))
    assert empty[3].shape == (2, 0)


def test_2d_moving_ring_warm(fg):
    mesh, q = synth.walsh_2d(N=5, n_box=12, ring=(12, 2))
    h = _setup(fg, mesh.coords, mesh.N, mesh.sub, mesh.dist)
    dev = torch.device("cuda:0")
    qs = torch.from_numpy(q.qsess).to(dev)
    out = fg.fp_find(h, torch.from_numpy(q.pts).to(dev), qs)
    mv = q.qsess == 1
    for k in range(1, 4):
        ang, sh = 5.0 * k, (0.02 * k, -0.01 * k, 0.0)
        c3 = np.concatenate([mesh.coords, np.zeros_like(mesh.coords[:1])])
        ck = synth.rigid_motion(c3, mesh.sub, 1, ang, sh, (np.pi, np.pi, 0.0))[:2]
        p3 = np.concatenate([q.pts, np.zeros_like(q.pts[:1])])
        pk = p3.copy()
        pk[:, mv] = synth.rigid_motion(p3[:, mv][:, None, :], np.array([1]), 1, ang, sh, (np.pi, np.pi, 0.0))[:, 0]
        pk = np.ascontiguousarray(pk[:2])
        fg.fp_update_coords(h, torch.from_numpy(np.ascontiguousarray(ck)).to(dev))
        hf = _setup(fg, ck, mesh.N, mesh.sub, mesh.dist)
        for x, y in zip(fg.fp_debug_boxes(h), fg.fp_debug_boxes(hf)):
            assert torch.equal(x, y)
        pt = torch.from_numpy(pk).to(dev)
        out = fg.fp_find_warm(h, pt, warm=(out[2], out[3]), qsess=qs, out=out)
        cold = fg.fp_find(h, pt, qs)
        for a in (0, 1, 2):
            assert torch.equal(out[a], cold[a])
        assert (out[3] - cold[3]).abs().max().item() <= TOL_RST[0]
        g = {"code": out[0].cpu().numpy(), "sub": out[1].cpu().numpy(), "elem": out[2].cpu().numpy(),
             "rst": out[3].cpu().numpy(), "dist2": out[4].cpu().numpy()}
        assert_parity(g, oracle.find(ck, mesh.N, mesh.sub, pk, qsess=q.qsess, dist=mesh.dist), 0)


def test_2d_rejections(fg):
    coords = synth.quad_mesh((2, 2), 3)
    E = coords.shape[1]
    dev = torch.device("cuda:0")
    ct = torch.from_numpy(coords).to(dev)
    with pytest.raises(fg.FindptsError):
        fg.fp_setup_2d(ct, 3, opts=fg.default_opts(precision=fg.PREC_MIXED))
    h = fg.fp_setup_2d(ct, 3)
    with pytest.raises(Exception):
        fg.Workspace(h, 100)
    pts = torch.from_numpy(synth.uniform_points_2d(10, 1)).to(dev)
    with pytest.raises(fg.FindptsError):
        fg.fp_find_static(h, pts)
    with pytest.raises(Exception):
        fg.Fields(h, torch.zeros((1, E, 16), dtype=torch.float64, device=dev))


@pytest.mark.parametrize("N", [3, 6])
def test_2d_default_distance_owner(fg, N):
    """No D passed: the library's default field (boundary edges of each
    subdomain) decides the owner exactly as the oracle's default field does."""
    mesh = synth.tiny_overlap_2d(N)                         # three overlapping rectangles
    h = _setup(fg, mesh.coords, N, mesh.sub)                # dist = None
    D = oracle.dist_default(mesh.coords, N, mesh.sub)
    pts = synth.uniform_points_2d(4000, seed=N, lo=(0.0, 0.0), hi=(2.0, 1.0))
    g = _run(fg, h, pts)
    ref = oracle.find(mesh.coords, N, mesh.sub, pts, dist=D)
    assert_parity(g, ref, 0)
    assert len(np.unique(g["sub"][g["code"] == 0])) == 3
    mesh, q = synth.walsh_2d(N=N, n_box=10, ring=(12, 2))
    h = _setup(fg, mesh.coords, N, mesh.sub)
    g = _run(fg, h, q.pts, q.qsess)
    ref = oracle.find(mesh.coords, N, mesh.sub, q.pts, qsess=q.qsess, dist=oracle.dist_default(mesh.coords, N, mesh.sub))
    assert_parity(g, ref, 0)
