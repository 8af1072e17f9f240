"""GPU tests of the moving-mesh path: fp_update_coords must leave the handle
exactly as a fresh fp_setup on the new coordinates would, and fp_find_warm
over a sequence of mesh positions must agree with the oracle and with a
cold find, whatever the warm hints hold."""
import numpy as np
import pytest
import torch

import synth
from gpu_util import TOL_RST, assert_parity, oracle_find

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_04891_gb300 as fg
    fg.lib()
    return fg


def _setup(fg, coords, N, sub, prec, dist=None):
    dev = torch.device("cuda:0")
    return fg.fp_setup(torch.from_numpy(np.ascontiguousarray(coords)).to(dev), N, torch.from_numpy(sub).to(dev),
                       None if dist is None else torch.from_numpy(dist).to(dev),
                       opts=fg.default_opts(precision=prec))


def _same(a, b):
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("prec", [0, 1])
def test_update_equals_fresh_setup(fg, prec):
    N = 5
    shape = (4, 3, 3)
    c0 = synth.box_mesh(shape, N, amp_frac=0.05)
    sub = np.zeros(c0.shape[1], np.int32)
    pts = torch.from_numpy(synth.uniform_points(5000, seed=5, lo=(-0.1, -0.1, -0.1), hi=(1.7, 1.1, 1.1))).cuda()
    h = _setup(fg, c0, N, sub, prec)
    seq = [synth.box_mesh(shape, N, amp_frac=0.12),                                      # deformation
           synth.rigid_motion(c0, sub, 0, 7.0, (0.05, -0.02, 0.01), (0.5, 0.5, 0.0)),    # rigid motion
           synth.box_mesh(shape, N, hi=(1.6, 1.0, 1.0), amp_frac=0.1)]                   # larger box
    for k, c in enumerate(seq):
        ct = torch.from_numpy(c)
        fg.fp_update_coords(h, ct.cuda() if k % 2 == 0 else ct)        # device and host sources
        hf = _setup(fg, c, N, sub, prec)
        assert h.info() == hf.info()
        _same(fg.fp_debug_boxes(h), fg.fp_debug_boxes(hf))
        _same(fg.fp_find(h, pts), fg.fp_find(hf, pts))
    torch.cuda.synchronize()


def test_update_rejects_nonfinite_and_keeps_mesh(fg):
    N = 4
    c0 = synth.box_mesh((3, 3, 3), N, amp_frac=0.05)
    sub = np.zeros(c0.shape[1], np.int32)
    h = _setup(fg, c0, N, sub, 0)
    pts = torch.from_numpy(synth.uniform_points(2000, seed=6)).cuda()
    before = [x.clone() for x in fg.fp_find(h, pts)]
    bad = c0.copy()
    bad[1, 5, 7] = np.nan
    for src in (torch.from_numpy(bad).cuda(), torch.from_numpy(bad)):
        with pytest.raises(fg.FindptsError) as ei:
            fg.fp_update_coords(h, src)
        assert ei.value.status == fg.FP_ERR_INVALID_ARG
    _same(before, fg.fp_find(h, pts))
    with pytest.raises(ValueError):
        fg.fp_update_coords(h, torch.from_numpy(c0[:, :-1]).cuda())


@pytest.mark.parametrize("prec", [0, 1])
def test_warm_find_moving_cylinder(fg, prec):
    """The annulus of the box+annulus overlap turns and drifts; its boundary
    nodes move with it, the box's stay.  Each step: update, then a warm find
    in place from the previous step's (e, r); parity with the oracle on the
    moved mesh and with a cold find on the same handle."""
    mesh, q = synth.box_annulus(n_az=16, n_rad=2, n_ax=4, box_shape=(8, 4, 4), N=5)
    h = _setup(fg, mesh.coords, mesh.N, mesh.sub, prec, mesh.dist)
    dev = torch.device("cuda:0")
    qs = torch.from_numpy(q.qsess).to(dev)
    ptsn = q.pts
    out = fg.fp_find(h, torch.from_numpy(ptsn).to(dev), qs)
    moving_pts = q.qsess == 1
    center = synth.meshes.BOX_ANNULUS_CYL["center"]
    for k in range(1, 4):
        ang, sh = 4.0 * k, (0.01 * k, 0.005 * k, 0.0)
        ck = synth.rigid_motion(mesh.coords, mesh.sub, 1, ang, sh, center)
        pk = ptsn.copy()
        # the annulus's own boundary nodes move with it
        pk[:, moving_pts] = synth.rigid_motion(ptsn[:, moving_pts][:, None, :], np.array([1]), 1, ang, sh,
                                               center)[:, 0, :]
        fg.fp_update_coords(h, torch.from_numpy(ck).to(dev))
        pt = torch.from_numpy(np.ascontiguousarray(pk)).to(dev)
        out = fg.fp_find_warm(h, pt, warm=(out[2], out[3]), qsess=qs, out=out)
        cold = fg.fp_find(h, pt, qs)
        torch.cuda.synchronize()
        g = {"code": out[0].cpu().numpy(), "sub": out[1].cpu().numpy(), "elem": out[2].cpu().numpy(),
             "rst": out[3].cpu().numpy(), "dist2": out[4].cpu().numpy()}
        moved = synth.Mesh(coords=ck, N=mesh.N, sub=mesh.sub, dist=mesh.dist)
        ref = oracle_find(moved, pk, q.qsess)
        assert_parity(g, ref, prec)
        for a in (0, 1, 2):
            assert torch.equal(out[a], cold[a])
        assert (out[3] - cold[3]).abs().max().item() <= TOL_RST[prec]
        assert (ref["code"] == 0).mean() > 0.5


@pytest.mark.parametrize("prec", [0, 1])
def test_warm_hints_do_not_change_results(fg, prec):
    """Wrong, out-of-range and non-finite hints only change where Newton
    starts: codes, subdomains and elements stay those of the cold find."""
    mesh, q = synth.cube4_small()
    h = _setup(fg, mesh.coords, mesh.N, mesh.sub, prec)
    pts = torch.from_numpy(np.concatenate([q.pts[:, :4000],
                                           synth.near_face_points(mesh.coords, mesh.N, 1000, seed=3)], 1)).cuda()
    P = pts.shape[1]
    cold = fg.fp_find(h, pts)
    rng = np.random.default_rng(7)
    we = torch.from_numpy(rng.integers(-1, mesh.E, P).astype(np.int32)).cuda()
    we[::3] = cold[2][::3]                                    # a third with the right element
    wr = torch.from_numpy(rng.uniform(-3, 3, (3, P))).cuda()
    wr[0, ::7] = float("nan")
    wr[1, ::11] = float("inf")
    warm = fg.fp_find_warm(h, pts, warm=(we, wr))
    for a in (0, 1, 2):
        assert torch.equal(warm[a], cold[a])
    assert (warm[3] - cold[3]).abs().max().item() <= TOL_RST[prec]
    # warm from the exact answer, in place, with the fused eval
    f = torch.from_numpy(q.fields).cuda()
    out = [x.clone() for x in cold]
    r = fg.fp_find_warm(h, pts, warm=(out[2], out[3]), fields=f, out=out)
    ref_v = fg.fp_eval(h, cold[0], cold[2], cold[3], f)
    for a in (0, 1, 2):
        assert torch.equal(r[a], cold[a])
    scale = f.abs().max().item()
    ok = ~torch.isnan(ref_v)
    assert torch.equal(ok, ~torch.isnan(r[5]))
    assert ((r[5] - ref_v)[ok].abs().max().item()) <= 1e-11 * scale
    st = fg.lib().fp_find_warm(h.ptr, P, fg._ptr(pts), None, fg._ptr(we), None, 0, None, None,
                               *[fg._ptr(x) for x in cold], None, None)
    assert st == fg.FP_ERR_INVALID_ARG


def test_interface_exchange_on_moving_annulus(fg):
    """Sub-iterations captured once keep replaying correctly after the
    annulus moves: move() refreshes the face geometry and relocates the
    interface points in the buffers the graph reads."""
    from paper_1811_04891_gb300.schwarz import InterfaceExchange
    n_az, n_rad, n_ax, box = 16, 2, 4, (8, 4, 4)
    mesh, q = synth.box_annulus(n_az=n_az, n_rad=n_rad, n_ax=n_ax, box_shape=box, N=5)
    nb = box[0] * box[1] * box[2]
    kind = np.zeros((mesh.E, 6), np.int8)
    for e in range(nb, mesh.E):
        el = e - nb
        er, ez = el % n_rad, el // (n_rad * n_az)
        kind[e, 0] = 2 if er == 0 else 0
        kind[e, 1] = 2 if er == n_rad - 1 else 0
        kind[e, 4] = 1 if ez == 0 else 0
        kind[e, 5] = 1 if ez == n_ax - 1 else 0
    dev = torch.device("cuda:0")
    hs, xs = [], []
    for graph in (True, False):
        h = _setup(fg, mesh.coords, mesh.N, mesh.sub, 1, mesh.dist)
        bf = fg.BFaces(h, torch.from_numpy(kind).to(dev))
        x = InterfaceExchange(h, bf, 1, torch.from_numpy(q.fields[:3]).to(dev).clone(), order=2)
        hs.append(h)
        xs.append(x)
    xg, xe = xs
    center = synth.meshes.BOX_ANNULUS_CYL["center"]
    for k in range(4):
        if k:
            ck = torch.from_numpy(synth.rigid_motion(mesh.coords, mesh.sub, 1, 3.0 * k, (0.01 * k, 0.0, 0.0),
                                                     center)).to(dev)
            xg.move(ck)
            xe.move(ck)
        ug = xg.step(kappa=2).clone()
        xe.predict()
        for _ in range(2):
            xe._correct_eager()
        xe.commit()
        torch.cuda.synchronize()
        assert torch.equal(ug, xe.u)
        # the relocated interface points equal a cold find on the moved mesh
        cold = fg.fp_find(hs[0], xg.pts, xg.qs)
        for a in (0, 1, 2):
            assert torch.equal(xg.found[a], cold[a])
        assert (xg.found[0] == 0).all()
        x_, nr, dA, nk = xg.bf.nodes()
        assert abs(((ug * nr).sum(0) * dA).sum().item()) < 1e-10
