"""GPU tests of the interface-data pipeline over Schwarz steps: temporal
extrapolation against the oracle, the split-input flux correction against
the plain one, and the graph-replayed sub-iteration loop against eager
calls."""
import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_flux import _gpu_faces
from test_oracle_flux import box_kind

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_04891_gb300 as fg
    fg.lib()
    return fg


@pytest.mark.parametrize("m", [1, 2, 3])
def test_extrapolate_parity(fg, m):
    rng = np.random.default_rng(10 + m)
    hist = [rng.uniform(-1, 1, (3, 1001)) for _ in range(m)]
    out = fg.fp_extrapolate([torch.from_numpy(h).cuda() for h in hist]).cpu().numpy()
    np.testing.assert_allclose(out, oracle.extrapolate(hist), atol=1e-14 * 2 ** m)


def test_flux_correct_iface_equals_scattered(fg):
    N = 4
    shp = (2, 2, 2)
    coords = synth.box_mesh(shp, N, amp_frac=0.15)
    kind = box_kind(shp, {(0, 0): 2, (0, 1): 2, (1, 0): 1, (1, 1): 2, (2, 0): 1, (2, 1): 1})
    h, bf = _gpu_faces(fg, coords, N, kind)
    x, nr, dA, nk = bf.nodes()
    ip = bf.iface_points()
    np.testing.assert_array_equal(ip.cpu().numpy(), x[:, nk == 2].cpu().numpy())
    rng = np.random.default_rng(0)
    ui = torch.from_numpy(rng.uniform(-1, 1, (3, bf.Mi))).cuda()
    up = torch.from_numpy(rng.uniform(-1, 1, (3, bf.M))).cuda()
    u = up.clone()
    u[:, nk == 2] = ui
    a = fg.fp_flux_correct(bf, u)
    b = fg.fp_flux_correct_iface(bf, ui, up)
    for p, q in zip(a, b):
        assert torch.equal(p, q)


def test_graph_replayed_subiterations_match_eager(fg):
    from paper_1811_04891_gb300.schwarz import InterfaceExchange
    mesh, q = synth.box_annulus()
    n_rad, n_az, n_ax = 4, 32, 8
    kind = np.zeros((mesh.E, 6), np.int8)
    for e in range(1024, mesh.E):
        el = e - 1024
        er, ez = el % n_rad, el // (n_rad * n_az)
        kind[e, 0] = 2 if er == 0 else 0
        kind[e, 1] = 2 if er == n_rad - 1 else 0
        kind[e, 4] = 1 if ez == 0 else 0
        kind[e, 5] = 1 if ez == n_ax - 1 else 0
    dev = torch.device("cuda:0")
    h = fg.fp_setup(torch.from_numpy(mesh.coords).to(dev), mesh.N, torch.from_numpy(mesh.sub).to(dev),
                    torch.from_numpy(mesh.dist).to(dev), opts=fg.default_opts(precision=fg.PREC_MIXED))
    base = torch.from_numpy(q.fields[:3]).to(dev)
    fields_g = base.clone()
    fields_e = base.clone()
    # each exchange renumbers the interface nodes of its own face set
    xg = InterfaceExchange(h, fg.BFaces(h, torch.from_numpy(kind).to(dev)), 1, fields_g, order=2)
    xe = InterfaceExchange(h, fg.BFaces(h, torch.from_numpy(kind).to(dev)), 1, fields_e, order=2)
    bf = xg.bf
    for step in range(3):
        # the donors' solution changes between steps (a stand-in for the solver)
        fields_g.copy_(base * (1.0 + 0.1 * step))
        fields_e.copy_(base * (1.0 + 0.1 * step))
        ug = xg.step(kappa=3).clone()
        # eager reference: the same operations without the graph
        xe.predict()
        for _ in range(3):
            xe._correct_eager()
        xe.commit()
        torch.cuda.synchronize()
        assert torch.equal(ug, xe.u)
        # the corrected flux vanishes
        x, nr, dA, nk = bf.nodes()
        assert abs(((ug * nr).sum(0) * dA).sum().item()) < 1e-10


def test_sort_iface_renumbers_without_changing_results(fg):
    N = 4
    shp = (3, 3, 2)
    coords = synth.box_mesh(shp, N, amp_frac=0.1)
    kind = box_kind(shp, {(0, 0): 2, (0, 1): 2, (1, 0): 2, (1, 1): 1, (2, 0): 1, (2, 1): 2})
    h, bf = _gpu_faces(fg, coords, N, kind)
    pts0 = bf.iface_points()
    found0 = fg.fp_find(h, pts0)
    f = torch.from_numpy(np.stack([synth.field_u(coords), coords[0] * coords[1], coords[2] ** 2])).cuda()
    up = torch.from_numpy(np.random.default_rng(2).uniform(-1, 1, (3, bf.M))).cuda()
    u0 = fg.fp_eval(h, found0[0], found0[2], found0[3], f)
    a = fg.fp_flux_correct_iface(bf, u0, up)
    bf.sort_iface(found0[2])
    pts1 = bf.iface_points()
    found1 = fg.fp_find(h, pts1)
    e1 = found1[2].cpu().numpy()
    assert (np.diff(e1) >= 0).all()                                  # grouped by donor element
    key0 = np.lexsort(pts0.cpu().numpy())
    key1 = np.lexsort(pts1.cpu().numpy())
    assert torch.equal(pts0[:, key0], pts1[:, key1])                 # the same points, reordered
    u1 = fg.fp_eval(h, found1[0], found1[2], found1[3], f)
    b = fg.fp_flux_correct_iface(bf, u1, up)
    for p, q in zip(a, b):
        assert torch.equal(p, q)


def test_posted_points_equal_eval_df(fg):
    """Posted points (cached basis values) evaluate posted fields exactly as
    fp_eval_df does at the same located points, including NaN for points
    not found; updating them in place tracks a new find."""
    mesh, q = synth.cube4_small()
    dev = torch.device("cuda:0")
    h = fg.fp_setup(torch.from_numpy(mesh.coords).to(dev), mesh.N, torch.from_numpy(mesh.sub).to(dev),
                    opts=fg.default_opts(precision=fg.PREC_MIXED))
    f = fg.Fields(h, torch.from_numpy(np.stack([q.fields[0], q.fields[0] ** 2])).to(dev))
    pts = np.concatenate([q.pts[:, :3000], np.array([[1.5, 0.5, 0.5]]).T], axis=1)
    r = fg.fp_find(h, torch.from_numpy(pts).to(dev))
    pp = fg.Points(h, pts.shape[1])
    for k in range(2):
        pp.set(r[0], r[2], r[3])
        a = pp.eval(f)
        b = fg.fp_eval_df(h, f, r[0], r[2], r[3])
        torch.testing.assert_close(a, b, rtol=0, atol=0, equal_nan=True)
        assert torch.isnan(a[:, r[0] == fg.NOT_FOUND]).all() and (r[0] == fg.NOT_FOUND).sum() == 1
        r = fg.fp_find(h, torch.from_numpy(np.ascontiguousarray(pts[:, ::-1])).to(dev))
