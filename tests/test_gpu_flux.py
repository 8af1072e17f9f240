"""GPU parity of the mass-flux correction (Sec. 2.2, Eqs. consv1, corr,
consv2) against the oracle: face quadrature, gamma and the corrected data,
and the whole interface update of the box + annulus overlap (interpolate the
cylinder's interface velocity from the box, keep prescribed data on its end
walls, correct the flux)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from test_oracle_flux import box_kind

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_04891_gb300 as fg
    fg.lib()
    return fg


def _gpu_faces(fg, coords, N, kind, sub=None):
    dev = torch.device("cuda:0")
    E = coords.shape[1]
    h = fg.fp_setup(torch.from_numpy(coords).to(dev), N,
                    torch.from_numpy(np.zeros(E, np.int32) if sub is None else sub).to(dev))
    bf = fg.BFaces(h, torch.from_numpy(np.ascontiguousarray(kind, dtype=np.int8)).to(dev))
    return h, bf


@pytest.mark.parametrize("N", [1, 3, 7])
def test_face_quadrature_and_correction_parity(fg, N):
    shp = (3, 2, 2)
    coords = synth.box_mesh(shp, N, lo=(0, 0, 0), hi=(1.5, 1, 1), amp_frac=0.2)
    coords[0] += 0.03 * np.sin(3 * coords[1]) * np.sin(2 * coords[2])   # curve the outer faces too
    marks = {(0, 0): 2, (0, 1): 2, (1, 0): 1, (1, 1): 2, (2, 0): 1, (2, 1): 2}
    kind = box_kind(shp, marks)
    h, bf = _gpu_faces(fg, coords, N, kind)
    x, nr, dA, nk = [t.cpu().numpy() for t in bf.nodes()]
    rx, rn, rdA, rk = oracle.bfaces(coords, N, kind)
    np.testing.assert_array_equal(x, rx)
    np.testing.assert_array_equal(nk, rk)
    np.testing.assert_allclose(nr, rn, atol=1e-13)
    np.testing.assert_allclose(dA, rdA, rtol=1e-13, atol=0)
    rng = np.random.default_rng(N)
    u = rng.uniform(-1, 1, (3, x.shape[1]))
    uo, g, fl = fg.fp_flux_correct(bf, torch.from_numpy(u).cuda())
    ru, rg, rfl = oracle.flux_correct(u, rn, rdA, rk)
    assert abs(g.item() - rg) <= 1e-12 * abs(rg)
    assert abs(fl.item() - rfl) <= 1e-12 * np.abs((u * rn).sum(axis=0) * rdA).sum()
    np.testing.assert_allclose(uo.cpu().numpy(), ru, atol=1e-13)
    # the corrected flux vanishes (Eq. consv1)
    assert abs((uo.cpu().numpy() * rn).sum(axis=0) @ rdA) < 1e-12


def test_interface_update_box_annulus(fg):
    """Cylinder (session 1) boundary: radial faces are interface faces whose
    velocity comes from the box (session 0); the end walls carry prescribed
    data.  Interpolate, then correct the flux -- against the oracle chain."""
    mesh, q = synth.box_annulus()
    n_rad, n_az, n_ax = 4, 32, 8
    E = mesh.E
    kind = np.zeros((E, 6), np.int8)
    for e in range(1024, E):
        el = e - 1024
        er, ez = el % n_rad, el // (n_rad * n_az)
        if er == 0:
            kind[e, 0] = 2
        if er == n_rad - 1:
            kind[e, 1] = 2
        if ez == 0:
            kind[e, 4] = 1
        if ez == n_ax - 1:
            kind[e, 5] = 1
    dev = torch.device("cuda:0")
    h = fg.fp_setup(torch.from_numpy(mesh.coords).to(dev), mesh.N, torch.from_numpy(mesh.sub).to(dev),
                    torch.from_numpy(mesh.dist).to(dev), opts=fg.default_opts(precision=fg.PREC_MIXED))
    bf = fg.BFaces(h, torch.from_numpy(kind).to(dev))
    x, nr, dA, nk = bf.nodes()
    iface = (nk == 2).nonzero().squeeze(1)
    pts = x[:, iface].contiguous()
    qs = torch.ones(pts.shape[1], dtype=torch.int32, device=dev)
    vel = torch.from_numpy(q.fields[:3]).to(dev)
    code, sub, elem, rst, d2, vals = fg.fp_find_eval(h, pts, qs, fields=vel)
    u = torch.empty((3, bf.M), dtype=torch.float64, device=dev)
    # prescribed data on the end walls: the nodal values of the cylinder's own fields
    xn = x.cpu().numpy()
    rng = np.random.default_rng(1)
    terms = [synth.random_poly_field(mesh.coords[:, :1], 5, rng)[1] for _ in range(4)]   # same draws as box_annulus
    pres = np.stack([sum(c * xn[0] ** i * xn[1] ** j * xn[2] ** k for c, (i, j, k) in terms[f]) for f in range(3)])
    u.copy_(torch.from_numpy(pres))
    u[:, iface] = vals
    uo, g, fl = fg.fp_flux_correct(bf, u)
    torch.cuda.synchronize()
    assert (code == 0).all() and (sub == 0).all()
    # oracle chain
    rx, rn, rdA, rk = oracle.bfaces(mesh.coords, mesh.N, kind)
    rif = rk == 2
    ref = oracle.find(mesh.coords, mesh.N, mesh.sub, rx[:, rif], qsess=np.ones(rif.sum(), np.int32), dist=mesh.dist)
    rv = oracle.evaluate(mesh.N, ref["code"], ref["elem"], ref["rst"], q.fields[:3])
    ru = pres.copy()
    ru[:, rif] = rv
    ruo, rg, rfl = oracle.flux_correct(ru, rn, rdA, rk)
    scale = np.abs(q.fields[:3]).max()
    assert abs(g.item() - rg) <= 1e-11 * scale
    np.testing.assert_allclose(uo.cpu().numpy(), ruo, atol=1e-11 * scale)
    # the interpolated flux was not zero before the correction, and is after
    assert abs(rfl) > 1e-8 and abs((uo.cpu().numpy() * rn).sum(axis=0) @ rdA) < 1e-10 * scale
