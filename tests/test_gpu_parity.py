"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  Codes, subdomains and elements must match bit for bit;
|delta r| <= 1e-12 in the FP64 form and <= 1e-10 in the mixed form; eval
within 1e-12 of the field's max nodal magnitude."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import NO_BAND, assert_parity, gpu_find, oracle_find

pytestmark = pytest.mark.gpu
PRECS = [0, 1]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_04891_gb300 as fg
    fg.lib()


@pytest.mark.parametrize("prec", PRECS)
def test_cube4_full(prec):
    mesh, q = synth.cube4_small()
    g = gpu_find(mesh, q.pts, prec=prec, fields=q.fields)
    r = oracle_find(mesh, q.pts, fields=q.fields)
    assert (r["code"] == oracle.INSIDE).all()
    assert_parity(g, r, prec, fields=q.fields, band=NO_BAND)


@pytest.mark.parametrize("prec", PRECS)
def test_box_annulus_interface_points(prec):
    mesh, q = synth.box_annulus()
    g = gpu_find(mesh, q.pts, q.qsess, prec=prec, fields=q.fields)
    r = oracle_find(mesh, q.pts, q.qsess, fields=q.fields)
    assert_parity(g, r, prec, fields=q.fields, band=NO_BAND)
    # session exclusion: a tagged point never comes back from its own session
    found = r["code"] != oracle.NOT_FOUND
    assert np.all(g["sub"][found] != q.qsess[found])
    assert found.mean() > 0.99


@pytest.mark.parametrize("prec", PRECS)
def test_box_annulus_untagged_owner_rule(prec):
    """Untagged points in the box/cylinder overlap: owner = argmax delta^k."""
    mesh, _ = synth.box_annulus()
    rng = np.random.default_rng(11)
    th = rng.uniform(0, 2 * np.pi, 4000)
    rho = rng.uniform(0.14, 0.36, 4000)
    pts = np.stack([1 + rho * np.cos(th), 0.5 + rho * np.sin(th), rng.uniform(0.0, 1.0, 4000)])
    g = gpu_find(mesh, pts, prec=prec)
    r = oracle_find(mesh, pts)
    assert_parity(g, r, prec, band=NO_BAND)
    assert set(np.unique(r["sub"][r["code"] == 0])) == {0, 1}


@pytest.mark.parametrize("refine", [0, 1, 2, 3])
def test_mixed_final_steps_and_full_fp64_fallback(refine):
    """Every route out of the mixed form's FP32 phase gives the oracle's
    results: refine = 0 sends every pair that converged near its element to
    the full FP64 Newton; with 1 the first compensated residual's step is
    too large to finish most pairs (they fall back); 2 finishes most of
    them; 3 is the default."""
    mesh, q = synth.deformed_cube(ne=8, P_uniform=30011, P_face=5003)
    g = gpu_find(mesh, q.pts, prec=1, fields=q.fields, refine=refine, paths=True)
    r = oracle_find(mesh, q.pts, fields=q.fields)
    assert_parity(g, r, 1, fields=q.fields, band=NO_BAND)
    p = g["paths"]
    near = p["fp64_step_converged"] + p["fallback"] - p["fp32_not_converged"]
    assert near > 0.9 * q.pts.shape[1]
    if refine == 0:
        assert p["fp64_step_converged"] == 0 and p["fallback"] >= near
    if refine == 1:
        assert p["fallback"] > 0.5 * near
    if refine >= 2:
        assert p["fp64_step_converged"] > 0.5 * near
    if refine == 3:
        assert p["fallback"] <= 1e-3 * near


def test_mixed_full_fp64_fallback_sessions_and_borders():
    """The full FP64 Newton behind the mixed form on tagged interface points
    of the box + annulus mesh (session exclusion, border points, owner rule)."""
    mesh, q = synth.box_annulus()
    g = gpu_find(mesh, q.pts, q.qsess, prec=1, fields=q.fields, refine=0, paths=True)
    r = oracle_find(mesh, q.pts, q.qsess, fields=q.fields)
    assert_parity(g, r, 1, fields=q.fields, band=NO_BAND)
    assert g["paths"]["fp64_step_converged"] == 0 and g["paths"]["fallback"] > 0


@pytest.mark.parametrize("prec", PRECS)
def test_deformed_cube_reduced_with_near_face(prec):
    mesh, q = synth.deformed_cube(ne=8, P_uniform=30011, P_face=5003)
    g = gpu_find(mesh, q.pts, prec=prec, fields=q.fields)
    r = oracle_find(mesh, q.pts, fields=q.fields)
    assert_parity(g, r, prec, fields=q.fields, band=NO_BAND)
    assert (r["code"] == oracle.INSIDE).all()


@pytest.mark.parametrize("N", [1, 2, 3, 5, 9, 12, 15])
@pytest.mark.parametrize("prec", PRECS)
def test_forward_recovery_all_orders(N, prec):
    coords = synth.box_mesh((3, 2, 3), N, amp_frac=0.1)
    mesh = synth.Mesh(coords=coords, N=N, sub=np.zeros(coords.shape[1], np.int32))
    rng = np.random.default_rng(100 + N)
    E = coords.shape[1]
    P = 257
    els = rng.integers(0, E, P)
    r = rng.uniform(-0.97, 0.97, (3, P))
    pts = np.empty((3, P))
    for e in np.unique(els):
        sel = els == e
        x, _ = oracle.map_points(coords, N, int(e), r[:, sel])
        pts[:, sel] = x
    fields = synth.field_u(coords)[None]
    g = gpu_find(mesh, pts, prec=prec, fields=fields)
    ref = oracle_find(mesh, pts, fields=fields)
    assert_parity(g, ref, prec, fields=fields)
    np.testing.assert_array_equal(g["elem"], els)
    assert np.abs(g["rst"] - r).max() <= 1e-11


@pytest.mark.parametrize("prec", PRECS)
def test_edge_cases(prec):
    import paper_1811_04891_gb300 as fg
    N = 4
    coords = synth.box_mesh((2, 2, 2), N)
    mesh = synth.Mesh(coords=coords, N=N, sub=np.zeros(8, np.int32))
    h_e = np.sqrt(3) * 0.5
    xi = oracle.gll(N)[0]
    pts = np.array([
        [0.3, 0.3, 1.0 + 0.2e-6 * h_e],        # border
        [0.3, 0.3, 1.0 + 10e-6 * h_e],         # not found
        [-5.0, 0.0, 0.0],
        [np.nan, 0.5, 0.5],
        [0.5, np.inf, 0.5],
        [1.0, 1.0, 1.0],                       # mesh corner
        [0.5, 0.5, 0.5],                       # vertex shared by 8 elements
        [0.25 * (1 + xi[1]), 0.5, 0.75],       # GLL node on a shared face
        [1.0 + 0.5e-6 * h_e, 1.0 + 0.5e-6 * h_e, 0.5],   # border near an edge
    ]).T
    g = gpu_find(mesh, pts, prec=prec)
    r = oracle_find(mesh, pts)
    # the last point lies 0.71e-6 h_e from an edge shared by two elements:
    # a BORDER tie between them, near the border threshold
    assert_parity(g, r, prec, band={"accept": 0, "border": 1, "owner": 0})
    np.testing.assert_array_equal(g["code"], [1, 2, 2, 2, 2, 0, 0, 0, 1])
    # empty query
    h = g["handle"]
    dev = torch.device("cuda:0")
    out = fg.fp_find(h, torch.zeros((3, 0), dtype=torch.float64, device=dev))
    assert out[0].numel() == 0
    ev = fg.fp_eval(h, out[0], out[2], out[3], torch.zeros((1, 8, 125), dtype=torch.float64, device=dev))
    assert ev.shape == (1, 0)


@pytest.mark.parametrize("prec", PRECS)
def test_tiny_overlap_owner_rule_all_tags(prec):
    mesh = synth.tiny_overlap(N=4)
    rng = np.random.default_rng(12)
    xs = np.concatenate([rng.uniform(-0.05, 2.05, 600), [0.8, 0.8, 0.6, 1.0, 1.6]])
    P = xs.size
    pts = np.stack([xs, rng.uniform(0.02, 0.98, P), rng.uniform(0.02, 0.98, P)])
    L = np.sqrt(2.0 ** 2 + 1 + 1)
    band = 1e-10 * L
    for tag in (-1, 0, 1, 2):
        qs = np.full(P, tag, np.int32)
        g = gpu_find(mesh, pts, qs, prec=prec)
        r = oracle_find(mesh, pts, qs)
        # owner near-ties from the closed-form delta^k = min(x - a_k, b_k - x)
        # of the subdomains that contain each point (x = 0.8: delta_0 = delta_1)
        ties = 0
        for x in xs:
            d = [min(x - a, b - x) for k, (a, b) in enumerate(synth.meshes.TINY_X) if k != tag and a <= x <= b]
            ties += len(d) > 1 and sum(v >= max(d) - 2 * band for v in d) > 1
        assert ties > 0 or tag >= 0
        assert_parity(g, r, prec, band={"accept": 0, "border": 0, "owner": ties})


@pytest.mark.parametrize("prec", PRECS)
def test_default_distance_field(prec):
    """No D supplied: both sides compute the nodal distance to boundary-face
    nodes of each subdomain (oracle brute force, device hash-accelerated)."""
    N = 3
    a = synth.box_mesh((3, 2, 2), N, lo=(0, 0, 0), hi=(1.2, 1, 1), amp_frac=0.05)
    b = synth.box_mesh((2, 2, 2), N, lo=(0.7, 0.1, 0.2), hi=(1.9, 0.9, 1.1), amp_frac=0.05)
    c = synth.box_mesh((2, 2, 1), N, lo=(0.9, -0.2, 0.3), hi=(1.5, 1.2, 0.8))
    mesh = synth.concat_meshes([a, b, c], N, [0, 1, 2])
    D = oracle.dist_default(mesh.coords, N, mesh.sub)
    pts = synth.uniform_points(3000, 13, lo=(0, -0.2, 0), hi=(1.9, 1.2, 1.1))
    g = gpu_find(mesh, pts, prec=prec, dist=None)
    r = oracle_find(mesh, pts, dist=D)
    assert_parity(g, r, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_spiral_element_N15(prec):
    N = 15
    coords, amap = synth.spiral_element(N)
    mesh = synth.Mesh(coords=coords, N=N, sub=np.zeros(1, np.int32))
    rng = np.random.default_rng(8)
    r = rng.uniform(-0.98, 0.98, (3, 1000))
    pts = amap(r[0], r[1], r[2])
    g = gpu_find(mesh, pts, prec=prec, tol_accept=1e-10)
    ref = oracle_find(mesh, pts, params=oracle.Params(tol_accept=1e-10, prefilter=False, n_restarts=8))
    assert_parity(g, ref, prec)
    assert (g["code"] == 0).all()


@pytest.mark.parametrize("prec", PRECS)
def test_invariance_hash_and_block(prec):
    """Hash size and block size change nothing.  0.02 cells per element
    makes cell lists longer than the screen's 31-entry candidate mask, so
    the emit pass tests those points again instead of reading the mask."""
    mesh, q = synth.deformed_cube(ne=6, P_uniform=20000, P_face=2000)
    base = gpu_find(mesh, q.pts, prec=prec)
    for kw in ({"hash_cells_per_elem": 0.2}, {"hash_cells_per_elem": 4.0}, {"hash_cells_per_elem": 0.02},
               {"points_per_block": 64}, {"points_per_block": 256}):
        g = gpu_find(mesh, q.pts, prec=prec, **kw)
        for k in ("code", "sub", "elem", "rst", "dist2"):
            np.testing.assert_array_equal(g[k], base[k], err_msg=str(kw))
    # the coarse grid does give lists longer than 31 entries
    import paper_1811_04891_gb300 as fg
    g = gpu_find(mesh, q.pts[:, :10], prec=prec, hash_cells_per_elem=0.02)
    cs = fg.fp_debug_boxes(g["handle"])[2].cpu().numpy()
    assert np.diff(cs).max() > 31


def test_hull_and_hash_contain_elements():
    import paper_1811_04891_gb300 as fg
    N = 7
    coords = synth.box_mesh((3, 3, 2), N, amp_frac=0.3)
    coords[0] += 0.02 * np.sin(7 * coords[1])
    E = coords.shape[1]
    dev = torch.device("cuda:0")
    h = fg.fp_setup(torch.from_numpy(coords).to(dev), N, torch.zeros(E, dtype=torch.int32, device=dev))
    aabb, grid, cs, ce = [t.cpu().numpy() for t in fg.fp_debug_boxes(h)]
    rng = np.random.default_rng(3)
    for e in range(E):
        r = rng.uniform(-1, 1, (3, 2000))
        r[:, :8] = np.array(np.meshgrid([-1, 1], [-1, 1], [-1, 1])).reshape(3, 8)
        x, _ = oracle.map_points(coords, N, e, r)
        assert np.all(x >= aabb[e, :3, None]) and np.all(x <= aabb[e, 3:, None])
    # brute-force overlap: every cell an element's box touches lists it
    org, inv, dims = grid[:3], grid[3:6], grid[6:].astype(int)
    lists = [set(ce[cs[c]:cs[c + 1]]) for c in range(len(cs) - 1)]
    for e in range(E):
        lo = np.clip(np.floor((aabb[e, :3] - org) * inv).astype(int), 0, dims - 1)
        hi = np.clip(np.floor((aabb[e, 3:] - org) * inv).astype(int), 0, dims - 1)
        for k in range(lo[2], hi[2] + 1):
            for j in range(lo[1], hi[1] + 1):
                for i in range(lo[0], hi[0] + 1):
                    assert e in lists[i + dims[0] * (j + dims[1] * k)]
    assert sum(len(s) for s in lists) == h.info()["nnz"]


def test_errors_are_reported():
    import paper_1811_04891_gb300 as fg
    dev = torch.device("cuda:0")
    bad = torch.zeros((3, 2, 8), dtype=torch.float64, device=dev)
    bad[0, 0, 0] = float("nan")
    with pytest.raises(fg.FindptsError) as ei:
        fg.fp_setup(bad, 1)
    assert ei.value.status == fg.FP_ERR_INVALID_ARG
    with pytest.raises(fg.FindptsError):
        fg.fp_setup(torch.zeros((3, 2, 8), dtype=torch.float64, device=dev), 1,
                    torch.tensor([0, 70000], dtype=torch.int32, device=dev))


@pytest.mark.parametrize("cfg", ["cube4_small", "box_annulus", "cube_small", "N3", "N15"])
def test_eval_double_float_parity(cfg):
    """fp_eval_df (double-float on the FP32 pipes) against the oracle's FP64
    triple sums and the FP64 kernel, on located points."""
    import paper_1811_04891_gb300 as fg
    if cfg == "cube4_small":
        mesh, q = synth.cube4_small()
        pts, fields = q.pts, q.fields
    elif cfg == "box_annulus":
        mesh, q = synth.box_annulus()
        pts, fields = q.pts, q.fields
    elif cfg == "cube_small":
        mesh, q = synth.deformed_cube(ne=6, P_uniform=20000, P_face=3000)
        pts, fields = q.pts, q.fields
    else:
        N = 3 if cfg == "N3" else 15
        coords = synth.box_mesh((2, 2, 2), N, amp_frac=0.1)
        mesh = synth.Mesh(coords=coords, N=N, sub=np.zeros(8, np.int32))
        fields = np.stack([synth.field_u(coords), synth.sine_product_field(coords, 3)])
        pts = synth.uniform_points(3001, 17, lo=(-0.01,) * 3, hi=(1.01,) * 3)
    dev = torch.device("cuda:0")
    g = gpu_find(mesh, pts, prec=1)
    h = g["handle"]
    f = fg.Fields(h, torch.from_numpy(fields).to(dev))
    code = torch.from_numpy(g["code"]).to(dev)
    elem = torch.from_numpy(g["elem"]).to(dev)
    rst = torch.from_numpy(g["rst"]).to(dev)
    vdf = fg.fp_eval_df(h, f, code, elem, rst).cpu().numpy()
    v64 = fg.fp_eval(h, code, elem, rst, torch.from_numpy(fields).to(dev)).cpu().numpy()
    ref = oracle.evaluate(mesh.N, g["code"], g["elem"], g["rst"], fields)
    assert np.array_equal(np.isnan(vdf), np.isnan(ref))
    scale = np.abs(fields).reshape(fields.shape[0], -1).max(axis=1)[:, None]
    ok = ~np.isnan(ref)
    err_df = (np.where(ok, np.abs(vdf - ref), 0.0) / scale).max()
    err_64 = (np.where(ok, np.abs(v64 - ref), 0.0) / scale).max()
    assert err_df <= 1e-12, err_df
    assert err_64 <= 1e-12, err_64


def test_fp64_two_pass_newton_equals_one_pass():
    """The FP64 form pauses solves that are still iterating after a fixed
    budget and resumes them in a second, denser pass; a paused solve keeps
    everything its next iteration depends on, so every output equals the
    one-pass solve (fp_find_static runs one pass) bit for bit."""
    import paper_1811_04891_gb300 as fg
    dev = torch.device("cuda:0")
    cases = []
    coords, amap = synth.spiral_element(15)
    rng = np.random.default_rng(21)
    cases.append((synth.Mesh(coords=coords, N=15, sub=np.zeros(1, np.int32)),
                  amap(*rng.uniform(-0.98, 0.98, (3, 3000))), {"tol_accept": 1e-10}))
    mesh, q = synth.deformed_cube(ne=6, P_uniform=12000, P_face=3000, with_fields=False)
    cases.append((mesh, q.pts, {}))
    for m, pts, opt in cases:
        h = fg.fp_setup(torch.from_numpy(m.coords).to(dev), m.N, torch.from_numpy(m.sub).to(dev),
                        opts=fg.default_opts(precision=0, **opt))
        t = torch.from_numpy(np.ascontiguousarray(pts)).to(dev)
        two = [x.cpu().numpy() for x in fg.fp_find(h, t)]
        one = [x.cpu().numpy() for x in fg.fp_find_static(h, t)]
        for a, b in zip(two, one):
            np.testing.assert_array_equal(a, b)
