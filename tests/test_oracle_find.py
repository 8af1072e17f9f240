"""Pins for the oracle's findpts / findpts_eval (Sec. 2.1): forward-map
recovery of known (e, r), affine closed forms, face ties, border / not-found
classification, session exclusion, polynomial exactness of eval, and the
N=15 spiral robustness case modelled on Sec. 3.1's spiral element."""
import numpy as np
import pytest

import oracle
import synth
from test_oracle_basis import vander_map

INSIDE, BORDER, NOT_FOUND = oracle.INSIDE, oracle.BORDER, oracle.NOT_FOUND


def _zeros(E):
    return np.zeros(E, np.int32)


@pytest.mark.parametrize("N", [1, 2, 5, 7, 9])
def test_forward_map_recovery_deformed(N):
    coords = synth.box_mesh((3, 3, 3), N, amp_frac=0.1)
    E = coords.shape[1]
    rng = np.random.default_rng(N)
    els = rng.integers(0, E, 40)
    r = rng.uniform(-0.95, 0.95, (3, 40))
    pts = np.stack([vander_map(coords, N, e, r[:, [m]])[:, 0] for m, e in enumerate(els)], axis=1)
    res = oracle.find(coords, N, _zeros(E), pts)
    assert (res["code"] == INSIDE).all()
    np.testing.assert_array_equal(res["elem"], els)
    np.testing.assert_allclose(res["rst"], r, atol=1e-12)


def test_affine_box_closed_form():
    N, shp = 4, (4, 3, 2)
    lo, hi = np.array([0.0, -1.0, 2.0]), np.array([2.0, 0.5, 3.0])
    coords = synth.box_mesh(shp, N, lo=lo, hi=hi)
    E = coords.shape[1]
    rng = np.random.default_rng(2)
    pts = (lo[:, None] + (hi - lo)[:, None] * rng.uniform(0.001, 0.999, (3, 300)))
    # closed form: element index and reference coordinates of an affine box
    width = (hi - lo) / np.array(shp)
    u = (pts - lo[:, None]) / width[:, None]
    cell = np.floor(u).astype(int)
    frac = u - cell
    keep = np.all((frac > 1e-6) & (frac < 1 - 1e-6), axis=0)
    pts, cell, frac = pts[:, keep], cell[:, keep], frac[:, keep]
    e_ref = cell[0] + shp[0] * (cell[1] + shp[1] * cell[2])
    res = oracle.find(coords, N, _zeros(E), pts)
    np.testing.assert_array_equal(res["code"], INSIDE)
    np.testing.assert_array_equal(res["elem"], e_ref)
    np.testing.assert_allclose(res["rst"], 2 * frac - 1, atol=1e-12)


def test_shared_face_lowest_element_id_and_nodes():
    N = 3
    coords = synth.box_mesh((2, 2, 1), N)
    E = coords.shape[1]
    # points on the x = 0.5 face shared by elements 0 and 1, and on the edge
    # x = 0.5, y = 0.5 shared by 0,1,2,3
    pts = np.array([[0.5, 0.5, 0.5], [0.3, 0.5, 0.5], [0.5, 0.25, 0.7]]).T
    res = oracle.find(coords, N, _zeros(E), pts)
    np.testing.assert_array_equal(res["code"], INSIDE)
    np.testing.assert_array_equal(res["elem"], [0, 0, 0])
    np.testing.assert_allclose(res["rst"][:, 0], [1, 1, 0], atol=1e-12)
    np.testing.assert_allclose(res["rst"][:, 1], [0.2, 1, 0], atol=1e-12)
    np.testing.assert_allclose(res["rst"][:, 2], [1, 0, 0.4], atol=1e-12)


def test_border_not_found_nan():
    N = 4
    coords = synth.box_mesh((2, 2, 2), N)
    E = coords.shape[1]
    h_e = np.sqrt(3) * 0.5
    pts = np.array([
        [0.3, 0.3, 1.0 + 0.2e-6 * h_e],    # just outside the top face: border
        [0.3, 0.3, 1.0 + 10e-6 * h_e],     # too far: not found
        [-5.0, 0.0, 0.0],                  # far outside
        [np.nan, 0.5, 0.5],
        [0.5, np.inf, 0.5],
        [1.0, 1.0, 1.0],                   # corner of the mesh: inside
    ]).T
    res = oracle.find(coords, N, _zeros(E), pts)
    np.testing.assert_array_equal(res["code"], [BORDER, NOT_FOUND, NOT_FOUND, NOT_FOUND, NOT_FOUND, INSIDE])
    assert res["elem"][0] == 4 and res["elem"][5] == 7
    np.testing.assert_allclose(res["rst"][:, 0], [0.2, 0.2, 1.0], atol=1e-12)
    np.testing.assert_allclose(np.sqrt(res["dist2"][0]), 0.2e-6 * h_e, rtol=1e-6)
    assert np.isinf(res["dist2"][1]) and res["elem"][1] == -1 and res["sub"][1] == -1
    np.testing.assert_array_equal(res["rst"][:, 1], 0.0)
    out = oracle.evaluate(N, res["code"], res["elem"], res["rst"], synth.field_u(coords))
    assert np.isnan(out[0, 1:5]).all() and np.isfinite(out[0, [0, 5]]).all()


def test_session_exclusion():
    mesh = synth.tiny_overlap(N=3)
    rng = np.random.default_rng(3)
    pts = np.stack([rng.uniform(0.85, 0.95, 60), rng.uniform(0.1, 0.9, 60), rng.uniform(0.1, 0.9, 60)])
    for tag in (0, 1, 2):
        qs = np.full(60, tag, np.int32)
        res = oracle.find(mesh.coords, mesh.N, mesh.sub, pts, qsess=qs, dist=mesh.dist)
        assert (res["code"] == INSIDE).all()
        assert (res["sub"] != tag).all()


@pytest.mark.parametrize("N", [3, 7])
def test_eval_reproduces_reference_QN_polynomial(N):
    coords = synth.box_mesh((2, 2, 2), N, amp_frac=0.15)
    E = coords.shape[1]
    vals, c = synth.reference_poly_field(N, E, seed=4)
    rng = np.random.default_rng(5)
    P = 50
    elem = rng.integers(0, E, P).astype(np.int32)
    r = rng.uniform(-1, 1, (3, P))
    out = oracle.evaluate(N, np.zeros(P, np.int32), elem, r, vals[None])
    ref = np.polynomial.polynomial.polyval3d(r[0], r[1], r[2], c)
    np.testing.assert_allclose(out[0], ref, atol=1e-12 * np.abs(vals).max())


def test_eval_physical_polynomial_on_affine_mesh():
    N = 5
    coords = synth.box_mesh((3, 2, 2), N, lo=(0, 0, 0), hi=(2, 1, 1))
    E = coords.shape[1]
    rng = np.random.default_rng(6)
    vals, terms = synth.random_poly_field(coords, 5, rng)
    pts = synth.uniform_points(200, 7, lo=(0, 0, 0), hi=(2, 1, 1))
    res = oracle.find(coords, N, _zeros(E), pts)
    out = oracle.evaluate(N, res["code"], res["elem"], res["rst"], vals[None])[0]
    ref = sum(cf * pts[0] ** i * pts[1] ** j * pts[2] ** k for cf, (i, j, k) in terms)
    np.testing.assert_allclose(out, ref, atol=1e-12 * np.abs(vals).max())


def test_spiral_element_robustness():
    """Sec. 3.1: single N=15 spiral element, 1000 random points, tolerance
    1e-14; nearest-GLL-node seeding must avoid false minima.  Points are the
    analytic spiral map at random r; the polynomial element reproduces it to
    about 1e-12, so every point is found with r close to the one drawn."""
    N = 15
    coords, amap = synth.spiral_element(N)
    rng = np.random.default_rng(8)
    r = rng.uniform(-0.98, 0.98, (3, 1000))
    pts = amap(r[0], r[1], r[2])
    res = oracle.find(coords, N, _zeros(1), pts, params=oracle.Params(tol_accept=1e-10, prefilter=False))
    assert (res["code"] == INSIDE).all()
    np.testing.assert_allclose(res["rst"], r, atol=1e-9)
    # multi-start from the 8 next-nearest nodes finds nothing better
    res2 = oracle.find(coords, N, _zeros(1), pts[:, :100],
                       params=oracle.Params(tol_accept=1e-10, prefilter=False, n_restarts=8))
    np.testing.assert_allclose(res2["rst"], res["rst"][:, :100], atol=1e-12)


def test_border_projection_on_skewed_element():
    """A point just outside a face of a skewed (affine) element: the
    constrained minimiser is its orthogonal projection onto the face plane
    (reference r = 1 and the face coordinates of the foot point), and the
    border distance is the distance to that plane -- the active set must
    freeze r and keep minimising over (s, t)."""
    N = 3
    xi = synth.reference_grid(N)
    A = np.array([[0.5, 0.0, 0.0], [0.25, 0.5, 0.0], [0.15, -0.1, 0.5]])   # columns: x_r, x_s, x_t
    c = np.array([1.0, 2.0, 3.0])
    R, S, T = np.meshgrid(xi, xi, xi, indexing="ij")
    ref = np.stack([R, S, T]).reshape(3, -1)                     # node (i,j,k) with i slowest here
    X = c[:, None] + A @ ref
    n = N + 1
    coords = X.reshape(3, n, n, n).transpose(0, 3, 2, 1).reshape(3, 1, n ** 3)   # i fastest
    he = np.linalg.norm(coords[:, 0].max(axis=1) - coords[:, 0].min(axis=1))
    nrm = np.cross(A[:, 1], A[:, 2])
    nrm /= np.linalg.norm(nrm)
    if nrm @ A[:, 0] < 0:
        nrm = -nrm                                               # outward at r = +1
    s0, t0 = 0.3, -0.4
    foot = c + A @ np.array([1.0, s0, t0])
    d = 0.3e-6 * he
    pts = (foot + d * nrm)[:, None]
    res = oracle.find(coords, N, _zeros(1), pts)
    assert res["code"][0] == BORDER and res["elem"][0] == 0
    np.testing.assert_allclose(res["rst"][:, 0], [1.0, s0, t0], atol=1e-9)
    np.testing.assert_allclose(np.sqrt(res["dist2"][0]), d, rtol=1e-6)


@pytest.mark.parametrize("case", ["deformed", "curved_border", "overlap_tags", "quad"])
def test_prefilter_never_changes_a_result(case):
    """The oracle's optional prefilter (node box grown by 25 % of its extent
    plus the border tolerance) may only skip elements that cannot hold the
    answer: with it and without it every output is identical, on strongly
    deformed and curved elements, at border distances and with session tags."""
    rng = np.random.default_rng(31)
    qsess = None
    if case == "deformed":
        N = 5
        coords = synth.box_mesh((3, 3, 2), N, amp_frac=0.45)
        coords[0] += 0.04 * np.sin(5 * coords[1]) * np.cos(3 * coords[2])
        mesh = synth.Mesh(coords=coords, N=N, sub=_zeros(coords.shape[1]))
        pts = rng.uniform(-0.02, 1.02, (3, 1500))
    elif case == "curved_border":
        N = 6
        mesh, _ = synth.box_annulus(n_az=12, n_rad=2, n_ax=2, box_shape=(4, 2, 2), N=N)
        th = rng.uniform(0, 2 * np.pi, 1200)
        # just outside and inside the annulus's curved faces, at border distances
        rho = np.where(rng.random(1200) < 0.5, 0.15, 0.35) + rng.choice([-1, 1], 1200) * 10.0 ** rng.uniform(-9, -6, 1200)
        pts = np.stack([1 + rho * np.cos(th), 0.5 + rho * np.sin(th), rng.uniform(0.0, 1.0, 1200)])
        qsess = np.zeros(1200, np.int32)           # search the annulus only
    elif case == "overlap_tags":
        mesh = synth.tiny_overlap(N=4)
        pts = np.stack([rng.uniform(-0.05, 2.05, 900), rng.uniform(-0.01, 1.01, 900), rng.uniform(0.0, 1.0, 900)])
        qsess = rng.integers(-1, 3, 900).astype(np.int32)
    else:
        N = 7
        mesh = synth.Mesh(coords=synth.quad_mesh((4, 3), N, amp_frac=0.4), N=N, sub=_zeros(12))
        pts = rng.uniform(-0.02, 1.02, (2, 1500))
    on = oracle.find(mesh.coords, mesh.N, mesh.sub, pts, qsess=qsess, dist=mesh.dist,
                     params=oracle.Params(prefilter=True))
    off = oracle.find(mesh.coords, mesh.N, mesh.sub, pts, qsess=qsess, dist=mesh.dist,
                      params=oracle.Params(prefilter=False))
    for k in ("code", "sub", "elem", "rst", "dist2"):
        np.testing.assert_array_equal(on[k], off[k], err_msg=k)
    assert (on["code"] == INSIDE).any() and (on["code"] != INSIDE).any()
