"""Pins for the oracle's 2D (quadrilateral) variant (the paper's 2D overset
examples, Sec. 3; the same findpts / findpts_eval steps with the double sum
x^e(r,s) = sum_ij x_ij h_i(r) h_j(s)): the map against an independent
Vandermonde evaluation and finite differences, forward-map recovery of known
(e, r), affine closed forms, edge ties, border / not-found classification,
polynomial exactness of eval, the owner rule with closed-form delta, and the
default distance field against closed forms."""
import numpy as np
import pytest

import oracle
import synth

INSIDE, BORDER, NOT_FOUND = oracle.INSIDE, oracle.BORDER, oracle.NOT_FOUND


def vander_map_2d(coords, N, e, r):
    """x^e(r) through monomial coefficients fitted to the GLL nodes (an
    evaluation independent of the product-formula Lagrange basis)."""
    n = N + 1
    xi = synth.reference_grid(N)
    Vi = np.linalg.inv(np.vander(xi, n, increasing=True))
    X = coords[:, e].reshape(2, n, n)                    # [d][j][i]
    C = np.einsum("ai,bj,dji->dab", Vi, Vi, X)           # coefficients of r^a s^b
    pr = np.vander(r[0], n, increasing=True)
    ps = np.vander(r[1], n, increasing=True)
    return np.einsum("dab,ma,mb->dm", C, pr, ps)


def _zeros(E):
    return np.zeros(E, np.int32)


@pytest.mark.parametrize("N", [2, 5, 7])
def test_map_2d_against_vandermonde_and_fd_jacobian(N):
    coords = synth.quad_mesh((3, 2), N, amp_frac=0.2)
    coords[0] += 0.05 * coords[1] ** 2                   # anisotropic: an i/j mixup shows
    rng = np.random.default_rng(1)
    r = rng.uniform(-1, 1, (2, 20))
    for e in (0, 4):
        x, J = oracle.map_points(coords, N, e, r)
        np.testing.assert_allclose(x, vander_map_2d(coords, N, e, r), atol=1e-12)
        h = 1e-6
        for b in range(2):
            dr = np.zeros((2, 1))
            dr[b] = h
            fd = (vander_map_2d(coords, N, e, r + dr) - vander_map_2d(coords, N, e, r - dr)) / (2 * h)
            for a in range(2):
                np.testing.assert_allclose(J[2 * a + b], fd[a], atol=1e-7)


@pytest.mark.parametrize("N", [1, 2, 5, 7, 9])
def test_forward_map_recovery_2d(N):
    coords = synth.quad_mesh((4, 3), N, amp_frac=0.1)
    E = coords.shape[1]
    rng = np.random.default_rng(N)
    els = rng.integers(0, E, 60)
    r = rng.uniform(-0.95, 0.95, (2, 60))
    pts = np.stack([vander_map_2d(coords, N, e, r[:, [m]])[:, 0] for m, e in enumerate(els)], axis=1)
    res = oracle.find(coords, N, _zeros(E), pts)
    assert (res["code"] == INSIDE).all()
    np.testing.assert_array_equal(res["elem"], els)
    np.testing.assert_allclose(res["rst"], r, atol=1e-12)


def test_ring_recovery_2d():
    """Curved (annular) quads: points drawn by forward-mapping known (e, r)."""
    N = 7
    coords, _ = synth.ring_mesh(12, 2, N, 0.5, 1.0, center=(0.2, -0.1))
    E = coords.shape[1]
    rng = np.random.default_rng(3)
    els = rng.integers(0, E, 40)
    r = rng.uniform(-0.9, 0.9, (2, 40))
    pts = np.stack([vander_map_2d(coords, N, e, r[:, [m]])[:, 0] for m, e in enumerate(els)], axis=1)
    res = oracle.find(coords, N, _zeros(E), pts)
    assert (res["code"] == INSIDE).all()
    np.testing.assert_array_equal(res["elem"], els)
    np.testing.assert_allclose(res["rst"], r, atol=1e-12)


def test_affine_rect_closed_form_2d():
    N, shp = 4, (4, 3)
    lo, hi = np.array([0.0, -1.0]), np.array([2.0, 0.5])
    coords = synth.quad_mesh(shp, N, lo=lo, hi=hi)
    E = coords.shape[1]
    rng = np.random.default_rng(2)
    pts = lo[:, None] + (hi - lo)[:, None] * rng.uniform(0.001, 0.999, (2, 300))
    width = (hi - lo) / np.array(shp)
    u = (pts - lo[:, None]) / width[:, None]
    cell = np.floor(u).astype(int)
    frac = u - cell
    keep = np.all((frac > 1e-6) & (frac < 1 - 1e-6), axis=0)
    pts, cell, frac = pts[:, keep], cell[:, keep], frac[:, keep]
    res = oracle.find(coords, N, _zeros(E), pts)
    np.testing.assert_array_equal(res["code"], INSIDE)
    np.testing.assert_array_equal(res["elem"], cell[0] + shp[0] * cell[1])
    np.testing.assert_allclose(res["rst"], 2 * frac - 1, atol=1e-12)


def test_shared_edge_and_vertex_lowest_id_2d():
    N = 3
    coords = synth.quad_mesh((2, 2), N)
    E = coords.shape[1]
    pts = np.array([[0.5, 0.5], [0.3, 0.5], [0.5, 0.25]]).T
    res = oracle.find(coords, N, _zeros(E), pts)
    np.testing.assert_array_equal(res["code"], INSIDE)
    np.testing.assert_array_equal(res["elem"], [0, 0, 0])
    np.testing.assert_allclose(res["rst"][:, 0], [1, 1], atol=1e-12)
    np.testing.assert_allclose(res["rst"][:, 1], [0.2, 1], atol=1e-12)
    np.testing.assert_allclose(res["rst"][:, 2], [1, 0], atol=1e-12)


def test_border_not_found_nan_2d():
    N = 4
    coords = synth.quad_mesh((2, 2), N)
    E = coords.shape[1]
    h_e = np.sqrt(2) * 0.5
    pts = np.array([
        [0.3, 1.0 + 0.2e-6 * h_e],      # just outside the top edge: border
        [0.3, 1.0 + 10e-6 * h_e],       # too far: not found
        [-5.0, 0.0],
        [np.nan, 0.5],
        [1.0, 1.0],                     # corner of the mesh: inside
    ]).T
    res = oracle.find(coords, N, _zeros(E), pts)
    np.testing.assert_array_equal(res["code"], [BORDER, NOT_FOUND, NOT_FOUND, NOT_FOUND, INSIDE])
    assert res["elem"][0] == 2 and res["elem"][4] == 3
    np.testing.assert_allclose(res["rst"][:, 0], [0.2, 1.0], atol=1e-12)
    np.testing.assert_allclose(np.sqrt(res["dist2"][0]), 0.2e-6 * h_e, rtol=1e-6)
    out = oracle.evaluate(N, res["code"], res["elem"], res["rst"], synth.field_u_2d(coords)[None])
    assert np.isnan(out[0, 1:4]).all() and np.isfinite(out[0, [0, 4]]).all()


@pytest.mark.parametrize("N", [3, 7])
def test_eval_reproduces_reference_QN_polynomial_2d(N):
    coords = synth.quad_mesh((2, 2), N, amp_frac=0.15)
    E = coords.shape[1]
    vals, c = synth.reference_poly_field_2d(N, E, seed=4)
    rng = np.random.default_rng(5)
    P = 50
    elem = rng.integers(0, E, P).astype(np.int32)
    r = rng.uniform(-1, 1, (2, P))
    out = oracle.evaluate(N, np.zeros(P, np.int32), elem, r, vals[None])
    ref = np.polynomial.polynomial.polyval2d(r[0], r[1], c)
    np.testing.assert_allclose(out[0], ref, atol=1e-12 * np.abs(vals).max())


def test_eval_physical_polynomial_on_affine_mesh_2d():
    N = 5
    coords = synth.quad_mesh((3, 2), N, lo=(0, 0), hi=(2, 1))
    E = coords.shape[1]
    rng = np.random.default_rng(6)
    terms = [(rng.uniform(-1, 1), (i, j)) for i in range(6) for j in range(6 - i)]
    vals = sum(cf * coords[0] ** i * coords[1] ** j for cf, (i, j) in terms)
    pts = synth.uniform_points_2d(200, 7, lo=(0, 0), hi=(2, 1))
    res = oracle.find(coords, N, _zeros(E), pts)
    out = oracle.evaluate(N, res["code"], res["elem"], res["rst"], vals[None])[0]
    ref = sum(cf * pts[0] ** i * pts[1] ** j for cf, (i, j) in terms)
    np.testing.assert_allclose(out, ref, atol=1e-12 * np.abs(vals).max())


def _delta(k, x):
    a, b = synth.meshes.TINY_X[k]
    return np.minimum(x - a, b - x) if a <= x <= b else -np.inf


@pytest.mark.parametrize("N", [2, 4])
def test_owner_by_max_distance_closed_form_2d(N):
    mesh = synth.tiny_overlap_2d(N)
    xs = np.array([0.05, 0.3, 0.62, 0.75, 0.8, 0.9, 0.95, 1.05, 1.25, 1.45, 1.7, 1.99])
    y = np.random.default_rng(0).uniform(0.05, 0.95, xs.size)
    pts = np.stack([xs, y])
    for tag in (-1, 0, 1, 2):
        qs = np.full(xs.size, tag, np.int32)
        res = oracle.find(mesh.coords, N, mesh.sub, pts, qsess=qs, dist=mesh.dist)
        for m, x in enumerate(xs):
            cand = [(k, _delta(k, x)) for k in range(3) if k != tag and _delta(k, x) > -np.inf]
            if not cand:
                assert res["code"][m] != INSIDE
                continue
            dmax = max(d for _, d in cand)
            owner = min(k for k, d in cand if d >= dmax - 1e-9)
            assert res["code"][m] == INSIDE
            assert res["sub"][m] == owner, (tag, x, cand)


def test_exact_tie_goes_to_lower_subdomain_2d():
    mesh = synth.tiny_overlap_2d(3)
    pts = np.array([[0.8, 0.5], [0.8, 0.2]]).T
    res = oracle.find(mesh.coords, 3, mesh.sub, pts, qsess=np.array([2, 2], np.int32), dist=mesh.dist)
    np.testing.assert_array_equal(res["code"], INSIDE)
    np.testing.assert_array_equal(res["sub"], [0, 0])


def test_default_distance_field_2d_closed_form():
    N = 3
    lo, hi = (0.0, 0.0), (2.0, 1.5)
    coords = synth.quad_mesh((3, 2), N, lo=lo, hi=hi)
    E = coords.shape[1]
    D = oracle.dist_default(coords, N, np.zeros(E, np.int32))
    np.testing.assert_allclose(D, synth.rect_distance(coords, lo, hi), atol=1e-14)
    a = synth.quad_mesh((2, 1), N, lo=(0, 0), hi=(1, 1))
    b = synth.quad_mesh((1, 2), N, lo=(0.5, 0), hi=(1.5, 1))
    mesh = synth.concat_meshes([a, b], N, [0, 1])
    D = oracle.dist_default(mesh.coords, N, mesh.sub)
    np.testing.assert_allclose(D[:2], synth.rect_distance(a, (0, 0), (1, 1)), atol=1e-14)
    np.testing.assert_allclose(D[2:], synth.rect_distance(b, (0.5, 0), (1.5, 1)), atol=1e-14)


def test_walsh_workload_all_found():
    """The 2D overset workload: every query lies in the other subdomain."""
    mesh, q = synth.walsh_2d(N=5, n_box=8, ring=(12, 2))
    res = oracle.find(mesh.coords, mesh.N, mesh.sub, q.pts, qsess=q.qsess, dist=mesh.dist)
    assert (res["code"] == INSIDE).all()
    assert (res["sub"] != q.qsess).all()
    out = oracle.evaluate(mesh.N, res["code"], res["elem"], res["rst"], q.fields)
    exact = np.stack([-np.cos(q.pts[0]) * np.sin(q.pts[1]), np.sin(q.pts[0]) * np.cos(q.pts[1])])
    assert np.abs(out[:2] - exact).max() < 1e-3          # spectral interpolation of the eddy


def test_border_projection_on_skewed_quad():
    """2D analogue: a point just outside an edge of a skewed quad projects
    orthogonally onto the edge line (r = 1, s of the foot point)."""
    N = 3
    xi = synth.reference_grid(N)
    A = np.array([[0.5, 0.2], [0.3, 0.5]])                       # columns x_r, x_s
    c = np.array([1.0, -2.0])
    R, S = np.meshgrid(xi, xi, indexing="xy")                    # R[j][i] = xi_i, S[j][i] = xi_j
    ref = np.stack([R.reshape(-1), S.reshape(-1)])               # node (i,j) at i + n j
    coords = (c[:, None] + A @ ref)[:, None, :]
    he = np.linalg.norm(coords[:, 0].max(axis=1) - coords[:, 0].min(axis=1))
    t = A[:, 1] / np.linalg.norm(A[:, 1])
    nrm = np.array([t[1], -t[0]])
    if nrm @ A[:, 0] < 0:
        nrm = -nrm
    s0 = 0.35
    foot = c + A @ np.array([1.0, s0])
    d = 0.3e-6 * he
    res = oracle.find(coords, N, _zeros(1), (foot + d * nrm)[:, None])
    assert res["code"][0] == BORDER and res["elem"][0] == 0
    np.testing.assert_allclose(res["rst"][:, 0], [1.0, s0], atol=1e-9)
    np.testing.assert_allclose(np.sqrt(res["dist2"][0]), d, rtol=1e-6)


@pytest.mark.parametrize("angle0", [0.0, 0.7])
def test_default_distance_field_ring_closed_form(angle0):
    """Curved edges: every node of a ring shares its angle with GLL nodes of
    both circles and no point of a circle is nearer, so the distance to the
    boundary-edge nodes is min(rho - r_in, r_out - rho); the periodic seam is
    interior."""
    N, r_in, r_out = 4, 0.2, 0.5
    coords, rho = synth.meshes.ring_mesh(10, 3, N, r_in, r_out, center=(0.1, 0.3), angle0=angle0)
    E = coords.shape[1]
    D = oracle.dist_default(coords, N, np.zeros(E, np.int32))
    np.testing.assert_allclose(D, np.minimum(rho - r_in, r_out - rho), atol=1e-13)


def test_owner_with_default_distance_on_curved_overlap_2d():
    """2D ownership with the default distance field: a ring that crosses the
    top edge of a rectangle; for ring points inside the rectangle the owner
    is the subdomain with the larger exact boundary distance (rectangle: the
    four lines; ring: min(rho - r_in, r_out - rho)) wherever the two differ by
    more than 0.01.  Both subdomains own some of them."""
    N, C, R0, R1 = 5, (1.0, 0.8), 0.1, 0.3
    cb = synth.quad_mesh((8, 4), N, lo=(0, 0), hi=(2, 1))
    cr, _ = synth.meshes.ring_mesh(16, 2, N, R0, R1, center=C)
    mesh = synth.concat_meshes([cb, cr], N, [0, 1])
    D = oracle.dist_default(mesh.coords, N, mesh.sub)
    rng = np.random.default_rng(6)
    r = np.sqrt(rng.uniform(R0 ** 2, R1 ** 2, 4000))
    th = rng.uniform(0, 2 * np.pi, 4000)
    pts = np.stack([C[0] + r * np.cos(th), C[1] + r * np.sin(th)])
    inside = pts[1] <= 1.0
    pts, r = np.ascontiguousarray(pts[:, inside]), r[inside]
    d_box = np.minimum.reduce([pts[0], 2 - pts[0], pts[1], 1 - pts[1]])
    d_ring = np.minimum(r - R0, R1 - r)
    res = oracle.find(mesh.coords, N, mesh.sub, pts, dist=D)
    assert (res["code"] == INSIDE).all()
    keep = np.abs(d_box - d_ring) > 0.01
    want = np.where(d_ring > d_box, 1, 0)
    np.testing.assert_array_equal(res["sub"][keep], want[keep])
    assert 0.05 < want[keep].mean() < 0.95
