"""Pins for the oracle's multi-subdomain rules (Sec. 2.1, Fig. 4): session
exclusion, owner = argmax_k delta^k(x*) with lower-id tie break, and the
default nodal distance field against closed forms on undeformed boxes and
curved annular cylinders, and ownership with that field on a curved overlap."""
import numpy as np
import pytest

import oracle
import synth

INSIDE = oracle.INSIDE


def _delta(k, x):
    a, b = synth.meshes.TINY_X[k]
    return np.minimum(x - a, b - x) if a <= x <= b else -np.inf


@pytest.mark.parametrize("N", [2, 4])
def test_owner_by_max_distance_closed_form(N):
    mesh = synth.tiny_overlap(N)
    xs = np.array([0.05, 0.3, 0.62, 0.75, 0.8, 0.9, 0.95, 1.05, 1.25, 1.45, 1.7, 1.99])
    rng = np.random.default_rng(0)
    y = rng.uniform(0.05, 0.95, xs.size)
    z = rng.uniform(0.05, 0.95, xs.size)
    pts = np.stack([xs, y, z])
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
            # the element lies in the owner's x-range
            a, b = synth.meshes.TINY_X[owner]
            mid = 0.5 * (a + b)
            e_loc = int(res["elem"][m]) - 2 * owner
            assert e_loc == (0 if x < mid or (x == mid) else 1)


def test_exact_tie_goes_to_lower_subdomain():
    mesh = synth.tiny_overlap(3)
    # x = 0.8 lies on the boundary of subdomain 2: delta0 = delta1 = 0.2
    pts = np.array([[0.8, 0.5, 0.5], [0.8, 0.2, 0.7]]).T
    res = oracle.find(mesh.coords, 3, mesh.sub, pts, qsess=np.array([2, 2], np.int32), dist=mesh.dist)
    np.testing.assert_array_equal(res["code"], INSIDE)
    np.testing.assert_array_equal(res["sub"], [0, 0])


def test_default_distance_field_box_closed_form():
    N = 3
    lo, hi = (0.0, 0.0, 0.0), (2.0, 1.0, 1.5)
    coords = synth.box_mesh((3, 2, 2), N, lo=lo, hi=hi)
    E = coords.shape[1]
    D = oracle.dist_default(coords, N, np.zeros(E, np.int32))
    ref = synth.box_distance(coords, lo, hi)
    np.testing.assert_allclose(D, ref, atol=1e-14)


def test_default_distance_field_two_subdomains_independent():
    N = 2
    a = synth.box_mesh((2, 1, 1), N, lo=(0, 0, 0), hi=(1, 1, 1))
    b = synth.box_mesh((1, 2, 1), N, lo=(0.5, 0, 0), hi=(1.5, 1, 1))
    mesh = synth.concat_meshes([a, b], N, [0, 1])
    D = oracle.dist_default(mesh.coords, N, mesh.sub)
    np.testing.assert_allclose(D[:2], synth.box_distance(a, (0, 0, 0), (1, 1, 1)), atol=1e-14)
    np.testing.assert_allclose(D[2:], synth.box_distance(b, (0.5, 0, 0), (1.5, 1, 1)), atol=1e-14)


@pytest.mark.parametrize("rot", [(0.0, 0.0), (15.0, -20.0)])
def test_default_distance_field_annulus_closed_form(rot):
    """Curved boundaries: on an annular cylinder every node shares its (theta,
    z) with GLL nodes of both cylindrical faces and its (rho, theta) with nodes
    of both end faces, and no point of a face is nearer than those, so the
    distance to the boundary-face nodes is exactly min(rho - r_in, r_out - rho,
    z - z0, z1 - z).  The periodic seam in theta must not count as boundary."""
    N, r_in, r_out, z0, z1 = 3, 0.2, 0.5, -0.25, 0.35
    coords, rho, zl = synth.annulus_mesh(8, 2, 3, N, r_in, r_out, z0, z1, center=(0.3, -0.1, 0.2), rot=rot)
    E = coords.shape[1]
    D = oracle.dist_default(coords, N, np.zeros(E, np.int32))
    ref = synth.annulus_distance(rho, zl, r_in, r_out, z0, z1)
    np.testing.assert_allclose(D, ref, atol=1e-13)


def test_default_distance_field_annulus_beside_box():
    """Two subdomains, one curved: each node's distance is to its own
    subdomain's boundary only (the cylinder inside the box changes neither)."""
    N = 2
    cb = synth.box_mesh((4, 2, 2), N, lo=(0.0, 0.0, 0.0), hi=(2.0, 1.0, 1.0))
    cc, rho, zl = synth.annulus_mesh(8, 1, 2, N, 0.15, 0.35, 0.0, 1.0, center=(1.0, 0.5, 0.0))
    mesh = synth.concat_meshes([cb, cc], N, [0, 1])
    D = oracle.dist_default(mesh.coords, N, mesh.sub)
    Eb = cb.shape[1]
    np.testing.assert_allclose(D[:Eb], synth.box_distance(cb, (0, 0, 0), (2, 1, 1)), atol=1e-14)
    np.testing.assert_allclose(D[Eb:], synth.annulus_distance(rho, zl, 0.15, 0.35, 0.0, 1.0), atol=1e-13)


def test_owner_with_default_distance_on_curved_overlap():
    """Ownership on a curved overlap with the default (computed) distance
    field: an annular cylinder that crosses the y = 1 face of a box.  For
    cylinder points inside the box the owner is the subdomain whose exact
    boundary distance is larger (box: the six planes; cylinder:
    min(rho - r_in, r_out - rho, z, 1 - z)) wherever the two differ by more
    than the interpolation error of D near its kinks (margin 0.01); both
    subdomains own some of them."""
    N, C, R0, R1 = 5, (1.0, 0.8, 0.0), 0.1, 0.3
    cb = synth.box_mesh((8, 4, 4), N, lo=(0, 0, 0), hi=(2, 1, 1))
    cc, _, _ = synth.annulus_mesh(16, 2, 4, N, R0, R1, 0.0, 1.0, center=C)
    mesh = synth.concat_meshes([cb, cc], N, [0, 1])
    D = oracle.dist_default(mesh.coords, N, mesh.sub)
    rng = np.random.default_rng(5)
    P = 4000
    r = np.sqrt(rng.uniform(R0 ** 2, R1 ** 2, P))
    th = rng.uniform(0, 2 * np.pi, P)
    z = rng.uniform(0, 1, P)
    pts = np.stack([C[0] + r * np.cos(th), C[1] + r * np.sin(th), z])
    inside = pts[1] <= 1.0
    pts, r, z = np.ascontiguousarray(pts[:, inside]), r[inside], z[inside]
    d_box = np.minimum.reduce([pts[0], 2 - pts[0], pts[1], 1 - pts[1], pts[2], 1 - pts[2]])
    d_cyl = np.minimum.reduce([r - R0, R1 - r, z, 1 - z])
    res = oracle.find(mesh.coords, N, mesh.sub, pts, dist=D)
    assert (res["code"] == INSIDE).all()
    keep = np.abs(d_box - d_cyl) > 0.01
    want = np.where(d_cyl > d_box, 1, 0)
    assert keep.sum() > 1500
    np.testing.assert_array_equal(res["sub"][keep], want[keep])
    assert 0.05 < want[keep].mean() < 0.95
    # a query tagged with the cylinder's session sees only the box
    res_b = oracle.find(mesh.coords, N, mesh.sub, pts[:, :50], qsess=np.ones(50, np.int32), dist=D)
    np.testing.assert_array_equal(res_b["sub"], 0)
