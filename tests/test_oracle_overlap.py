"""Pins for the oracle's multi-subdomain rules (Sec. 2.1, Fig. 4): session
exclusion, owner = argmax_k delta^k(x*) with lower-id tie break, and the
default nodal distance field against closed forms on undeformed boxes."""
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
