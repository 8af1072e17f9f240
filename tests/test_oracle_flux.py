"""Pins for the oracle's mass-flux correction (Sec. 2.2, Eqs. consv1, corr,
consv2): boundary-face quadrature against closed-form areas, closure of a
watertight surface (sum of n dA = 0), the divergence theorem, outward
orientation on left-handed elements, and the corrected flux."""
import numpy as np
import pytest

import oracle
import synth


def box_kind(shape, marks):
    """[E][6] face kinds of a structured box: marks[(axis, end)] for outer faces."""
    ex, ey, ez = shape
    E = ex * ey * ez
    kind = np.zeros((E, 6), np.int8)
    for e in range(E):
        idx = (e % ex, (e // ex) % ey, e // (ex * ey))
        for ax in range(3):
            if idx[ax] == 0 and (ax, 0) in marks:
                kind[e, 2 * ax] = marks[(ax, 0)]
            if idx[ax] == shape[ax] - 1 and (ax, 1) in marks:
                kind[e, 2 * ax + 1] = marks[(ax, 1)]
    return kind


ALL2 = {(a, s): 2 for a in range(3) for s in (0, 1)}


@pytest.mark.parametrize("N", [1, 3, 6])
def test_box_area_closure_divergence(N):
    lo, hi = np.array([0.0, -1.0, 0.5]), np.array([2.0, 0.5, 1.75])
    shp = (3, 2, 2)
    coords = synth.box_mesh(shp, N, lo=lo, hi=hi, amp_frac=0.2)   # interior deformed, boundary flat
    x, nr, dA, nk = oracle.bfaces(coords, N, box_kind(shp, ALL2))
    L = hi - lo
    assert abs(dA.sum() - 2 * (L[0] * L[1] + L[1] * L[2] + L[0] * L[2])) < 1e-12
    np.testing.assert_allclose((nr * dA).sum(axis=1), 0.0, atol=1e-13)
    vol = L.prod()
    for a in range(3):
        assert abs((x[a] * nr[a] * dA).sum() - vol) < 1e-12
    np.testing.assert_allclose(np.linalg.norm(nr, axis=0), 1.0, atol=1e-14)


def test_left_handed_elements_still_outward():
    N = 3
    coords = synth.box_mesh((2, 2, 1), N, amp_frac=0.1)
    mirrored = coords.copy()
    mirrored[0] = -mirrored[0]                     # left-handed elements, box [-1,0]x[0,1]^2
    x, nr, dA, nk = oracle.bfaces(mirrored, N, box_kind((2, 2, 1), ALL2))
    assert abs((x[0] * nr[0] * dA).sum() - 1.0) < 1e-12   # divergence theorem: volume > 0
    np.testing.assert_allclose((nr * dA).sum(axis=1), 0.0, atol=1e-13)


def test_annulus_closure_and_areas():
    N = 7
    coords, rho, zl = synth.annulus_mesh(16, 2, 3, N, 0.15, 0.35, 0.0, 1.0, center=(1.0, 0.5, 0.0))
    E = coords.shape[1]
    kind = np.zeros((E, 6), np.int8)
    for e in range(E):
        er, ea, ez = e % 2, (e // 2) % 16, e // 32
        if er == 0:
            kind[e, 0] = 2
        if er == 1:
            kind[e, 1] = 2
        if ez == 0:
            kind[e, 4] = 1
        if ez == 2:
            kind[e, 5] = 1
    x, nr, dA, nk = oracle.bfaces(coords, N, kind)
    radial = nk == 2
    assert abs(dA[radial].sum() - 2 * np.pi * (0.15 + 0.35)) < 1e-8
    assert abs(dA[~radial].sum() - 2 * np.pi * (0.35 ** 2 - 0.15 ** 2)) < 1e-8
    np.testing.assert_allclose((nr * dA).sum(axis=1), 0.0, atol=1e-12)
    # div (x-1, y-0.5, 0) = 2: flux = 2 x volume
    flux = ((x[0] - 1.0) * nr[0] + (x[1] - 0.5) * nr[1]) @ dA
    assert abs(flux - 2 * np.pi * (0.35 ** 2 - 0.15 ** 2)) < 1e-8
    # outer radial normal points away from the axis, inner one towards it
    rad = np.stack([x[0] - 1.0, x[1] - 0.5])
    proj = (rad * nr[:2]).sum(axis=0) / np.linalg.norm(rad, axis=0)
    r_node = np.linalg.norm(rad, axis=0)
    assert np.all(proj[radial & (r_node > 0.3)] > 0.99) and np.all(proj[radial & (r_node < 0.2)] < -0.99)


def test_flux_correction_zeroes_flux_and_moves_only_interface():
    N = 4
    shp = (2, 2, 2)
    coords = synth.box_mesh(shp, N, amp_frac=0.1)
    marks = {(0, 0): 2, (0, 1): 2, (1, 0): 1, (1, 1): 1, (2, 0): 2, (2, 1): 1}
    x, nr, dA, nk = oracle.bfaces(coords, N, box_kind(shp, marks))
    rng = np.random.default_rng(0)
    u = rng.uniform(-1, 1, (3, x.shape[1]))
    u_out, g, fl = oracle.flux_correct(u, nr, dA, nk)
    assert abs(fl - ((u * nr).sum(axis=0) @ dA)) < 1e-13
    assert abs(g + fl / dA[nk == 2].sum()) < 1e-14
    assert abs((u_out * nr).sum(axis=0) @ dA) < 1e-13                 # Eq. consv1 holds after the correction
    np.testing.assert_array_equal(u_out[:, nk == 1], u[:, nk == 1])     # prescribed data untouched
    d = u_out[:, nk == 2] - u[:, nk == 2]
    np.testing.assert_allclose(d, g * nr[:, nk == 2], atol=1e-15)      # correction along n (Eq. corr)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_extrapolation_exact_for_degree_m_minus_1(m):
    """Order-m extrapolation over equal steps reproduces polynomials in time
    of degree m-1 exactly and keeps constants."""
    rng = np.random.default_rng(m)
    coef = rng.uniform(-1, 1, (m, 5))
    def val(t):
        return sum(coef[d] * t ** d for d in range(m))
    hist = [val(float(-j)) for j in range(m)]         # t_n = 0, t_{n-1} = -1, ...
    np.testing.assert_allclose(oracle.extrapolate(hist), val(1.0), atol=1e-13)
    np.testing.assert_allclose(oracle.extrapolate([np.full(5, 2.5)] * m), 2.5, atol=1e-15)
    if m > 1:   # degree m is not reproduced (guards against a wrong order)
        hist = [np.full(5, float(-j) ** m) for j in range(m)]
        assert np.abs(oracle.extrapolate(hist) - 1.0).max() > 0.5
