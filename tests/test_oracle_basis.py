"""Pins for the oracle's GLL points, Lagrange basis and isoparametric map
(Sec. 1-2: Q_N tensor-product map on GLL nodes) against closed forms,
quadrature exactness, library routines and an independent Vandermonde
evaluation."""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.txt")


def _parse(tok):
    return float(eval(tok, {"sqrt": math.sqrt}))


def _golden():
    rows = {}
    for line in open(GOLD):
        line = line.split("#")[0].strip()
        if not line:
            continue
        parts = line.split()
        N = int(parts[0])
        vals = [_parse(t) for t in parts[1:]]
        rows[N] = (np.array(vals[:N + 1]), np.array(vals[N + 1:]))
    return rows


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_gll_closed_forms(N):
    x, w = oracle.gll(N)
    gx, gw = _golden()[N]
    np.testing.assert_allclose(x, gx, atol=1e-15, rtol=0)
    np.testing.assert_allclose(w, gw, atol=1e-15, rtol=1e-14)


@pytest.mark.parametrize("N", range(1, 16))
def test_gll_quadrature_exact_and_symmetric(N):
    x, w = oracle.gll(N)
    assert np.all(np.diff(x) > 0)
    np.testing.assert_array_equal(x, -x[::-1])
    for k in range(2 * N):          # GLL is exact through degree 2N-1
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 2e-14, k
    # degree 2N is NOT integrated exactly (guards against Gauss-type mixups)
    if N <= 8:
        assert abs(np.dot(w, x ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-6


@pytest.mark.parametrize("N", range(2, 16))
def test_gll_against_numpy_legendre_roots(N):
    x, _ = oracle.gll(N)
    ref = np.sort(np.polynomial.legendre.Legendre.basis(N).deriv().roots().real)
    np.testing.assert_allclose(x[1:-1], ref, atol=5e-14)


@pytest.mark.parametrize("N", [1, 3, 7, 15])
def test_lagrange_kronecker_partition_and_derivative(N):
    x, _ = oracle.gll(N)
    for m in range(N + 1):
        h, _ = oracle.lagrange(N, x[m])
        e = np.zeros(N + 1)
        e[m] = 1.0
        np.testing.assert_allclose(h, e, atol=1e-13)
    rng = np.random.default_rng(0)
    for r in rng.uniform(-1, 1, 5):
        h, dh = oracle.lagrange(N, r)
        assert abs(h.sum() - 1.0) < 1e-12
        assert abs(dh.sum()) < 1e-9
        # derivative against numpy's polynomial through (x_i, delta_im)
        for i in range(N + 1):
            y = np.zeros(N + 1)
            y[i] = 1.0
            c = np.linalg.solve(np.vander(x, N + 1, increasing=True), y)
            dpoly = np.polynomial.polynomial.polyder(c)
            assert abs(np.polynomial.polynomial.polyval(r, dpoly) - dh[i]) < 1e-8 * max(1, abs(dh[i]))
            assert abs(np.polynomial.polynomial.polyval(r, c) - h[i]) < 1e-10


def vander_map(coords, N, e, r):
    """Independent evaluation of x^e(r): monomial coefficients from the 1-D
    Vandermonde matrix at numpy's GLL abscissae, applied per direction."""
    n = N + 1
    xi = synth.reference_grid(N)
    Vi = np.linalg.inv(np.vander(xi, n, increasing=True))     # coefficients = Vi @ values
    X = coords[:, e, :].reshape(3, n, n, n)                   # [a][k][j][i]
    C = np.einsum("ai,bj,ck,dkji->dabc", Vi, Vi, Vi, X)       # [d][a(r)][b(s)][c(t)]
    pr = np.vander(r[0], n, increasing=True)
    ps = np.vander(r[1], n, increasing=True)
    pt = np.vander(r[2], n, increasing=True)
    return np.einsum("dabc,ma,mb,mc->dm", C, pr, ps, pt)


@pytest.mark.parametrize("N", [2, 5, 7])
def test_map_against_vandermonde_and_fd_jacobian(N):
    coords = synth.box_mesh((2, 3, 2), N, amp_frac=0.2)
    # make the geometry anisotropic so that an i/j/k mixup shows
    coords[0] += 0.05 * coords[1] ** 2
    coords[2] += 0.03 * np.sin(3 * coords[0])
    rng = np.random.default_rng(1)
    r = rng.uniform(-1, 1, (3, 20))
    for e in (0, 5, 11):
        x, J = oracle.map_points(coords, N, e, r)
        np.testing.assert_allclose(x, vander_map(coords, N, e, r), atol=1e-12)
        h = 1e-6
        for b in range(3):
            dr = np.zeros((3, 1))
            dr[b] = h
            fd = (vander_map(coords, N, e, r + dr) - vander_map(coords, N, e, r - dr)) / (2 * h)
            for a in range(3):
                np.testing.assert_allclose(J[3 * a + b], fd[a], atol=1e-7)
