"""CPU tests that the seeded generators produce the workloads the input
recipe describes: the deformed cube's displacement rule, the near-face
points' offsets, the batch's size ranges and totals, the box + annulus
queries and tags, and the served request stream."""
import numpy as np

import synth


def _undeformed(shape, N=7):
    """Undeformed node positions of a unit-cube box mesh of that shape."""
    return synth.box_mesh(shape, N)


def test_deformed_cube_displacement_rule():
    """One scalar 0.1 h sin(2 pi x) sin(2 pi y) sin(2 pi z) added to each
    coordinate of every node not on the cube boundary; boundary nodes stay;
    nodes shared by neighbouring elements stay bit-identical."""
    mesh, _ = synth.deformed_cube(ne=4, P_uniform=10, P_face=0, with_fields=False)
    x0 = _undeformed((4, 4, 4))
    d = mesh.coords - x0
    h = 1.0 / 4
    want = 0.1 * h * np.sin(2 * np.pi * x0[0]) * np.sin(2 * np.pi * x0[1]) * np.sin(2 * np.pi * x0[2])
    onb = np.zeros(x0.shape[1:], bool)
    for a in range(3):
        onb |= (x0[a] == 0.0) | (x0[a] == 1.0)
    for a in range(3):
        np.testing.assert_allclose(d[a][~onb], want[~onb], rtol=0, atol=1e-15)
        assert np.all(d[a][onb] == 0.0)
    assert np.abs(d).max() > 0.02 * h
    # shared nodes: the same undeformed point maps to the same deformed point everywhere
    key = np.round(x0.reshape(3, -1).T * 2 ** 20).astype(np.int64)
    pts = mesh.coords.reshape(3, -1).T
    order = np.lexsort(key.T)
    ks, ps = key[order], pts[order]
    same = np.all(ks[1:] == ks[:-1], axis=1)
    assert same.any()
    assert np.array_equal(ps[1:][same], ps[:-1][same])


def test_near_face_points_offsets():
    """Face-interior GLL nodes moved along the face's axis by 10^U(-11,-9)
    (90 %) or by exactly 0 (10 %), all inside the unit cube."""
    mesh, _ = synth.deformed_cube(ne=4, P_uniform=10, P_face=0, with_fields=False)
    M = 20000
    p = synth.near_face_points(mesh.coords, mesh.N, M, seed=1)
    assert p.shape == (3, M)
    assert np.all((p >= 0.0) & (p <= 1.0))
    nodes = mesh.coords.reshape(3, -1)
    # distance to the nearest node: exactly 0 for ~10 %, else in [1e-11, 1e-9]
    from scipy.spatial import cKDTree
    dist, _ = cKDTree(nodes.T).query(p.T)
    zero = dist == 0.0
    assert 0.08 < zero.mean() < 0.12
    assert np.all((dist[~zero] >= 0.99e-11) & (dist[~zero] <= 1.01e-9))


def test_instance_batch_sizes():
    insts = synth.instance_batch()
    assert len(insts) == 64
    Es = np.array([m.E for m, _ in insts])
    Ns = {m.N for m, _ in insts}
    Ps = np.array([q.P for _, q in insts])
    assert Ns == {5, 7, 9}
    assert Es.min() >= 27 and Es.max() <= 2 * 8192          # log-U[64, 8192] rounded to near-cubic shapes
    assert Ps.min() >= 1000 and Ps.max() <= 10 ** 6
    assert int(Es.sum()) == 94980 and int(Ps.sum()) == 7825127


def test_box_annulus_queries():
    mesh, q = synth.box_annulus(n_az=16, n_rad=2, n_ax=4, box_shape=(8, 4, 4), N=5)
    assert set(np.unique(mesh.sub)) == {0, 1}
    assert set(np.unique(q.qsess)) == {0, 1}
    assert np.all(mesh.dist >= 0.0)
    # cylinder-tagged queries are cylinder boundary nodes: rho = r_in or r_out, or z on an end
    cyl = q.qsess == 1
    rho = np.hypot(q.pts[0, cyl] - 1.0, q.pts[1, cyl] - 0.5)
    z = q.pts[2, cyl]
    on = (np.abs(rho - 0.15) < 1e-12) | (np.abs(rho - 0.35) < 1e-12) | (z == 0.0) | (z == 1.0)
    assert on.all()


def test_poisson_requests():
    _, iface = synth.box_two_annuli(box_shape=(10, 5, 5), cyl_shape=(8, 2, 8), N=3)
    reqs = synth.poisson_requests(iface, 50, seed=4, size_range=(100, 10000), rate_hz=100.0)
    t = np.array([r["t_arrive"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    for r in reqs:
        P = r["pts"].shape[1]
        assert 100 <= P <= 10000 and r["qsess"].shape == (P,)
        untagged = r["qsess"] == -1
        assert untagged.sum() == P // 2
        assert set(np.unique(r["qsess"][~untagged])) <= {1, 2}
