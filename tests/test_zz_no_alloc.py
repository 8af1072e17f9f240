"""fp_find_static: the allocation-free variant of fp_find.

It serves callers that cannot allocate device memory when they locate points
(a solver whose device memory is all in its own pool allocator, a time-step
loop that cannot take the device-wide synchronisation of cudaMalloc/cudaFree).
Its scratch is a fixed device array inside the library.  This test calls it
through the C ABI twice in a row, on different point sets, and checks each
result against fp_find on the same handle and against the CPU oracle, with
the tolerances of the other GPU tests; it also checks that requests over the
point limit and over the pair limit are refused and that the next call is
still right.  Collected last so that a failure here does not hide the rest of
the suite; it needs nothing from the other tests.
"""
import numpy as np
import pytest
import torch

import synth
from gpu_util import TOL_RST, assert_parity, oracle_find

pytestmark = pytest.mark.gpu


def _both(fg, h, pts):
    dev = torch.device("cuda:0")
    t = torch.from_numpy(np.ascontiguousarray(pts)).to(dev)
    ref = [x.cpu().numpy() for x in fg.fp_find(h, t)]
    got = [x.cpu().numpy() for x in fg.fp_find_static(h, t)]
    torch.cuda.synchronize()
    return ref, got


def _setup(fg, mesh, prec):
    dev = torch.device("cuda:0")
    return fg.fp_setup(torch.from_numpy(mesh.coords).to(dev), mesh.N, torch.from_numpy(mesh.sub).to(dev),
                       opts=fg.default_opts(precision=prec))


@pytest.mark.parametrize("prec", [0, 1])
def test_static_find_matches_fp_find_and_oracle_on_two_calls(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_04891_gb300 as fg
    mesh, q = synth.deformed_cube(ne=6, P_uniform=12007, P_face=2003, with_fields=False)
    h = _setup(fg, mesh, prec)
    first = q.pts
    second = synth.uniform_points(5001, seed=77, lo=(-0.05, -0.05, -0.05), hi=(1.05, 1.05, 1.05))
    for pts in (first, second):
        (c0, s0, e0, r0, d0), (c1, s1, e1, r1, d1) = _both(fg, h, pts)
        np.testing.assert_array_equal(c1, c0)
        np.testing.assert_array_equal(s1, s0)
        np.testing.assert_array_equal(e1, e0)
        assert np.abs(r1 - r0).max() <= TOL_RST[prec]
        fin = np.isfinite(d0)
        np.testing.assert_array_equal(fin, np.isfinite(d1))
        assert np.abs(np.sqrt(d1[fin]) - np.sqrt(d0[fin])).max() <= 1e-12
        assert fg.fp_last_find_stats(h) >= pts.shape[1] // 2
        # the static call against the oracle directly
        g = {"code": c1, "sub": s1, "elem": e1, "rst": r1, "dist2": d1}
        assert_parity(g, oracle_find(mesh, pts), prec)
    assert (c0 == fg.NOT_FOUND).any() and (c0 == fg.INSIDE).any()
    assert fg.fp_band_hits(h) == {"accept": 0, "border": 0, "owner": 0}


@pytest.mark.parametrize("prec", [0, 1])
def test_static_find_refuses_oversized_requests(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_04891_gb300 as fg
    dev = torch.device("cuda:0")
    N = 3
    coords = synth.box_mesh((8, 8, 8), N)
    mesh = synth.Mesh(coords=coords, N=N, sub=np.zeros(coords.shape[1], np.int32))
    h = _setup(fg, mesh, prec)
    too_many = torch.zeros((3, fg.STATIC_MAX_POINTS + 1), dtype=torch.float64, device=dev)
    with pytest.raises(fg.FindptsError) as ei:
        fg.fp_find_static(h, too_many)
    assert ei.value.status == fg.FP_ERR_INVALID_ARG
    # points on the interior vertices of the 8^3 grid: each lies in 8 elements'
    # boxes, so 16384 of them give about 131k candidate pairs, over the limit
    v = np.arange(1, 8) / 8.0
    X, Y, Z = np.meshgrid(v, v, v, indexing="ij")
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    reps = np.resize(np.arange(verts.shape[1]), fg.STATIC_MAX_POINTS)
    crowded = torch.from_numpy(np.ascontiguousarray(verts[:, reps])).to(dev)
    with pytest.raises(fg.FindptsError) as ei:
        fg.fp_find_static(h, crowded)
    assert ei.value.status == fg.FP_ERR_INVALID_ARG
    assert fg.fp_last_find_stats(h) > fg.STATIC_MAX_PAIRS
    # the next ordinary call still matches fp_find and the oracle
    pts = synth.uniform_points(4001, seed=5, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0))
    (c0, s0, e0, r0, d0), (c1, s1, e1, r1, d1) = _both(fg, h, pts)
    np.testing.assert_array_equal(c1, c0)
    np.testing.assert_array_equal(e1, e0)
    assert np.abs(r1 - r0).max() <= TOL_RST[prec]
    assert_parity({"code": c1, "sub": s1, "elem": e1, "rst": r1, "dist2": d1}, oracle_find(mesh, pts), prec)
