"""GPU tests of fp_find_eval_host (points and results in host memory,
streamed through the device in chunks): results identical to the device
entry point for several chunk sizes with a ragged last chunk, with and
without session tags and fields, in both forms, from pinned and pageable
memory, when a chunk's candidate pairs overflow the workspace (its RETRY
points are searched again before the call returns), and when a call has far
more pairs per point than the previous call its launches were sized on."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_04891_gb300 as fg
    fg.lib()
    return fg


def _same(dev, host):
    """Bit-for-bit equal, NaN where the other has NaN (points not found)."""
    for a, b in zip(dev, host):
        torch.testing.assert_close(a.cpu(), b, rtol=0, atol=0, equal_nan=True)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("chunk,max_pairs", [(2500, 0), (3000, 0), (4096, 0), (10 ** 6, 0), (2500, 300)])
def test_host_stream_equals_device(fg, prec, chunk, max_pairs):
    mesh, q = synth.cube4_small()
    dev = torch.device("cuda:0")
    h = fg.fp_setup(torch.from_numpy(mesh.coords).to(dev), mesh.N, torch.from_numpy(mesh.sub).to(dev),
                    opts=fg.default_opts(precision=prec))
    pts = np.concatenate([q.pts, synth.near_face_points(mesh.coords, mesh.N, 1500, seed=4),
                          np.array([[1.5, 0.5, 0.5], [np.nan, 0.2, 0.2]]).T], axis=1)
    f = torch.from_numpy(q.fields).to(dev)
    posted = fg.Fields(h, f) if prec == 1 else None
    ref = fg.fp_find_eval(h, torch.from_numpy(np.ascontiguousarray(pts)).to(dev), fields=f, posted=posted)
    ph = torch.from_numpy(np.ascontiguousarray(pts)).pin_memory()
    for _ in range(2):                                   # state kept in the handle: a second call reuses it
        got = fg.fp_find_eval_host(h, ph, fields=f, posted=posted, chunk=chunk, max_pairs=max_pairs)
        _same(ref, got)
    assert (got[0] != fg.RETRY).all()


def test_host_stream_sessions_find_only_pageable(fg):
    mesh, q = synth.box_annulus(n_az=16, n_rad=2, n_ax=4, box_shape=(8, 4, 4), N=5)
    dev = torch.device("cuda:0")
    h = fg.fp_setup(torch.from_numpy(mesh.coords).to(dev), mesh.N, torch.from_numpy(mesh.sub).to(dev),
                    torch.from_numpy(mesh.dist).to(dev))
    qs = torch.from_numpy(q.qsess)
    ref = fg.fp_find(h, torch.from_numpy(q.pts).to(dev), qs.to(dev))
    got = fg.fp_find_eval_host(h, torch.from_numpy(q.pts), qs, chunk=700)       # pageable host memory
    _same(ref, got)
    empty = fg.fp_find_eval_host(h, torch.zeros((3, 0), dtype=torch.float64))
    assert empty[0].numel() == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_host_stream_more_pairs_than_the_previous_call(fg, prec):
    """A call sizes its launches on the previous call's pairs per point; a
    call whose points have several times more candidates (mesh vertices, each
    in the boxes of up to eight elements) than that estimate covers is still
    solved completely, bit-identical to the device entry point."""
    mesh, q = synth.cube4_small()
    dev = torch.device("cuda:0")
    h = fg.fp_setup(torch.from_numpy(mesh.coords).to(dev), mesh.N, torch.from_numpy(mesh.sub).to(dev),
                    opts=fg.default_opts(precision=prec))
    f = torch.from_numpy(q.fields).to(dev)
    posted = fg.Fields(h, f) if prec == 1 else None
    C = 40000
    rng = np.random.default_rng(11)
    few = synth.uniform_points(C, seed=12)
    n = mesh.N + 1
    corners = [i + n * (j + n * k) for i in (0, n - 1) for j in (0, n - 1) for k in (0, n - 1)]
    verts = mesh.coords[:, :, corners].reshape(3, -1)
    many = verts[:, rng.integers(0, verts.shape[1], C)]
    many = np.ascontiguousarray(many)
    fg.fp_find(h, torch.from_numpy(few).to(dev))
    pairs_few = fg.fp_last_find_stats(h)
    ref = fg.fp_find_eval(h, torch.from_numpy(many).to(dev), fields=f, posted=posted)
    pairs_many = fg.fp_last_find_stats(h)
    assert pairs_many > 1.125 * pairs_few + 4096 + C      # beyond what the first call's estimate covers
    kw = dict(fields=f, posted=posted, chunk=C, max_pairs=10 * C)
    fg.fp_find_eval_host(h, torch.from_numpy(few).pin_memory(), **kw)
    got = fg.fp_find_eval_host(h, torch.from_numpy(many).pin_memory(), **kw)
    _same(ref, got)
    assert (got[0] != fg.RETRY).all()
