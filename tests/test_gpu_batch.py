"""GPU tests of the batched form: many independent deformed-box instances of
different E and N in one run must give, instance by instance, exactly what
fp_find + fp_eval give alone, and agree with the CPU oracle; the autotuned
schedule and the captured CUDA graph must not change any result."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_EVAL_REL, TOL_RST

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_04891_gb300 as fg
    fg.lib()
    return fg


_MIXED = set()


def h_mixed(fg, h):
    return id(h) in _MIXED


def _instances(n_inst, seed, prec, fg, with_empty=False):
    insts = synth.instance_batch(n_inst=n_inst, seed=seed, E_range=(8, 300), P_range=(50, 4000))
    dev = torch.device("cuda:0")
    handles, fields, pts = [], [], []
    for k, (mesh, q) in enumerate(insts):
        handles.append(fg.fp_setup(torch.from_numpy(mesh.coords).to(dev), mesh.N, torch.from_numpy(mesh.sub).to(dev),
                                   opts=fg.default_opts(precision=prec)))
        if prec == fg.PREC_MIXED:
            _MIXED.add(id(handles[-1]))
        fields.append(torch.from_numpy(q.fields).to(dev))
        p = q.pts if not (with_empty and k == 1) else np.zeros((3, 0))
        pts.append(p)
    return insts, handles, fields, pts


def _check_against_single(fg, insts, handles, fields, pts, outs):
    code, sub, elem, rst, d2, val = [x.cpu().numpy() for x in outs]
    off = np.concatenate([[0], np.cumsum([p.shape[1] for p in pts])])
    dev = torch.device("cuda:0")
    for k, h in enumerate(handles):
        if pts[k].shape[1] == 0:
            continue
        t = torch.from_numpy(np.ascontiguousarray(pts[k])).to(dev)
        r = fg.fp_find(h, t)
        if h_mixed(fg, h):   # the mixed form evaluates with double-float fields
            v = fg.fp_eval_df(h, fg.Fields(h, fields[k]), r[0], r[2], r[3]).cpu().numpy()
        else:
            v = fg.fp_eval(h, r[0], r[2], r[3], fields[k]).cpu().numpy()
        r = [x.cpu().numpy() for x in r]
        sl = slice(off[k], off[k + 1])
        np.testing.assert_array_equal(code[sl], r[0])
        np.testing.assert_array_equal(sub[sl], r[1])
        np.testing.assert_array_equal(elem[sl], r[2])
        np.testing.assert_array_equal(rst[:, sl], r[3])
        np.testing.assert_array_equal(d2[sl], r[4])
        np.testing.assert_array_equal(val[:, sl], v)


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_equals_single_instance_runs(fg, prec):
    insts, handles, fields, pts = _instances(9, 31, prec, fg, with_empty=True)
    assert len({m.N for m, _ in insts}) > 1
    batch = fg.Batch(handles, [p.shape[1] for p in pts], fields)
    allp = torch.from_numpy(np.ascontiguousarray(np.concatenate(pts, axis=1))).cuda()
    outs = batch.run(allp, batch.outputs())
    torch.cuda.synchronize()
    _check_against_single(fg, insts, handles, fields, pts, outs)
    # and against the oracle on two instances
    code, sub, elem, rst, d2, val = [x.cpu().numpy() for x in outs]
    off = np.concatenate([[0], np.cumsum([p.shape[1] for p in pts])])
    for k in (0, len(insts) - 1):
        mesh, q = insts[k]
        ref = oracle.find(mesh.coords, mesh.N, mesh.sub, pts[k])
        sl = slice(off[k], off[k + 1])
        np.testing.assert_array_equal(code[sl], ref["code"])
        np.testing.assert_array_equal(elem[sl], ref["elem"])
        assert np.abs(rst[:, sl] - ref["rst"]).max() <= TOL_RST[prec]
        rv = oracle.evaluate(mesh.N, ref["code"], ref["elem"], ref["rst"], q.fields)
        assert np.abs(val[:, sl] - rv).max() <= TOL_EVAL_REL * np.abs(q.fields).max()


def test_batch_tune_and_graph_replay(fg):
    insts, handles, fields, pts = _instances(7, 32, 1, fg)
    batch = fg.Batch(handles, [p.shape[1] for p in pts], fields)
    allp = torch.from_numpy(np.ascontiguousarray(np.concatenate(pts, axis=1))).cuda()
    outs = batch.outputs()
    ms = batch.tune(allp, outs, reps=1)
    assert ms > 0
    scheds = []
    for g in range(batch.groups()):
        blk, bps, tile = batch.schedule(g)
        assert blk in (64, 128, 256) and bps in (1, 2, 4, 8) and tile in (32, 128, 512)
        scheds.append((blk, bps, tile))
        info = batch.group_info(g)
        assert info["N"] in (5, 7, 9) and info["pairs"] >= info["P"] > 0 and info["newton_ms"] > 0
    # both modes give the same results
    mode = batch.mode()
    ref_mode = [x.clone() for x in batch.run(allp, batch.outputs())]
    batch.mode(1 - mode)
    other = batch.run(allp, batch.outputs())
    torch.cuda.synchronize()
    for a, c in zip(ref_mode, other):
        assert torch.equal(a, c)
    batch.mode(mode)
    # a second batch over the same instances takes the cached schedules
    again = fg.Batch(handles, [p.shape[1] for p in pts], fields)
    again.tune(allp, again.outputs(), reps=1)
    assert [again.schedule(g) for g in range(again.groups())] == scheds
    ref = [x.clone() for x in batch.run(allp, batch.outputs())]
    batch.capture(allp, outs)
    for x in outs:
        x.zero_()
    k0 = fg.fp_launch_count()
    batch.launch()
    torch.cuda.synchronize()
    # one graph: screen, scan, emit, sort, per group Newton (+ fallback) and eval, classification
    assert fg.fp_launch_count() - k0 <= 12 + 3 * batch.groups()
    for a, b in zip(ref, outs):
        assert torch.equal(a, b)
    # new contents in the captured input buffer
    pts2 = [synth.uniform_points(p.shape[1], seed=900 + k) for k, p in enumerate(pts)]
    allp.copy_(torch.from_numpy(np.concatenate(pts2, axis=1)))
    batch.launch()
    torch.cuda.synchronize()
    _check_against_single(fg, insts, handles, fields, pts2, outs)


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_with_overlapping_subdomains(fg, prec):
    """Instances with several subdomains (the owner rule, each instance with
    its own tie band) beside single-subdomain ones: every result equals the
    instance's own fp_find bit for bit and the oracle's at the tolerances."""
    dev = torch.device("cuda:0")
    overlap = synth.tiny_overlap(N=4)
    annulus, _ = synth.box_annulus(n_az=12, n_rad=2, n_ax=3, box_shape=(6, 3, 3), N=5)
    plain = synth.Mesh(coords=synth.box_mesh((3, 2, 2), 5, amp_frac=0.1), N=5, sub=np.zeros(12, np.int32))
    meshes = [overlap, annulus, plain]
    rng = np.random.default_rng(41)
    xs = np.concatenate([rng.uniform(-0.05, 2.05, 700), [0.8, 0.8, 1.0]])
    pts = [np.stack([xs, rng.uniform(0.02, 0.98, xs.size), rng.uniform(0.02, 0.98, xs.size)]),
           np.stack([rng.uniform(0.0, 2.0, 900), rng.uniform(0.0, 1.0, 900), rng.uniform(0.0, 1.0, 900)]),
           synth.uniform_points(500, seed=42)]
    handles = [fg.fp_setup(torch.from_numpy(m.coords).to(dev), m.N, torch.from_numpy(m.sub).to(dev),
                           None if m.dist is None else torch.from_numpy(m.dist).to(dev),
                           opts=fg.default_opts(precision=prec)) for m in meshes]
    batch = fg.Batch(handles, [p.shape[1] for p in pts])
    allp = torch.from_numpy(np.ascontiguousarray(np.concatenate(pts, axis=1))).to(dev)
    outs = [x.cpu().numpy() for x in batch.run(allp, batch.outputs())]
    off = np.concatenate([[0], np.cumsum([p.shape[1] for p in pts])])
    for k, (m, h) in enumerate(zip(meshes, handles)):
        sl = slice(off[k], off[k + 1])
        single = [x.cpu().numpy() for x in fg.fp_find(h, torch.from_numpy(np.ascontiguousarray(pts[k])).to(dev))]
        for a, b in zip(outs[:4], single[:4]):
            np.testing.assert_array_equal(a[..., sl], b)
        np.testing.assert_array_equal(outs[4][sl], single[4])
        ref = oracle.find(m.coords, m.N, m.sub, pts[k], dist=m.dist)
        np.testing.assert_array_equal(outs[0][sl], ref["code"])
        np.testing.assert_array_equal(outs[1][sl], ref["sub"])
        np.testing.assert_array_equal(outs[2][sl], ref["elem"])
        found = ref["code"] != oracle.NOT_FOUND
        assert np.abs(outs[3][:, sl][:, found] - ref["rst"][:, found]).max() <= TOL_RST[prec]
    assert set(np.unique(outs[1][off[1]:off[2]][outs[0][off[1]:off[2]] == 0])) == {0, 1}
    # the two points at x = 0.8 tie between the first and second box (lower id wins)
    assert batch.band_hits()["owner"] == 2
