"""GPU parity at the benchmark's full sizes, in the launch configurations the
benchmark times.  The deformed 32^3 cube (N = 7, 32,768 elements) with
1e7 uniform + 1e5 near-face points and five fields, one fused find + eval
call per form on a reserved handle (the mixed form with its fields posted as
double-float pairs); and the 64-instance batch in its captured graph.

Two checks.  (1) Sampled outputs against the oracle, computed one by one: a
strided sample of the whole range, the last 1000 points (the near-face block
and the ragged end) and 1000 random ones; codes, subdomains and elements bit
for bit, |delta r| and values within the tolerances of the smaller parity
tests.  (2) Every output, through properties that hold at any size: every
point lies in the mesh, so every code is INSIDE; and the forward map x^e(r),
evaluated by the oracle at each returned (e, r), gives the point back."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_EVAL_REL, TOL_RST, assert_parity

pytestmark = pytest.mark.gpu

# |x^e(r) - x*| over all points: the Newton tolerance in r (<= 1e-12 FP64,
# <= 1e-10 mixed) times |dx/dr| = h/2 = 1/64, with room for rounding
TOL_MAP = {0: 1e-12, 1: 1e-11}
TOL_MAP_BATCH = {0: 1e-12, 1: 2e-11}     # elements up to 1/4 wide: |dx/dr| <= 1/8


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_04891_gb300 as fg
    fg.lib()
    mesh, q = synth.deformed_cube()
    P = q.P
    rng = np.random.default_rng(2024)
    idx = np.unique(np.concatenate([np.arange(0, P, P // 4000), np.arange(P - 1000, P),
                                    rng.integers(0, P, 1000)]))
    pts_s = np.ascontiguousarray(q.pts[:, idx])
    ref = oracle.find(mesh.coords, mesh.N, mesh.sub, pts_s)
    ref["eval"] = oracle.evaluate(mesh.N, ref["code"], ref["elem"], ref["rst"], q.fields)
    return fg, mesh, q, idx, ref


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_bench_configuration(full, prec):
    fg, mesh, q, idx, ref = full
    dev = torch.device("cuda:0")
    P, F = q.P, q.fields.shape[0]
    coords = torch.from_numpy(mesh.coords).to(dev)
    fields = torch.from_numpy(q.fields).to(dev)
    pts = torch.from_numpy(q.pts).to(dev)
    h = fg.fp_setup(coords, mesh.N, torch.from_numpy(mesh.sub).to(dev), opts=fg.default_opts(precision=prec))
    fg.fp_reserve(h, P)
    posted = fg.Fields(h, fields) if prec == fg.PREC_MIXED else None
    outs = (torch.empty(P, dtype=torch.int32, device=dev), torch.empty(P, dtype=torch.int32, device=dev),
            torch.empty(P, dtype=torch.int32, device=dev), torch.empty((3, P), dtype=torch.float64, device=dev),
            torch.empty(P, dtype=torch.float64, device=dev))
    vals = torch.empty((F, P), dtype=torch.float64, device=dev)
    for _ in range(2):                      # a warm call, then the call checked, as the benchmark steps
        fg.fp_find_eval(h, pts, None, fields=fields, posted=posted, out=outs, values=vals)
    torch.cuda.synchronize()
    code, sub, elem, rst = (t.cpu().numpy() for t in outs[:4])
    dist2 = outs[4].cpu().numpy()
    out = vals.cpu().numpy()

    # (1) sampled outputs against the oracle
    g = {"code": code[idx], "sub": sub[idx], "elem": elem[idx], "rst": rst[:, idx], "dist2": dist2[idx],
         "eval": out[:, idx]}
    assert (ref["code"] == oracle.INSIDE).all()
    drst = assert_parity(g, ref, prec, fields=q.fields)
    assert drst <= TOL_RST[prec]

    # (2) every output
    assert (code == oracle.INSIDE).all()
    x = oracle.evaluate(mesh.N, code, elem, rst, mesh.coords)
    res = np.abs(x - q.pts).max()
    assert res <= TOL_MAP[prec], f"max |x(e, r) - x*| = {res:.3e}"
    assert np.isfinite(out).all()
    # no decision of either call fell near a threshold or a tie band
    assert fg.fp_band_hits(h) == {"accept": 0, "border": 0, "owner": 0}
    del h


@pytest.fixture(scope="module")
def batch_full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_04891_gb300 as fg
    fg.lib()
    return fg, synth.instance_batch()


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_batched_configuration(batch_full, prec):
    """The batched workload at full size (64 deformed-cube instances, E from
    64 to 8192, N in {5, 7, 9}, 7.8e6 points) run as the benchmark runs it:
    schedule autotuned, one captured graph replayed.  Per instance, 60 strided
    points and its last one against the oracle; every output by code INSIDE
    and the forward map (|dx/dr| <= h/2 <= 1/8 here)."""
    fg, insts = batch_full
    dev = torch.device("cuda:0")
    pts = torch.from_numpy(np.ascontiguousarray(np.concatenate([q.pts for _, q in insts], axis=1))).to(dev)
    fields = [torch.from_numpy(q.fields).to(dev) for _, q in insts]
    handles = [fg.fp_setup(torch.from_numpy(m.coords).to(dev), m.N, torch.from_numpy(m.sub).to(dev),
                           opts=fg.default_opts(precision=prec)) for m, _ in insts]
    b = fg.Batch(handles, [q.P for _, q in insts], fields)
    outs = b.outputs(dev)
    b.tune(pts, outs, reps=1)
    b.capture(pts, outs)
    for _ in range(2):
        b.launch()
    torch.cuda.synchronize()
    code, sub, elem, rst, d2, val = [x.cpu().numpy() for x in outs]
    assert (code == oracle.INSIDE).all()
    off = np.concatenate([[0], np.cumsum([q.P for _, q in insts])])
    worst_map = 0.0
    for k, (mesh, q) in enumerate(insts):
        lo, hi = off[k], off[k + 1]
        s = np.unique(np.concatenate([np.linspace(0, q.P - 1, min(60, q.P)).astype(np.int64), [q.P - 1]]))
        ref = oracle.find(mesh.coords, mesh.N, mesh.sub, np.ascontiguousarray(q.pts[:, s]))
        g = lo + s
        np.testing.assert_array_equal(code[g], ref["code"])
        np.testing.assert_array_equal(sub[g], ref["sub"])
        np.testing.assert_array_equal(elem[g], ref["elem"])
        assert np.abs(rst[:, g] - ref["rst"]).max() <= TOL_RST[prec]
        rv = oracle.evaluate(mesh.N, ref["code"], ref["elem"], ref["rst"], q.fields)
        assert np.abs(val[:, g] - rv).max() <= TOL_EVAL_REL * np.abs(q.fields).max()
        x = oracle.evaluate(mesh.N, code[lo:hi], elem[lo:hi], rst[:, lo:hi], mesh.coords)
        worst_map = max(worst_map, float(np.abs(x - q.pts).max()))
    assert worst_map <= TOL_MAP_BATCH[prec], f"max |x(e, r) - x*| = {worst_map:.3e}"
    assert b.band_hits() == {"accept": 0, "border": 0, "owner": 0}
    del b, handles
