"""GPU test of the serving loop: a Poisson stream of uneven requests against a
resident three-subdomain overlap (box + two rotated annular cylinders) is
served with continuous batching over several stream slots; every request's
results must equal those of the same request served alone, and agree with the
CPU oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_EVAL_REL, TOL_RST

pytestmark = pytest.mark.gpu


def test_served_results_same_alone_and_in_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_04891_gb300 as fg
    from paper_1811_04891_gb300 import serve
    mesh, iface = synth.box_two_annuli(box_shape=(20, 10, 10), cyl_shape=(16, 3, 16))
    rng = np.random.default_rng(0)
    fields = np.stack([synth.random_poly_field(mesh.coords, 3, rng)[0] for _ in range(4)])
    dev = torch.device("cuda:0")
    h = fg.fp_setup(torch.from_numpy(mesh.coords).to(dev), mesh.N, torch.from_numpy(mesh.sub).to(dev),
                    torch.from_numpy(mesh.dist).to(dev), opts=fg.default_opts(precision=fg.PREC_MIXED))
    fd = torch.from_numpy(fields).to(dev)
    reqs = synth.poisson_requests(iface, 40, seed=9, size_range=(10, 6000), rate_hz=2000.0)

    def make():
        return [serve.Request(rid=i, t_arrive=r["t_arrive"], pts=r["pts"], qsess=r["qsess"])
                for i, r in enumerate(reqs)]

    srv = serve.Server(h, fd, slots=3, slot_points=4096)
    done, makespan = serve.run_stream(srv, make())
    assert len(done) == len(reqs) and srv.launches > 1
    stats = serve.latency_stats(done)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    by_id = {r.rid: r for r in done}
    alone = serve.Server(h, fd, slots=1, slot_points=8192)
    for r in make():
        alone.submit(r)
        while alone.step(0.0):
            pass
        a = alone.completed[-1]
        m = by_id[r.rid]
        np.testing.assert_array_equal(a.code, m.code)
        np.testing.assert_array_equal(a.elem, m.elem)
        np.testing.assert_array_equal(a.rst, m.rst)
        np.testing.assert_array_equal(a.values, m.values)
    # oracle parity on a few requests
    for rid in (0, 7, 21):
        r = by_id[rid]
        ref = oracle.find(mesh.coords, mesh.N, mesh.sub, r.pts, qsess=r.qsess, dist=mesh.dist)
        np.testing.assert_array_equal(r.code, ref["code"])
        np.testing.assert_array_equal(r.elem, ref["elem"])
        ok = ref["code"] != oracle.NOT_FOUND
        assert np.abs(r.rst[:, ok] - ref["rst"][:, ok]).max() <= TOL_RST[1]
        rv = oracle.evaluate(mesh.N, ref["code"], ref["elem"], ref["rst"], fields)
        assert np.array_equal(np.isnan(rv), np.isnan(r.values))
        err = np.nan_to_num(np.abs(rv - r.values)).max() / np.abs(fields).max()
        assert err <= TOL_EVAL_REL
