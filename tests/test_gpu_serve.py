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

    srv = serve.Server(h, fd, chunk_points=4096, streams=3)
    done, makespan = serve.run_stream(srv, make())
    assert len(done) == len(reqs) and srv.launches > 1
    stats = serve.latency_stats(done)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    by_id = {r.rid: r for r in done}
    # alone: one stream, results copied by the dispatcher itself (no copier threads)
    alone = serve.Server(h, fd, chunk_points=8192, streams=1, copy_threads=0)
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


@pytest.mark.parametrize("prec", [0, 1])
def test_memory_budget_holds_requests_back(prec):
    """A budget with room for little more than one chunk beside the resident
    mesh: requests that arrive while it is taken are held back and admitted
    as chunks complete; the memory in flight never exceeds the budget, and
    every result equals the same request served alone."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_04891_gb300 as fg
    from paper_1811_04891_gb300 import serve
    mesh, iface = synth.box_two_annuli(box_shape=(12, 6, 6), cyl_shape=(12, 2, 8))
    rng = np.random.default_rng(2)
    fields = np.stack([synth.random_poly_field(mesh.coords, 3, rng)[0] for _ in range(2)])
    dev = torch.device("cuda:0")
    h = fg.fp_setup(torch.from_numpy(mesh.coords).to(dev), mesh.N, torch.from_numpy(mesh.sub).to(dev),
                    torch.from_numpy(mesh.dist).to(dev), opts=fg.default_opts(precision=prec))
    fd = torch.from_numpy(fields).to(dev)
    resident = fd.numel() * 8
    chunk = 2048
    probe = serve.Server(h, fd, chunk_points=chunk)
    budget = resident + fg.fp_memory(h)["resident"] + 1.5 * probe.bytes_for(chunk)
    reqs = synth.poisson_requests(iface, 30, seed=3, size_range=(50, 5000), rate_hz=20000.0)

    def make():
        return [serve.Request(rid=i, t_arrive=r["t_arrive"], pts=r["pts"], qsess=r["qsess"])
                for i, r in enumerate(reqs)]

    srv = serve.Server(h, fd, budget_bytes=budget, resident_bytes=resident, chunk_points=chunk, streams=4,
                       min_chunk=256)
    done, _ = serve.run_stream(srv, make())
    assert len(done) == len(reqs)
    assert srv.held_back > 0
    assert 0 < srv.peak_inflight_bytes <= budget - srv.resident
    alone = serve.Server(h, fd, chunk_points=8192, streams=1)
    by_id = {r.rid: r for r in done}
    for r in make():
        alone.submit(r)
        while alone.step(0.0):
            pass
        a, m = alone.completed[-1], by_id[r.rid]
        np.testing.assert_array_equal(a.code, m.code)
        np.testing.assert_array_equal(a.elem, m.elem)
        np.testing.assert_array_equal(a.rst, m.rst)
        np.testing.assert_array_equal(a.values, m.values)
    r = by_id[5]
    ref = oracle.find(mesh.coords, mesh.N, mesh.sub, r.pts, qsess=r.qsess, dist=mesh.dist)
    np.testing.assert_array_equal(r.code, ref["code"])
    np.testing.assert_array_equal(r.elem, ref["elem"])
