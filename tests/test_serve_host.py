"""CPU tests of the serving loop's host logic: memory-budget admission, the
continuous-batching packer and the scatter of slot results back to their
requests.  A fake device computes each point's results from the point itself
(in the slot buffer), slots finish out of order, and every request must get
back exactly the results of its own points, once."""
import collections

import numpy as np
import pytest

from paper_1811_04891_gb300 import serve


def test_chunk_capacity_and_io_bytes():
    assert [serve.chunk_capacity(n, 1 << 17) for n in (1, 2, 3, 4096, 4097, 1 << 17, 10 ** 6)] == \
        [1, 2, 4, 4096, 8192, 1 << 17, 1 << 17]
    assert serve.io_bytes(1000, 4) == 1000 * (24 + 4 + 12 + 24 + 8 + 32)


class _Q:
    def __init__(self, P, taken=0):
        self.P, self.next_pt = P, taken


def test_admit_by_memory():
    per = 100                                   # bytes per point of capacity
    bf = lambda cap: per * cap + 1000           # noqa: E731
    big = collections.deque([_Q(10 ** 6)])
    # room for a full chunk: a full chunk
    assert serve.admit(big, 1 << 17, 1 << 12, bf(1 << 17), bf) == 1 << 17
    # room for less: the largest power of two that fits, not below min_chunk
    assert serve.admit(big, 1 << 17, 1 << 12, bf(1 << 15) + 5, bf) == 1 << 15
    assert serve.admit(big, 1 << 17, 1 << 12, bf(1 << 12) - 1, bf) == 0        # held back
    # a small head request is admitted whole when its capacity fits
    small = collections.deque([_Q(300)])
    assert serve.admit(small, 1 << 17, 1 << 12, bf(512), bf) == 300
    assert serve.admit(small, 1 << 17, 1 << 12, bf(512) - 1, bf) == 0          # 256 < the request
    # several requests: their total, up to a chunk
    many = collections.deque([_Q(3000), _Q(5000, 1000), _Q(100)])
    assert serve.admit(many, 1 << 17, 1 << 12, 1e12, bf) == 3000 + 4000 + 100
    assert serve.admit(collections.deque(), 1 << 17, 1 << 12, 1e12, bf) == 0


def test_budget_holds_work_back_and_every_request_gets_its_results():
    """A fake device with memory accounting: chunks are admitted only while
    their bytes fit the budget, requests that arrive while memory is taken
    wait and are admitted when chunks complete, and every request gets back
    exactly its own points' results."""
    rng = np.random.default_rng(7)
    per = 100
    bf = lambda cap: per * cap                  # noqa: E731
    chunk, min_chunk = 1 << 12, 1 << 8
    avail = 2.5 * bf(chunk)                     # two full chunks, or one and smaller ones
    reqs = [_request(i, float(i), int(P), rng) for i, P in enumerate(rng.integers(1, 3 * chunk, 60))]
    pending, completed, inflight = collections.deque(), [], []
    held = peak = 0
    arrivals = list(reqs)
    tick = 0
    while arrivals or pending or inflight:
        tick += 1
        for _ in range(int(rng.integers(0, 4))):
            if arrivals:
                pending.append(arrivals.pop(0))
        keep = []
        for c in inflight:                       # chunks complete in random order
            if rng.random() < 0.4:
                code, elem, rst, values = _device(c["pts"][:, :c["n"]], c["qs"][:c["n"]])
                serve.scatter_results(c["pieces"], code, elem, rst, values, float(tick), completed)
            else:
                keep.append(c)
        inflight = keep
        while pending and len(inflight) < 4:
            used = sum(bf(c["cap"]) for c in inflight)
            n = serve.admit(pending, chunk, min_chunk, avail - used, bf)
            if n == 0:
                held += 1
                break
            cap = serve.chunk_capacity(n, chunk)
            c = {"cap": cap, "pts": np.zeros((3, cap)), "qs": np.zeros(cap, np.int32)}

            def copy_in(req, lo, so, take, c=c):
                c["pts"][:, so:so + take] = req.pts[:, lo:lo + take]
                c["qs"][so:so + take] = req.qsess[lo:lo + take]
            c["pieces"], c["n"] = serve.pack_pending(pending, n, copy_in)
            assert c["n"] == n <= cap
            inflight.append(c)
            peak = max(peak, sum(bf(x["cap"]) for x in inflight))
        assert tick < 100000
    assert peak <= avail and held > 0
    assert sorted(r.rid for r in completed) == list(range(len(reqs)))
    for r in reqs:
        code, elem, rst, values = _device(r.pts, r.qsess)
        np.testing.assert_array_equal(r.code, code)
        np.testing.assert_array_equal(r.values, values)


def _request(rid, t, P, rng):
    r = serve.Request(rid=rid, t_arrive=t, pts=rng.uniform(0, 1, (3, P)), qsess=rng.integers(-1, 3, P).astype(np.int32))
    r.code = np.full(P, -7, np.int32)
    r.elem = np.full(P, -7, np.int32)
    r.rst = np.full((3, P), np.nan)
    r.values = np.full((2, P), np.nan)
    return r


def _device(pts, qs):
    """Stand-in for find + eval: results that depend on each point only."""
    code = (np.floor(pts[0] * 3).astype(np.int32) + qs) % 3
    elem = np.floor(pts[1] * 1000).astype(np.int32) + 7 * qs
    rst = 2 * pts - 1
    values = np.stack([pts.sum(0), pts[2] * qs])
    return code, elem, rst, values


@pytest.mark.parametrize("seed,capacity,nslots", [(0, 1000, 3), (1, 64, 1), (2, 4096, 4), (3, 1, 2)])
def test_pack_and_scatter_return_each_point_its_own_results(seed, capacity, nslots):
    rng = np.random.default_rng(seed)
    sizes = list(rng.integers(1, 3 * capacity + 2, 40)) + [1, capacity, capacity + 1, 5 * capacity]
    reqs = [_request(i, float(i), int(P), rng) for i, P in enumerate(sizes)]
    pending = collections.deque()
    completed = []
    slots = [{"busy": False, "pts": np.zeros((3, capacity)), "qs": np.zeros(capacity, np.int32)}
             for _ in range(nslots)]
    first_packed = {}
    arrivals = list(reqs)
    tick = 0
    while arrivals or pending or any(s["busy"] for s in slots):
        tick += 1
        for _ in range(int(rng.integers(0, 4))):            # requests arrive while slots are busy
            if arrivals:
                pending.append(arrivals.pop(0))
        for s in slots:                                      # slots finish in random order
            if s["busy"] and rng.random() < 0.5:
                n = s["n"]
                code, elem, rst, values = _device(s["pts"][:, :n], s["qs"][:n])
                serve.scatter_results(s["pieces"], code, elem, rst, values, float(tick), completed)
                s["busy"] = False
        for s in slots:
            if not s["busy"] and pending:
                def copy_in(req, lo, so, take, s=s):
                    s["pts"][:, so:so + take] = req.pts[:, lo:lo + take]
                    s["qs"][so:so + take] = req.qsess[lo:lo + take]
                pieces, n = serve.pack_pending(pending, capacity, copy_in)
                assert 0 < n <= capacity and sum(p[3] for p in pieces) == n
                slot_los = [p[2] for p in pieces]
                assert slot_los == sorted(slot_los) and slot_los[0] == 0
                for req, lo, so, take in pieces:
                    first_packed.setdefault(req.rid, tick * 1000 + len(first_packed))
                s.update(busy=True, pieces=pieces, n=n)
        assert tick < 100000
    # every request completed exactly once, with its own points' results
    assert sorted(r.rid for r in completed) == list(range(len(reqs)))
    for r in reqs:
        assert r.done_pts == r.P and r.next_pt == r.P and r.t_done is not None
        code, elem, rst, values = _device(r.pts, r.qsess)
        np.testing.assert_array_equal(r.code, code)
        np.testing.assert_array_equal(r.elem, elem)
        np.testing.assert_array_equal(r.rst, rst)
        np.testing.assert_array_equal(r.values, values)
    # first-come first-served: a request starts no later than the ones after it
    order = [first_packed[r.rid] for r in reqs]
    assert order == sorted(order)


def test_large_request_spans_slots_in_order():
    rng = np.random.default_rng(5)
    big = _request(0, 0.0, 2500, rng)
    small = _request(1, 0.0, 10, rng)
    pending = collections.deque([big, small])
    got = []
    for _ in range(3):
        pieces, n = serve.pack_pending(pending, 1000, lambda *a: None)
        got.append([(p[0].rid, p[1], p[2], p[3]) for p in pieces])
    assert got == [[(0, 0, 0, 1000)], [(0, 1000, 0, 1000)], [(0, 2000, 0, 500), (1, 0, 500, 10)]]
    assert not pending


def test_copied_chunks_complete_requests_at_their_latest_copy():
    """Results copied on several threads: chunks of one request copied out
    of order, concurrently; the request completes once, stamped with the
    latest copy's time, with every point's results in place."""
    from concurrent.futures import ThreadPoolExecutor
    P, n = 10_000, 1024
    req = serve.Request(0, 0.0, np.zeros((3, P)), np.zeros(P, np.int32))
    req.code, req.elem = np.empty(P, np.int32), np.empty(P, np.int32)
    req.rst, req.values = np.empty((3, P)), np.empty((2, P))
    chunks = []
    for lo in range(0, P, n):
        take = min(n, P - lo)
        ids = np.arange(lo, lo + take)
        chunks.append(([(req, lo, 0, take)], ids.astype(np.int32), -ids.astype(np.int32),
                       np.stack([ids * 1.0, ids * 2.0, ids * 3.0]), np.stack([ids + 0.5, ids - 0.5])))
    order = list(np.random.default_rng(3).permutation(len(chunks)))
    with ThreadPoolExecutor(4) as ex:
        futs = [ex.submit(serve.copy_results, *chunks[k]) for k in order]
        for f in futs:
            f.result()
    completed = []
    times = [7.0, 2.0, 9.5] + [1.0] * (len(chunks) - 3)
    for k, t in zip(order, times):
        assert req.t_done is None
        serve.account(chunks[k][0], t, completed)
    assert completed == [req] and req.t_done == 9.5 and req.done_pts == P
    ids = np.arange(P)
    np.testing.assert_array_equal(req.code, ids)
    np.testing.assert_array_equal(req.elem, -ids)
    np.testing.assert_array_equal(req.rst, np.stack([ids * 1.0, ids * 2.0, ids * 3.0]))
    np.testing.assert_array_equal(req.values, np.stack([ids + 0.5, ids - 0.5]))
