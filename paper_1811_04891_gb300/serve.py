"""Serving loop: point-location / interpolation requests against resident meshes.

The mesh, its hash grid and the fields stay resident on the device (one
handle).  Requests of uneven size arrive over time and are served with
continuous batching under a device-memory budget:

* Work is cut into chunks of at most `chunk_points` points: whole small
  requests packed together, or bounded pieces of a large one, taken in
  arrival order.
* A chunk holds device memory while it is in flight -- its points, tags,
  outputs and values, and an fp_workspace for its candidate pairs (bytes from
  chunk_bytes / fp_workspace_bytes).  It is admitted only when those bytes fit
  in what is left of the budget: budget - resident mesh - chunks in flight.
  With less room than a full chunk, a smaller chunk (never below
  `min_chunk` points, or the whole head request if smaller) is admitted
  instead; with less than that, the pending work waits until a chunk
  completes and frees its memory ("held back").
* Admitted chunks run on a pool of CUDA streams (copy in from pinned memory,
  fp_find_eval_ws, copy out), so the work of requests that arrived at
  different times overlaps on the device.  Buffers and workspaces are kept in
  pools by capacity (a power of two) and reused; the pools never hold more
  than the largest set of chunks the budget has let run at once.
* A finished chunk's results are copied from its pinned buffers into the
  requests on a few host threads (`copy_threads`; numpy copies release the
  GIL), so the dispatcher keeps admitting and launching meanwhile.  The
  chunk's buffers, and the device bytes they count for, go back to the pool
  when that copy is done.
* A request completes when all its chunks are back; latency = completion -
  arrival.

Every point is located and interpolated independently of what else shares
its launch, so a request's results are the same alone and in the mix.
"""
from __future__ import annotations

import collections
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np
import torch

import paper_1811_04891_gb300 as fg


@dataclass
class Request:
    rid: int
    t_arrive: float
    pts: np.ndarray                       # [3][P] float64
    qsess: np.ndarray                     # [P] int32
    code: np.ndarray = None
    elem: np.ndarray = None
    rst: np.ndarray = None
    values: np.ndarray = None             # [F][P]
    done_pts: int = 0
    next_pt: int = 0
    t_last: Optional[float] = None
    t_done: Optional[float] = None

    @property
    def P(self) -> int:
        return int(self.pts.shape[1])


def io_bytes(n: int, F: int) -> int:
    """Device bytes of a chunk's own buffers for n points and F fields:
    points (24), tags (4), code / sub / elem (12), r (24), dist^2 (8) and the
    values (8 F) per point."""
    return n * (24 + 4 + 12 + 24 + 8 + 8 * F)


def chunk_capacity(n: int, chunk_points: int) -> int:
    """Buffer class of a chunk of n points: the next power of two, at most
    chunk_points (chunks are never larger)."""
    c = 1
    while c < n:
        c <<= 1
    return min(c, chunk_points)


def admit(pending, chunk_points: int, min_chunk: int, avail: float, bytes_for) -> int:
    """Memory-budget admission of the next chunk: the points to take now from
    the head of `pending` -- a full chunk when its bytes fit in `avail`,
    else the largest power-of-two capacity that fits (at least min_chunk
    points, or the rest of the pending work if that is smaller), else 0 (the
    work waits).  bytes_for(capacity) gives the device bytes a chunk of that
    capacity holds."""
    want = min(chunk_points, sum(r.P - r.next_pt for r in pending))
    if want <= 0:
        return 0
    cap = chunk_capacity(want, chunk_points)
    floor = min(want, min_chunk)
    while cap > 1 and bytes_for(cap) > avail:
        cap >>= 1
    if bytes_for(cap) > avail or cap < floor:
        return 0
    return min(want, cap)


def pack_pending(pending: "collections.deque", capacity: int, copy_in) -> tuple:
    """Continuous batching: take the oldest pending work into one chunk of
    `capacity` points -- whole requests while they fit, then the next piece
    of the request at the head.  copy_in(req, lo, slot_lo, n) copies points
    [lo, lo + n) of req to chunk positions [slot_lo, slot_lo + n).  Requests
    whose last point is taken leave `pending`.  Returns (pieces, points used),
    pieces = [(request, req_lo, slot_lo, n)]."""
    n_used = 0
    pieces = []
    while pending and n_used < capacity:
        req = pending[0]
        take = min(req.P - req.next_pt, capacity - n_used)
        lo = req.next_pt
        copy_in(req, lo, n_used, take)
        pieces.append((req, lo, n_used, take))
        req.next_pt += take
        n_used += take
        if req.next_pt == req.P:
            pending.popleft()
    return pieces, n_used


def copy_results(pieces, code, elem, rst, values):
    """Copy one chunk's results (code, elem [n], rst [3][n], values [F][n],
    host arrays) back to the requests its pieces came from.  Pieces write
    disjoint slices, so chunks may be copied concurrently."""
    for req, lo, so, take in pieces:
        req.code[lo:lo + take] = code[so:so + take]
        req.elem[lo:lo + take] = elem[so:so + take]
        req.rst[:, lo:lo + take] = rst[:, so:so + take]
        req.values[:, lo:lo + take] = values[:, so:so + take]


def account(pieces, t: float, completed: list):
    """Count one chunk's copied pieces against their requests; a request
    whose every point is back is stamped with the latest time one of its
    chunks was copied (t for this one) and appended to `completed`."""
    for req, lo, so, take in pieces:
        req.done_pts += take
        req.t_last = t if req.t_last is None else max(req.t_last, t)
        if req.done_pts == req.P:
            req.t_done = req.t_last
            completed.append(req)


def scatter_results(pieces, code, elem, rst, values, now: float, completed: list):
    """copy_results then account, in the calling thread, stamped `now`."""
    copy_results(pieces, code, elem, rst, values)
    account(pieces, now, completed)


@dataclass
class _Buffers:
    """Device and pinned-host buffers and a workspace for chunks of up to
    `cap` points."""
    cap: int
    ws: "fg.Workspace"
    pts_h: torch.Tensor
    qs_h: torch.Tensor
    pts_d: torch.Tensor
    qs_d: torch.Tensor
    outs: tuple
    val_d: torch.Tensor
    code_h: torch.Tensor
    elem_h: torch.Tensor
    rst_h: torch.Tensor
    val_h: torch.Tensor


@dataclass
class _Chunk:
    buf: _Buffers
    stream: torch.cuda.Stream
    event: torch.cuda.Event
    n: int
    nbytes: int
    pieces: list = field(default_factory=list)   # (request, req_lo, slot_lo, n)


class Server:
    def __init__(self, handle, fields: torch.Tensor, budget_bytes: float = 40e9, resident_bytes: float = 0.0,
                 chunk_points: int = 1 << 17, streams: int = 4, min_chunk: int = 1 << 12, pairs_per_point: int = 4,
                 device=None, posted=None, copy_threads: int = 4):
        """handle: the resident mesh; fields [F][E][n^3] FP64 on the device
        (or `posted` double-float fields for the mixed form);
        budget_bytes: device memory the resident state and all chunks in
        flight may hold together; resident_bytes: what the resident state
        holds (fields, posted copies and anything else besides the handle's
        own mesh, which fp_memory counts); copy_threads: host threads that
        copy finished chunks' results into the requests (0: the dispatcher
        copies them itself)."""
        self.h = handle
        self.fields = fields
        self.posted = posted                  # fg.Fields (double-float) or None for FP64 eval
        self.F = int(fields.shape[0])
        self.dev = device or fields.device
        self.chunk_points = int(chunk_points)
        self.min_chunk = int(min_chunk)
        self.pairs_per_point = int(pairs_per_point)
        self.resident = float(resident_bytes) + fg.fp_memory(handle)["resident"]
        self.budget = float(budget_bytes)
        self.avail_total = self.budget - self.resident
        if self.avail_total < self.bytes_for(min(self.min_chunk, self.chunk_points)):
            raise ValueError("memory budget leaves no room for one chunk beside the resident state")
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(max(1, int(streams)))]
        self.free_streams = list(self.streams)
        self.pool: Dict[int, List[_Buffers]] = collections.defaultdict(list)
        self.inflight: List[_Chunk] = []
        self.inflight_bytes = 0
        self.peak_inflight_bytes = 0
        self.held_back = 0                    # passes where work waited for memory with a stream free
        self.pending = collections.deque()
        self.completed: List[Request] = []
        self.launches = 0
        self.chunk_sizes: List[int] = []
        self.copy_threads = max(0, int(copy_threads))
        self.copiers = ThreadPoolExecutor(self.copy_threads) if self.copy_threads else None
        self.copying: List[tuple] = []        # (future, chunk) of results being copied out
        self.t0 = time.perf_counter()         # origin of the times requests are stamped with
        self.idle = False                     # the last pass moved nothing

    def close(self):
        if self.copiers is not None:
            self.copiers.shutdown(wait=True)
            self.copiers = None

    def bytes_for(self, cap: int) -> int:
        """Device bytes a chunk of capacity `cap` holds: its buffers and its
        workspace."""
        return io_bytes(cap, self.F) + fg.fp_workspace_bytes(self.h, cap, self.pairs_per_point * cap)

    # -- request side ---------------------------------------------------------
    def submit(self, req: Request):
        P = req.P
        req.code = np.empty(P, np.int32)
        req.elem = np.empty(P, np.int32)
        req.rst = np.empty((3, P))
        req.values = np.empty((self.F, P))
        self.pending.append(req)

    # -- device side ------------------------------------------------------------
    def _buffers(self, cap: int) -> _Buffers:
        if self.pool[cap]:
            return self.pool[cap].pop()
        d, P, F = self.dev, cap, self.F
        outs = (torch.empty(P, dtype=torch.int32, device=d), torch.empty(P, dtype=torch.int32, device=d),
                torch.empty(P, dtype=torch.int32, device=d), torch.empty((3, P), dtype=torch.float64, device=d),
                torch.empty(P, dtype=torch.float64, device=d))
        return _Buffers(
            cap=cap, ws=fg.Workspace(self.h, P, self.pairs_per_point * P),
            pts_h=torch.empty((3, P), dtype=torch.float64).pin_memory(),
            qs_h=torch.empty(P, dtype=torch.int32).pin_memory(),
            pts_d=torch.empty((3, P), dtype=torch.float64, device=d),
            qs_d=torch.empty(P, dtype=torch.int32, device=d), outs=outs,
            val_d=torch.empty((F, P), dtype=torch.float64, device=d),
            code_h=torch.empty(P, dtype=torch.int32).pin_memory(),
            elem_h=torch.empty(P, dtype=torch.int32).pin_memory(),
            rst_h=torch.empty((3, P), dtype=torch.float64).pin_memory(),
            val_h=torch.empty((F, P), dtype=torch.float64).pin_memory())

    def _launch(self, n: int):
        cap = chunk_capacity(n, self.chunk_points)
        buf = self._buffers(cap)
        stream = self.free_streams.pop()

        def copy_in(req, lo, so, take):
            buf.pts_h[:, so:so + take].numpy()[...] = req.pts[:, lo:lo + take]
            buf.qs_h[so:so + take].numpy()[...] = req.qsess[lo:lo + take]
        pieces, n_used = pack_pending(self.pending, n, copy_in)
        F = self.F
        with torch.cuda.stream(stream):
            # packed [3][n] / [F][n] views of the buffers
            pts_c = buf.pts_d.view(-1)[:3 * n_used].view(3, n_used)
            rst_c = buf.outs[3].view(-1)[:3 * n_used].view(3, n_used)
            val_c = buf.val_d.view(-1)[:F * n_used].view(F, n_used)
            for a in range(3):
                pts_c[a].copy_(buf.pts_h[a, :n_used], non_blocking=True)
            qs_d = buf.qs_d[:n_used]
            qs_d.copy_(buf.qs_h[:n_used], non_blocking=True)
            code, osub, elem, d2 = buf.outs[0][:n_used], buf.outs[1][:n_used], buf.outs[2][:n_used], \
                buf.outs[4][:n_used]
            fg.fp_find_eval_ws(self.h, buf.ws, pts_c, qs_d, fields=self.fields, posted=self.posted,
                               out=(code, osub, elem, rst_c, d2), values=val_c, stream=stream)
            buf.code_h[:n_used].copy_(code, non_blocking=True)
            buf.elem_h[:n_used].copy_(elem, non_blocking=True)
            buf.rst_h.view(-1)[:3 * n_used].copy_(rst_c.view(-1), non_blocking=True)
            buf.val_h.view(-1)[:F * n_used].copy_(val_c.view(-1), non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        nbytes = self.bytes_for(cap)
        self.inflight.append(_Chunk(buf=buf, stream=stream, event=ev, n=n_used, nbytes=nbytes, pieces=pieces))
        self.inflight_bytes += nbytes
        self.peak_inflight_bytes = max(self.peak_inflight_bytes, self.inflight_bytes)
        self.launches += 1
        self.chunk_sizes.append(n_used)

    def _copy_out(self, ch: _Chunk) -> float:
        n = ch.n
        rst_h = ch.buf.rst_h.view(-1)[:3 * n].view(3, n).numpy()
        val_h = ch.buf.val_h.view(-1)[:self.F * n].view(self.F, n).numpy()
        copy_results(ch.pieces, ch.buf.code_h[:n].numpy(), ch.buf.elem_h[:n].numpy(), rst_h, val_h)
        return time.perf_counter() - self.t0

    def _release(self, ch: _Chunk, t: float):
        account(ch.pieces, t, self.completed)
        self.pool[ch.buf.cap].append(ch.buf)
        self.inflight_bytes -= ch.nbytes

    def _harvest(self, ch: _Chunk, now: float):
        """A chunk whose device work and copies are done gives its stream back
        at once; its results are copied into the requests (on a copier
        thread if there are any) before its buffers are released."""
        self.free_streams.append(ch.stream)
        if self.copiers is None:
            self._release(ch, self._copy_out(ch))
        else:
            self.copying.append((self.copiers.submit(self._copy_out, ch), ch))

    def step(self, now: float) -> bool:
        """One dispatcher pass: harvest finished chunks (freeing their
        streams), release chunks whose results are copied out (their memory),
        then admit chunks while a stream is free and the budget has room.
        Returns True if any chunk is in flight or being copied out, or work
        is pending."""
        still = []
        for ch in self.inflight:
            if ch.event.query():
                self._harvest(ch, now)
            else:
                still.append(ch)
        moved = len(still) < len(self.inflight)
        self.inflight = still
        left = []
        for fut, ch in self.copying:
            if fut.done():
                self._release(ch, fut.result())
            else:
                left.append((fut, ch))
        moved = moved or len(left) < len(self.copying)
        self.copying = left
        launched = self.launches
        while self.pending and self.free_streams:
            n = admit(self.pending, self.chunk_points, self.min_chunk, self.avail_total - self.inflight_bytes,
                      self.bytes_for)
            if n == 0:
                self.held_back += 1
                break
            self._launch(n)
        self.idle = not moved and self.launches == launched
        return bool(self.inflight) or bool(self.copying) or bool(self.pending)


def run_stream(server: Server, requests: List[Request], time_scale: float = 1.0):
    """Replay a request stream in real time (arrival times scaled by
    time_scale) and return (completed requests, makespan in s)."""
    order = sorted(requests, key=lambda r: r.t_arrive)
    i = 0
    t0 = time.perf_counter()
    server.t0 = t0
    while True:
        now = time.perf_counter() - t0
        while i < len(order) and order[i].t_arrive * time_scale <= now:
            order[i].t_arrive = order[i].t_arrive * time_scale
            server.submit(order[i])
            i += 1
        busy = server.step(now)
        if i == len(order) and not busy:
            break
        if busy and server.idle:
            time.sleep(5e-5)          # let the copier threads take the interpreter
        if not busy and i < len(order):
            wait = order[i].t_arrive * time_scale - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.001))
    return server.completed, time.perf_counter() - t0


def latency_stats(done: List[Request]):
    lat = np.array([(r.t_done - r.t_arrive) * 1e3 for r in done])
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "requests": int(len(done))}
