"""Serving loop: point-location / interpolation requests against resident meshes.

The mesh, its hash grid and the fields stay resident on the device (one
handle).  Requests of uneven size arrive over time.  The server keeps `slots`
execution slots; each slot owns a CUDA stream, an fp_workspace and device /
pinned-host buffers for up to `slot_points` points.  How many slots may hold
work at once is set by the device-memory budget: budget minus the resident
mesh and fields, divided by the bytes one slot holds.

Continuous batching: whenever a slot is free, the dispatcher packs the oldest
pending work into it -- whole small requests, or the next chunk of a large
one -- copies the points in from pinned memory, runs fp_find_ws + fp_eval on
the slot's stream, and copies the codes and values back.  Requests that
arrive while other slots are on the GPU are admitted as soon as a slot (and
its memory) frees up, so their work overlaps on the device.  A request is
complete when all its chunks are; its latency is completion minus arrival.

Every point is located and interpolated independently of what else shares
its launch, so a request's results are the same alone and in the mix.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from typing import List, Optional

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
    t_done: Optional[float] = None

    @property
    def P(self) -> int:
        return int(self.pts.shape[1])


def slot_bytes(slot_points: int, F: int) -> int:
    """Device + pinned-host bytes one slot holds for `slot_points` points and
    F fields: points, tags, the five outputs and values on both sides, plus
    the workspace's per-point scan arrays and 4 pairs per point of pair
    records (element, point, order, residual, r)."""
    return slot_points * (24 + 4 + 24 + 4 * 3 + 8 + 8 * F) + 2 * slot_points * (4 * 3 + 8 + 24) + \
        slot_points * 12


def slots_for_budget(slots: int, slot_points: int, F: int, budget_bytes: float, resident_bytes: float) -> int:
    """Memory-budget admission: how many slots may hold work at once -- the
    budget left after the resident mesh and fields, divided by the bytes of
    one slot, at least one and at most `slots`."""
    avail = max(0.0, budget_bytes - resident_bytes)
    return max(1, min(slots, int(avail // slot_bytes(slot_points, F))))


def pack_pending(pending: "collections.deque", capacity: int, copy_in) -> tuple:
    """Continuous batching: take the oldest pending work into one slot of
    `capacity` points -- whole requests while they fit, then the next chunk of
    the request at the head.  copy_in(req, lo, slot_lo, n) copies points
    [lo, lo + n) of req to slot positions [slot_lo, slot_lo + n).  Requests
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


def scatter_results(pieces, code, elem, rst, values, now: float, completed: list):
    """Copy one slot's results (code, elem [n], rst [3][n], values [F][n],
    host arrays) back to the requests its pieces came from; a request whose
    every point is back is stamped `now` and appended to `completed`."""
    for req, lo, so, take in pieces:
        req.code[lo:lo + take] = code[so:so + take]
        req.elem[lo:lo + take] = elem[so:so + take]
        req.rst[:, lo:lo + take] = rst[:, so:so + take]
        req.values[:, lo:lo + take] = values[:, so:so + take]
        req.done_pts += take
        if req.done_pts == req.P:
            req.t_done = now
            completed.append(req)


@dataclass
class _Slot:
    stream: torch.cuda.Stream
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
    event: torch.cuda.Event
    pieces: list = field(default_factory=list)   # (request, req_lo, slot_lo, n)
    busy: bool = False


class Server:
    def __init__(self, handle, fields: torch.Tensor, slots: int = 4, slot_points: int = 1 << 20,
                 budget_bytes: float = 40e9, resident_bytes: float = 0.0, device=None, posted=None):
        self.h = handle
        self.fields = fields
        self.posted = posted                  # fg.Fields (double-float) or None for FP64 eval
        self.F = int(fields.shape[0])
        self.dev = device or fields.device
        self.slot_bytes = slot_bytes(slot_points, self.F)
        self.max_slots = slots_for_budget(slots, slot_points, self.F, budget_bytes, resident_bytes)
        self.slot_points = slot_points
        self.slots: List[_Slot] = []
        for _ in range(self.max_slots):
            P = slot_points
            d = self.dev
            outs = (torch.empty(P, dtype=torch.int32, device=d), torch.empty(P, dtype=torch.int32, device=d),
                    torch.empty(P, dtype=torch.int32, device=d), torch.empty((3, P), dtype=torch.float64, device=d),
                    torch.empty(P, dtype=torch.float64, device=d))
            self.slots.append(_Slot(
                stream=torch.cuda.Stream(device=d), ws=fg.Workspace(handle, P, 4 * P),
                pts_h=torch.empty((3, P), dtype=torch.float64).pin_memory(),
                qs_h=torch.empty(P, dtype=torch.int32).pin_memory(),
                pts_d=torch.empty((3, P), dtype=torch.float64, device=d),
                qs_d=torch.empty(P, dtype=torch.int32, device=d), outs=outs,
                val_d=torch.empty((self.F, P), dtype=torch.float64, device=d),
                code_h=torch.empty(P, dtype=torch.int32).pin_memory(),
                elem_h=torch.empty(P, dtype=torch.int32).pin_memory(),
                rst_h=torch.empty((3, P), dtype=torch.float64).pin_memory(),
                val_h=torch.empty((self.F, P), dtype=torch.float64).pin_memory(),
                event=torch.cuda.Event()))
        self.pending = collections.deque()
        self.completed: List[Request] = []
        self.launches = 0

    # -- request side ---------------------------------------------------------
    def submit(self, req: Request):
        P = req.P
        req.code = np.empty(P, np.int32)
        req.elem = np.empty(P, np.int32)
        req.rst = np.empty((3, P))
        req.values = np.empty((self.F, P))
        self.pending.append(req)

    # -- device side ------------------------------------------------------------
    def _fill(self, slot: _Slot) -> int:
        def copy_in(req, lo, so, take):
            slot.pts_h[:, so:so + take].numpy()[...] = req.pts[:, lo:lo + take]
            slot.qs_h[so:so + take].numpy()[...] = req.qsess[lo:lo + take]
        slot.pieces, n_used = pack_pending(self.pending, self.slot_points, copy_in)
        return n_used

    def _launch(self, slot: _Slot, n: int):
        F = self.F
        with torch.cuda.stream(slot.stream):
            # packed [3][n] / [F][n] views of the slot's buffers
            pts_c = slot.pts_d.view(-1)[:3 * n].view(3, n)
            rst_c = slot.outs[3].view(-1)[:3 * n].view(3, n)
            val_c = slot.val_d.view(-1)[:F * n].view(F, n)
            for a in range(3):
                pts_c[a].copy_(slot.pts_h[a, :n], non_blocking=True)
            qs_d = slot.qs_d[:n]
            qs_d.copy_(slot.qs_h[:n], non_blocking=True)
            code, osub, elem, d2 = slot.outs[0][:n], slot.outs[1][:n], slot.outs[2][:n], slot.outs[4][:n]
            fg.fp_find_eval_ws(self.h, slot.ws, pts_c, qs_d, fields=self.fields, posted=self.posted,
                               out=(code, osub, elem, rst_c, d2), values=val_c, stream=slot.stream)
            slot.code_h[:n].copy_(code, non_blocking=True)
            slot.elem_h[:n].copy_(elem, non_blocking=True)
            slot.rst_h.view(-1)[:3 * n].copy_(rst_c.view(-1), non_blocking=True)
            slot.val_h.view(-1)[:F * n].copy_(val_c.view(-1), non_blocking=True)
            slot.event.record(slot.stream)
        slot.busy = True
        slot.n = n
        self.launches += 1

    def _harvest(self, slot: _Slot, now: float):
        n = slot.n
        rst_h = slot.rst_h.view(-1)[:3 * n].view(3, n).numpy()
        val_h = slot.val_h.view(-1)[:self.F * n].view(self.F, n).numpy()
        scatter_results(slot.pieces, slot.code_h[:n].numpy(), slot.elem_h[:n].numpy(), rst_h, val_h, now,
                        self.completed)
        slot.pieces = []
        slot.busy = False

    def step(self, now: float) -> bool:
        """One dispatcher pass: harvest finished slots, refill free ones.
        Returns True if any slot is busy or work is pending."""
        for slot in self.slots:
            if slot.busy and slot.event.query():
                self._harvest(slot, now)
        for slot in self.slots:
            if not slot.busy and self.pending:
                n = self._fill(slot)
                if n:
                    self._launch(slot, n)
        return any(s.busy for s in self.slots) or bool(self.pending)


def run_stream(server: Server, requests: List[Request], time_scale: float = 1.0):
    """Replay a request stream in real time (arrival times scaled by
    time_scale) and return (completed requests, makespan in s)."""
    order = sorted(requests, key=lambda r: r.t_arrive)
    i = 0
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while i < len(order) and order[i].t_arrive * time_scale <= now:
            order[i].t_arrive = order[i].t_arrive * time_scale
            server.submit(order[i])
            i += 1
        busy = server.step(now)
        if i == len(order) and not busy:
            break
        if not busy and i < len(order):
            wait = order[i].t_arrive * time_scale - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.001))
    return server.completed, time.perf_counter() - t0


def latency_stats(done: List[Request]):
    lat = np.array([(r.t_done - r.t_arrive) * 1e3 for r in done])
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "requests": int(len(done))}
