"""Interface data of one receiving subdomain across Schwarz time steps.

The paper advances each subdomain with boundary data interpolated from its
donors (Sec. 2): either lagged donor values, or values extrapolated in time
to order m and then refined by kappa predictor-corrector sub-iterations, each
of which re-interpolates the donors' new solution at the interface points and
corrects the mass flux (Sec. 2.2).  This class keeps the located interface
points (found once per mesh position), the history of corrected interface
velocities, and a CUDA graph of one sub-iteration (eval at the interface
points + flux correction), replayed kappa times per step.  Every operation is
a call into the library's kernels.
"""
from __future__ import annotations

import collections
from typing import Optional

import torch

import paper_1811_04891_gb300 as fg


class InterfaceExchange:
    def __init__(self, h, bfaces: "fg.BFaces", session: int, fields: torch.Tensor,
                 posted: Optional["fg.Fields"] = None, order: int = 1):
        """`bfaces` belongs to this exchange: locate() renumbers its interface
        nodes by donor element, so it must not be shared with another one."""
        if order not in (1, 2, 3):
            raise ValueError("order must be 1, 2 or 3")
        self.h, self.bf, self.fields, self.posted, self.order = h, bfaces, fields, posted, order
        dev = fields.device
        self.pts = bfaces.iface_points(dev)
        Mi, M = bfaces.Mi, bfaces.M
        self.qs = torch.full((Mi,), int(session), dtype=torch.int32, device=dev)
        self.F = int(fields.shape[0])
        self.found = None
        self.vals = torch.empty((self.F, Mi), dtype=torch.float64, device=dev)
        self.u_pres = torch.zeros((3, M), dtype=torch.float64, device=dev)   # prescribed data (caller fills)
        self.u = torch.zeros((3, M), dtype=torch.float64, device=dev)        # current boundary velocity
        self.gamma = torch.zeros(1, dtype=torch.float64, device=dev)
        self.flux = torch.zeros(1, dtype=torch.float64, device=dev)
        self.history = collections.deque(maxlen=order)
        self.graph = None
        self.locate()

    def locate(self):
        """Locate the interface points in the donors, then renumber them by
        donor element (neighbouring threads of the sub-iteration's eval then
        share an element's field rows) and locate them in that order."""
        f = None if self.posted else self.fields
        self.found = fg.fp_find_eval(self.h, self.pts, self.qs, fields=f, posted=self.posted, values=self.vals)
        self.bf.sort_iface(self.found[2])
        self.bf.iface_points(out=self.pts)
        self.found = fg.fp_find_eval(self.h, self.pts, self.qs, fields=f, posted=self.posted,
                                     out=self.found[:5], values=self.vals)
        if self.posted is not None:     # basis values kept for the sub-iterations
            self.ppts = fg.Points(self.h, self.pts.shape[1])
            self.ppts.set(self.found[0], self.found[2], self.found[3])
        self.graph = None

    def move(self, coords: torch.Tensor, dist: Optional[torch.Tensor] = None):
        """The meshes moved (Sec. 1: donors are found again after every step
        on moving meshes): post the new coordinates, refresh the face
        geometry and the interface points, and relocate them warm-started
        from the previous donors.  Results are written into the buffers the
        captured sub-iteration reads, so the graph stays valid."""
        fg.fp_update_coords(self.h, coords, dist)
        self.bf.refresh()
        self.bf.iface_points(out=self.pts)
        fg.fp_find_warm(self.h, self.pts, warm=(self.found[2], self.found[3]), qsess=self.qs, fields=self.fields,
                        posted=self.posted, out=self.found[:5], values=self.vals)
        if self.posted is not None:     # same buffers: a captured sub-iteration stays valid
            self.ppts.set(self.found[0], self.found[2], self.found[3])

    def _correct_eager(self):
        code, elem, rst = self.found[0], self.found[2], self.found[3]
        if self.posted is not None:
            self.ppts.eval(self.posted, out=self.vals)
        else:
            fg.fp_eval(self.h, code, elem, rst, self.fields, out=self.vals)
        st = fg.lib().fp_flux_correct_iface(self.bf.ptr, fg._ptr(self.vals), fg._ptr(self.u_pres), fg._ptr(self.u),
                                            fg._ptr(self.gamma), fg._ptr(self.flux), fg._stream(None))
        if st != fg.FP_OK:
            raise fg.FindptsError(st, "fp_flux_correct_iface failed")

    def capture(self):
        """Record one sub-iteration (eval + correction) as a CUDA graph."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self._correct_eager()
        torch.cuda.current_stream().wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._correct_eager()

    def correct(self):
        """One sub-iteration: re-interpolate the donors at the interface
        points and correct the flux; self.u holds the new boundary data."""
        if self.graph is None:
            self.capture()
        self.graph.replay()
        return self.u

    def predict(self):
        """Boundary data for the next step: lagged (m=1) or extrapolated in
        time from the m newest corrected values; before m values exist the
        order drops to what is available."""
        if not self.history:
            return self.correct()
        fg.fp_extrapolate(list(self.history)[::-1], out=self.u)
        return self.u

    def commit(self):
        """Store the current (corrected) boundary data as the newest value."""
        self.history.append(self.u.clone())

    def step(self, kappa: int = 1):
        """predict, then kappa sub-iterations (the solver runs in between in
        a full Schwarz code; here the donors' fields are whatever the caller
        has put in `fields`), then commit."""
        self.predict()
        for _ in range(kappa):
            self.correct()
        self.commit()
        return self.u
