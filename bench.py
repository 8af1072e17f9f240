#!/usr/bin/env python
"""Throughput of the findpts + findpts_eval hot path on GB300.

Workload: the precision-form-at-scale configuration -- a 32^3 = 32768-element
deformed hex cube at N=7 (interior nodes displaced by 0.1 h sin sin sin),
1e7 uniform query points plus 1e5 points within 1e-9 of element faces, five
FP64 fields.  One step = fp_find over all 10,100,000 points followed by
fp_eval of the five fields, with the mesh, hash grid and inputs resident in
HBM (setup is timed separately).  Metric: located+interpolated points/s.

The headline `value` is the mixed form (FP32 seed and early Newton steps,
FP64 final step, residual, classification and eval); the FP64 form is timed
in the same run under `forms`.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (brute force, FP64, OpenMP on the
host cores) on bounded samples of the same workload.  Under torchrun each
rank processes its own copy of the workload (weak scaling, no collective on
the data path); `value` is all ranks' points / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "located+interpolated points/s (mixed vs FP64 form, N=7); serving p50/p99 ms"
UNIT = "points/s"
# Algorithmic work per located point at N=7 (n = 8), counting the true
# element only: the nearest-node seed (512 nodes x 8 flops = 4.1 kflop), the
# K Newton iterations with Jacobian (6n^3 + 9n^2 + 12n FMA + ~6n^2 basis, 8.4
# kflop each) that the oracle needs from that seed, the final step (a
# value-only residual 3 (n^3 + n^2 + n) FMA + basis values = 3.8 kflop), and
# one field evaluation (n^3 + n^2 + n FMA = 1.17 kflop) per field.
# K = 3.43: the mean iteration count of the oracle's Newton on the true
# element, measured on a 22,000-point sample of this workload (20,000 uniform
# + 2,000 near-face points).
SEED, ITER, FINAL, EVAL1 = 4.1e3, 8.4e3, 3.8e3, 1.17e3
K_ORACLE = 3.43
# Where each part of that work runs, and at which measured peak its
# roofline time is taken:
#   FP64 form:  seed + K iterations, all on the FP64 pipe              -> P64
#   mixed form: seed + K iterations in FP32                            -> P32
#               the final step at FP64 accuracy: on whichever of the
#               FP64 pipe and double-float arithmetic on the FP32
#               pipes this GPU runs faster                             -> max(P64, Pdf)
#   eval:       FP64 form on the FP64 pipe; mixed form at FP64
#               accuracy                                               -> P64 / max(P64, Pdf)
# The refinement steps the mixed form adds between its FP32 iterations and
# its final step are the implementation's precision technique, not the
# method's work, and are not counted.
def work_for_order(n: int) -> dict:
    """The per-point algorithmic work above for n = N + 1 GLL points per
    direction, scaled from the N = 7 figures by each part's operation count
    (seed n^3, iteration 6n^3 + 9n^2 + 12n, residual and eval n^3 + n^2 + n)."""
    it = (6 * n ** 3 + 9 * n ** 2 + 12 * n) / (6 * 512 + 9 * 64 + 12 * 8)
    ev = (n ** 3 + n ** 2 + n) / (512 + 64 + 8)
    return {"seed": SEED * n ** 3 / 512, "iter": ITER * it, "final": FINAL * ev, "eval1": EVAL1 * ev}


WORK = {"fp64": {"f64": SEED + K_ORACLE * ITER, "f32": 0.0, "f64acc": 0.0},
        "mixed": {"f64": 0.0, "f32": SEED + K_ORACLE * ITER, "f64acc": FINAL}}
# DRAM bytes (read + written) per (point, candidate element) pair of the Newton
# stage, from one-pass ncu captures of the stage at this full size
# (dram__bytes_read.sum + dram__bytes_write.sum of k_newton_mixed, and of
# k_newton + k_newton_resume, over the 10.24 M pairs of one launch).
TRAFFIC_PER_PAIR = {"mixed": 622.0, "fp64": 620.0}
HBM_FALLBACK_GBS = 6800.0


def measured_hbm_gbs():
    """Measured copy bandwidth (GB/s) of the GB300s, else the
    fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except Exception:  # noqa: BLE001
        return HBM_FALLBACK_GBS, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--forms", default="mixed,fp64")
    ap.add_argument("--ne", type=int, default=32)
    ap.add_argument("--points", type=int, default=10 ** 7)
    ap.add_argument("--face-points", type=int, default=10 ** 5)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-interface", action="store_true")
    ap.add_argument("--no-moving", action="store_true")
    ap.add_argument("--no-planar", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--stage-eval", action="store_true",
                    help="mixed form: time the eval with element fields staged in shared memory")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the peak probes (profiling runs); the line then has no roofline")
    ap.add_argument("--served-requests", type=int, default=200)
    ap.add_argument("--served-load", type=float, default=0.7)
    ap.add_argument("--served-chunk", type=int, default=1 << 17)
    ap.add_argument("--served-scale", type=float, default=1.0,
                    help="element-count scale of the served mesh (1.0 = 193,536 elements)")
    return ap.parse_args()


def make_collectives(dist, world: int, device):
    """barrier() and max_over_ranks(x) of the replica runs: every rank runs its
    own copy of the workload (no collective on the data path); the job's time
    is the slowest rank's."""
    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return barrier, max_over_ranks


def replica_rate(world: int, points_per_rank: int, steps: int, ms_slowest: float) -> float:
    """Weak scaling: all ranks' points over the slowest rank's time (points/s)."""
    return world * points_per_rank * steps / (ms_slowest / 1e3)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(args):
    import synth
    mesh, q = synth.deformed_cube(ne=args.ne, P_uniform=args.points, P_face=args.face_points)
    return mesh, q


def config_dict(args, mesh, q, form_note=""):
    return {"workload": f"deformed cube {args.ne}^3 hex N=7 (amp 0.1h), {args.points} uniform + "
                        f"{args.face_points} near-face points, 5 FP64 fields; find + eval per step",
            "E": int(mesh.E), "N": int(mesh.N), "points_per_step": int(q.P), "fields": 5,
            "l2_flush": "inputs larger than L2 (points 242 MB, coords 403 MB, fields 671 MB)",
            "setup": "mesh, boxes and hash grid resident; setup timed separately"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[4 + i] and "Not" not in r[4 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# measured arithmetic peaks (the roofline's denominators)
# ---------------------------------------------------------------------------
def measure_peaks(fg, dev, uuid, target_ms: float = 60.0, blocks_per_sm: int = 4):
    """FP64, FP32 and double-float multiply-add rates of this GPU from the
    library's chain probes (fp_fma_probe: 8 independent fma chains per thread,
    blocks_per_sm blocks of 256 threads on every SM), each timed with CUDA
    events on the launching stream, best of three launches of ~target_ms,
    with the SM clock sampled meanwhile.  Returns TFLOP/s."""
    import torch
    stream = torch.cuda.current_stream(dev)
    sink = torch.empty(fg.fp_probe_threads(blocks_per_sm), dtype=torch.float64, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def once(kind, iters):
        ev0.record(stream)
        fl = fg.fp_fma_probe(kind, iters, sink, blocks_per_sm, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        return fl, ev0.elapsed_time(ev1)

    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.3)
    rates, launches = {}, {}
    for kind in ("f64", "f32", "df", "f32x2", "df2"):
        iters = 256
        fl, ms = once(kind, iters)
        while ms < 5.0 and iters < (1 << 30):
            iters *= 4
            fl, ms = once(kind, iters)
        iters = max(1, int(iters * target_ms / max(ms, 1e-3)))
        best = 0.0
        for _ in range(3):
            fl, ms = once(kind, iters)
            best = max(best, fl / (ms / 1e3))
        rates[kind] = best / 1e12
        launches[kind] = {"iters": iters, "flops": fl, "ms": ms}
    clk = clocks.stop()
    return {"p64": rates["f64"], "p32": max(rates["f32"], rates["f32x2"]), "pdf": max(rates["df"], rates["df2"]),
            "unit": "TFLOP/s", "clocks": clk, "launches": launches, "by_kind": rates,
            "method": f"fp_fma_probe: {blocks_per_sm} x 256 threads per SM, 8 independent chains per thread, "
                      "best of 3 launches (CUDA events); df = double-float multiply-add on the FP32 pipes "
                      "(exact leading product + two-sum), counted as 2 FP64-class flops; p32 and pdf are the "
                      "faster of the scalar and the packed-pair (float2) instruction forms"}


def roofline_form(form, P, F, kernel_ms, ms_per_step, peaks, hbm_gbs, pairs, coords_bytes, field_bytes):
    """Roofline of one form from the algorithmic work (WORK, EVAL1) and the
    measured peaks.  Dominant kernel: the Newton stage.  Whole step: find +
    eval of F fields, with the step's compulsory HBM bytes beside it."""
    p64, p32, pdf = peaks["p64"] * 1e12, peaks["p32"] * 1e12, peaks["pdf"] * 1e12
    pacc = max(p64, pdf)                     # FP64-accuracy work of the mixed form
    w = WORK[form]
    kn = kernel_ms["newton"] / 1e3
    if form == "fp64":
        t_newton = P * w["f64"] / p64
        achieved, peak, unit = P * w["f64"] / kn, p64, "TFLOP/s (FP64)"
        t_eval = P * F * EVAL1 / p64
    else:
        t_newton = P * (w["f32"] / p32 + w["f64acc"] / pacc)
        # FP32-equivalent flops: FP64-accuracy flops scaled by P32 / max(P64, Pdf)
        achieved, peak = P * (w["f32"] + w["f64acc"] * p32 / pacc) / kn, p32
        unit = "TFLOP/s (FP32-equivalent: FP32 flops + FP64-accuracy flops x P32/max(P64,Pdf))"
        t_eval = P * F * EVAL1 / pacc
    step_bytes = P * (24 + 44 + 8 * F) + coords_bytes + field_bytes
    t_bytes = step_bytes / (hbm_gbs * 1e9)
    t_step = max(t_newton + t_eval, t_bytes)
    traffic = TRAFFIC_PER_PAIR.get(form)
    fp64_view = P * (SEED + K_ORACLE * ITER + F * EVAL1) / p64
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": unit,
            "frac": t_newton / kn, "traffic": None if traffic is None else traffic * pairs,
            "kernel": "k_newton_mixed<8> + k_newton64_full<8>" if form == "mixed" else "k_newton<8>",
            "kernel_ms": kernel_ms["newton"], "units_per_launch": P, "work_unit": "located point (true element only)",
            "unit_work": w, "pairs_per_launch": pairs, "roofline_ms": 1e3 * t_newton,
            "peaks_tflops": {"p64": peaks["p64"], "p32": peaks["p32"], "pdf": peaks["pdf"],
                             "by_instruction_form": peaks.get("by_kind")},
            "peak_source": "measured in this run (fp_fma_probe, CUDA events), SM clock "
                           f"{peaks['clocks'].get('sm_mhz')} MHz",
            "traffic_source": None if traffic is None else
            "ncu dram__bytes_read.sum + dram__bytes_write.sum per pair, full-size one-pass capture, x pairs",
            "step": {"frac": t_step / (ms_per_step / 1e3), "roofline_ms": 1e3 * t_step,
                     "eval_roofline_ms": 1e3 * t_eval, "bytes": step_bytes, "bytes_ms": 1e3 * t_bytes,
                     "note": f"find + eval of {F} fields: Newton roofline + eval roofline "
                             f"({EVAL1:.0f} flop per field per point at "
                             f"{'P64' if form == 'fp64' else 'max(P64, Pdf)'}), against the measured step"},
            "frac_final_step_on_fp64_pipe": (None if form == "fp64" else
                                             P * (w["f32"] / p32 + w["f64acc"] / p64) / kn),
            "fp64_roofline": {"ms": 1e3 * fp64_view, "frac": fp64_view / (ms_per_step / 1e3),
                              "note": "the whole step's algorithmic work (seed + K iterations + evals) at the "
                                      "FP64 peak, against the measured step: above 1 means faster than any "
                                      "FP64-only implementation can be"}}


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_rate(mesh, q, seconds: float, stride_seed: int = 0):
    """Time the oracle's find + eval on a strided sample of the workload
    sized to take about `seconds`; returns (points/s, sample size, cores, s)."""
    import oracle
    P = q.P

    def run(idx):
        pts = np.ascontiguousarray(q.pts[:, idx])
        t0 = time.perf_counter()
        r = oracle.find(mesh.coords, mesh.N, mesh.sub, pts)
        oracle.evaluate(mesh.N, r["code"], r["elem"], r["rst"], q.fields)
        return time.perf_counter() - t0

    m0 = min(P, 2000)
    idx0 = np.arange(stride_seed % max(1, P // m0), P, max(1, P // m0))[:m0]
    dt0 = run(idx0)
    rate0 = len(idx0) / max(dt0, 1e-9)
    m = int(min(P, max(len(idx0), rate0 * seconds)))
    idx = np.arange(0, P, max(1, P // m))[:m]
    dt = run(idx)
    return len(idx) / dt, len(idx), oracle.num_threads(), dt


def oracle_rate_one_core(mesh, q, seconds: float):
    """The oracle on one core (OpenMP threads set to 1, then restored) on a
    strided sample sized to take about `seconds`; returns (points/s, sample
    size, s)."""
    import oracle
    n0 = oracle.num_threads()
    oracle.set_threads(1)
    try:
        rate, m, _, dt = oracle_rate(mesh, q, seconds, stride_seed=1)
    finally:
        oracle.set_threads(n0)
    return rate, m, dt


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    mesh, q = workload(args)
    vals = []
    per_step = max(2.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    for s in range(args.warmup):
        oracle_rate(mesh, q, per_step, stride_seed=s)
    samples, times = [], []
    for s in range(args.steps):
        rate, m, cores, dt = oracle_rate(mesh, q, per_step, stride_seed=args.warmup + s)
        vals.append(rate)
        samples.append(m)
        times.append(dt)
    value = sum(samples) / sum(times)
    # one step of this arm is one bounded sample: its measured time, not the
    # time the oracle would need for all of the workload's points
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "points_per_step": statistics.mean(samples),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args, mesh, q),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"strided samples of {min(samples)}-{max(samples)} of the {q.P} points per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# configurations 0 and 1: small, latency-bound find + eval calls
# ---------------------------------------------------------------------------
def run_small_configs(args, fg, dev, peaks, with_oracle: bool):
    """The plain single-subdomain cube (4^3 elements, 1e4 points, one field)
    and the box + annulus overlap (2048 elements, its ~4e4 tagged interface
    nodes, four fields, owner rule): one fp_find_eval call per step, both
    forms, CUDA events over 50 calls after 5 warm-up calls.  The step
    roofline uses the iteration count K of the 32^3 workload."""
    import torch

    import synth
    out = {}
    p64, p32 = peaks["p64"] * 1e12, peaks["p32"] * 1e12
    pacc = max(p64, peaks["pdf"] * 1e12)
    for name, (mesh, q) in (("cube4_small", synth.cube4_small()), ("box_annulus", synth.box_annulus())):
        pts = torch.from_numpy(q.pts).to(dev)
        qs = None if q.qsess is None else torch.from_numpy(q.qsess).to(dev)
        fields = torch.from_numpy(q.fields).to(dev)
        coords = torch.from_numpy(mesh.coords).to(dev)
        sub = torch.from_numpy(mesh.sub).to(dev)
        dist = None if mesh.dist is None else torch.from_numpy(mesh.dist).to(dev)
        F, P = fields.shape[0], q.P
        res = {"E": int(mesh.E), "N": int(mesh.N), "points": int(P), "fields": int(F)}
        for form, prec in (("fp64", fg.PREC_FP64), ("mixed", fg.PREC_MIXED)):
            h = fg.fp_setup(coords, mesh.N, sub, dist, opts=fg.default_opts(precision=prec))
            fg.fp_reserve(h, P)
            posted = fg.Fields(h, fields) if form == "mixed" else None
            outs = fg._find_outs(P, dev)
            vals = torch.empty((F, P), dtype=torch.float64, device=dev)
            for _ in range(5):
                fg.fp_find_eval(h, pts, qs, fields=fields, posted=posted, out=outs, values=vals)
            torch.cuda.synchronize()
            fg.fp_band_hits(h)
            reps = 50
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fg.fp_find_eval(h, pts, qs, fields=fields, posted=posted, out=outs, values=vals)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            band = fg.fp_band_hits(h)
            if form == "fp64":
                t_roof = P * (SEED + K_ORACLE * ITER + F * EVAL1) / p64
            else:
                t_roof = P * ((SEED + K_ORACLE * ITER) / p32 + (FINAL + F * EVAL1) / pacc)
            codes = torch.bincount(outs[0].long(), minlength=3).tolist()
            res[form] = {"points_per_s": P / (ms / 1e3), "ms_per_call": ms, "step_roofline_frac": t_roof / (ms / 1e3),
                         "band_hits_per_call": {k: v / reps for k, v in band.items()},
                         "codes": {"inside": codes[0], "border": codes[1], "not_found": codes[2]}}
            del posted, h
        if with_oracle:
            import oracle
            t0 = time.perf_counter()
            r = oracle.find(mesh.coords, mesh.N, mesh.sub, q.pts, qsess=q.qsess, dist=mesh.dist)
            oracle.evaluate(mesh.N, r["code"], r["elem"], r["rst"], q.fields)
            dt = time.perf_counter() - t0
            res["oracle"] = {"points_per_s": P / dt, "cores": oracle.num_threads(), "sample": "all points"}
        out[name] = res
    out["note"] = ("latency-bound calls (few points): one fused find + eval call per step; step_roofline_frac = "
                   "algorithmic work at the measured peaks over the call's time")
    return out


# ---------------------------------------------------------------------------
# batched form: 64 deformed-box instances, E logU[64,8192], N in {5,7,9}
# ---------------------------------------------------------------------------
def run_batched(args, fg, dev, barrier, max_over_ranks, world, peaks):
    import torch

    import synth
    insts = synth.instance_batch()
    out = {"instances": len(insts), "elements": int(sum(m.E for m, _ in insts)),
           "points_per_step": int(sum(q.P for _, q in insts)), "orders": sorted({m.N for m, _ in insts})}
    pts = torch.from_numpy(np.ascontiguousarray(np.concatenate([q.pts for _, q in insts], axis=1))).to(dev)
    fields = [torch.from_numpy(q.fields).to(dev) for _, q in insts]
    P = pts.shape[1]
    for form, prec in (("mixed", fg.PREC_MIXED), ("fp64", fg.PREC_FP64)):
        handles = [fg.fp_setup(torch.from_numpy(m.coords).to(dev), m.N, torch.from_numpy(m.sub).to(dev),
                               opts=fg.default_opts(precision=prec)) for m, _ in insts]
        b = fg.Batch(handles, [q.P for _, q in insts], fields)
        outs = b.outputs(dev)
        t0 = time.perf_counter()
        tuned_ms = b.tune(pts, outs, reps=1)
        tune_s = time.perf_counter() - t0
        b.capture(pts, outs)
        for _ in range(max(1, args.warmup)):
            b.launch()
        torch.cuda.synchronize()
        b.band_hits()
        barrier()
        l0 = fg.fp_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            b.launch()
        e1.record()
        torch.cuda.synchronize()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1)) / args.steps
        launches = (fg.fp_launch_count() - l0) // max(1, args.steps)
        band = b.band_hits()
        codes = torch.bincount(outs[0].long(), minlength=4).tolist()
        # one profiled (eager) run: per-order Newton and eval times, the groups one after another
        b.profile(True)
        b.run(pts, outs)
        torch.cuda.synchronize()
        b.profile(False)
        per_order = {}
        for g in range(b.groups()):
            gi = b.group_info(g)
            n = gi["N"] + 1
            w = work_for_order(n)
            blk, bps, tile = b.schedule(g)
            row = {"elements": gi["E"], "points": gi["P"], "pairs": gi["pairs"], "newton_ms": gi["newton_ms"],
                   "eval_ms": gi["eval_ms"],
                   "points_per_s_newton_eval": gi["P"] / max(1e-9, (gi["newton_ms"] + gi["eval_ms"]) / 1e3),
                   "schedule": {"threads_per_block": blk, "blocks_per_sm": bps, "pairs_per_item": tile}}
            if peaks is not None and gi["newton_ms"] > 0:
                p64, p32 = peaks["p64"] * 1e12, peaks["p32"] * 1e12
                pacc = max(p64, peaks["pdf"] * 1e12)
                if form == "fp64":
                    t = gi["P"] * (w["seed"] + K_ORACLE * w["iter"]) / p64
                else:
                    t = gi["P"] * ((w["seed"] + K_ORACLE * w["iter"]) / p32 + w["final"] / pacc)
                row["newton_roofline_frac"] = t / (gi["newton_ms"] / 1e3)
            per_order[f"N{gi['N']}"] = row
        out[form] = {"value": world * P / (ms / 1e3), "ms_per_step": ms, "tuned_ms": tuned_ms, "tune_s": tune_s,
                     "groups_sequential": bool(b.mode()),
                     "gpu_launches": launches, "per_order": per_order, "band_hits_per_step": band,
                     "codes": {"inside": codes[0], "border": codes[1], "not_found": codes[2], "retry": codes[3]}}
        del b, handles
    out["unit"] = UNIT
    out["note"] = ("one CUDA-graph launch per step: batch-wide screen, scan, emit, pair sort and classification; "
                   "per order N one persistent work-queue Newton launch (concurrent streams) and one eval launch; "
                   "schedule autotuned per order; per-order times from one profiled eager run; roofline with the "
                   "N=7 oracle iteration count K")
    return out


# ---------------------------------------------------------------------------
# interface update of the box + annulus overlap (box + annulus): the cylinder's
# radial faces take velocity and pressure interpolated from the box, its end
# walls keep prescribed data, and the interpolated velocity is flux-corrected
# ---------------------------------------------------------------------------
def run_interface(args, fg, dev):
    import torch

    import synth
    mesh, q = synth.box_annulus()
    n_rad, n_az, n_ax = 4, 32, 8
    kind = np.zeros((mesh.E, 6), np.int8)
    for e in range(1024, mesh.E):
        el = e - 1024
        er, ez = el % n_rad, el // (n_rad * n_az)
        kind[e, 0] = 2 if er == 0 else 0
        kind[e, 1] = 2 if er == n_rad - 1 else 0
        kind[e, 4] = 1 if ez == 0 else 0
        kind[e, 5] = 1 if ez == n_ax - 1 else 0
    out = {}
    for form, prec in (("mixed", fg.PREC_MIXED), ("fp64", fg.PREC_FP64)):
        h = fg.fp_setup(torch.from_numpy(mesh.coords).to(dev), mesh.N, torch.from_numpy(mesh.sub).to(dev),
                        torch.from_numpy(mesh.dist).to(dev), opts=fg.default_opts(precision=prec))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bf = fg.BFaces(h, torch.from_numpy(kind).to(dev))
        torch.cuda.synchronize()
        bf_ms = 1e3 * (time.perf_counter() - t0)
        x, nr, dA, nk = bf.nodes(dev)
        iface = (nk == 2).nonzero().squeeze(1)
        pts = x[:, iface].contiguous()
        qs = torch.ones(pts.shape[1], dtype=torch.int32, device=dev)
        fields = torch.from_numpy(q.fields).to(dev)            # u, v, w, p
        posted = fg.Fields(h, fields) if form == "mixed" else None
        P = pts.shape[1]
        found = fg.fp_find_eval(h, pts, qs, fields=fields, posted=posted)
        code, elem, rst = found[0], found[2], found[3]
        vals = torch.empty((4, P), dtype=torch.float64, device=dev)
        u = torch.zeros((3, bf.M), dtype=torch.float64, device=dev)
        uo = torch.empty_like(u)

        def find_step():
            fg.fp_find_eval(h, pts, qs, fields=fields, posted=posted, out=found[:5], values=vals)

        def iterate():      # one Schwarz sub-iteration: re-interpolate at the found points, correct
            if posted is not None:
                fg.fp_eval_df(h, posted, code, elem, rst, out=vals)
            else:
                fg.fp_eval(h, code, elem, rst, fields, out=vals)
            u[:, iface] = vals[:3]
            fg.fp_flux_correct(bf, u, uo)

        res = {}
        for name, fn, reps in (("find_eval", find_step, 20), ("iteration", iterate, 200)):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            res[name + "_ms"] = e0.elapsed_time(e1) / reps
        # the Schwarz step through the graph-replayed pipeline: predict
        # (order-m extrapolation), kappa captured eval + correction
        # sub-iterations, commit; (m, kappa) = (1, 1), (2, 4), (3, 7)
        from paper_1811_04891_gb300.schwarz import InterfaceExchange
        steps = {}
        for m, kappa in ((1, 1), (2, 4), (3, 7)):
            xch = InterfaceExchange(h, bf, 1, fields, posted=posted, order=m)
            for _ in range(m + 2):
                xch.step(kappa)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 50
            e0.record()
            for _ in range(reps):
                xch.step(kappa)
            e1.record()
            torch.cuda.synchronize()
            steps[f"m{m}_kappa{kappa}_ms"] = e0.elapsed_time(e1) / reps
            del xch
        out[form] = {"interface_points": int(P), "face_nodes": int(bf.M), "bfaces_setup_ms": bf_ms,
                     **res, "iteration_points_per_s": P / (res["iteration_ms"] / 1e3),
                     "graph_step": steps}
        del bf, h
    out["note"] = ("per Schwarz sub-iteration: eval of u,v,w,p at the found interface points + flux "
                   "correction (Eq. consv2); find_eval = locate + eval once (static mesh); graph_step = "
                   "extrapolation of order m + kappa graph-replayed sub-iterations + history update")
    return out


def run_moving(args, fg, dev, mesh, coords, sub, pts, fields):
    return {form: _moving_form(args, fg, dev, mesh, coords, sub, pts, fields, form) for form in ("mixed", "fp64")}


def _moving_form(args, fg, dev, mesh, coords, sub, pts, fields, form):
    """Moving mesh: the deformed cube turns about its vertical axis by 0.02
    degrees and drifts by 2e-4 (0.6 % of an element) per time step while the
    query points stay, so every donor is found again each step.  Per step:
    fp_update_coords (boxes, hash grid, FP32 geometry rebuilt in place) and a
    find + eval warm-started from the previous step's (e, r); the cold find +
    eval on the same moved mesh and a fresh fp_setup are timed beside it."""
    import math

    import torch
    P = pts.shape[1]
    prec = fg.PREC_MIXED if form == "mixed" else fg.PREC_FP64
    h = fg.fp_setup(coords, mesh.N, sub, opts=fg.default_opts(precision=prec))
    fg.fp_reserve(h, P)
    posted = fg.Fields(h, fields) if form == "mixed" else None
    moved = torch.empty_like(coords)

    def position(k):                 # the mesh motion itself (the flow solver's job, untimed)
        a = math.radians(0.02 * k)
        x, y = coords[0] - 0.5, coords[1] - 0.5
        moved[0].copy_(x).mul_(math.cos(a)).add_(y, alpha=-math.sin(a)).add_(0.5 + 2e-4 * k)
        moved[1].copy_(y).mul_(math.cos(a)).add_(x, alpha=math.sin(a)).add_(0.5)
        moved[2].copy_(coords[2])

    F = fields.shape[0]
    outs = fg._find_outs(P, dev)
    vals = torch.empty((F, P), dtype=torch.float64, device=dev)
    fg.fp_find_eval(h, pts, None, fields=fields, posted=posted, out=outs, values=vals)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_upd = t_find = 0.0
    k = 0
    for it in range(args.warmup + args.steps):
        k += 1
        position(k)
        ev[0].record()
        fg.fp_update_coords(h, moved)
        ev[1].record()
        fg.fp_find_warm(h, pts, warm=(outs[2], outs[3]), fields=fields, posted=posted, out=outs, values=vals)
        ev[2].record()
        torch.cuda.synchronize()
        if it >= args.warmup:
            t_upd += ev[0].elapsed_time(ev[1])
            t_find += ev[1].elapsed_time(ev[2])
    K = args.steps
    counts = torch.bincount(outs[0].long(), minlength=3).tolist()
    cold = fg._find_outs(P, dev)
    for _ in range(2):
        fg.fp_find_eval(h, pts, None, fields=fields, posted=posted, out=cold, values=vals)
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(K):
        fg.fp_find_eval(h, pts, None, fields=fields, posted=posted, out=cold, values=vals)
    ev[1].record()
    torch.cuda.synchronize()
    t_cold = ev[0].elapsed_time(ev[1]) / K
    same = all(bool(torch.equal(outs[a], cold[a])) for a in (0, 1, 2))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2 = fg.fp_setup(moved, mesh.N, sub, opts=fg.default_opts(precision=prec))
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t0)
    del h2
    step_ms = (t_upd + t_find) / K
    return {"update_ms": t_upd / K, "find_eval_warm_ms": t_find / K, "find_eval_cold_ms": t_cold,
            "step_ms": step_ms, "points_per_s": P / (step_ms / 1e3), "fresh_setup_ms": setup_ms,
            "codes": {"inside": counts[0], "border": counts[1], "not_found": counts[2]},
            "warm_equals_cold_ids": same,
            "note": "deformed cube 32^3 N=7 turning 0.02 deg + drifting 2e-4 per step, 1.01e7 fixed points, "
                    "step = update + warm find + eval"}


def run_planar(args, fg, dev):
    """2D variant (quadrilaterals, the paper's 2D overset examples): a
    512 x 512 deformed quad mesh at N=7 (amplitude 0.1 h) with 1e7 uniform
    points and three fields, find + eval per step (FP64 form); and the
    box + annulus overset workload (session tags, owner rule), whose few
    thousand interface points make it latency-bound."""
    import torch

    import synth
    out = {}
    ne = 512
    coords = torch.from_numpy(synth.quad_mesh((ne, ne), 7, amp_frac=0.1)).to(dev)
    E = coords.shape[1]
    P = args.points
    pts = torch.from_numpy(synth.uniform_points_2d(P, seed=0)).to(dev)
    x, y = coords[0], coords[1]
    fields = torch.stack([torch.sin(torch.pi * x) * torch.cos(torch.pi * y), x * y, torch.exp(x - y)]).contiguous()
    h = fg.fp_setup_2d(coords, 7, torch.zeros(E, dtype=torch.int32, device=dev))
    fg.fp_reserve(h, P)
    outs = fg._find_outs(P, dev, 2)
    vals = torch.empty((3, P), dtype=torch.float64, device=dev)
    for _ in range(max(args.warmup, 1)):
        fg.fp_find_eval(h, pts, None, fields=fields, out=outs, values=vals)
    torch.cuda.synchronize()
    fg.fp_profile(h, True)
    for k in fg.PROF_KINDS:
        fg.fp_profile_read(h, k)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fg.fp_find_eval(h, pts, None, fields=fields, out=outs, values=vals)
    e1.record()
    torch.cuda.synchronize()
    fg.fp_profile(h, False)
    kt = {k: fg.fp_profile_read(h, k) for k in fg.PROF_KINDS}
    ms = e0.elapsed_time(e1) / args.steps
    counts = torch.bincount(outs[0].long(), minlength=3).tolist()
    out["quad512_N7"] = {"E": E, "points": P, "fields": 3, "ms_per_step": ms, "points_per_s": P / (ms / 1e3),
                         "pairs_per_point": fg.fp_last_find_stats(h) / P,
                         "kernel_ms": {k: (v[0] / max(v[1], 1)) for k, v in kt.items()},
                         "codes": {"inside": counts[0], "border": counts[1], "not_found": counts[2]}}
    del h
    mesh, q = synth.walsh_2d(N=7, n_box=16, ring=(16, 3))
    h = fg.fp_setup_2d(torch.from_numpy(mesh.coords).to(dev), mesh.N, torch.from_numpy(mesh.sub).to(dev),
                       torch.from_numpy(mesh.dist).to(dev))
    pq = torch.from_numpy(q.pts).to(dev)
    qs = torch.from_numpy(q.qsess).to(dev)
    fq = torch.from_numpy(q.fields).to(dev)
    found = fg.fp_find_eval(h, pq, qs, fields=fq)
    for _ in range(3):
        fg.fp_find_eval(h, pq, qs, fields=fq, out=found[:5], values=found[5])
    torch.cuda.synchronize()
    reps = 50
    e0.record()
    for _ in range(reps):
        fg.fp_find_eval(h, pq, qs, fields=fq, out=found[:5], values=found[5])
    e1.record()
    torch.cuda.synchronize()
    out["walsh_overset_N7"] = {"E": mesh.E, "points": q.P, "ms_per_call": e0.elapsed_time(e1) / reps,
                               "note": "box 16x16 + annulus 16x3, tagged interface points, find + eval of u, v, p"}
    return out


# ---------------------------------------------------------------------------
# served form: resident box + two rotated annular cylinders, Poisson requests
# ---------------------------------------------------------------------------
def run_served(args, fg, dev):
    """Served form: the box + two rotated annular cylinders resident (config
    4), a Poisson stream of requests served with continuous batching under a
    40 GB device-memory budget, both forms.  Capacity = 1e6-point requests
    served back to back; the stream runs at args.served_load of it.  Beside
    them, fp_find_eval on the same resident mesh over 4e6 points of the same
    mix in one device-resident call (what the loop's own overhead is measured
    against)."""
    import torch

    import synth
    from paper_1811_04891_gb300 import serve
    sc = args.served_scale
    box = tuple(max(2, int(round(v * sc ** (1 / 3)))) for v in (80, 40, 40))
    cyl = tuple(max(2, int(round(v * sc ** (1 / 3)))) for v in (64, 8, 64))
    mesh, iface = synth.box_two_annuli(box_shape=box, cyl_shape=cyl)
    F = 4
    coords_d = torch.from_numpy(mesh.coords).to(dev)
    x, y, z = coords_d[0], coords_d[1], coords_d[2]
    # u, v, w, p: closed-form fields sampled at the nodes (evaluated on the device)
    fields_d = torch.stack([torch.sin(np.pi * x) * torch.cos(np.pi * y) * torch.exp(z),
                            -torch.cos(np.pi * x) * torch.sin(np.pi * y) * torch.exp(z),
                            torch.sin(np.pi * z) * x, x * x + y * y - z * z]).contiguous()
    del x, y, z
    sub_d = torch.from_numpy(mesh.sub).to(dev)
    dist_d = torch.from_numpy(mesh.dist).to(dev)
    out = {"elements": int(mesh.E), "N": mesh.N, "budget_bytes": 40e9, "chunk_points": args.served_chunk}
    cal = synth.poisson_requests(iface, 4, seed=40, size_range=(10 ** 6, 10 ** 6))
    mean_size = (10 ** 6 - 10 ** 2) / np.log(10 ** 4)
    for form, prec in (("mixed", fg.PREC_MIXED), ("fp64", fg.PREC_FP64)):
        h = fg.fp_setup(coords_d, mesh.N, sub_d, dist_d, opts=fg.default_opts(precision=prec))
        posted = fg.Fields(h, fields_d) if form == "mixed" else None
        resident = fields_d.numel() * 8 * (2 if posted is not None else 1)
        # the same points through one fused device-resident call
        allp = torch.from_numpy(np.ascontiguousarray(np.concatenate([r["pts"] for r in cal], axis=1))).to(dev)
        allq = torch.from_numpy(np.concatenate([r["qsess"] for r in cal])).to(dev)
        fg.fp_reserve(h, allp.shape[1])
        o5 = fg._find_outs(allp.shape[1], dev)
        vals = torch.empty((F, allp.shape[1]), dtype=torch.float64, device=dev)
        for _ in range(2):
            fg.fp_find_eval(h, allp, allq, fields=fields_d, posted=posted, out=o5, values=vals)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            fg.fp_find_eval(h, allp, allq, fields=fields_d, posted=posted, out=o5, values=vals)
        e1.record()
        torch.cuda.synchronize()
        direct = 3 * allp.shape[1] / (e0.elapsed_time(e1) / 1e3)
        del o5, vals, allp, allq
        srv = serve.Server(h, fields_d, budget_bytes=40e9, resident_bytes=resident, chunk_points=args.served_chunk,
                           streams=4, posted=posted, copy_threads=4)
        # capacity: 1e6-point requests back to back (the first pass also fills the buffer pools)
        for _ in range(2):
            srv.completed = []
            done, span = serve.run_stream(srv, [serve.Request(i, 0.0, r["pts"], r["qsess"])
                                                for i, r in enumerate(cal)])
        capacity = sum(r.P for r in done) / span
        rate = args.served_load * capacity / mean_size
        reqs = synth.poisson_requests(iface, args.served_requests, seed=4, rate_hz=rate)
        srv.completed, srv.launches, srv.held_back, srv.peak_inflight_bytes = [], 0, 0, 0
        srv.chunk_sizes = []
        done, span = serve.run_stream(srv, [serve.Request(i, r["t_arrive"], r["pts"], r["qsess"])
                                            for i, r in enumerate(reqs)])
        st = serve.latency_stats(done)
        tot = sum(r.P for r in done)
        codes = np.bincount(np.concatenate([r.code for r in done]), minlength=4).tolist()
        out[form] = {"p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                     "requests": st["requests"], "points": int(tot), "points_per_s": tot / span,
                     "capacity_points_per_s": capacity, "direct_fp_find_eval_points_per_s": direct,
                     "capacity_over_direct": capacity / direct, "arrival_rate_hz": rate, "load": args.served_load,
                     "chunks": srv.launches, "mean_chunk_points": float(np.mean(srv.chunk_sizes)),
                     "held_back_passes": srv.held_back, "peak_inflight_bytes": srv.peak_inflight_bytes,
                     "copy_threads": srv.copy_threads,
                     "resident_bytes": srv.resident,
                     "codes": {"inside": codes[0], "border": codes[1], "not_found": codes[2], "retry": codes[3]}}
        srv.close()
        del srv, posted, h
    out["note"] = ("Poisson arrivals, sizes logU[1e2,1e6], 50% uniform untagged + 50% cylinder interface nodes "
                   "tagged with their session; chunks of at most chunk_points admitted while their device bytes "
                   "fit the 40 GB budget beside the resident state; 4 streams; results copied into the requests "
                   "on 4 host threads; latency = arrival to results in "
                   "host memory; direct = one fp_find_eval over 4e6 device-resident points of the same mix")
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    import paper_1811_04891_gb300 as fg

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    barrier, max_over_ranks = make_collectives(dist, world, dev)

    mesh, q = workload(args)
    P = q.P
    coords = torch.from_numpy(mesh.coords).to(dev)
    sub = torch.from_numpy(mesh.sub).to(dev)
    fields = torch.from_numpy(q.fields).to(dev)
    pts = torch.from_numpy(q.pts).to(dev)
    F = fields.shape[0]
    stream = torch.cuda.current_stream(dev)
    code = torch.empty(P, dtype=torch.int32, device=dev)
    osub = torch.empty_like(code)
    elem = torch.empty_like(code)
    rst = torch.empty((3, P), dtype=torch.float64, device=dev)
    d2 = torch.empty(P, dtype=torch.float64, device=dev)
    out = torch.empty((F, P), dtype=torch.float64, device=dev)
    outs = (code, osub, elem, rst, d2)

    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None

    forms = [f.strip() for f in args.forms.split(",") if f.strip()]
    results = {}
    handles = {}
    for form in forms:
        prec = fg.PREC_MIXED if form == "mixed" else fg.PREC_FP64
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = fg.fp_setup(coords, mesh.N, sub, opts=fg.default_opts(precision=prec))
        torch.cuda.synchronize()
        setup_ms = 1e3 * (time.perf_counter() - t0)
        fg.fp_reserve(h, P)
        handles[form] = h
        # mixed form: fields posted once as double-float pairs, evaluated on the FP32 pipes
        posted = fg.Fields(h, fields) if form == "mixed" else None
        handles[form + "_fields"] = posted
        if posted is not None and args.stage_eval:
            fg.fp_set_eval_staging(h, True)

        def step(h=h, posted=posted):
            # one fused call: find, then eval in the element-sorted pair order
            fg.fp_find_eval(h, pts, None, fields=fields, posted=posted, out=outs, values=out)

        for _ in range(max(args.warmup, 1)):
            step()
        torch.cuda.synchronize()
        fg.fp_profile(h, True)
        for k in fg.PROF_KINDS:
            fg.fp_profile_read(h, k)
        fg.fp_band_hits(h)                      # reset: count the timed steps only
        clocks = ClockSampler(uuid)
        clocks.start()
        time.sleep(0.3)
        barrier()
        torch.cuda.synchronize()
        l0 = fg.fp_launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        launches = fg.fp_launch_count() - l0
        ms = ev0.elapsed_time(ev1)
        clk = clocks.stop()
        band = fg.fp_band_hits(h)
        paths = fg.fp_newton_paths(h) if form == "mixed" else None
        fg.fp_profile(h, False)
        kt = {k: fg.fp_profile_read(h, k) for k in fg.PROF_KINDS}
        ms_max = max_over_ranks(ms)
        counts = torch.bincount(code.long(), minlength=3).tolist()
        npairs = fg.fp_last_find_stats(h)
        results[form] = {"ms_per_step": ms_max / args.steps, "value": replica_rate(world, P, args.steps, ms_max),
                         "setup_ms": setup_ms, "gpu_launches": launches, "clocks": clk,
                         "kernel_ms": {k: (v[0] / max(v[1], 1)) for k, v in kt.items()},
                         "codes": {"inside": counts[0], "border": counts[1], "not_found": counts[2]},
                         "pairs_per_point": npairs / P, "newton_paths_per_step": None if paths is None else
                         {k: v // max(1, args.steps) for k, v in paths.items()},
                         "band_hits_per_step": {k: v / max(1, args.steps) for k, v in band.items()}}
        if posted is not None:
            # the other eval design beside the timed one: element fields staged
            # in shared memory per block, or read through L1 (same values)
            fg.fp_set_eval_staging(h, not args.stage_eval)
            for _ in range(2):
                step()
            torch.cuda.synchronize()
            fg.fp_profile(h, True)
            fg.fp_profile_read(h, "eval")
            for _ in range(args.steps):
                step()
            other = fg.fp_profile_read(h, "eval")
            fg.fp_profile(h, False)
            fg.fp_set_eval_staging(h, args.stage_eval)
            results[form]["eval_staging"] = {
                "timed_design": "staged in shared memory" if args.stage_eval else "L1 (rows shared by an element's threads)",
                "eval_ms_staged": other[0] / max(other[1], 1) if not args.stage_eval else results[form]["kernel_ms"]["eval"],
                "eval_ms_l1": results[form]["kernel_ms"]["eval"] if not args.stage_eval else other[0] / max(other[1], 1)}

    head = "mixed" if "mixed" in results else forms[0]
    R = results[head]

    peaks = None if args.no_peaks else measure_peaks(fg, dev, uuid)
    hbm_gbs, hbm_src = measured_hbm_gbs()
    coords_bytes, field_bytes = mesh.coords.nbytes, q.fields.nbytes
    roofs = {} if peaks is None else {
        f: roofline_form(f, P, F, results[f]["kernel_ms"], results[f]["ms_per_step"], peaks, hbm_gbs,
                         results[f]["pairs_per_point"] * P, coords_bytes, field_bytes) for f in results}
    roof = roofs.get(head)
    roof_other = {f: v for f, v in roofs.items() if f != head}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        h = handles[head]
        posted = handles.get(head + "_fields")
        # the library's host-memory entry point: points in, codes, ids, r,
        # dist^2 and values out, streamed in chunks with the copies
        # overlapping the search
        pts_h = torch.from_numpy(q.pts).pin_memory()
        outs_h = (torch.empty(P, dtype=torch.int32).pin_memory(), torch.empty(P, dtype=torch.int32).pin_memory(),
                  torch.empty(P, dtype=torch.int32).pin_memory(), torch.empty((3, P), dtype=torch.float64).pin_memory(),
                  torch.empty(P, dtype=torch.float64).pin_memory())
        out_h = torch.empty((F, P), dtype=torch.float64).pin_memory()

        def e2e_step():
            fg.fp_find_eval_host(h, pts_h, None, fields=fields, posted=posted, out=outs_h, values=out_h)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": replica_rate(world, P, args.steps, 1e3 * dt), "unit": UNIT, "h2d_bytes_per_step": int(pts_h.numel() * 8),
               "d2h_bytes_per_step": int(out_h.numel() * 8 + sum(t.numel() * t.element_size() for t in outs_h)),
               "api": "fp_find_eval_host (host buffers, chunks of 2^22 points, copies overlapped)"}

    small = None
    if rank == 0 and not args.no_small and peaks is not None:
        small = run_small_configs(args, fg, dev, peaks, with_oracle=not args.no_cpu_baseline)
    batched = None
    moving = None
    planar = None
    if rank == 0 and not args.no_planar:
        planar = run_planar(args, fg, dev)
    if not args.no_moving:
        moving = run_moving(args, fg, dev, mesh, coords, sub, pts, fields)
    if not args.no_batched:
        del handles
        batched = run_batched(args, fg, dev, barrier, max_over_ranks, world, peaks)
    served = None
    if rank == 0 and not args.no_served:
        served = run_served(args, fg, dev)
    interface = None
    if rank == 0 and not args.no_interface:
        interface = run_interface(args, fg, dev)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, m, cores, dt = oracle_rate(mesh, q, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{m} of the {P} points (strided), find + eval, {dt:.1f} s"}
        try:    # a side figure: its failure must not cost the measurement line
            r1, m1, dt1 = oracle_rate_one_core(mesh, q, min(5.0, args.cpu_seconds))
            cpu["one_core"] = {"value": r1, "unit": UNIT, "sample": f"{m1} strided points, {dt1:.1f} s"}
        except Exception as ex:  # noqa: BLE001
            cpu["one_core"] = {"error": str(ex)[:200]}

    if rank == 0:
        line = {"metric": METRIC, "value": R["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": R["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32" if head == "mixed" else "f64",
                "data": "synthetic", "config": config_dict(args, mesh, q), "form": head,
                "forms": {k: {"value": v["value"], "ms_per_step": v["ms_per_step"], "setup_ms": v["setup_ms"],
                              "kernel_ms": v["kernel_ms"], "codes": v["codes"],
                              "pairs_per_point": v["pairs_per_point"],
                              "newton_paths_per_step": v["newton_paths_per_step"],
                              "band_hits_per_step": v["band_hits_per_step"],
                              "eval_staging": v.get("eval_staging")} for k, v in results.items()},
                "roofline": roof, "roofline_other_forms": roof_other, "peaks": peaks,
                "hbm_peak": {"gbs": hbm_gbs, "source": hbm_src}, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": R["gpu_launches"],
                "clocks": R["clocks"], "small_configs": small, "batched": batched, "serving": served, "interface": interface,
                "moving": moving, "planar": planar}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
