"""Benchmark: complex double-double f + Jacobian evaluations per second.

Workload (one "step" = one evaluation of f and the full Jacobian at a batch
of points, i.e. the whole hot path: power table, common factors, Speelpenning
gradients, coefficient products and sums):
  n = 128 variables, 128 polynomials, m = 1024 monomials each, k = 32
  variables per monomial, exponents 1..4, unit-circle complex double-double
  coefficients and points, 16384 points per GPU (seeded synthetic data).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  With N > 1 (launched by torch.distributed.run) every
rank evaluates its own batch of points on its own GPU (weak scaling, no
collective on the data path); the reported time is the maximum over ranks and
`value` counts the points of all ranks.  `--impl reference` times the CPU
double-double oracle on the host cores on bounded samples of the same
workload instead.

Besides the headline (double-double on the FP64 pipe) the line carries the
same workload in complex double, in double-double with integer-pipe products
and in quad-double, and under "secondary" the smaller workloads: n = 32 at
1024 points (with Newton steps, the paper's three-kernel design and path
tracking), n = 64 at 4096 points, and the batch of 200 uneven systems in one
launch.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "complex-dd f+Jacobian evals/s on 1 GB300; %FP64 peak; dd/FP64 time ratio"
CONFIG_INDEX = 5
WORKLOAD = ("n=128 variables, 128 polynomials, m=1024 monomials, k=32, exponents 1..4, unit-circle complex "
            "double-double coefficients and points, 16384 points per GPU")
L2_FLUSH_BYTES = 256 << 20
SMS = 152
DFMA_PER_SM_CLK = 2  # nominal FP64 FMA lanes per SM per clock on GB300

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch
# of the double-double main kernel on the first 512 points of the n = 128
# workload, from one ncu capture, per point: a launch's traffic grows with its
# points (points and power table in, f and J out, the J rows read and written
# while they are summed), so it scales to the 16384-point launch by the points.
# The figure belongs to the kernel sources it was taken on (their fingerprint,
# kernel_sources_sha()); with other sources the line reports null.
MAIN_TRAFFIC_PER_POINT = (19_233_778_176 + 35_684_915_200) / 512  # read + write bytes of the capture / points
MAIN_TRAFFIC_SOURCES = "daec4a2983d22163"
KERNEL_SOURCES = ("kernels.cu", "dd.cuh", "arith.cuh", "items.cuh", "internal.h")


def kernel_sources_sha() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1201_0499_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def env_dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_points_seed(cfg: int, rank: int) -> int:
    """Each rank evaluates its own batch: the points seed depends on the rank
    (rank 0 draws the workload's own points)."""
    return synth.SEED_BASE + cfg + 1000 + 7919 * rank


def max_over_ranks(value: float, dist) -> float:
    """Largest value over all ranks (timings: the slowest rank sets the time)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, points_per_rank: int, ms_per_step: float) -> float:
    """Evaluations per second of the whole job (weak scaling: every rank has its own points)."""
    return world * points_per_rank / (ms_per_step * 1e-3)


def peaks_file():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh)
    return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 200):
        self.gpu = gpu_index
        self.period = period_ms
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.period)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self, t0, t1):
        rows = []
        for ts, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((ts, float(parts[1]), float(parts[2]), float(parts[3]), parts[4:]))
            except ValueError:
                continue
        inside = [r for r in rows if t0 <= r[0] <= t1]
        window = "timed region"
        if not inside:  # timed region shorter than the sampling period: nearest samples under the same load
            inside = sorted(rows, key=lambda r: min(abs(r[0] - t0), abs(r[0] - t1)))[:3]
            window = "nearest samples to the timed region"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in inside:
            for name, val in zip(names, r[4][1:]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "power_w_median": statistics.median(r[3] for r in inside),
                "reasons": sorted(reasons), "samples": len(inside), "window": window}


def cpu_oracle_rate(system, pts, seconds: float = 10.0, max_points=None, threads=None):
    """The C double-double oracle on the host cores (all of them, or
    `threads`): evaluations per second, repeating the batch (or its first
    max_points points) for ~`seconds`."""
    import oracle

    P = pts.shape[1] if max_points is None else min(max_points, pts.shape[1])
    sub = np.ascontiguousarray(pts[:, :P])
    threads = oracle.max_threads() if threads is None else threads
    out = (np.zeros((system.n_polys, P, 4)), np.zeros((system.n_polys, system.n_vars, P, 4)))
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.dd_eval(system, sub, threads=threads, out=out)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return reps * P / el, threads, f"{P} points of the workload, evaluated {reps} times ({el:.1f} s)"


# points of the workload the oracle arm evaluates per step: one tile, about a
# point per host core
REFERENCE_POINTS_PER_STEP = 16


def run_reference(args, rank, world):
    """The oracle arm: the C double-double oracle on the host cores."""
    if rank != 0:
        return
    import oracle

    system, pts = synth.config(CONFIG_INDEX, n_points=args.reference_points)
    P_step = pts.shape[1]
    sub = np.ascontiguousarray(pts)
    threads = oracle.max_threads()
    out = (np.zeros((system.n_polys, P_step, 4)), np.zeros((system.n_polys, system.n_vars, P_step, 4)))
    for _ in range(args.warmup):
        oracle.dd_eval(system, sub, threads=threads, out=out)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.dd_eval(system, sub, threads=threads, out=out)
    el = time.perf_counter() - t0
    value = args.steps * P_step / el
    sample = f"the first {P_step} of the 16384 points of the workload per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "points_per_step": P_step, "oracle": "C double-double, term by term"},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


QD_SEED = synth.SEED_BASE + 500  # lower parts of the quad-double copy of a workload
POINTS = {2: 1024, 3: 4096, 5: 16384}  # points per GPU of the single-system workloads
PRECS = ("dd", "ddint", "f64", "qd")


def buf_fmt(prec):
    """Buffer set a precision reads and writes."""
    return {"f64": "f64", "qd": "qd"}.get(prec, "dd")


class Workload:
    """The batch one step evaluates, with an evaluator per precision
    ("dd": double-double on the FP64 pipe, "ddint": integer-pipe products,
    "f64": complex double, "qd": quad-double on the integer pipes, on the same
    data widened by two random lower parts), device buffers and, with
    `host`, pinned host buffers for the end-to-end leg."""

    def __init__(self, cfg, rank, dev, host=False, points=0):
        import torch

        import paper_1201_0499_gb300 as pkg

        self.pkg, self.torch, self.dev, self.cfg = pkg, torch, dev, cfg
        codes = {"dd": pkg.PE_DD, "ddint": pkg.PE_DD_INT, "f64": pkg.PE_F64, "qd": pkg.PE_QD_INT}
        rng = np.random.Generator(np.random.PCG64(QD_SEED + cfg))

        def inputs(fmt, system, p):
            if fmt == "f64":
                return system.as_fp64(), np.ascontiguousarray(p[..., [0, 2]])
            if fmt == "qd":
                return system.to_qd(QD_SEED + 1), synth.widen_qd(rng, p)
            return system, p

        self.host = None
        if cfg == 4:
            systems, pts = synth.config(4)
            self.text = synth.CONFIG_TEXT[4] + ", one launch"
            npts = [p.shape[1] for p in pts]
            self.ev, self.bufs = {}, {}
            for k, code in codes.items():
                ins = [inputs(buf_fmt(k), s_, p_) for s_, p_ in zip(systems, pts)]
                self.ev[k] = pkg.PolyEvalMany([a for a, _ in ins], npts, code)
                if k in ("dd", "f64", "qd"):
                    b = self.ev[k].buffers(dev)
                    self.ev[k].pack_points([torch.from_numpy(np.ascontiguousarray(b_)) for _, b_ in ins], b[0])
                    self.bufs[k] = b
            self.points = sum(npts)
            if host:
                self.host = [t.cpu().pin_memory() for t in self.bufs["dd"]]
            self.system, self.pts = systems, pts
        else:
            system, _ = synth.config(cfg, n_points=1)
            P = POINTS[cfg] if points <= 0 else min(points, POINTS[cfg])
            mod = (-1, 0) if cfg == 3 else None
            pts = synth.points(rank_points_seed(cfg, rank), system.n_vars, P, modulus_octaves=mod)
            self.text = WORKLOAD if cfg == CONFIG_INDEX else synth.CONFIG_TEXT[cfg]
            n, N = system.n_vars, system.n_polys
            self.system, self.pts, self.points = system, pts, P
            self.ev, self.bufs = {}, {}
            for k, code in codes.items():
                fmt = buf_fmt(k)
                sk, pk = inputs(fmt, system, pts)
                self.ev[k] = pkg.PolyEval(sk, code, max_points=P)
                if k == fmt:
                    c = pk.shape[-1]
                    self.bufs[fmt] = (torch.from_numpy(pk).to(dev),
                                      torch.empty((N, P, c), dtype=torch.float64, device=dev),
                                      torch.empty((N, n, P, c), dtype=torch.float64, device=dev))
            if host:
                self.host = [torch.from_numpy(pts).pin_memory(),
                             torch.empty((N, P, 4), dtype=torch.float64, pin_memory=True),
                             torch.empty((N, n, P, 4), dtype=torch.float64, pin_memory=True)]
        if self.host is not None:
            self.h2d_bytes = int(self.host[0].numel() * 8)
            self.d2h_bytes = int((self.host[1].numel() + self.host[2].numel()) * 8)

    def handle(self, prec):
        return self.ev[prec].handle

    def eval(self, prec):
        x, f, J = self.bufs[buf_fmt(prec)]
        if self.cfg == 4:
            self.ev[prec].eval_buffers(x, f, J)
        else:
            self.ev[prec].eval(x, f, J)

    def eval_host(self, prec):
        """Host points in, host f and J out, through the public entry points."""
        if self.cfg == 4:
            x, f, J = self.bufs["dd"]
            x.copy_(self.host[0], non_blocking=True)
            self.ev[prec].eval_buffers(x, f, J)
            self.host[1].copy_(f, non_blocking=True)
            self.host[2].copy_(J, non_blocking=True)
            self.torch.cuda.current_stream().synchronize()
        else:
            hp, hf, hJ = self.host
            self.pkg.polyeval_eval_host(self.ev[prec].handle, hp, self.points, hf, hJ,
                                        self.torch.cuda.current_stream())

    def autotune(self, prec, stream):
        x, f, J = self.bufs[buf_fmt(prec)]
        if self.cfg == 4:
            return self.ev[prec].autotune(x, f, J, stream)
        return self.pkg.polyeval_autotune(self.handle(prec), x, self.points, f, J, stream)

    def cost_per_launch(self, prec):
        """FP64 instructions and flops of one main-kernel launch."""
        if self.cfg == 4:
            return self.ev[prec].cost()  # a batch handle reports whole-evaluation totals
        ops, flops = self.ev[prec].cost()
        return ops * self.points, flops * self.points

    def close(self):
        for ev in self.ev.values():
            ev.close()
        self.ev, self.bufs, self.host = {}, {}, None


def nominal_paper_flops(system, points):
    """Flops of one evaluation batch by the paper's operation counts: per
    monomial 6k - 5 complex products (k - 1 for the common factor, 5k - 4 for
    the Speelpenning gradient, value and coefficients, Sections 3.1-3.2) and
    k + 1 complex sums, a complex double-double product counted as 88 flops
    (four double-double products of 12 and two double-double sums of 20) and a
    sum as 40; plus n (d - 2) products per point for the powers."""
    k = np.diff(system.mono_ptr)
    per_point = float(np.sum(np.where(k > 0, (6 * k - 5) * 88 + (k + 1) * 40, 40)))
    per_point += system.n_vars * max(system.max_exp - 2, 0) * 88
    return per_point * points


class Timer:
    """Steps of one precision timed with CUDA events on the launching stream,
    the L2 flushed before each step outside its events."""

    def __init__(self, torch, stream, dev):
        self.torch, self.stream = torch, stream
        self.flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def run(self, fn, steps):
        torch = self.torch
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        stops = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for i in range(steps):
            self.flush.zero_()
            starts[i].record(self.stream)
            fn()
            stops[i].record(self.stream)
        torch.cuda.synchronize()
        self.last = [a.elapsed_time(b) for a, b in zip(starts, stops)]
        return sum(self.last)


def leg_ms(timer, wl, prec, warmup, reps, dist):
    """Mean step time of one precision on a workload (max over ranks)."""
    for _ in range(warmup):
        wl.eval(prec)
    return max_over_ranks(timer.run(lambda: wl.eval(prec), reps) / reps, dist)


TRACK_N = 10  # variables of the path-tracking system (dense quadrics: 2^10 paths)


def track_leg(pkg, torch):
    """Solve a generic system of TRACK_N dense quadrics (every monomial of
    degree <= 2) by following all 2^TRACK_N paths of the total-degree
    homotopy: in double, in double-double (evaluations on the FP64 pipe and
    on the integer pipes; linear solves in double with double-double
    residuals), and adaptively (double, then double-double refinement and
    re-tracking of failed paths)."""
    s = synth.dense_system(synth.SEED_BASE + 700, TRACK_N, [2] * TRACK_N)
    B = 2 ** TRACK_N
    out = {"system": f"{TRACK_N} dense quadrics in {TRACK_N} variables (66 monomials each), {B} paths"}
    hs = {}
    for name, code in (("f64", pkg.PE_F64), ("dd", pkg.PE_DD), ("ddint", pkg.PE_DD_INT)):
        ev = pkg.PolyEval(s.as_fp64() if code == pkg.PE_F64 else s, code, max_points=B)
        hs[name] = ev
        ev.track(ev.start_points(B))  # warm-up (allocates the tracker's scratch)
        x = ev.start_points(B)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, _t, it = ev.track(x)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        # iterations of the batch (each one evaluation of f and J at every
        # running path, the batch compacted as paths end)
        out[name] = {"ms": el * 1e3, "paths_per_s": B / el, "iterations": it,
                     "success": int((st == 1).sum().item())}
    lo, hi = hs["f64"], hs["ddint"]
    prm_lo, prm_hi = pkg.polyeval_track_defaults(pkg.PE_F64), pkg.polyeval_track_defaults(pkg.PE_DD)
    status = torch.empty(B, dtype=torch.int32, device="cuda")
    x = hi.start_points(B)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    esc = pkg.polyeval_track_adaptive(lo.handle, hi.handle, prm_lo, prm_hi, x, B, status)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    out["adaptive"] = {"ms": el * 1e3, "paths_per_s": B / el, "escalated_to_dd": esc,
                       "success": int((status == 1).sum().item()),
                       "what": "every path in double, end points refined by 3 Newton steps in double-double "
                               "(integer-pipe evaluation), failed paths tracked again in double-double "
                               "(polyeval_track_adaptive)"}
    for ev in hs.values():
        ev.close()
    return out


def newton_leg(pkg, torch, timer, wl, prec, ms_eval, warmup, reps, dist, world):
    """Newton steps from the same start (x restored before each, outside the
    events); the solve's share is the step time less the evaluation's."""
    P = wl.points
    ev_p = wl.ev[prec]
    xb, fb, Jb = wl.bufs[buf_fmt(prec)]
    x0 = xb.clone()
    xn = x0.clone()
    dx = torch.empty_like(fb)
    lu = torch.empty_like(Jb)
    nrm = torch.empty((P, 2), dtype=torch.float64, device=xb.device)
    for _ in range(max(warmup, 1)):  # the first quad-double call at n > 22 allocates its scratch
        xn.copy_(x0)
        pkg.polyeval_newton(ev_p.handle, xn, P, dx, lu, nrm, timer.stream)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    for i in range(reps):
        xn.copy_(x0)
        timer.flush.zero_()
        starts[i].record(timer.stream)
        pkg.polyeval_newton(ev_p.handle, xn, P, dx, lu, nrm, timer.stream)
        stops[i].record(timer.stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(starts, stops)) / reps, dist)
    return {"ms_per_step": ms, "solve_ms": ms - ms_eval, "points_per_s": job_throughput(world, P, ms)}


def paper_leg(pkg, torch, timer, wl, ms_dd, reps, dist, world):
    """The paper's three-kernel design on the same batch (double-double)."""
    P = wl.points
    ev_paper = pkg.PolyEval(wl.system, pkg.PE_DD, max_points=P, flags=pkg.PE_PAPER_KERNELS)
    xd, fd, Jd = wl.bufs["dd"]
    ev_paper.eval(xd, fd, Jd)
    ms = max_over_ranks(timer.run(lambda: ev_paper.eval(xd, fd, Jd), reps) / reps, dist)
    ev_paper.close()
    return {"ms_per_step": ms, "evals_per_s": job_throughput(world, P, ms), "fused_fp64_dd_speedup": ms / ms_dd,
            "what": "the paper's K1 common factors / K2 Speelpenning + coefficients into zero-padded Mons / "
                    "K3 one thread per output, complex double-double (PE_PAPER_KERNELS)"}


def secondary(cfg, pkg, torch, timer, rank, world, dev, dist, reps, sm_max):
    """One of the smaller workloads: every precision after autotuning, and on
    the n = 32 workload the Newton step, the paper's three kernels and the
    path tracker."""
    wl = Workload(cfg, rank, dev)
    out = {"workload": wl.text, "points_per_gpu": wl.points}
    tuned = {}
    for prec in PRECS:
        c, m, g = wl.autotune(prec, timer.stream)
        tuned[prec] = {"chunks": c, "shape": "one wave" if m == 1 else "persistent",
                       ("partial_tile_groups_cap" if cfg == 4 else "monomial_groups_per_warp"): g}
    torch.cuda.synchronize()
    out["autotuned_launch"] = tuned
    ms = {}
    for prec in PRECS:
        ms[prec] = leg_ms(timer, wl, prec, 1, reps, dist)
        out[prec] = {"evals_per_s": job_throughput(world, wl.points, ms[prec]), "ms_per_step": ms[prec]}
    ops, _flops = wl.cost_per_launch("dd")
    out["dd"]["fp64_issue_frac_of_step"] = ops / (ms["dd"] * 1e-3) / (SMS * DFMA_PER_SM_CLK * sm_max * 1e6)
    out["dd_fp64_time_ratio"] = ms["dd"] / ms["f64"]
    out["ddint_speedup_vs_fp64_dd"] = ms["dd"] / ms["ddint"]
    for prec in PRECS:
        assert pkg.polyeval_status(wl.handle(prec)) == pkg.PE_OK
    # the double-double evaluation captured once in a CUDA graph and replayed
    # (the library queues only kernels and a memset on the caller's stream)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        wl.eval("dd")
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(g):
        wl.eval("dd")
    g.replay()
    ms_g = max_over_ranks(timer.run(g.replay, reps) / reps, dist)
    out["dd"]["graph_replay"] = {"evals_per_s": job_throughput(world, wl.points, ms_g), "ms_per_step": ms_g}
    del g
    if cfg == 2:
        newton = newton_leg(pkg, torch, timer, wl, "dd", ms["dd"], 1, reps, dist, world)
        newton["what"] = "f, J, LU with partial pivoting per point, x += dx (polyeval_newton)"
        newton["qd"] = newton_leg(pkg, torch, timer, wl, "qd", ms["qd"], 1, reps, dist, world)
        newton["qd"]["what"] = ("quad-double f and J, LU in double-double from their leading parts, x + dx "
                                "rounded to quad-double")
        out["newton_step"] = newton
        out["paper_three_kernels"] = paper_leg(pkg, torch, timer, wl, ms["dd"], reps, dist, world)
        out["path_tracker"] = track_leg(pkg, torch)
    wl.close()
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--reference-points", type=int, default=REFERENCE_POINTS_PER_STEP,
                    help="points of the workload the oracle arm evaluates per step")
    ap.add_argument("--precision", default="dd", choices=["dd", "ddint"],
                    help="dd: double-double on the FP64 pipe; ddint: products in 128-bit integer block "
                         "floating point, sums in double-double (same inputs, outputs and accuracy bar)")
    ap.add_argument("--graph", action="store_true",
                    help="replay the evaluation from a captured CUDA graph in the timed steps")
    ap.add_argument("--no-secondary", action="store_true", help="skip the smaller workloads")
    ap.add_argument("--only-tracker", action="store_true",
                    help="run only the path-tracking leg and print its JSON object (for profiling the tracker)")
    ap.add_argument("--only-newton", action="store_true",
                    help="run only the Newton-step legs on the n = 32 workload and print their JSON object "
                         "(for profiling the solve)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in launch of a smaller headline workload instead of autotuning it")
    ap.add_argument("--points", type=int, default=0,
                    help="evaluate only the first POINTS points of a single-system workload (profiling of "
                         "smaller launches; 0: all)")
    ap.add_argument("--config", type=int, default=CONFIG_INDEX, choices=[2, 3, 4, 5],
                    help="headline workload (default 5, n = 128 at 16384 points; 2, 3, 4: the smaller and "
                         "ragged ones, for experiments)")
    args = ap.parse_args()
    rank, world, local = env_dist()
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist is not None:
            dist.destroy_process_group()
        return

    import torch

    import paper_1201_0499_gb300 as pkg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    if args.only_tracker:
        out = track_leg(pkg, torch)
        if rank == 0:
            print(json.dumps({"path_tracker": out}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.only_newton:
        wl2 = Workload(2, rank, dev)
        timer2 = Timer(torch, stream, dev)
        out = {}
        for prec in ("dd", "qd"):
            ms_eval = leg_ms(timer2, wl2, prec, 1, 3, dist)
            out[prec] = newton_leg(pkg, torch, timer2, wl2, prec, ms_eval, 1, 3, dist, world)
        if rank == 0:
            print(json.dumps({"newton_step": out}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    cfg = args.config
    wl = Workload(cfg, rank, dev, host=True, points=args.points)
    prim = args.precision
    other = "ddint" if prim == "dd" else "dd"
    timer = Timer(torch, stream, dev)
    peaks = peaks_file()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))

    tuned = {}
    if cfg != CONFIG_INDEX and not args.no_autotune:
        # pick the launch per precision on this batch, before any timed step
        for prec in PRECS:
            c, m, g = wl.autotune(prec, stream)
            tuned[prec] = {"chunks": c, "shape": "one wave" if m == 1 else "persistent", "groups": g}
        torch.cuda.synchronize()
        launch_note = "autotuned per precision (polyeval_autotune)"
    elif cfg != CONFIG_INDEX:
        launch_note = "built-in (autotuning skipped)"
    else:
        # 128 x 1024 (polynomial, tile) items fill many waves and one chunk of
        # outputs (8.7 GB) exceeds the chunk scratch: the tuner's only
        # candidate is the built-in persistent launch, so it is not run
        launch_note = "built-in: one monomial chunk, persistent grid of 4-warp blocks (the only candidate here)"

    graphs = {}

    def step(prec):
        if prec in graphs:
            graphs[prec].replay()
        else:
            wl.eval(prec)

    if args.graph:
        # capture one evaluation; the library call queues only kernels and a
        # memset on the capturing stream
        wl.eval(prim)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            wl.eval(prim)
        graphs[prim] = g
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(prim)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.5)
    pkg.polyeval_timing(wl.handle(prim), True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    total_ms = timer.run(lambda: step(prim), args.steps)
    step_ms = list(timer.last)
    t_wall1 = time.time()
    if dist is not None:
        dist.barrier()
    kern_ms, launches, kernels = pkg.polyeval_timing_read(wl.handle(prim))
    pkg.polyeval_timing(wl.handle(prim), False)
    sampler.stop()
    if graphs:
        # graph replays record no library events: time the main kernel on an
        # eager pass of the same evaluation, and count the graph's kernels
        pkg.polyeval_timing(wl.handle(prim), True)
        kt = min(args.steps, 3)
        timer.run(lambda: wl.eval(prim), kt)
        kern_ms, launches, k_eager = pkg.polyeval_timing_read(wl.handle(prim))
        pkg.polyeval_timing(wl.handle(prim), False)
        kernels = (k_eager // max(kt, 1)) * args.steps
    clocks = sampler.summary(t_wall0, t_wall1)
    assert pkg.polyeval_status(wl.handle(prim)) == pkg.PE_OK

    P = wl.points
    ms_per_step = max_over_ranks(total_ms / args.steps, dist)
    value = job_throughput(world, P, ms_per_step)

    # roofline of the main (monomial) kernel: FP64 pipe bound
    ops_launch, flops_launch = wl.cost_per_launch(prim)
    kern_avg_ms = kern_ms / max(launches, 1)
    achieved_tflops = flops_launch / (kern_avg_ms * 1e-3) / 1e12
    peak_nominal = SMS * DFMA_PER_SM_CLK * 2 * sm_max * 1e6 / 1e12
    # the paper's method at its own cost (6k - 5 complex products and k + 1
    # complex sums per monomial, dd product 88 flops, dd sum 40): what the same
    # evaluations would cost done the paper's way, per second of this kernel
    nominal_flops = nominal_paper_flops(wl.system, P) if cfg != 4 else None
    fma_rate, probe_mhz = pkg.polyeval_fp64_peak(stream)
    peak_probe = 2 * fma_rate / 1e12
    issue_rate = ops_launch / (kern_avg_ms * 1e-3)
    traffic = None
    if (cfg == CONFIG_INDEX and prim == "dd" and MAIN_TRAFFIC_PER_POINT is not None
            and MAIN_TRAFFIC_SOURCES == kernel_sources_sha()):
        traffic = MAIN_TRAFFIC_PER_POINT * P
    paper_tflops = nominal_flops / (kern_avg_ms * 1e-3) / 1e12 if nominal_flops else None

    # complex double path and the other double-double paths on the same
    # workload, same harness (one warm-up step and a few timed ones each: the
    # headline workload takes seconds per step)
    reps = min(args.steps, 3) if cfg == CONFIG_INDEX else max(args.steps, 10)
    legs = {leg: leg_ms(timer, wl, leg, 1, reps if leg != "qd" else max(min(reps, 2), 1), dist)
            for leg in ("f64", other, "qd")}
    for leg in legs:
        assert pkg.polyeval_status(wl.handle(leg)) == pkg.PE_OK
    ms64 = legs["f64"]
    ms_dd = ms_per_step if prim == "dd" else legs["dd"]

    # end to end through the public API: pinned host in, pinned host out
    wl.eval_host(prim)
    if dist is not None:
        dist.barrier()
    e2e_steps = min(args.steps, 3) if cfg == CONFIG_INDEX else args.steps
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        wl.eval_host(prim)
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / e2e_steps, dist)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and cfg != 4:
        rate, cores, sample = cpu_oracle_rate(wl.system, wl.pts, seconds=15.0, max_points=16)
        rate1, _c1, sample1 = cpu_oracle_rate(wl.system, wl.pts, seconds=5.0, max_points=1, threads=1)
        cpu = {"value": rate, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample,
               "single_core": {"value": rate1, "sample": sample1}}

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "step_ms_median": statistics.median(step_ms),
        "step_ms_min_max": [min(step_ms), max(step_ms)],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.text, "points_per_gpu": P, "gpu": torch.cuda.get_device_name(dev),
                   "precision": ("complex double-double" if prim == "dd" else
                                 "complex double-double in/out, products in 128-bit integer block floating point"),
                   "l2": "flushed between timed steps (256 MiB write outside the step events); the step's "
                         "outputs alone exceed the L2",
                   "cuda_graph": bool(args.graph),
                   "launch": launch_note,
                   "autotuned_launch": tuned or None,
                   "kernels_per_step": kernels // max(args.steps, 1)},
        "e2e": {"value": job_throughput(world, P, e2e_ms), "unit": "evals/s",
                "h2d_bytes_per_step": wl.h2d_bytes, "d2h_bytes_per_step": wl.d2h_bytes, "steps": e2e_steps,
                "what": "polyeval_eval_host: pinned host points in, pinned host f and J out, synchronous"},
        "gpu_launches": kernels,
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": peak_nominal, "unit": "TFLOP/s",
                     "frac": achieved_tflops / peak_nominal, "traffic": traffic,
                     "traffic_basis": ("ncu DRAM bytes per point of a 512-point launch of the same kernel on this "
                                       "workload, times the points" if traffic is not None else
                                       "no capture on the current kernel sources"),
                     "kernel": "main_kernel<ArithDD>" if prim == "dd" else "main_wide",
                     "kernel_ms": kern_avg_ms,
                     "achieved_basis": "FP64 flops the kernel executes (polyeval_cost: FMA = 2, add and "
                                       "multiply = 1), equal to the ncu instruction count",
                     "peak_basis": f"nominal: {SMS} SMs x {DFMA_PER_SM_CLK} FP64 FMA/clk x 2 flops x {sm_max:.0f} MHz",
                     "peak_probe": peak_probe, "frac_of_probe": achieved_tflops / peak_probe,
                     "probe_sm_mhz": probe_mhz,
                     "fp64_issue_frac": issue_rate / (SMS * DFMA_PER_SM_CLK * sm_max * 1e6),
                     "paper_method_equiv_tflops": paper_tflops,
                     "paper_method_frac": paper_tflops / peak_nominal if paper_tflops else None},
        "fp64_path": {"evals_per_s": job_throughput(world, P, ms64), "ms_per_step": ms64,
                      # FP64 instructions of the step's main kernel over the whole step time
                      "fp64_issue_frac": (wl.cost_per_launch("f64")[0] / (ms64 * 1e-3)
                                          / (SMS * DFMA_PER_SM_CLK * sm_max * 1e6))},
        "dd_fp64_time_ratio": ms_dd / ms64,
        ("int_pipe_path" if other == "ddint" else "fp64_dd_path"): {
            "evals_per_s": job_throughput(world, P, legs[other]), "ms_per_step": legs[other],
            "speedup_vs_fp64_dd": (ms_per_step / legs[other]) if other == "ddint" else (legs[other] / ms_per_step),
            "precision": ("complex double-double in/out, products in 128-bit integer block floating point, "
                          "sums in double-double" if other == "ddint" else "complex double-double on the FP64 pipe")},
        "qd_int_path": {
            "evals_per_s": job_throughput(world, P, legs["qd"]), "ms_per_step": legs["qd"],
            "time_vs_fp64_dd": legs["qd"] / ms_dd,
            "precision": "complex quad-double in/out (the same data with two random lower parts), products in "
                         "256-bit integer block floating point, sums in 224-bit integer accumulators"},
        "fp64_peak_frac": achieved_tflops / peak_nominal,
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    wl.close()
    del wl
    torch.cuda.empty_cache()

    if not args.no_secondary:
        sec = {}
        for c2 in (2, 3, 4):
            if c2 != cfg:
                sec[f"config{c2}"] = secondary(c2, pkg, torch, timer, rank, world, dev, dist, 5 if c2 != 2 else 10,
                                               sm_max)
        line["secondary"] = sec
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
