"""Benchmark: complex double-double f + Jacobian evaluations per second.

Workload (one "step" = one evaluation of f and the full Jacobian at a batch
of points, i.e. the whole hot path: power table, common factors, Speelpenning
gradients, coefficient products and sums):
  n = 32 variables, 32 polynomials, m = 64 monomials each, k = 9 variables
  per monomial, exponents 1..5, unit-circle complex double-double
  coefficients and points, 1024 points per GPU (seeded synthetic data).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  With N > 1 (launched by torch.distributed.run) every
rank evaluates its own batch of 1024 points on its own GPU (weak scaling, no
collective on the data path); the reported time is the maximum over ranks and
`value` counts the points of all ranks.  `--impl reference` times the CPU
double-double oracle on the host cores on the same workload instead.
"""
from __future__ import annotations

import argparse
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
CONFIG_INDEX = 2
WORKLOAD = ("n=32 variables, 32 polynomials, m=64 monomials, k=9, exponents 1..5, unit-circle complex "
            "double-double coefficients and points, 1024 points per GPU")
L2_FLUSH_BYTES = 256 << 20
SMS = 152
DFMA_PER_SM_CLK = 2  # nominal FP64 FMA lanes per SM per clock on GB300
# DRAM bytes (read + write) of one main-kernel launch on this workload (two monomial chunks,
# one wave), from the ncu capture summarised in profiles/main_kernel_dd_n32_m64_k9_p1024.md:
# 5.45 MB read + 70.14 MB written. Set to None when the kernel changes.
MAIN_KERNEL_DRAM_BYTES = 5_449_984 + 70_139_648


def env_dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_points_seed(rank: int) -> int:
    """Each rank evaluates its own batch: the points seed depends on the rank."""
    return synth.SEED_BASE + CONFIG_INDEX + 1000 + 7919 * rank


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

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.gpu = gpu_index
        self.period = period_ms
        self.lines = []
        self.proc = None
        self.windows = []

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

    def mark(self, t0, t1):
        self.windows.append((t0, t1))

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
                rows.append((ts, float(parts[1]), float(parts[2]), parts[4:]))
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
            for name, val in zip(names, r[3][1:]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
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


def run_reference(args, rank, world):
    """The oracle arm: the C double-double oracle on the host cores."""
    if rank != 0:
        return
    import oracle

    system, pts = synth.config(CONFIG_INDEX)
    P_step = 256  # one step = a bounded sample of the workload
    sub = np.ascontiguousarray(pts[:, :P_step])
    threads = oracle.max_threads()
    out = (np.zeros((system.n_polys, P_step, 4)), np.zeros((system.n_polys, system.n_vars, P_step, 4)))
    for _ in range(args.warmup):
        oracle.dd_eval(system, sub, threads=threads, out=out)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.dd_eval(system, sub, threads=threads, out=out)
    el = time.perf_counter() - t0
    value = args.steps * P_step / el
    sample = f"{P_step} of the 1024 points of the workload per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "points_per_step": P_step, "oracle": "C double-double, term by term"},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


QD_SEED = synth.SEED_BASE + 500  # lower parts of the quad-double copy of the workload


def buf_fmt(prec):
    """Buffer set a precision reads and writes."""
    return {"f64": "f64", "qd": "qd"}.get(prec, "dd")


class Workload:
    """The batch one step evaluates, with an evaluator per precision
    ("dd": double-double on the FP64 pipe, "ddint": integer-pipe products,
    "f64": complex double, "qd": quad-double on the integer pipes, on the same
    data widened by two random lower parts), device buffers and pinned host
    buffers."""

    def __init__(self, cfg, rank, dev):
        import torch

        import paper_1201_0499_gb300 as pkg

        self.pkg, self.torch, self.dev, self.cfg = pkg, torch, dev, cfg
        codes = {"dd": pkg.PE_DD, "ddint": pkg.PE_DD_INT, "f64": pkg.PE_F64, "qd": pkg.PE_QD_INT}
        rng = np.random.Generator(np.random.PCG64(QD_SEED))

        def inputs(fmt, system, p):
            if fmt == "f64":
                return system.as_fp64(), np.ascontiguousarray(p[..., [0, 2]])
            if fmt == "qd":
                return system.to_qd(QD_SEED + 1), synth.widen_qd(rng, p)
            return system, p

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
            self.host = [t.cpu().pin_memory() for t in self.bufs["dd"]]
            self.system, self.pts = systems, pts
        else:
            if cfg == CONFIG_INDEX:
                system, _ = synth.config(cfg, n_points=1)
                P = 1024
                pts = synth.points(rank_points_seed(rank), system.n_vars, P)
                self.text = WORKLOAD
            else:
                system, pts = synth.config(cfg)
                P = pts.shape[1]
                self.text = synth.CONFIG_TEXT[cfg]
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
            self.host = [torch.from_numpy(pts).pin_memory(), torch.empty((N, P, 4), dtype=torch.float64).pin_memory(),
                         torch.empty((N, n, P, 4), dtype=torch.float64).pin_memory()]
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

    def cost_per_launch(self, prec):
        """FP64 instructions and flops of one main-kernel launch."""
        if self.cfg == 4:
            return self.ev[prec].cost()  # a batch handle reports whole-evaluation totals
        ops, flops = self.ev[prec].cost()
        return ops * self.points, flops * self.points


TRACK_N = 10  # variables of the path-tracking system (dense quadrics: 2^10 paths)


def nominal_paper_flops(wl):
    """Flops of one evaluation batch by the paper's operation counts: per
    monomial 6k - 5 complex products (k - 1 for the common factor, 5k - 4 for
    the Speelpenning gradient, value and coefficients, Sections 3.1-3.2) and
    k + 1 complex sums, a complex double-double product counted as 88 flops
    (four double-double products of 12 and two double-double sums of 20) and a
    sum as 40; plus n (d - 2) products per point for the powers."""
    s = wl.system
    k = np.diff(s.mono_ptr)
    per_point = float(np.sum(np.where(k > 0, (6 * k - 5) * 88 + (k + 1) * 40, 40)))
    per_point += s.n_vars * max(s.max_exp - 2, 0) * 88
    return per_point * wl.points


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


# The experiment shapes of the paper's Tables 1 and 2 (Section 4): n = 32,
# k = 9 with powers at most 2, and k = 16 with powers at most 10, each with 22,
# 32 and 48 monomials per polynomial; the paper times 100,000 evaluations.
PAPER_SHAPES = [(9, 2, 22), (9, 2, 32), (9, 2, 48), (16, 10, 22), (16, 10, 32), (16, 10, 48)]
PAPER_EVALS = 100_000


def paper_tables(pkg, torch):
    """Time PAPER_EVALS evaluations (one batch) of a synthetic system of each
    shape in double-double (FP64 pipe and integer pipes) and in double."""
    rows = []
    for i, (k, d, m) in enumerate(PAPER_SHAPES):
        s = synth.regular_system(synth.SEED_BASE + 800 + i, 32, m, k, d)
        pts = synth.points(synth.SEED_BASE + 900 + i, 32, PAPER_EVALS)
        row = {"k": k, "max_power": d, "monomials": 32 * m}
        for name, code in (("dd", pkg.PE_DD), ("ddint", pkg.PE_DD_INT), ("f64", pkg.PE_F64)):
            sk = s.as_fp64() if code == pkg.PE_F64 else s
            x = torch.from_numpy(np.ascontiguousarray(pts[..., [0, 2]]) if code == pkg.PE_F64 else pts).cuda()
            ev = pkg.PolyEval(sk, code, max_points=PAPER_EVALS)
            f, J = ev.eval(x)  # warm-up
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 3
            e0.record()
            for _ in range(reps):
                ev.eval(x, f, J)
            e1.record()
            torch.cuda.synchronize()
            assert ev.status() == pkg.PE_OK
            ms = e0.elapsed_time(e1) / reps
            row[name] = {"ms": ms, "us_per_eval": 1e3 * ms / PAPER_EVALS, "evals_per_s": PAPER_EVALS / (ms * 1e-3)}
            ev.close()
            del x, f, J
        rows.append(row)
    return {"evaluations": PAPER_EVALS, "n": 32, "shapes": rows,
            "data": "synthetic systems of the shapes of Tables 1-2, unit-circle points, one batch"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="dd", choices=["dd", "ddint"],
                    help="dd: double-double on the FP64 pipe; ddint: products in 128-bit integer block "
                         "floating point, sums in double-double (same inputs, outputs and accuracy bar)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip polyeval_autotune (launch choices from the built-in heuristic)")
    ap.add_argument("--graph", action="store_true",
                    help="replay the evaluation from a captured CUDA graph in the timed steps")
    ap.add_argument("--no-tracker", action="store_true", help="skip the path-tracking leg")
    ap.add_argument("--paper-tables", action="store_true",
                    help="time the experiment shapes of the paper's Tables 1-2 and print their JSON object")
    ap.add_argument("--only-tracker", action="store_true",
                    help="run only the path-tracking leg and print its JSON object (for profiling the tracker)")
    ap.add_argument("--config", type=int, default=CONFIG_INDEX, choices=[2, 3, 4, 5],
                    help="workload (default 2, the benchmark workload; 3, 4, 5: the larger and ragged ones)")
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
    if args.paper_tables:
        out = paper_tables(pkg, torch)
        if rank == 0:
            print(json.dumps({"paper_tables": out}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.only_tracker:
        out = track_leg(pkg, torch)
        if rank == 0:
            print(json.dumps({"path_tracker": out}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    wl = Workload(args.config, rank, dev)
    prim = args.precision
    other = "ddint" if prim == "dd" else "dd"
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    tuned = {}
    if not args.no_autotune and args.config != 4:
        # pick the launch per precision on this batch, before any timed step
        for prec in ("dd", "ddint", "f64", "qd"):
            x, f, J = wl.bufs[buf_fmt(prec)]
            tuned[prec] = pkg.polyeval_autotune(wl.handle(prec), x, wl.points, f, J, stream)
        torch.cuda.synchronize()

    graphs = {}

    def step(prec):
        if prec in graphs:
            graphs[prec].replay()
        else:
            wl.eval(prec)

    def timed_loop(prec, steps):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        stops = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for i in range(steps):
            flush.zero_()  # L2 flush between timed steps (outside the step's events)
            starts[i].record(stream)
            step(prec)
            stops[i].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in zip(starts, stops))

    if args.graph:
        # capture one evaluation per precision; the library call queues only
        # kernels and a memset on the capturing stream
        for prec in ("dd", "ddint", "f64", "qd"):
            wl.eval(prec)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                wl.eval(prec)
            graphs[prec] = g
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(prim)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    pkg.polyeval_timing(wl.handle(prim), True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    total_ms = timed_loop(prim, args.steps)
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
        kt = min(args.steps, 20)
        for _ in range(kt):
            flush.zero_()
            wl.eval(prim)
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
    peaks = peaks_file()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_nominal = SMS * DFMA_PER_SM_CLK * 2 * sm_max * 1e6 / 1e12
    # the paper's method at its own cost (6k - 5 complex products and k + 1
    # complex sums per monomial, dd product 88 flops, dd sum 40): what the same
    # evaluations would cost done the paper's way, per second of this kernel
    nominal_flops = nominal_paper_flops(wl) if args.config != 4 else None
    fma_rate, probe_mhz = pkg.polyeval_fp64_peak(stream)
    peak_probe = 2 * fma_rate / 1e12
    issue_rate = ops_launch / (kern_avg_ms * 1e-3)

    # complex double path and the other double-double path on the same workload, same harness
    legs = {}
    for leg in ("f64", other, "qd"):
        for _ in range(args.warmup):
            step(leg)
        kl = max(args.steps, 10) if args.config == CONFIG_INDEX else args.steps
        legs[leg] = max_over_ranks(timed_loop(leg, kl) / kl, dist)
    ms64 = legs["f64"]

    def newton_leg(prec, ms_eval):
        """Newton steps from the same start (x restored before each, outside
        the events); the solve's share is the step time less the evaluation's."""
        ev_p = wl.ev[prec]
        xb, fb, Jb = wl.bufs[buf_fmt(prec)]
        x0 = xb.clone()
        xn = x0.clone()
        dx = torch.empty_like(fb)
        lu = torch.empty_like(Jb)
        nrm = torch.empty((P, 2), dtype=torch.float64, device=dev)
        for _ in range(max(args.warmup, 1)):  # the first quad-double call at n > 22 allocates its scratch
            xn.copy_(x0)
            pkg.polyeval_newton(ev_p.handle, xn, P, dx, lu, nrm, stream)
        kn = max(min(args.steps, 50), 3)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(kn)]
        stops = [torch.cuda.Event(enable_timing=True) for _ in range(kn)]
        for i in range(kn):
            xn.copy_(x0)
            flush.zero_()
            starts[i].record(stream)
            pkg.polyeval_newton(ev_p.handle, xn, P, dx, lu, nrm, stream)
            stops[i].record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(starts, stops)) / kn, dist)
        return {"ms_per_step": ms, "solve_ms": ms - ms_eval, "points_per_s": job_throughput(world, P, ms)}

    # Newton step (evaluation + LU solve per point + update) with the primary
    # precision, and with quad-double (quad-double f and J, double-double solve)
    newton = None
    if args.config != 4:
        newton = newton_leg(prim, ms_per_step)
        newton["what"] = "f, J, LU with partial pivoting per point, x += dx (polyeval_newton)"
        newton["qd"] = newton_leg("qd", legs["qd"])
        newton["qd"]["what"] = ("quad-double f and J, LU in double-double from their leading parts, x + dx "
                                "rounded to quad-double")

    # the paper's three-kernel design on the same batch (double-double), for comparison
    paper = None
    if args.config == CONFIG_INDEX:
        ev_paper = pkg.PolyEval(wl.system, pkg.PE_DD, max_points=P, flags=pkg.PE_PAPER_KERNELS)
        xd, fd, Jd = wl.bufs["dd"]
        for _ in range(args.warmup):
            ev_paper.eval(xd, fd, Jd)
        kp = max(min(args.steps, 50), 3)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(kp)]
        stops = [torch.cuda.Event(enable_timing=True) for _ in range(kp)]
        for i in range(kp):
            flush.zero_()
            starts[i].record(stream)
            ev_paper.eval(xd, fd, Jd)
            stops[i].record(stream)
        torch.cuda.synchronize()
        ms_paper = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(starts, stops)) / kp, dist)
        paper = {"ms_per_step": ms_paper, "evals_per_s": job_throughput(world, P, ms_paper),
                 "fused_fp64_dd_speedup": ms_paper / (ms_per_step if prim == "dd" else legs["dd"]),
                 "what": "the paper's K1 common factors / K2 Speelpenning + coefficients into zero-padded Mons / "
                         "K3 one thread per output, complex double-double (PE_PAPER_KERNELS)"}
        ev_paper.close()

    # path tracking on top of the evaluation (total-degree homotopy)
    tracker = None
    if args.config == CONFIG_INDEX and not args.no_tracker:
        tracker = track_leg(pkg, torch)

    # end to end through the public API: pinned host in, pinned host out
    for _ in range(max(args.warmup, 1)):
        wl.eval_host(prim)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        wl.eval_host(prim)
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, dist)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.config == CONFIG_INDEX:
        rate, cores, sample = cpu_oracle_rate(wl.system, wl.pts, seconds=10.0)
        rate1, _c1, sample1 = cpu_oracle_rate(wl.system, wl.pts, seconds=5.0, max_points=64, threads=1)
        cpu = {"value": rate, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample,
               "single_core": {"value": rate1, "sample": sample1}}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value,
            "unit": "evals/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_per_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl.text, "points_per_gpu": P, "gpu": torch.cuda.get_device_name(dev),
                       "precision": ("complex double-double" if args.precision == "dd" else
                                     "complex double-double in/out, products in 128-bit integer block floating point"),
                       "l2": "flushed between timed steps (256 MiB write outside the step events)",
                       "cuda_graph": bool(args.graph),
                       "autotuned_launch": {k: {"chunks": v[0], "shape": "one wave" if v[1] == 1 else "persistent",
                                                "monomial_groups_per_warp": v[2]}
                                            for k, v in tuned.items()},
                       "launch": f"{kernels // max(args.steps, 1)} kernels per step (power table, monomial "
                                 "kernel, combine of monomial chunks when the call has few items)"},
            "e2e": {"value": job_throughput(world, P, e2e_ms), "unit": "evals/s",
                    "h2d_bytes_per_step": wl.h2d_bytes, "d2h_bytes_per_step": wl.d2h_bytes},
            "gpu_launches": kernels,
            "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": peak_nominal, "unit": "TFLOP/s",
                         "frac": achieved_tflops / peak_nominal,
                         "traffic": MAIN_KERNEL_DRAM_BYTES if args.config == CONFIG_INDEX else None,
                         "kernel": "main_kernel<ArithDD>" if args.precision == "dd" else "main_wide",
                         "kernel_ms": kern_avg_ms,
                         "peak_basis": f"nominal: {SMS} SMs x {DFMA_PER_SM_CLK} FP64 FMA/clk x 2 flops x {sm_max:.0f} MHz",
                         "peak_probe": peak_probe, "frac_of_probe": achieved_tflops / peak_probe,
                         "probe_sm_mhz": probe_mhz,
                         "fp64_issue_frac": issue_rate / (SMS * DFMA_PER_SM_CLK * sm_max * 1e6),
                         "paper_method_equiv_tflops": (nominal_flops / (kern_avg_ms * 1e-3) / 1e12
                                                       if nominal_flops else None)},
            "fp64_path": {"evals_per_s": job_throughput(world, P, ms64), "ms_per_step": ms64,
                          # FP64 instructions of the step's main kernel over the whole step time
                          "fp64_issue_frac": (wl.cost_per_launch("f64")[0] / (ms64 * 1e-3)
                                              / (SMS * DFMA_PER_SM_CLK * sm_max * 1e6))},
            "dd_fp64_time_ratio": (ms_per_step if prim == "dd" else legs["dd"]) / ms64,
            ("int_pipe_path" if other == "ddint" else "fp64_dd_path"): {
                "evals_per_s": job_throughput(world, P, legs[other]), "ms_per_step": legs[other],
                "speedup_vs_fp64_dd": (ms_per_step / legs[other]) if other == "ddint" else (legs[other] / ms_per_step),
                "precision": ("complex double-double in/out, products in 128-bit integer block floating point, "
                              "sums in double-double" if other == "ddint" else "complex double-double on the FP64 pipe")},
            "qd_int_path": {
                "evals_per_s": job_throughput(world, P, legs["qd"]), "ms_per_step": legs["qd"],
                "time_vs_fp64_dd": legs["qd"] / (ms_per_step if prim == "dd" else legs["dd"]),
                "precision": "complex quad-double in/out (the same data with two random lower parts), products in "
                             "256-bit integer block floating point, sums in 224-bit integer accumulators"},
            "fp64_peak_frac": achieved_tflops / peak_nominal,
            "newton_step": newton,
            "path_tracker": tracker,
            "paper_three_kernels": paper,
            "clocks": clocks,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
