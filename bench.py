"""Throughput of canonical DMPT solves on GB300 (one JSON line on rank 0).

Workload (one step): the mixed-precision configuration, two systems solved canonically at
beta = 20 with n = 14 recursion steps and one dipole perturbation each:
  - the 20 x 20 x 20 periodic simple-cubic tight-binding lattice (N = 8000, on-site
    N(0, 0.3^2), hopping -1 +- 10 %, seed 1003), dipole along x;
  - a random symmetric banded matrix, N = 8192, bandwidth 64, entries N(0,1)/8 (seed 1004),
    perturbation diag(i - (N-1)/2).
A solve is the whole path: the occupation loop, the refinement, the first-order response,
mu1 and the polarizability, with P0 and P1 written out.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp32|fp64]
                  [--impl ours|reference] [--no-compare] [--no-cpu-baseline] [--no-extras]

The timed precision defaults to mixed (TF32 sweeps; refinement of the pair-stored
trajectory with split-TF32 and Ozaki-sliced FP64-class residuals; split-TF32 response).
One step in FP32 with split-TF32 products is timed beside it ("fp32"), and both precisions'
P0, P1, mu1 and alpha are compared with the FP64 oracle ("error"). Extras: the 16^3 lattice
at beta 5, 20 and 80 (N = 4096), the 96-cluster batch, and one FP64 solve.

--impl reference times the FP64 CPU oracle (exact diagonalisation) on the host cores, one
solve of the workload (alternating the two systems) per step.
Under torchrun every rank solves its own copy (weak scaling, no collective on the data
path); times are max-reduced over ranks.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("DMPT response solves/sec and tensor TFLOP/s vs peak, mixed vs FP32 at "
          "≤1e-6 err")
C3 = ("cubic20_b20", "banded8192")
WORKLOAD = ("mixed-precision config: 20x20x20 lattice (N=8000) and banded N=8192 (bandwidth 64), "
            "beta 20, n 14, D=1 dipole; one step = one canonical solve of each")
C2_BETAS = (5.0, 20.0, 80.0)
ENGINE_NAMES = {1: "CUDA-core FFMA/DFMA", 2: "tcgen05 TF32", 3: "tcgen05 3xTF32",
                4: "tcgen05 BF16", 5: "tcgen05 Ozaki BF16 digits"}
# tensor-pipe products per algorithmic product of each engine
PIPE_FACTOR = {2: 1.0, 3: 3.0, 4: 1.0, 5: 15.0}
# DRAM bytes (read + write) of one launch and its algorithmic flops, from the ncu captures
# summarised in profiles/ (engine 3: k_gemm_split2sm, D = Z Z^T + I at N = 8192); the roofline
# scales it to the mean launch of the step by algorithmic flops
TRAFFIC = {3: (3849249024 + 271198464, 2.0 * 8192.0 ** 3)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(pg, x, device):
    """Maximum of a host scalar over all ranks (x itself without a process group)."""
    if not pg:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": d["hbm_gbs"], "bf16": d["bf16_tflops"],
                "bf16_sustained": d.get("bf16_tflops_sustained", d["bf16_tflops"]),
                "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}


def measure_peaks(dev):
    """TF32 and FP64 tensor-library rates of this GPU, measured the way the driver measures the
    BF16 one: torch.matmul at 8192^3 (TF32, FP32 inputs) as the best of 10 and back to back for
    3 s, and at 4096^3 in FP64 (best of 3), with CUDA events."""
    import torch
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        n = 8192
        a = torch.randn((n, n), device=dev, dtype=torch.float32)
        b = torch.randn((n, n), device=dev, dtype=torch.float32)
        c = torch.empty_like(a)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(3):
            torch.matmul(a, b, out=c)
        best = 1e30
        for _ in range(10):
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out["tf32_tflops"] = 2.0 * n ** 3 / (best / 1e3) / 1e12
        reps = max(1, int(3000.0 / best))
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        out["tf32_tflops_sustained"] = 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) / 1e3) / 1e12
        del a, b, c
        n = 4096
        a = torch.randn((n, n), device=dev, dtype=torch.float64)
        b = torch.randn((n, n), device=dev, dtype=torch.float64)
        c = torch.empty_like(a)
        torch.matmul(a, b, out=c)
        best = 1e30
        for _ in range(3):
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out["fp64_tflops"] = 2.0 * n ** 3 / (best / 1e3) / 1e12
        del a, b, c
        torch.cuda.empty_cache()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    out["how"] = ("torch.matmul: TF32 8192^3 best of 10 and back to back for 3 s; FP64 4096^3 "
                  "best of 3; CUDA events, in this run")
    return out


# --------------------------------------------------------------------------- oracle timing

def oracle_solve(p, eig=None):
    """The FP64 oracle's solve of problem p (recursion-exact function), and its wall time."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", eig=eig)
    return r, time.perf_counter() - t0


def time_oracle_one_core():
    """The oracle's solve of the 16 x 16 x 8 lattice (N = 2048, beta 20) on one host core, in a
    child process whose BLAS pools are limited to one thread; scaled to the workload's mean N
    of 8096 by the N^3 cost of the eigendecomposition and the Daleckii-Krein products. A bounded
    sample: about 10 s on one core."""
    code = ("import time, oracle, synthetic\n"
            "p = synthetic.cubic_lattice((16, 16, 8), seed=1002, beta=20.0, n=14)\n"
            "t = time.perf_counter()\n"
            "oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind='rec')\n"
            "print(time.perf_counter() - t)\n")
    env = dict(os.environ)
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS",
              "BLIS_NUM_THREADS", "VECLIB_MAXIMUM_THREADS"):
        env[k] = "1"
    here = os.path.dirname(os.path.abspath(__file__))
    try:
        out = subprocess.run([sys.executable, "-c", code], cwd=here, env=env, capture_output=True,
                             text=True, timeout=300, check=True)
        dt = float(out.stdout.strip().splitlines()[-1])
    except Exception as e:   # a missing baseline must not fail the bench
        return {"unavailable": f"one-core oracle run failed: {e}"[:200]}
    scale = (8096.0 / 2048.0) ** 3
    return {"value": 1.0 / (scale * dt), "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"beta=20 solve of the 16x16x8 lattice (N=2048) in {dt:.1f} s on one core, "
                      f"scaled by (8096/2048)^3 to the workload's mean N"}


def blas_threads():
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return os.cpu_count()


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import synthetic
    probs = [synthetic.workload(c) for c in C3]
    seq = [probs[i % len(probs)] for i in range(args.warmup + args.steps)]
    for p in seq[:args.warmup]:
        oracle_solve(p)
    t0 = time.perf_counter()
    for p in seq[args.warmup:]:
        oracle_solve(p)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "fp64 exact diagonalisation (oracle)",
                   "step": "one solve of one of the two systems (alternating)"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": blas_threads(),
                         "kind": "oracle",
                         "sample": "one system per step: dsyevd N=8000 or 8192, bisection on mu, "
                                   "Daleckii-Krein P1, mu1, alpha"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- our path

def _errors(res, ref, D):
    """Errors of one solve's outputs against the oracle: P0, P1 (relative Frobenius, worst
    direction), alpha (relative, worst direction) and mu1 (worst direction, relative to
    max(|mu1|, 1): mu1 is an energy per unit field, and the hopping, 1, sets the scale where
    the dipole fields cancel and mu1 itself is near zero)."""
    import numpy as np

    import oracle
    e = {"P0": oracle.rel_frobenius(res["P0"], ref["P0"]),
         "P1": max(oracle.rel_frobenius(res["P1"][d], ref["P1"][d]) for d in range(D)),
         "mu1": max(abs(res["mu1"][d] - ref["mu1"][d]) / max(abs(ref["mu1"][d]), 1.0)
                    for d in range(D)),
         "alpha": max(abs(res["alpha"][d] - ref["alpha"][d]) / abs(ref["alpha"][d])
                      for d in range(D))}
    e["max"] = max(e["P0"], e["P1"], e["mu1"], e["alpha"])
    return {k: float(v) for k, v in e.items()}


def run_ours(args):
    import ctypes

    import numpy as np
    import torch

    import paper_1503_07037_gb300 as pkg
    import synthetic

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return reduce_max(pg, x, dev)

    stream = torch.cuda.current_stream()
    mpk = measure_peaks(dev)
    pk = peaks()
    probs = [synthetic.workload(c) for c in C3]
    bufs = []
    for p in probs:
        N, D = p.N, p.D
        bufs.append({"H0": torch.from_numpy(p.H0).to(dev), "H1": torch.from_numpy(p.H1).to(dev),
                     "P0": torch.empty((N, N), dtype=torch.float64, device=dev),
                     "P1": torch.empty((D, N, N), dtype=torch.float64, device=dev),
                     "mu": ctypes.c_double(), "mu1": np.zeros(D)})

    def make(precision, engine="auto"):
        hs = []
        for p, b in zip(probs, bufs):
            h = pkg.Handle(precision=precision, engine=engine, profile=True, stream=stream)
            h.set_H(b["H0"], b["H1"])       # resident in HBM before any timed region
            hs.append(h)
        return hs

    def step(hs, stats_acc=None, outs=None):
        for h, p, b in zip(hs, probs, bufs):
            pkg.solve_raw(h.h, p.beta, p.nocc, p.n, b["P0"].data_ptr(), b["P1"].data_ptr(),
                          ctypes.addressof(b["mu"]), b["mu1"].ctypes.data, 1)
            if stats_acc is not None:
                stats_acc.append(h.stats())
            if outs is not None:
                outs.append({"P0": b["P0"].cpu().numpy(), "P1": b["P1"].cpu().numpy(),
                             "mu1": b["mu1"].copy(), "alpha": h.polarizability()})

    def timed_steps(hs, k, stats_acc):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        for _ in range(k):
            step(hs, stats_acc)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1)

    hs = make(args.precision)
    for _ in range(args.warmup):
        step(hs)
    clocks = ClockSampler(local)
    clocks.start()
    st_all = []
    ms = timed_steps(hs, args.steps, st_all)
    clk = clocks.stop()
    ms = max_over_ranks(ms)
    barrier()
    solves = args.steps * len(probs) * world
    value = solves / (ms / 1000.0)
    outs_main = []
    step(hs, None, outs_main)

    # roofline of the dominant kernel: the GEMM engine with the most device time
    n_eng = len(st_all[0]["engine_ms"])
    eng_ms = [sum(s["engine_ms"][e] for s in st_all) for e in range(n_eng)]
    eng_n = [sum(s["engine_launches"][e] for s in st_all) for e in range(n_eng)]
    eng_fl = [sum(s["engine_flops"][e] for s in st_all) for e in range(n_eng)]
    dom = max(range(n_eng), key=lambda e: eng_ms[e])
    avg_s = eng_ms[dom] / 1000.0 / max(1, eng_n[dom])
    # mean algorithmic flops per launch: 2 M N K for a full product, N (N + 1) N for a
    # symmetric one (upper-triangular tiles only)
    per_launch = eng_fl[dom] / max(1, eng_n[dom])
    achieved = per_launch / avg_s / 1e12
    if dom == 1:
        peak, pnote = mpk["fp64_tflops"], "measured FP64 cuBLAS 4096^3 in this run"
        roof = {"bound": "alu"}
    elif dom == 5:
        peak, pnote = pk["bf16_sustained"], f"{pk['source']} sustained bf16 (MEASURED_PEAKS.json)"
        roof = {"bound": "tensor"}
    else:
        peak, pnote = mpk["tf32_tflops_sustained"], "measured sustained TF32 cuBLAS 8192^3 in this run"
        roof = {"bound": "tensor"}
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                 "traffic": (TRAFFIC[dom][0] * per_launch / TRAFFIC[dom][1]
                             if dom in TRAFFIC else None),
                 "traffic_note": ("DRAM bytes of one N = 8192 launch (ncu, profiles/"
                                  "gemm_split2sm_n4096.md) scaled by the mean launch's flops"
                                  if dom in TRAFFIC else None),
                 "kernel": f"{ENGINE_NAMES.get(dom)}: mean {per_launch:.3e} algorithmic flop per "
                           f"launch (2 M N K full, N^2 (N + 1) symmetric), mean "
                           f"{avg_s * 1e3:.3f} ms over {eng_n[dom]} launches",
                 "peak_note": pnote + " (of measured)",
                 "tensor_pipe_frac": achieved * PIPE_FACTOR.get(dom, 1.0) / peak})
    launches = sum(s["kernel_launches"] for s in st_all)
    engines = {}
    for e in range(n_eng):
        if not eng_n[e]:
            continue
        ach = eng_fl[e] / (eng_ms[e] / 1e3) / 1e12 if eng_ms[e] else None
        pe = (mpk["fp64_tflops"] if e == 1 else pk["bf16_sustained"] if e in (4, 5)
              else mpk["tf32_tflops_sustained"])
        engines[ENGINE_NAMES.get(e, str(e))] = {
            "ms_per_step": eng_ms[e] / args.steps, "launches_per_step": eng_n[e] / args.steps,
            "algorithmic_tflops": ach, "frac_of_peak": ach / pe if ach else None,
            "tensor_pipe_frac": ach * PIPE_FACTOR.get(e, 1.0) / pe if ach else None}

    # end to end through the public API with host buffers (pinned), copies inside the region
    host = []
    for p in probs:
        host.append({"H0": torch.from_numpy(p.H0).pin_memory(),
                     "H1": torch.from_numpy(p.H1).pin_memory(),
                     "P0": torch.empty((p.N, p.N), dtype=torch.float64).pin_memory(),
                     "P1": torch.empty((p.D, p.N, p.N), dtype=torch.float64).pin_memory(),
                     "mu": ctypes.c_double(), "mu1": np.zeros(p.D)})
    ke = max(1, min(args.steps, 2))
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        for h, p, b in zip(hs, probs, host):
            pkg.set_H(h.h, p.N, b["H0"].data_ptr(), p.D, b["H1"].data_ptr(), 0)
            pkg.solve_raw(h.h, p.beta, p.nocc, p.n, b["P0"].data_ptr(), b["P1"].data_ptr(),
                          ctypes.addressof(b["mu"]), b["mu1"].ctypes.data, 0)
    torch.cuda.synchronize()
    dte = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": ke * len(probs) * world / dte, "unit": "solves/s",
           "h2d_bytes_per_step": sum((b["H0"].numel() + b["H1"].numel()) * 8 for b in host),
           "d2h_bytes_per_step": sum((b["P0"].numel() + b["P1"].numel()) * 8 for b in host),
           "steps": ke}

    # FP32 (split-TF32 products) on the same workload, for "mixed vs FP32"
    fp32 = None
    outs_fp32 = []
    if not args.no_compare and args.precision != "fp32":
        hf = make("fp32")
        step(hf)                    # warm-up (allocations)
        stf = []
        msf = max_over_ranks(timed_steps(hf, 1, stf))
        step(hf, None, outs_fp32)
        fp32 = {"solves_per_s": len(probs) * world / (msf / 1000.0), "ms_per_step": msf,
                "speedup_of_timed_precision": value / (len(probs) * world / (msf / 1000.0))}
        for h in hf:
            h.close()
    for h in hs:
        h.close()
    torch.cuda.empty_cache()

    extras = {}
    if not args.no_extras:
        extras["cubic16_n4096"] = run_c2(pkg, args, barrier, max_over_ranks, world, rank)
        if not args.no_batch:
            extras["batched"] = run_batched(pkg, args, barrier, max_over_ranks, rank, world)
        extras["fp64_n2048"] = run_fp64(pkg, mpk, rank)
    if args.screen and rank == 0:
        extras["screened_chain"] = run_screened(
            pkg, sizes=[int(x) for x in args.screen_sizes.split(",") if x])

    cpu = cpu1 = err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        refs, t_or = [], 0.0
        for p in probs:
            r, dt = oracle_solve(p)
            refs.append(r)
            t_or += dt
        cpu = {"value": len(probs) / t_or, "unit": "solves/s", "cores": blas_threads(),
               "kind": "oracle",
               "sample": f"one oracle solve of each system (dsyevd N=8000 and 8192, bisection on "
                         f"mu, Daleckii-Krein P1, mu1, alpha) in {t_or:.1f} s"}
        cpu1 = time_oracle_one_core()
        err = {"vs": "oracle, recursion-exact function: P0, P1 relative Frobenius; alpha "
                     "relative; mu1 relative to max(|mu1|, 1); worst direction"}
        for label, outs in ((args.precision, outs_main), ("fp32", outs_fp32)):
            if outs:
                err[label] = {c: _errors(o, r, p.D) for c, o, r, p in zip(C3, outs, refs, probs)}
                err[label]["max"] = max(v["max"] for v in err[label].values())

    if rank == 0:
        s_last = st_all[-len(probs):]
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32 (3xtf32 products)", "fp64": "f64",
                      "mixed": "tf32 + bf16-digit products, f32-pair storage"}[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": args.precision,
                       "gemm": {"fp32": "tcgen05 3xTF32", "fp64": "CUDA-core DFMA",
                                "mixed": "tcgen05 TF32 sweeps and CG iterations; 3xTF32 "
                                         "refinement of early steps, response right-hand sides "
                                         "and restarts; Ozaki BF16-digit (FP64-class) residuals "
                                         "of the late steps and of dP0/dmu"}[args.precision],
                       "l2": "no flush: working set (trajectory of 29 N x N matrices as pairs "
                             "with their TF32 splits, about 30 GiB) exceeds the 129 MB L2",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "cpu_baseline_one_core": cpu1,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "fp32": fp32,
            "error": err,
            "peaks": {**mpk, "bf16_tflops": pk["bf16"], "bf16_tflops_sustained": pk["bf16_sustained"],
                      "hbm_gbs": pk["hbm_gbs"], "bf16_hbm_source": pk["source"]},
            "engines": engines,
            "extras": extras,
            "detail": {
                "gemm_share_of_step_time": sum(eng_ms) / (ms / world) if ms else None,
                "gemm_launches_per_step": sum(eng_n) / args.steps,
                "algorithmic_tflop_per_step": sum(eng_fl) / args.steps / 1e12,
                "per_system": [{"system": c, "mu_iterations": s["mu_iterations"],
                                "cg_sweeps": s["cg_iterations_sweeps"],
                                "cg_refine": s["cg_iterations_refine"],
                                "refine_passes": s["refine_passes"],
                                "fp64_residual_passes": s["fp64_residual_passes"],
                                "fp64_residual_first_step": s["fp64_residual_first_step"],
                                "cg_response": s["cg_iterations_response"],
                                "cg_q": s["cg_iterations_q"],
                                "phase_ms": dict(zip(("sweeps", "refine", "response", "q_mu1_alpha",
                                                      "output"), s["phase_ms"])),
                                "seconds": s["seconds"]} for c, s in zip(C3, s_last)],
            },
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def run_c2(pkg, args, barrier, max_over_ranks, world, rank):
    """The 16^3 lattice (N = 4096, n 14) at beta 5, 20 and 80: one step (three solves) in mixed
    precision, in FP32 and in FP64 (tensor-core FP64 products), with every output against the
    oracle."""
    import numpy as np
    import torch

    import synthetic
    probs = [synthetic.cubic_lattice((16, 16, 16), seed=1002, beta=b, n=14) for b in C2_BETAS]
    out = {"workload": "16x16x16 lattice, N=4096, n=14, D=1, beta 5, 20, 80; one step = 3 solves"}
    res = {}
    for prec in ("mixed", "fp32", "fp64"):
        with pkg.Handle(precision=prec) as h:
            h.set_H(probs[0].H0, probs[0].H1)
            for p in probs:
                h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)   # warm-up
            barrier()
            t0 = time.perf_counter()
            rs = []
            for p in probs:
                r = h.solve(p.beta, p.nocc, p.n)
                torch.cuda.synchronize()
                rs.append({"P0": r["P0"].cpu().numpy(), "P1": r["P1"].cpu().numpy(),
                           "mu1": np.asarray(r["mu1"]), "alpha": h.polarizability()})
            dt = max_over_ranks(time.perf_counter() - t0)
        out[prec] = {"solves_per_s": len(probs) * world / dt}
        res[prec] = rs
    out["mixed_vs_fp32"] = out["mixed"]["solves_per_s"] / out["fp32"]["solves_per_s"]
    if rank == 0 and not args.no_cpu_baseline:
        eig = np.linalg.eigh(probs[0].H0)
        refs = [oracle_solve(p, eig)[0] for p in probs]
        for prec, rs in res.items():
            out[prec]["error"] = {f"beta={p.beta:g}": _errors(r, ref, p.D)
                                  for p, r, ref in zip(probs, rs, refs)}
    return out


def run_fp64(pkg, mpk, rank):
    """FP64 solves of the 16 x 16 x 8 lattice (N = 2048) at beta 20 with each FP64 product
    engine: the tensor-core Ozaki engine (seven BF16 digits, the default) and CUDA-core DFMA,
    with their product rates against the measured cuBLAS FP64 rate and their errors against
    the oracle."""
    import numpy as np
    import torch

    import oracle
    import synthetic
    p = synthetic.cubic_lattice((16, 16, 8), seed=1002, beta=20.0, n=14)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec") if rank == 0 else None
    out = {"workload": "16x16x8 lattice, N=2048, beta 20, n 14, FP64",
           "fp64_peak_tflops": mpk["fp64_tflops"]}
    for engine, eng_id, label in (("auto", 5, "tensor_core_ozaki"), ("simt", 1, "cuda_core_dfma")):
        with pkg.Handle(precision="fp64", engine=engine, profile=True) as h:
            h.set_H(p.H0, p.H1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = h.solve(p.beta, p.nocc, p.n)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            st = h.stats()
            alpha = h.polarizability()
        ms = st["engine_ms"][eng_id]
        ach = st["engine_flops"][eng_id] / (ms / 1e3) / 1e12 if ms else None
        o = {"solve_s": dt, "gemm_ms": ms, "gemm_launches": st["engine_launches"][eng_id],
             "gemm_tflops_fp64": ach,
             "frac_of_fp64_peak": ach / mpk["fp64_tflops"] if ach else None}
        if eng_id == 5 and ach:
            o["bf16_digit_tflops"] = 28 * ach
            o["frac_of_bf16_sustained"] = 28 * ach / peaks()["bf16_sustained"]
        if ref is not None:
            o["error"] = _errors({"P0": r["P0"].cpu().numpy(), "P1": r["P1"].cpu().numpy(),
                                  "mu1": np.asarray(r["mu1"]), "alpha": alpha}, ref, p.D)
        out[label] = o
    if out["cuda_core_dfma"]["solve_s"]:
        out["speedup_tensor_core_vs_dfma"] = (out["cuda_core_dfma"]["solve_s"] /
                                              out["tensor_core_ozaki"]["solve_s"])
    return out


def run_screened(pkg, tau=1e-8, sizes=(4096, 8192, 16384)):
    """Block-sparse screened products (opts.screen_tau) on the Anderson-disordered 1D chain,
    beta 10, n 12, mixed precision: one dense and one screened solve per size after a warm-up
    of each, timed with CUDA events around the solve; the fraction of 128 x 32 k-slices
    the screened products computed, the screened-vs-dense change of alpha and P1, and (as in
    Fig. 3) the number of elements above 1e-5 in the screened P0, P1 and P2."""
    import numpy as np
    import torch

    import synthetic
    out = {"workload": f"1D chain (seed 1001), beta 10, n 12, mixed precision, tau {tau:g}",
           "sizes": {}}
    for N in sizes:
        p = synthetic.chain_1d(N, 1001, 10.0, 12)
        res = {}
        for label, t in (("screened", tau), ("dense", 0.0)):
            with pkg.Handle(precision="mixed", screen_tau=t) as h:
                h.set_H(p.H0, p.H1)
                h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)   # warm-up
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                r = h.solve(p.beta, p.nocc, p.n)
                e1.record()
                torch.cuda.synchronize()
                st = h.stats()
                res[label] = {"s": e0.elapsed_time(e1) / 1e3, "alpha": float(h.polarizability()[0]),
                              "P1": r["P1"][0].cpu().numpy(),
                              "computed": st["screen_slices_computed"],
                              "examined": st["screen_slices_examined"]}
                if label == "screened":
                    # Fig. 3: elements above the paper's threshold of 1e-5 in P0, P1 and P2
                    P2 = h.response2(want_grad=False)["P2"][0]
                    res[label]["nnz"] = {k: int((m.abs() > 1e-5).sum())
                                         for k, m in (("P0", r["P0"]), ("P1", r["P1"][0]),
                                                      ("P2", P2))}
        d, s_ = res["dense"], res["screened"]
        out["sizes"][str(N)] = {
            "dense_s": d["s"], "screened_s": s_["s"], "speedup": d["s"] / s_["s"],
            "slices_computed_frac": s_["computed"] / s_["examined"] if s_["examined"] else None,
            "nnz_above_1e-5": s_["nnz"],
            "alpha_rel_change": abs(s_["alpha"] - d["alpha"]) / abs(d["alpha"]),
            "P1_rel_change": float(np.linalg.norm(s_["P1"] - d["P1"]) / np.linalg.norm(d["P1"]))}
    return out


def run_batched(pkg, args, barrier, max_over_ranks=lambda x: x, rank=0, world=1):
    """The 96-cluster workload as one lockstep batch (FP32 and mixed precision), against the
    same systems solved one at a time (split-TF32 FP32 and CUDA-core FFMA FP32). With several
    ranks each solves its LPT share of the clusters (no exchange) and the time is the slowest
    rank's: the batch leg scales strongly."""
    import torch

    import synthetic
    from paper_1503_07037_gb300.shard import cube_weights, lpt_partition
    all_probs = synthetic.clusters(B=96, seed=1005, beta=20.0, n=12)
    share = lpt_partition(cube_weights([p.N for p in all_probs]), world)[rank]
    probs = [all_probs[i] for i in share]
    sizes = [p.N for p in probs]
    betas = [p.beta for p in probs]
    noccs = [p.nocc for p in probs]
    out = {"workload": "96 clusters, N_b ~ U{128..1536} (seed 1005), D = 3, beta 20, n 12; one "
                       "grouped tcgen05 launch per product, CG iterations as a CUDA graph, tile "
                       "width from the autotuner",
           "sum_N3": float(sum(float(p.N) ** 3 for p in all_probs)),
           "ranks": world, "systems_on_rank0": len(probs)}
    results = {}
    for prec in ("fp32", "mixed"):
        bt = pkg.Batch(sizes, 3, precision=prec, profile=1)
        bt.set_H([p.H0 for p in probs], [p.H1 for p in probs], 12)
        bt.solve(betas, noccs, 12)                 # warm-up (descriptor and map caches)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record()
        r = bt.solve(betas, noccs, 12)
        ev1.record()
        torch.cuda.synchronize()
        ms = max_over_ranks(ev0.elapsed_time(ev1))
        st = bt.stats()
        out[prec] = {"solves_per_s": 96 / (ms / 1e3), "ms": ms, "mu_sweeps": st["mu_iterations"],
                     "cg_sweeps": st["cg_iterations_sweeps"],
                     "cg_refine": st["cg_iterations_refine"],
                     "refine_passes": st["refine_passes"],
                     "fp64_residual_passes": st["fp64_residual_passes"],
                     "kernel_launches": st["kernel_launches"],
                     "phase_ms": dict(zip(("sweeps", "refine", "response", "q_mu1_alpha",
                                           "output"), st["phase_ms"])),
                     "algorithmic_tflops": st["gemm_flops"] / (ms / 1e3) / 1e12,
                     "tuning": bt.tuning()}
        results[prec] = r
        bt.close()
    if getattr(args, "batched_only", False):
        return out
    # the same systems solved one at a time through the single-system path
    t0 = time.perf_counter()
    with pkg.Handle(precision="fp32") as h:
        for p in probs:
            h.set_H(p.H0, p.H1)
            h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
    torch.cuda.synchronize()
    out["sequential_fp32_3xtf32_solves_per_s"] = 96 / max_over_ranks(time.perf_counter() - t0)
    # CUDA-core FFMA FP32 one at a time: a bounded sample (the first 24 systems)
    sample = probs[:24]
    t0 = time.perf_counter()
    with pkg.Handle(precision="fp32", engine="simt") as h:
        for p in sample:
            h.set_H(p.H0, p.H1)
            h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out["sequential_fp32_ffma_solves_per_s"] = world * len(sample) / max_over_ranks(dt) * (
        sum(float(p.N) ** 3 for p in sample) / len(sample)) / (out["sum_N3"] / 96)
    out["sequential_fp32_ffma_note"] = ("first 24 systems, scaled to the batch's mean N^3")
    out["mixed_batched_vs_sequential_fp32_ffma"] = (out["mixed"]["solves_per_s"] /
                                                    out["sequential_fp32_ffma_solves_per_s"])
    out["mixed_batched_vs_fp32_batched"] = (out["mixed"]["solves_per_s"] /
                                            out["fp32"]["solves_per_s"])
    if not args.no_cpu_baseline and rank == 0:
        import oracle
        for prec, r in results.items():
            worst = 0.0
            for i in range(0, len(probs), max(1, len(probs) // 4))[:4]:
                p = probs[i]
                ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
                worst = max(worst, oracle.rel_frobenius(r["P0"][i].cpu().numpy(), ref["P0"]),
                            max(oracle.rel_frobenius(r["P1"][i][d].cpu().numpy(), ref["P1"][d])
                                for d in range(3)))
            out[prec]["max_err_sampled_systems"] = worst
        out["sampled_systems"] = "4 evenly spaced systems of rank 0's share"
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["fp32", "fp64", "mixed"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the N = 4096 lattice, batch and FP64 measurements")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched 96-cluster measurement")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the FP32 step on the same workload")
    ap.add_argument("--screen", action="store_true",
                    help="add the screened-product (block-sparse) chain measurement")
    ap.add_argument("--screen-sizes", default="4096,8192,16384",
                    help="chain sizes of the screened-product measurement")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the lockstep batches (FP32 and mixed) of the 96-cluster "
                         "workload (one JSON line, no one-at-a-time comparison)")
    ap.add_argument("--screened-only", action="store_true",
                    help="run only the screened-product chain measurement (one JSON line)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.batched_only:
        import paper_1503_07037_gb300 as pkg
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(run_batched(pkg, args, torch.cuda.synchronize)), flush=True)
        return 0
    if args.screened_only:
        import paper_1503_07037_gb300 as pkg
        sizes = [int(x) for x in args.screen_sizes.split(",") if x]
        print(json.dumps(run_screened(pkg, sizes=sizes)), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
