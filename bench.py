"""Throughput of canonical DMPT solves on GB300 (one JSON line on rank 0).

Workload (one step): the 16 x 16 x 16 periodic simple-cubic tight-binding
lattice (N = 4096, on-site N(0, 0.3^2), hopping -1 +- 10 %, seed 1002), dipole
perturbation along x, N_occ = N/2, n = 14 recursion steps, solved canonically
at beta = 5, 20 and 80: three full solves (occupation loop, first-order
response, mu1, polarizability) per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp32|fp64]
                  [--impl ours|reference] [--no-compare] [--no-cpu-baseline]

The timed precision defaults to mixed (TF32 sweeps, split-TF32 refinement and
response); one step of FP32 with split-TF32 products and one with CUDA-core
FFMA products are timed beside it ("modes"), and every mode's P0 and P1 are
compared with the FP64 oracle at the three temperatures ("error").

--impl reference times the FP64 CPU oracle (exact diagonalisation) on the
host cores, one solve of the same workload per step.
Under torchrun every rank solves its own copy (weak scaling, no collective on
the data path); times are max-reduced over ranks.
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
BETAS = (5.0, 20.0, 80.0)
LATTICE = (16, 16, 16)
NSTEPS_REC = 14
WORKLOAD = "cubic16x16x16 tight-binding, N=4096, D=1 (x dipole), n=14, beta in {5,20,80}"
TF32_OVER_BF16 = 1.1 / 2.25     # nominal dense tf32 / bf16 tensor rate ratio
# DRAM bytes (read + write) of one GEMM launch at N = 4096 from the ncu captures summarised in
# profiles/ (per engine); None until the kernel's counters are re-taken after a change
TRAFFIC = {2: None, 3: 995.9e6}   # per launch at N = 4096 (3xTF32 captured on the current kernel)


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


def problems():
    import synthetic
    return [synthetic.cubic_lattice(LATTICE, seed=1002, beta=b, n=NSTEPS_REC) for b in BETAS]


# --------------------------------------------------------------------------- oracle timing

def time_oracle(sample_betas, cores_note=True):
    """Times the FP64 oracle on this host: returns (solves/s, seconds, results)."""
    import oracle
    import synthetic
    res = {}
    t0 = time.perf_counter()
    for b in sample_betas:
        p = synthetic.cubic_lattice(LATTICE, seed=1002, beta=b, n=NSTEPS_REC)
        res[b] = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    dt = time.perf_counter() - t0
    return len(sample_betas) / dt, dt, res


def time_oracle_one_core():
    """The oracle's beta = 20 solve of a 16 x 16 x 8 lattice (N = 2048) on one host core, in a
    child process whose BLAS pools are limited to one thread; scaled to the N = 4096 workload by
    the N^3 cost of the eigendecomposition and the Daleckii-Krein products (x 8). A bounded sample:
    about 10 s on one core."""
    import subprocess
    import sys
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
    return {"value": 1.0 / (8.0 * dt), "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"beta=20 solve of the 16x16x8 lattice (N=2048) in {dt:.1f} s on one core, "
                      f"scaled x8 (N^3) to N=4096"}


def blas_threads():
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return os.cpu_count()


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    betas = [BETAS[i % len(BETAS)] for i in range(args.warmup + args.steps)]
    for b in betas[:args.warmup]:
        time_oracle([b])
    t0 = time.perf_counter()
    for b in betas[args.warmup:]:
        time_oracle([b])
    dt = time.perf_counter() - t0
    value = args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "fp64 exact diagonalisation (oracle)",
                   "step": "one solve of the workload (cycling beta 5, 20, 80)"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": blas_threads(),
                         "kind": "oracle",
                         "sample": "one beta per step: dsyevd N=4096, bisection on mu, "
                                   "Daleckii-Krein P1, mu1, alpha"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- our path

def run_ours(args):
    import ctypes

    import numpy as np
    import torch

    import paper_1503_07037_gb300 as pkg

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

    probs = problems()
    N, D = probs[0].N, probs[0].D
    stream = torch.cuda.current_stream()
    H0 = torch.from_numpy(probs[0].H0).to(dev)
    H1 = torch.from_numpy(probs[0].H1).to(dev)
    P0 = torch.empty((N, N), dtype=torch.float64, device=dev)
    P1 = torch.empty((D, N, N), dtype=torch.float64, device=dev)
    mu = ctypes.c_double()
    mu1 = np.zeros(D)

    def make(precision, engine="auto"):
        h = pkg.Handle(precision=precision, engine=engine, profile=True, stream=stream)
        h.set_H(H0, H1)                 # resident in HBM before any timed region
        return h

    def step(h, stats_acc=None, outs=None):
        for p in probs:
            pkg.solve_raw(h.h, p.beta, p.nocc, p.n, P0.data_ptr(), P1.data_ptr(),
                          ctypes.addressof(mu), mu1.ctypes.data, 1)
            if stats_acc is not None:
                stats_acc.append(h.stats())
            if outs is not None:
                outs.append((P0.cpu().numpy(), P1[0].cpu().numpy()))

    def timed_steps(h, k, stats_acc):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        for _ in range(k):
            step(h, stats_acc)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1)

    h = make(args.precision)
    for _ in range(args.warmup):
        step(h)
    clocks = ClockSampler(local)
    clocks.start()
    st_all = []
    ms = timed_steps(h, args.steps, st_all)
    clk = clocks.stop()
    ms = max_over_ranks(ms)
    barrier()
    solves = args.steps * len(probs) * world
    value = solves / (ms / 1000.0)

    # roofline of the dominant kernel: the GEMM engine with the most device time
    n_eng = len(st_all[0]["engine_ms"])
    eng_ms = [sum(s["engine_ms"][e] for s in st_all) for e in range(n_eng)]
    eng_n = [sum(s["engine_launches"][e] for s in st_all) for e in range(n_eng)]
    eng_fl = [sum(s["engine_flops"][e] for s in st_all) for e in range(n_eng)]
    dom = max(range(n_eng), key=lambda e: eng_ms[e])
    names = {1: "CUDA-core FFMA/DFMA", 2: "tcgen05 TF32", 3: "tcgen05 3xTF32", 4: "tcgen05 BF16"}
    avg_s = eng_ms[dom] / 1000.0 / max(1, eng_n[dom])
    # mean algorithmic flops per launch: 2 N^3 for a full product, N (N + 1) N for a symmetric
    # one (upper-triangular tiles only)
    per_launch = eng_fl[dom] / max(1, eng_n[dom])
    achieved = per_launch / avg_s / 1e12
    pk = peaks()
    if args.precision == "fp64":
        roof = {"bound": "alu", "achieved": achieved, "peak": 1.25, "unit": "TFLOP/s",
                "frac": achieved / 1.25, "traffic": None,
                "peak_note": "nominal FP64 rate of GB300 (no measured FP64 peak)"}
    else:
        peak_tf32 = pk["bf16_sustained"] * TF32_OVER_BF16
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak_tf32, "unit": "TFLOP/s",
                "frac": achieved / peak_tf32, "traffic": TRAFFIC.get(dom),
                "kernel": f"k_gemm_tc ({names.get(dom)}), mean {per_launch:.3e} algorithmic flop "
                          f"per launch (2 N^3 full, N^2 (N + 1) symmetric), mean "
                          f"{avg_s * 1e3:.3f} ms over {eng_n[dom]} launches",
                "peak_note": f"tf32 = {pk['source']} sustained bf16 {pk['bf16_sustained']} x "
                             f"{TF32_OVER_BF16:.4f} (nominal 1.1/2.25) of measured",
                "tensor_pipe_frac": achieved * (3 if dom == 3 else 1) / peak_tf32}
    launches = sum(s["kernel_launches"] for s in st_all)
    gemm_ms_total = sum(eng_ms)

    # end to end through the public API with host buffers (pinned), copies inside the region
    H0h = torch.from_numpy(probs[0].H0).pin_memory()
    H1h = torch.from_numpy(probs[0].H1).pin_memory()
    P0h = torch.empty((N, N), dtype=torch.float64).pin_memory()
    P1h = torch.empty((D, N, N), dtype=torch.float64).pin_memory()
    ke = max(1, min(args.steps, 2))
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        pkg.set_H(h.h, N, H0h.data_ptr(), D, H1h.data_ptr(), 0)
        for p in probs:
            pkg.solve_raw(h.h, p.beta, p.nocc, p.n, P0h.data_ptr(), P1h.data_ptr(),
                          ctypes.addressof(mu), mu1.ctypes.data, 0)
    torch.cuda.synchronize()
    dte = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": ke * len(probs) * world / dte, "unit": "solves/s",
           "h2d_bytes_per_step": (H0h.numel() + H1h.numel()) * 8,
           "d2h_bytes_per_step": len(probs) * (P0h.numel() + P1h.numel()) * 8, "steps": ke}
    h.set_H(H0, H1)

    # the other precisions on the same workload (one step each), for "mixed vs FP32"
    modes = {}
    outs_by_mode = {}
    if not args.no_compare:
        for label, prec, eng in (("fp32_3xtf32", "fp32", "3xtf32"), ("fp32_ffma", "fp32", "simt"),
                                 (args.precision, args.precision, "auto")):
            hm = make(prec, eng) if label != args.precision else h
            step(hm)            # warm-up (allocations)
            stm = []
            msm = timed_steps(hm, 1, stm)
            outs = []
            step(hm, None, outs)
            outs_by_mode[label] = outs
            modes[label] = {"solves_per_s": len(probs) / (msm / 1000.0), "ms_per_step": msm}
            if hm is not h:
                hm.close()

    if "fp32_3xtf32" in modes and "fp32_ffma" in modes and args.precision in modes:
        me = modes[args.precision]["solves_per_s"]
        modes["speedup_vs_fp32_3xtf32"] = me / modes["fp32_3xtf32"]["solves_per_s"]
        modes["speedup_vs_fp32_ffma"] = me / modes["fp32_ffma"]["solves_per_s"]

    # batched workload: 96 disordered clusters, N_b ~ U{128..1536}, 3 directions, beta 20, n 12
    batched = None
    if not args.no_batch:
        batched = run_batched(pkg, args, barrier, max_over_ranks, rank, world)

    # the N = 8192 product chain: one mixed solve of the banded workload, per-engine rates
    chain = None
    if not args.no_chain:
        chain = run_chain(pkg, pk)

    # block-sparse screened products on the 1D chain (Sec. VI): dense against screened
    screened = None
    if not args.no_screen and rank == 0:
        screened = run_screened(pkg, sizes=[int(x) for x in args.screen_sizes.split(",") if x])

    cpu = None
    cpu1 = None
    err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # bounded oracle sample: the beta = 20 solve of the workload, eigendecomposition included
        import oracle
        v, dt, res = time_oracle([20.0])
        cpu = {"value": v, "unit": "solves/s", "cores": blas_threads(), "kind": "oracle",
               "sample": f"1 of the 3 solves of a step (beta=20, N=4096), {dt:.1f} s"}
        cpu1 = time_oracle_one_core()
        if outs_by_mode:
            eig = np.linalg.eigh(probs[0].H0)
            refs = {p.beta: oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", eig=eig)
                    for p in probs}
            err = {"vs": "oracle, recursion-exact function (relative Frobenius)"}
            for label, outs in outs_by_mode.items():
                err[label] = {f"beta={p.beta:g}": {
                    "P0": oracle.rel_frobenius(o[0], refs[p.beta]["P0"]),
                    "P1": oracle.rel_frobenius(o[1], refs[p.beta]["P1"][0])}
                    for p, o in zip(probs, outs)}

    if rank == 0:
        s_last = st_all[-len(probs):]
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64", "mixed": "tf32+f32"}[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": args.precision,
                       "gemm": {"fp32": "tcgen05 3xTF32", "fp64": "CUDA-core DFMA",
                                "mixed": "tcgen05 TF32 sweeps and response CG iterations, 3xTF32 "
                                         "refinement, response right-hand sides and restarts"
                                }[args.precision],
                       "l2": "no flush: working set (trajectory of 29 N x N matrices plus "
                             "their TF32 splits, 5.4 GiB) exceeds the 129 MB L2",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "cpu_baseline_one_core": cpu1,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "modes": modes,
            "batched": batched,
            "chain_n8192": chain,
            "screened_chain": screened,
            "error": err,
            "detail": {
                "gemm_share_of_step_time": gemm_ms_total / (ms / world) if ms else None,
                "gemm_ms_per_engine": {names.get(e, e): eng_ms[e] / args.steps for e in range(n_eng)
                                       if eng_n[e]},
                "gemm_launches_per_step": sum(eng_n) / args.steps,
                "algorithmic_tflop_per_step": sum(eng_fl) / args.steps / 1e12,
                "per_beta": [{"beta": p.beta, "mu_iterations": s["mu_iterations"],
                              "cg_sweeps": s["cg_iterations_sweeps"],
                              "cg_refine": s["cg_iterations_refine"],
                              "cg_response": s["cg_iterations_response"],
                              "cg_q": s["cg_iterations_q"],
                              "seconds": s["seconds"]} for p, s in zip(probs, s_last)],
            },
        }
        print(json.dumps(line), flush=True)
    h.close()
    if pg:
        pg.destroy_process_group()
    return 0


def run_chain(pkg, pk):
    """GEMM chain at N = 8192: one mixed-precision solve of the banded workload (bandwidth 64,
    beta 20, n 14) with every product timed; achieved rate per engine against the TF32 peak."""
    import torch

    import synthetic
    p = synthetic.workload("banded8192")
    names = {1: "CUDA-core", 2: "tcgen05 TF32", 3: "tcgen05 3xTF32"}
    peak = pk["bf16_sustained"] * TF32_OVER_BF16
    with pkg.Handle(precision="mixed", profile=True) as h:
        h.set_H(p.H0, p.H1)
        h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st = h.stats()
    out = {"workload": "banded N=8192 (bandwidth 64, seed 1004), beta 20, n 14, mixed precision",
           "solve_s": dt, "engines": {}}
    tensor_fl = 0.0
    gemm_s = 0.0
    for e in (2, 3):
        n_l = st["engine_launches"][e]
        if not n_l:
            continue
        ms = st["engine_ms"][e]
        fl = st["engine_flops"][e]
        ach = fl / (ms / 1e3) / 1e12
        tensor_fl += fl * (3 if e == 3 else 1)
        gemm_s += ms / 1e3
        out["engines"][names[e]] = {"launches": n_l, "ms": ms, "algorithmic_tflops": ach,
                                    "frac_of_tf32_peak": ach / peak,
                                    "tensor_pipe_frac": ach * (3 if e == 3 else 1) / peak}
    out["tensor_pipe_frac_all_products"] = (tensor_fl / gemm_s / 1e12 / peak) if gemm_s else None
    out["gemm_share_of_solve"] = gemm_s / dt if dt else None
    out["peak_note"] = (f"tf32 peak = {pk['source']} sustained bf16 {pk['bf16_sustained']} x "
                        f"{TF32_OVER_BF16:.4f}")
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
        bt = pkg.Batch(sizes, 3, precision=prec)
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
                     "kernel_launches": st["kernel_launches"],
                     "algorithmic_tflops": st["gemm_flops"] / (ms / 1e3) / 1e12,
                     "tuning": bt.tuning()}
        results[prec] = r
        bt.close()
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
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["fp32", "fp64", "mixed"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched 96-cluster measurement")
    ap.add_argument("--no-chain", action="store_true",
                    help="skip the N = 8192 product-chain measurement")
    ap.add_argument("--no-screen", action="store_true",
                    help="skip the screened-product (block-sparse) chain measurement")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the one-step runs of the other precisions")
    ap.add_argument("--screen-sizes", default="4096,8192,16384",
                    help="chain sizes of the screened-product measurement")
    ap.add_argument("--screened-only", action="store_true",
                    help="run only the screened-product chain measurement (one JSON line)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.screened_only:
        import paper_1503_07037_gb300 as pkg
        sizes = [int(x) for x in args.screen_sizes.split(",") if x]
        print(json.dumps(run_screened(pkg, sizes=sizes)), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
