"""Micro-benchmark of the recursion's product kernel through the C ABI.

  python -m paper_1503_07037_gb300.kernel_bench --n 4096 --engine tf32 --reps 5

Times D = Z Z^T + I (the step's system matrix A_k = I + Z_k^2) on an N x N
FP32 (or FP64) matrix with CUDA events on the launching stream, after three
warm-up launches, and prints one JSON line with the duration and the
algorithmic rate 2 N^3 / t. The input is a seeded symmetric matrix scaled like
a recursion iterate (spectrum in [-1, 1]); the tensor-core engines get its
TF32 split once, before timing, as the solver keeps splits resident. Engine
"oz" is the Ozaki-sliced product of a pair-stored matrix (hi + lo FP32),
D + Dl = Z Z^T; its timing includes slicing both operands into BF16 digits,
as every call of the solver's FP64-class residual does. "f64tc" is the FP64
product on the tensor cores (seven BF16 digits per element), slicing
included; "f64" the CUDA-core DFMA product. --check adds the error against a
cuBLAS FP64 product, on the signed input and on its absolute value.

  python -m paper_1503_07037_gb300.kernel_bench --batch 16 [--precision fp32]

instead solves one lockstep batch of the first B clusters of the batched workload (N_b drawn
from {128..1536}, seed 1005, D = 3) and prints the tile autotuner's per-launch times of its
first grouped product (W = Z^2 over all systems) for each tile width, with the solve's time:
the grouped tcgen05 products at a size a profiler capture can hold.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def run_batch(pkg, a):
    import torch

    import synthetic
    probs = synthetic.clusters(B=a.batch, seed=1005, beta=20.0, n=12)
    b = pkg.Batch([p.N for p in probs], 3, precision=a.precision)
    b.set_H([p.H0 for p in probs], [p.H1 for p in probs], 12)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    b.solve([p.beta for p in probs], [p.nocc for p in probs], 12)
    e1.record()
    torch.cuda.synchronize()
    out = {"kernel": "grouped", "clusters": a.batch, "precision": a.precision,
           "sum_N3": float(sum(float(p.N) ** 3 for p in probs)),
           "solve_ms_first": e0.elapsed_time(e1), "tuning": b.tuning()}
    b.close()
    print(json.dumps(out))


def main():
    import torch

    import paper_1503_07037_gb300 as pkg

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--engine", default="tf32", choices=["simt", "tf32", "3xtf32", "bf16", "f64", "f64tc", "oz"])
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=0,
                    help="solve a lockstep batch of this many clusters instead (see above)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "mixed"],
                    help="precision of the --batch solve")
    ap.add_argument("--epi", default="plain", choices=["plain", "cdot"],
                    help="epilogue of the tf32/3xtf32 products: D = X Y^T + I (plain), or "
                         "D = X Y^T + C with the dot sum(D * E) (cdot, as in the CG updates)")
    ap.add_argument("--check", action="store_true",
                    help="also report the error against an FP64 product (cuBLAS DGEMM), on the "
                         "signed input and on its absolute value (all-positive sums show the "
                         "bias of a truncating accumulation)")
    a = ap.parse_args()
    if a.batch > 0:
        return run_batch(pkg, a)
    dev = torch.device("cuda")
    g = torch.Generator(device=dev).manual_seed(1234)
    dt = torch.float64 if a.engine in ("f64", "f64tc") else torch.float32
    Z = torch.randn(a.n, a.n, device=dev, generator=g, dtype=torch.float64)
    Z64 = (Z + Z.T) / (2.0 * (2 * a.n) ** 0.5)
    Z = Z64.to(dt).contiguous()
    D = torch.empty_like(Z)
    if a.engine == "oz":
        Zl = (Z64 - Z.double()).float().contiguous()     # the pair's low part
        Dl = torch.empty_like(Z)
    if a.engine in ("tf32", "3xtf32"):
        Zs = pkg.split_tf32(Z)      # split once, outside the timed launches
        dsum = torch.zeros(1, device=dev, dtype=torch.float64)

    def run():
        if a.engine in ("f64", "f64tc"):
            pkg.gemm_f64(Z, Z, D, gamma=1.0, engine="tc" if a.engine == "f64tc" else "simt")
        elif a.engine == "oz":
            pkg.gemm_pair(Z, Zl, Z, Zl, D, Dl)
        elif a.engine in ("simt", "bf16"):
            # bf16: includes rounding the operand to BF16 (one pass, X is Y)
            pkg.gemm_f32(Z, Z, D, gamma=1.0, engine=a.engine)
        elif a.epi == "cdot":
            pkg.gemm_f32_split(Zs, Zs, D, beta=1.0, C=Z, dot=dsum, E=Z, engine=a.engine)
        else:
            pkg.gemm_f32_split(Zs, Zs, D, gamma=1.0, engine=a.engine)

    for _ in range(a.warmup):
        run()
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(a.reps):
        run()
    e1.record(s)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / a.reps / 1e3
    out = {"kernel": "gemm", "engine": a.engine, "n": a.n, "ms": t * 1e3,
           "alg_tflops": 2.0 * a.n ** 3 / t / 1e12}
    if a.engine in ("tf32", "3xtf32"):
        out["epi"] = a.epi
    if a.engine in ("oz", "f64tc"):
        # BF16 digit pairs: p + q <= 4 of 5 digits (pairs), p + q <= 6 of 7 digits (FP64)
        out["digit_products"] = 15 if a.engine == "oz" else 28
        out["bf16_tflops"] = out["alg_tflops"] * out["digit_products"]
    if a.check and a.engine != "oz":
        for label, src in (("signed", Z64), ("positive", Z64.abs())):
            Zc = src.to(dt).contiguous()
            if a.engine in ("tf32", "3xtf32"):
                Zs = pkg.split_tf32(Zc)
            ref = Zc.double() @ Zc.double().T + torch.eye(a.n, dtype=torch.float64, device=dev)
            if a.engine in ("f64", "f64tc"):
                pkg.gemm_f64(Zc, Zc, D, gamma=1.0, engine="tc" if a.engine == "f64tc" else "simt")
            elif a.engine in ("simt", "bf16"):
                pkg.gemm_f32(Zc, Zc, D, gamma=1.0, engine=a.engine)
            else:
                pkg.gemm_f32_split(Zs, Zs, D, gamma=1.0, engine=a.engine)
            torch.cuda.synchronize()
            err = D.double() - ref
            out[f"rel_err_{label}"] = float(err.norm() / ref.norm())
            out[f"rel_bias_{label}"] = float(err.sum() / ref.abs().sum())
    print(json.dumps(out))


if __name__ == "__main__":
    main()
