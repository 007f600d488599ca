"""GPU tests of trajectory checkpointing (the adjoint's sqrt(n) checkpoints).

With ckpt_stride s the solve keeps Z_k for k a multiple of s, Z_n and W_0
only; the first-order response, the adjoint's reverse sweep and the higher
orders recompute each segment of s steps from its checkpoint. The
recomputation repeats the final sweep's CG on the same data, so every result
must match the run that stores the whole trajectory up to the rounding of the
device reductions. Bars between the two runs: 1e-12 (FP64) and 1e-6 (FP32)
relative Frobenius; against the oracle the usual 1e-10 / 1e-5.
"""
import functools

import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


def _run(pkg, p, precision, ckpt, G0=None, order=3):
    import torch
    with pkg.Handle(precision=precision, ckpt_stride=ckpt) as h:
        h.set_H(p.H0, p.H1)
        r = h.solve(p.beta, p.nocc, p.n)
        out = {"P0": r["P0"].cpu().numpy(), "P1": r["P1"].cpu().numpy(), "mu": r["mu"],
               "mu1": r["mu1"], "stats": h.stats()}
        if G0 is not None:
            out["vjp"] = h.vjp_P0(torch.from_numpy(G0).cuda()).cpu().numpy()
        if order >= 2:
            r2 = h.response2()
            out["P2"] = r2["P2"].cpu().numpy()
            out["grad"] = r2["grad"].cpu().numpy()
        if order >= 3:
            out["P3"] = h.response3()["P3"].cpu().numpy()
    return out


def _sym(seed, N, scale):
    A = np.random.default_rng(seed).standard_normal((N, N)) * scale
    return 0.5 * (A + A.T)


@functools.lru_cache(maxsize=None)
def _fp64_full():
    import paper_1503_07037_gb300 as pkg
    p = syn.cubic_lattice((5, 5, 5), seed=7, beta=8.0, n=12)
    return p, _run(pkg, p, "fp64", 0, _sym(3, p.N, 1.0))


@pytest.mark.parametrize("ckpt,stride", [(1, 1), (3, 3), (5, 5), ("sqrt", 4)])
def test_checkpointed_fp64_matches_full_trajectory(cuda, cdmpt_lib, ckpt, stride):
    """n = 12: strides 3 and 4 divide it, 5 leaves a ragged last segment of 2 steps, 1 keeps
    every Z_k and recomputes only W_k."""
    p, full = _fp64_full()
    ck = _run(cdmpt_lib, p, "fp64", ckpt, _sym(3, p.N, 1.0))
    assert ck["stats"]["checkpoint_stride"] == stride
    assert full["stats"]["checkpoint_stride"] == 0
    if stride > 1:
        assert ck["stats"]["cg_iterations_recompute"] > 0
    assert abs(ck["mu"] - full["mu"]) < 1e-13
    for key in ("P0", "P1", "vjp", "P2", "grad", "P3"):
        assert oracle.rel_frobenius(ck[key], full[key]) < 1e-12, key


def test_checkpointed_fp64_against_oracle(cuda, cdmpt_lib):
    p, _ = _fp64_full()
    ck = _run(cdmpt_lib, p, "fp64", "sqrt", order=3)
    ref = oracle.response3(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", close=0.2, quad=0.2)
    assert oracle.rel_frobenius(ck["P1"][0], ref["P1"][0]) < 1e-10
    assert oracle.rel_frobenius(ck["grad"], ref["grad_alpha"][0]) < 1e-10
    assert oracle.rel_frobenius(ck["P3"][0], ref["P3"][0]) < 1e-10


def test_checkpointed_fp32_differentiation_workload(cuda, cdmpt_lib):
    """16 x 16 x 8 lattice (N = 2048), beta 20, n = 16, FP32 forward and adjoint with
    sqrt(n) = 4 checkpoints: the polarizability gradient and a P0 loss gradient."""
    p = syn.workload("cubic16x16x8")
    G0 = _sym(4, p.N, 1.0)
    full = _run(cdmpt_lib, p, "fp32", 0, G0, order=2)
    ck = _run(cdmpt_lib, p, "fp32", "sqrt", G0, order=2)
    assert ck["stats"]["checkpoint_stride"] == 4
    for key in ("P0", "P1", "vjp", "grad"):
        assert oracle.rel_frobenius(ck[key], full[key]) < 1e-6, key
    ref = oracle.response2(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    assert oracle.rel_frobenius(ck["grad"], ref["grad_alpha"][0]) < 1e-5


def test_checkpointing_reduces_device_memory(cuda, cdmpt_lib):
    """Device memory held by a handle after an FP32 solve at N = 2048, n = 16: the whole
    trajectory (33 matrices with their TF32 splits) against sqrt(n) checkpoints (13)."""
    import torch
    p = syn.workload("cubic16x16x8")

    def footprint(ckpt):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        h = cdmpt_lib.Handle(precision="fp32", ckpt_stride=ckpt)
        h.set_H(p.H0, p.H1)
        h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
        torch.cuda.synchronize()
        used = free0 - torch.cuda.mem_get_info()[0]
        h.close()
        return used

    full = footprint(0)
    ck = footprint("sqrt")
    assert ck < 0.6 * full, (ck, full)


def test_checkpointing_rejected_in_mixed_precision(cuda, cdmpt_lib):
    with pytest.raises(cdmpt_lib.CdmptError):
        cdmpt_lib.Handle(precision="mixed", ckpt_stride=-1)
