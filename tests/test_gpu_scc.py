"""GPU tests of the self-consistent charge layer (Sec. IV with a synthetic G(D)).

cdmpt_scc_solve iterates the Mulliken charges to self-consistency (Anderson
mixing; each step a canonical solve of F = h + G(D) in the non-orthogonal
basis), then solves the coupled-perturbed equations D1 = R(h1 + G(D1)) per
direction on the converged trajectory, and returns Omega_SCF^(1) = 2 Tr[h1 D0]
and Omega_SCF^(2) = Tr[h1 D1] (Eq. Resp_Omega). Reference: the oracle's SCF
(linear mixing to 1e-13) and its CPSCF by a direct solve of the linear charge
equations, pinned on the CPU by finite differences of the self-consistent D and
of the SCF free energy. Bars: 1e-9 (FP64, SCF stopped at 1e-12 in the charges),
1e-5 (FP32).
"""
import functools

import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def _case(N, seed):
    p = syn.nonorthogonal_cluster(N, seed=seed, beta=20.0, n=14)
    m = p.meta
    ref = oracle.scc_solve(p.H0, p.H1, m["S"], m["gamma"], m["q0"], p.beta, p.nocc, n=p.n,
                           order=2)
    return p, ref


def _run(pkg, p, precision, tol, order=1):
    m = p.meta
    with pkg.Handle(precision=precision) as h:
        h.set_overlap(m["S"])
        return h.scc_solve(p.H0, p.H1, m["gamma"], p.beta, p.nocc, p.n, q0=m["q0"], tol=tol,
                           order=order)


def test_scc_fp64_cluster(cuda, cdmpt_lib):
    p, ref = _case(120, 3001)
    r = _run(cdmpt_lib, p, "fp64", 1e-12)
    assert r["iters"][0] < 60 and r["iters"][1] < 3 * 60, r["iters"]
    assert oracle.rel_frobenius(r["D0"], ref["D0"]) < 1e-9
    assert abs(r["mu"] - ref["mu"]) < 1e-9
    for d in range(3):
        assert oracle.rel_frobenius(r["D1"][d], ref["D1"][d]) < 1e-9
        assert abs(r["mu1"][d] - ref["mu1"][d]) < 1e-9 * max(1.0, abs(ref["mu1"][d]))
        assert abs(r["omega1"][d] - ref["omega1"][d]) < 1e-9 * max(1.0, abs(ref["omega1"][d]))
        assert abs(r["omega2"][d] - ref["omega2"][d]) < 1e-9 * abs(ref["omega2"][d])


def test_scc_fp32_cluster(cuda, cdmpt_lib):
    p, ref = _case(120, 3001)
    r = _run(cdmpt_lib, p, "fp32", 0.0)
    assert oracle.rel_frobenius(r["D0"], ref["D0"]) < 1e-5
    for d in range(3):
        assert oracle.rel_frobenius(r["D1"][d], ref["D1"][d]) < 1e-5
        assert abs(r["omega2"][d] - ref["omega2"][d]) < 1e-5 * abs(ref["omega2"][d])


def test_scc_orthogonal_without_coupling_equals_plain_solve(cuda, cdmpt_lib):
    """gamma = 0 in the orthogonal mode: F = h whatever the charges, so the mixer settles the
    charges within a few steps and D0, D1 equal the plain solve."""
    q = syn.workload("chain64")
    with cdmpt_lib.Handle(precision="fp64") as h:
        h.set_H(q.H0, q.H1)
        base = h.solve(q.beta, q.nocc, q.n)
        r = h.scc_solve(q.H0, q.H1, np.zeros((q.N, q.N)), q.beta, q.nocc, q.n, tol=1e-12)
    assert r["iters"][0] <= 4, r["iters"]
    assert oracle.rel_frobenius(r["D0"], base["P0"].cpu().numpy()) < 1e-13
    assert oracle.rel_frobenius(r["D1"][0], base["P1"][0].cpu().numpy()) < 1e-11


@pytest.mark.parametrize("precision,bar,wbar", [("fp64", 1e-9, 1e-12), ("fp32", 1e-5, 1e-6)])
def test_scc_second_order(cuda, cdmpt_lib, precision, bar, wbar):
    """The second-order self-consistent response D2 and Omega_SCF^(3) = (2/3) Tr[h1 D2].
    Omega_SCF^(3) is a trace that cancels: (2/3) ||h1||_F ||D2||_F is 27 to 4000 times
    |Omega_SCF^(3)| for these directions, so its bar is normwise, wbar (2/3) ||h1|| ||D2||, at
    the storage rounding of each precision (FP32: 1e-6, about 16 ulp)."""
    p, ref = _case(120, 3001)
    r = _run(cdmpt_lib, p, precision, 1e-12 if precision == "fp64" else 0.0, order=2)
    for d in range(3):
        assert oracle.rel_frobenius(r["D2"][d], ref["D2"][d]) < bar
        norm = 2.0 / 3.0 * np.linalg.norm(p.H1[d]) * np.linalg.norm(ref["D2"][d])
        assert abs(r["omega3"][d] - ref["omega3"][d]) < wbar * norm
        assert abs(r["mu2"][d] - ref["mu2"][d]) < bar * max(1.0, abs(ref["mu2"][d]))
