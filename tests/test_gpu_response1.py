"""GPU tests of cdmpt_response1: first-order responses to new perturbations on the trajectory
of a finished solve (no new solve). References: the oracle's canonical Daleckii-Krein response
(kind="rec") and the solve's own response for the same directions. Bars: 1e-10 (FP64) against
the oracle, 1e-12 against the solve's own P1; 1e-5 in mixed precision.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


def _dirs(p, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((p.N, p.N)) * 0.1
    return np.stack([p.H1[0], 0.5 * (A + A.T)])


def test_response1_fp64_matches_oracle_and_solve(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    H1 = _dirs(p, 3)
    ref = oracle.solve(p.H0, H1, p.beta, p.nocc, n=p.n, kind="rec")
    with cdmpt_lib.Handle(precision="fp64") as h:
        h.set_H(p.H0, None)
        h.solve(p.beta, p.nocc, p.n, want_P0=False)
        r = h.response1(H1)
        rh = h.response1(H1, device="cpu")            # host outputs
        h.set_H(p.H0, H1)
        s = h.solve(p.beta, p.nocc, p.n, want_P0=False)
        a = h.polarizability()
    for d in range(2):
        P1 = r["P1"][d].cpu().numpy()
        assert oracle.rel_frobenius(P1, ref["P1"][d]) < 1e-10
        assert oracle.rel_frobenius(P1, s["P1"][d].cpu().numpy()) < 1e-12
        assert oracle.rel_frobenius(rh["P1"][d].numpy(), P1) < 1e-14
        assert abs(r["mu1"][d] - ref["mu1"][d]) < 1e-10 * max(1.0, abs(ref["mu1"][d]))
        assert abs(r["alpha"][d] - a[d]) < 1e-12 * abs(a[d])


def test_response1_mixed_lattice(cuda, cdmpt_lib):
    p = syn.cubic_lattice((8, 8, 8), seed=1002, beta=20.0, n=14)
    H1 = _dirs(p, 4)
    ref = oracle.solve(p.H0, H1, p.beta, p.nocc, n=p.n, kind="rec")
    with cdmpt_lib.Handle(precision="mixed") as h:
        h.set_H(p.H0, None)
        h.solve(p.beta, p.nocc, p.n, want_P0=False)
        r = h.response1(H1)
    for d in range(2):
        assert oracle.rel_frobenius(r["P1"][d].cpu().numpy(), ref["P1"][d]) < 1e-5


def test_response1_non_orthogonal(cuda, cdmpt_lib):
    p = syn.nonorthogonal_cluster(150, seed=2003, beta=10.0, n=12)
    ref = oracle.solve_nonorthogonal(p.H0, p.H1, p.meta["S"], p.beta, p.nocc, n=p.n)
    with cdmpt_lib.Handle(precision="fp64") as h:
        h.set_overlap(p.meta["S"])
        h.set_H(p.H0, None)
        h.solve(p.beta, p.nocc, p.n, want_P0=False)
        r = h.response1(p.H1)
    for d in range(3):
        assert oracle.rel_frobenius(r["P1"][d].cpu().numpy(), ref["D1"][d]) < 1e-10
        assert abs(r["alpha"][d] - ref["alpha"][d]) < 1e-10 * abs(ref["alpha"][d])


def test_response1_errors(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    with cdmpt_lib.Handle(precision="fp64") as h:
        with pytest.raises(cdmpt_lib.CdmptError):
            h.response1(p.H1)                     # no solve yet
