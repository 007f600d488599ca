"""GPU tests of the non-orthogonal basis (Sec. IV, Eq. Fermi_D).

cdmpt_set_overlap computes the Loewdin factor Z = S^(-1/2) by Newton-Schulz;
set_H then takes F and h1, the solve works on Z F Z and Z h1 Z, and outputs are
mapped back (D = Z P Z and likewise for D1, D2, the gradients). The oracle
orthogonalises with the inverse Cholesky factor instead (another Z with
Z^T S Z = I), so agreement checks the basis independence as well. Bars: 1e-10
(FP64); FP32 1e-5; mixed 1e-6.
"""
import functools

import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def _case(N, seed, beta, n):
    p = syn.nonorthogonal_cluster(N, seed=seed, beta=beta, n=n)
    ref = oracle.solve_nonorthogonal(p.H0, p.H1, p.meta["S"], p.beta, p.nocc, n=p.n, order=2)
    return p, ref


def _run(pkg, p, precision, want2=True):
    with pkg.Handle(precision=precision) as h:
        h.set_overlap(p.meta["S"])
        it, res = h.overlap_info()
        h.set_H(p.H0, p.H1)
        r = h.solve(p.beta, p.nocc, p.n)
        out = {"D0": r["P0"].cpu().numpy(), "D1": r["P1"].cpu().numpy(), "mu": r["mu"],
               "mu1": r["mu1"], "alpha": h.polarizability(), "ns": (it, res)}
        if want2:
            r2 = h.response2()
            out["D2"] = r2["P2"].cpu().numpy()
            out["grad_alpha"] = r2["grad"].cpu().numpy()
            out["grad_omega"] = h.free_energy()["grad"].cpu().numpy()
    return out


def test_overlap_fp64_cluster(cuda, cdmpt_lib):
    p, ref = _case(201, 2001, 20.0, 14)
    r = _run(cdmpt_lib, p, "fp64")
    it, res = r["ns"]
    assert res < 1e-12 and 3 <= it <= 60, r["ns"]
    assert oracle.rel_frobenius(r["D0"], ref["D0"]) < 1e-10
    S = p.meta["S"]
    assert abs(np.trace(r["D0"] @ S) - p.nocc) < 1e-9
    for d in range(3):
        assert oracle.rel_frobenius(r["D1"][d], ref["D1"][d]) < 1e-10
        assert oracle.rel_frobenius(r["D2"][d], ref["D2"][d]) < 1e-10
        assert abs(r["alpha"][d] - ref["alpha"][d]) < 1e-10 * abs(ref["alpha"][d])
    g = ref["grad_alpha"].sum(axis=0)
    assert oracle.rel_frobenius(r["grad_alpha"], g) < 1e-10
    assert oracle.rel_frobenius(r["grad_omega"], ref["grad_omega"]) < 1e-10
    assert abs(r["mu"] - ref["mu"]) < 1e-10


def test_overlap_fp64_vjp_against_response(cuda, cdmpt_lib):
    """dL/dF for L = Tr[G D]: the adjoint in the orthogonal basis between the two congruences.
    Reference: the oracle's canonical response to the perturbation Z^T G Z in the orthogonal
    basis (the adjoint's tangent), mapped back as a gradient."""
    import torch
    p, _ = _case(150, 2002, 10.0, 12)
    S = p.meta["S"]
    rng = np.random.default_rng(3)
    A = rng.standard_normal((p.N, p.N))
    G = 0.5 * (A + A.T)
    with cdmpt_lib.Handle(precision="fp64") as h:
        h.set_overlap(S)
        h.set_H(p.H0, None)
        h.solve(p.beta, p.nocc, p.n, want_P0=False)
        g = h.vjp_P0(torch.from_numpy(G).cuda()).cpu().numpy()
    Linv = oracle.cholesky_factor(S)
    Fp = oracle.to_orthogonal(p.H0, Linv)
    Gp = Linv @ G @ Linv.T            # dL/dP_perp for D = Linv^T P_perp Linv
    ref = oracle.solve(Fp, Gp, p.beta, p.nocc, n=p.n, kind="rec")["P1"][0]
    assert oracle.rel_frobenius(g, oracle.from_orthogonal(ref, Linv)) < 1e-10


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_overlap_float_cluster(cuda, cdmpt_lib, precision):
    p, ref = _case(201, 2001, 20.0, 14)
    r = _run(cdmpt_lib, p, precision, want2=False)
    bar0 = bar1 = 1e-5 if precision == "fp32" else 1e-6
    assert oracle.rel_frobenius(r["D0"], ref["D0"]) < bar0
    for d in range(3):
        assert oracle.rel_frobenius(r["D1"][d], ref["D1"][d]) < bar1


def test_overlap_identity_and_reset(cuda, cdmpt_lib):
    """S = I reproduces the orthogonal solve; set_overlap(None) returns to the orthogonal mode."""
    q = syn.workload("chain64")
    with cdmpt_lib.Handle(precision="fp64") as h:
        h.set_H(q.H0, q.H1)
        base = h.solve(q.beta, q.nocc, q.n)
        h.set_overlap(np.eye(q.N))
        assert h.overlap_info()[1] < 1e-12
        h.set_H(q.H0, q.H1)
        ident = h.solve(q.beta, q.nocc, q.n)
        h.set_overlap(None)
        assert h.overlap_info() == (0, 0.0)
        h.set_H(q.H0, q.H1)
        back = h.solve(q.beta, q.nocc, q.n)
    for r in (ident, back):
        assert oracle.rel_frobenius(r["P0"].cpu().numpy(), base["P0"].cpu().numpy()) < 1e-13
        assert oracle.rel_frobenius(r["P1"].cpu().numpy(), base["P1"].cpu().numpy()) < 1e-12


def test_overlap_errors(cuda, cdmpt_lib):
    q = syn.workload("chain64")
    with cdmpt_lib.Handle(precision="fp64") as h:
        S = np.eye(q.N)
        S[0, 0] = -1.0                     # indefinite: Newton-Schulz cannot converge
        with pytest.raises(cdmpt_lib.CdmptError):
            h.set_overlap(S)
        h.set_overlap(np.eye(q.N))
        with pytest.raises(cdmpt_lib.CdmptError):
            h.set_H(q.H0[:32, :32], None)  # size differs from the overlap's
