"""GPU tests of the Fermi-Dirac-exact start (opts.fd_exact).

Starting the recursion from Z_0 = tanh(-beta (H0 - mu I) / 2^(n+1)) instead of the
linear X_0 makes the n steps reproduce the Fermi-Dirac density matrix itself
(Appendix A: Z_n = tanh(2^n atanh Z_0)). Reference: the oracle with
kind="fd" (eigenvalues of H0, the Fermi-Dirac function, Daleckii-Krein), the
plain definition. Bars: 1e-10 (FP64); FP32 1e-5; mixed 1e-6 for P0 and max(1e-6,
1.3 x the FP32 error) for P1 (the FP32 storage floor). The linear start misses
the Fermi-Dirac reference by its truncation error, which the first test shows.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


def _solve(pkg, p, precision, **kw):
    with pkg.Handle(precision=precision, **kw) as h:
        h.set_H(p.H0, p.H1)
        r = h.solve(p.beta, p.nocc, p.n)
        return {"P0": r["P0"].cpu().numpy(), "P1": r["P1"].cpu().numpy(), "mu": r["mu"],
                "mu1": r["mu1"], "alpha": h.polarizability()}


def test_fd_exact_fp64_chain64_matches_fermi_dirac(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, kind="fd")
    r = _solve(cdmpt_lib, p, "fp64", fd_exact=True)
    assert oracle.rel_frobenius(r["P0"], ref["P0"]) < 1e-10
    assert oracle.rel_frobenius(r["P1"][0], ref["P1"][0]) < 1e-10
    assert abs(r["mu"] - ref["mu"]) < 1e-11
    assert abs(r["mu1"][0] - ref["mu1"][0]) < 1e-10 * max(1.0, abs(ref["mu1"][0]))
    assert abs(r["alpha"][0] - ref["alpha"][0]) < 1e-10 * abs(ref["alpha"][0])
    lin = _solve(cdmpt_lib, p, "fp64")
    assert oracle.rel_frobenius(lin["P1"][0], ref["P1"][0]) > 1e-9   # the truncation gap


@pytest.mark.parametrize("beta", [5.0, 80.0])
def test_fd_exact_fp64_lattice(cuda, cdmpt_lib, beta):
    p = syn.cubic_lattice((6, 6, 6), seed=91, beta=beta, n=14)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, kind="fd")
    r = _solve(cdmpt_lib, p, "fp64", fd_exact=True)
    assert oracle.rel_frobenius(r["P0"], ref["P0"]) < 1e-10
    assert oracle.rel_frobenius(r["P1"][0], ref["P1"][0]) < 1e-10


def test_fd_exact_fp64_checkpointed_and_grand_canonical(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, kind="fd")
    r = _solve(cdmpt_lib, p, "fp64", fd_exact=True, ckpt_stride="sqrt")
    assert oracle.rel_frobenius(r["P1"][0], ref["P1"][0]) < 1e-10
    mu = ref["mu"] + 0.05
    refg = oracle.solve(p.H0, p.H1, p.beta, p.nocc, kind="fd", canonical=False, mu=mu)
    g = _solve(cdmpt_lib, p, "fp64", fd_exact=True, mu_guess=mu, grand_canonical=True)
    assert oracle.rel_frobenius(g["P0"], refg["P0"]) < 1e-10
    assert oracle.rel_frobenius(g["P1"][0], refg["P1"][0]) < 1e-10


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_fd_exact_float_lattice_512(cuda, cdmpt_lib, precision):
    p = syn.cubic_lattice((8, 8, 8), seed=1002, beta=20.0, n=14)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, kind="fd")
    r = _solve(cdmpt_lib, p, precision, fd_exact=True)
    if precision == "fp32":
        b0 = b1 = 1e-5
    else:
        f = _solve(cdmpt_lib, p, "fp32", fd_exact=True)
        b0 = 1e-6
        b1 = max(1e-6, 1.3 * oracle.rel_frobenius(f["P1"][0], ref["P1"][0]))
    assert oracle.rel_frobenius(r["P0"], ref["P0"]) < b0
    assert oracle.rel_frobenius(r["P1"][0], ref["P1"][0]) < b1


def test_fd_exact_refuses_the_other_derivatives(cuda, cdmpt_lib):
    import torch
    p = syn.workload("chain64")
    with cdmpt_lib.Handle(precision="fp64", fd_exact=True) as h:
        h.set_H(p.H0, p.H1)
        h.solve(p.beta, p.nocc, p.n)
        for call in (lambda: h.vjp_P0(torch.eye(p.N, dtype=torch.float64).cuda()),
                     lambda: h.response2(), lambda: h.free_energy()):
            with pytest.raises(cdmpt_lib.CdmptError) as e:
                call()
            assert e.value.status == 1
