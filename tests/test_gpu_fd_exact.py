"""GPU tests of the Fermi-Dirac-exact start (opts.fd_exact).

Starting the recursion from Z_0 = tanh(-beta (H0 - mu I) / 2^(n+1)) instead of the
linear X_0 makes the n steps reproduce the Fermi-Dirac density matrix itself
(Appendix A: Z_n = tanh(2^n atanh Z_0)). Reference: the oracle with
kind="fd" (eigenvalues of H0, the Fermi-Dirac function, Daleckii-Krein), the
plain definition. Bars: 1e-10 (FP64); FP32 1e-5; mixed 1e-6. The linear start misses
the Fermi-Dirac reference by its truncation error, which the first test shows.
The derivatives of the last solve (adjoint, free energy, orders 1 to 3 with the
higher perturbation terms, and the self-consistent charge layer) go through the
tangent and the Taylor coefficients of the tanh start; their references are the
oracle's Fermi-Dirac free energy, Daleckii-Krein orders and SCC solve.
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
    b0 = b1 = 1e-5 if precision == "fp32" else 1e-6
    assert oracle.rel_frobenius(r["P0"], ref["P0"]) < b0
    assert oracle.rel_frobenius(r["P1"][0], ref["P1"][0]) < b1


def _sym(N, seed, scale=1.0):
    A = np.random.default_rng(seed).standard_normal((N, N)) * scale
    return 0.5 * (A + A.T)


def _gc_args(p, gc):
    """Grand canonical: mu fixed 0.05 above the canonical one."""
    if not gc:
        return None, {}
    mu = oracle.solve(p.H0, p.H1, p.beta, p.nocc, kind="fd")["mu"] + 0.05
    return mu, dict(mu_guess=mu, grand_canonical=True)


@pytest.mark.parametrize("gc", [False, True])
def test_fd_exact_adjoint_fp64(cuda, cdmpt_lib, gc):
    """d Tr[G P0] / d H0 through the reverse sweep and the tanh start equals the first-order
    Fermi-Dirac response to G (the response operator is self-adjoint)."""
    import torch
    p = syn.workload("chain64")
    G = _sym(p.N, 17)
    mu, kw = _gc_args(p, gc)
    ref = oracle.solve(p.H0, G, p.beta, p.nocc, kind="fd", canonical=not gc, mu=mu)["P1"][0]
    with cdmpt_lib.Handle(precision="fp64", fd_exact=True, **kw) as h:
        h.set_H(p.H0, p.H1)
        h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
        g = h.vjp_P0(torch.from_numpy(G).cuda()).cpu().numpy()
    assert oracle.rel_frobenius(g, ref) < 1e-10


@pytest.mark.parametrize("gc", [False, True])
def test_fd_exact_free_energy_fp64(cuda, cdmpt_lib, gc):
    """The Mermin free energy of the Fermi-Dirac P0 (R = atanh Z_0 - Y vanishes) and its
    gradient: P0 itself (canonical) or P0 + mu dTr P0/dH0 (fixed mu)."""
    p = syn.workload("chain64")
    mu, kw = _gc_args(p, gc)
    ref = oracle.free_energy(p.H0, p.beta, p.nocc, kind="fd", canonical=not gc, mu=mu)
    with cdmpt_lib.Handle(precision="fp64", fd_exact=True, **kw) as h:
        h.set_H(p.H0, None)
        h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
        r = h.free_energy()
    assert abs(r["omega"] - ref["omega"]) < 1e-10 * abs(ref["omega"])
    assert oracle.rel_frobenius(r["grad"].cpu().numpy(), ref["grad"]) < 1e-10


@pytest.mark.parametrize("gc", [False, True])
def test_fd_exact_orders_1_to_3_fp64(cuda, cdmpt_lib, gc):
    """response1/2/3 from the Taylor coefficients of the tanh start against the Fermi-Dirac
    Daleckii-Krein orders, with mu2, mu3, Omega^(3), Omega^(4) and d alpha / d H0."""
    p = syn.workload("chain64")
    mu, kw = _gc_args(p, gc)
    ref = oracle.response3(p.H0, p.H1, p.beta, p.nocc, kind="fd", canonical=not gc, mu=mu)
    with cdmpt_lib.Handle(precision="fp64", fd_exact=True, **kw) as h:
        h.set_H(p.H0, p.H1)
        h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
        r1 = h.response1(p.H1)
        r2 = h.response2()
        r3 = h.response3()
    assert oracle.rel_frobenius(r1["P1"][0].cpu().numpy(), ref["P1"][0]) < 1e-10
    assert oracle.rel_frobenius(r2["P2"][0].cpu().numpy(), ref["P2"][0]) < 1e-10
    assert oracle.rel_frobenius(r3["P3"][0].cpu().numpy(), ref["P3"][0]) < 1e-10
    assert oracle.rel_frobenius(r2["grad"].cpu().numpy(), ref["grad_alpha"][0]) < 1e-10
    assert abs(r2["mu2"][0] - ref["mu2"][0]) < 1e-10 * max(1.0, abs(ref["mu2"][0]))
    assert abs(r3["mu3"][0] - ref["mu3"][0]) < 1e-10 * max(1.0, abs(ref["mu3"][0]))
    assert abs(r2["omega3"][0] - ref["omega3"][0]) < 1e-10 * abs(ref["omega3"][0])
    assert abs(r3["omega4"][0] - ref["omega4"][0]) < 1e-10 * abs(ref["omega4"][0])


def test_fd_exact_higher_terms_fp64_lattice(cuda, cdmpt_lib):
    """H(lambda) = H0 + lambda H1 + lambda^2 H2 + lambda^3 H3: the Y^(2), Y^(3) of the start."""
    p = syn.cubic_lattice((5, 5, 5), seed=23, beta=8.0, n=12)
    H2, H3 = _sym(p.N, 4, 0.05)[None], _sym(p.N, 5, 0.03)[None]
    ref = oracle.response3(p.H0, p.H1, p.beta, p.nocc, kind="fd", close=0.2, quad=0.2, H2=H2,
                           H3=H3)
    with cdmpt_lib.Handle(precision="fp64", fd_exact=True) as h:
        h.set_H(p.H0, p.H1)
        h.set_H_orders(H2, H3)
        h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
        r2 = h.response2(want_grad=False)
        r3 = h.response3()
    assert oracle.rel_frobenius(r2["P2"][0].cpu().numpy(), ref["P2"][0]) < 1e-10
    assert oracle.rel_frobenius(r3["P3"][0].cpu().numpy(), ref["P3"][0]) < 1e-10
    assert abs(r2["omega3"][0] - ref["omega3"][0]) < 1e-10 * abs(ref["omega3"][0])
    assert abs(r3["omega4"][0] - ref["omega4"][0]) < 1e-10 * abs(ref["omega4"][0])


def test_fd_exact_fp32_lattice_512_derivatives(cuda, cdmpt_lib):
    import torch
    p = syn.cubic_lattice((8, 8, 8), seed=1002, beta=20.0, n=14)
    G = _sym(p.N, 29, 0.1)
    ref1 = oracle.solve(p.H0, G, p.beta, p.nocc, kind="fd")
    ref2 = oracle.response2(p.H0, p.H1, p.beta, p.nocc, kind="fd", close=0.2, quad=0.2)
    reff = oracle.free_energy(p.H0, p.beta, p.nocc, kind="fd")
    with cdmpt_lib.Handle(precision="fp32", fd_exact=True) as h:
        h.set_H(p.H0, p.H1)
        h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
        g = h.vjp_P0(torch.from_numpy(G).cuda()).cpu().numpy()
        r2 = h.response2(want_grad=False)
        fe = h.free_energy()
    assert oracle.rel_frobenius(g, ref1["P1"][0]) < 1e-5
    assert oracle.rel_frobenius(r2["P2"][0].cpu().numpy(), ref2["P2"][0]) < 1e-5
    assert abs(fe["omega"] - reff["omega"]) < 1e-6 * abs(reff["omega"])
    assert oracle.rel_frobenius(fe["grad"].cpu().numpy(), reff["grad"]) < 1e-5


def test_fd_exact_scc_second_order_fp64(cuda, cdmpt_lib):
    """The self-consistent charge layer on the Fermi-Dirac start, through its CPSCF orders."""
    p = syn.nonorthogonal_cluster(120, seed=3001, beta=20.0, n=14)
    m = p.meta
    ref = oracle.scc_solve(p.H0, p.H1, m["S"], m["gamma"], m["q0"], p.beta, p.nocc,
                           kind="fd", order=2)
    with cdmpt_lib.Handle(precision="fp64", fd_exact=True) as h:
        h.set_overlap(m["S"])
        r = h.scc_solve(p.H0, p.H1, m["gamma"], p.beta, p.nocc, p.n, q0=m["q0"], tol=1e-12,
                        order=2)
    assert oracle.rel_frobenius(r["D0"], ref["D0"]) < 1e-9
    for d in range(p.H1.shape[0]):
        assert oracle.rel_frobenius(r["D1"][d], ref["D1"][d]) < 1e-9
        assert oracle.rel_frobenius(r["D2"][d], ref["D2"][d]) < 1e-9
        assert abs(r["omega2"][d] - ref["omega2"][d]) < 1e-9 * abs(ref["omega2"][d])
