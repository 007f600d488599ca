"""GPU tests of the grand-canonical (fixed-mu) mode against the oracle.

With opts.grand_canonical = 1 the chemical potential stays at mu_guess: one
occupation sweep, mu1 = mu2 = 0, and the adjoint drops the dmu/dH0 term.
Reference: the oracle with canonical=False at the same mu (itself pinned on the
CPU against Algorithm 1's recursion with mu1 = mu2 = 0).
"""
import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


def _sym(rng, N, scale=1.0):
    A = rng.standard_normal((N, N)) * scale
    return 0.5 * (A + A.T)


def _mu(p, shift):
    return oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")["mu"] + shift


def test_grand_canonical_fp64_chain64(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    mu = _mu(p, 0.05)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", canonical=False, mu=mu)
    with cdmpt_lib.Handle(precision="fp64", grand_canonical=True, mu_guess=mu) as h:
        h.set_H(p.H0, p.H1)
        r = h.solve(p.beta, p.nocc, p.n)
        alpha = h.polarizability()
        st = h.stats()
    assert st["mu_iterations"] == 1
    assert r["mu"] == pytest.approx(mu, abs=0.0)
    assert r["mu1"][0] == 0.0
    assert oracle.rel_frobenius(r["P0"].cpu().numpy(), ref["P0"]) < 1e-10
    assert oracle.rel_frobenius(r["P1"][0].cpu().numpy(), ref["P1"][0]) < 1e-10
    assert abs(alpha[0] - ref["alpha"][0]) < 1e-9 * abs(ref["alpha"][0])


def test_grand_canonical_adjoint_and_second_order(cuda, cdmpt_lib):
    import torch
    p = syn.cubic_lattice((5, 5, 5), seed=17, beta=8.0, n=12)
    mu = _mu(p, -0.1)
    rng = np.random.default_rng(4)
    G = _sym(rng, p.N)
    with cdmpt_lib.Handle(precision="fp64", grand_canonical=True, mu_guess=mu) as h:
        h.set_H(p.H0, p.H1)
        h.solve(p.beta, p.nocc, p.n)
        g = h.vjp_P0(torch.from_numpy(G).cuda()).cpu().numpy()
        r2 = h.response2()
    # fixed mu: d Tr[G P0]/dH0 is the grand-canonical response to sym(G)
    ref = oracle.solve(p.H0, G, p.beta, p.nocc, n=p.n, kind="rec", canonical=False, mu=mu)
    assert oracle.rel_frobenius(g, ref["P1"][0]) < 1e-9
    ref2 = oracle.response2(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", canonical=False,
                            mu=mu)
    assert r2["mu2"][0] == 0.0
    assert oracle.rel_frobenius(r2["P2"][0].cpu().numpy(), ref2["P2"][0]) < 1e-10
    assert oracle.rel_frobenius(r2["grad"].cpu().numpy(), ref2["grad_alpha"][0]) < 1e-10


def test_grand_canonical_mixed_lattice_1000(cuda, cdmpt_lib):
    p = syn.cubic_lattice((10, 10, 10), seed=7, beta=20.0, n=14)
    mu = _mu(p, 0.02)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", canonical=False, mu=mu)
    with cdmpt_lib.Handle(precision="mixed", grand_canonical=True, mu_guess=mu) as h:
        h.set_H(p.H0, p.H1)
        r = h.solve(p.beta, p.nocc, p.n)
    assert oracle.rel_frobenius(r["P0"].cpu().numpy(), ref["P0"]) < 1e-6
    assert oracle.rel_frobenius(r["P1"][0].cpu().numpy(), ref["P1"][0]) < 1e-6


def test_grand_canonical_errors(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    with pytest.raises(cdmpt_lib.CdmptError):           # needs mu_guess
        cdmpt_lib.Handle(precision="fp64", grand_canonical=True)
    with cdmpt_lib.Handle(precision="fp64", grand_canonical=True, mu_guess=1e4) as h:
        h.set_H(p.H0, p.H1)
        with pytest.raises(cdmpt_lib.CdmptError) as e:  # X_0 leaves [0, 1]
            h.solve(p.beta, p.nocc, p.n)
        assert e.value.status == 2
