"""GPU tests of the higher perturbation terms H(lambda) = H0 + lambda H1 + lambda^2 H2 +
lambda^3 H3 (Eq. H_prt; Algorithm 1's X_0^(i) with H^(i), i = 1..3) in the second and third
order and in Eq. Resp_0's Omega^(3) and Omega^(4).

Reference: the oracle's Daleckii-Krein orders with H2 and H3, pinned on the CPU against
Algorithm 1's recursion, a 60-digit brute force and free-energy derivatives. Bars: 1e-10
(FP64), 1e-5 (FP32 and mixed).
"""
import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


def _sym(N, seed, scale):
    A = np.random.default_rng(seed).standard_normal((N, N)) * scale
    return 0.5 * (A + A.T)


def _run(pkg, p, precision, H2, H3):
    with pkg.Handle(precision=precision) as h:
        h.set_H(p.H0, p.H1)
        h.set_H_orders(H2, H3)
        h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
        r2 = h.response2(want_grad=False)
        r3 = h.response3()
    return r2, r3


def _check(r2, r3, ref, D, bar):
    for d in range(D):
        assert oracle.rel_frobenius(r2["P2"][d].cpu().numpy(), ref["P2"][d]) < bar
        assert oracle.rel_frobenius(r3["P3"][d].cpu().numpy(), ref["P3"][d]) < bar
        assert abs(r2["omega3"][d] - ref["omega3"][d]) < bar * abs(ref["omega3"][d])
        assert abs(r3["omega4"][d] - ref["omega4"][d]) < bar * abs(ref["omega4"][d])


def test_higher_terms_fp64_chain64(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    H2, H3 = _sym(p.N, 1, 0.05)[None], _sym(p.N, 2, 0.03)[None]
    ref = oracle.response3(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", H2=H2, H3=H3)
    r2, r3 = _run(cdmpt_lib, p, "fp64", H2, H3)
    _check(r2, r3, ref, 1, 1e-10)
    assert abs(r2["mu2"][0] - ref["mu2"][0]) < 1e-10 * max(1.0, abs(ref["mu2"][0]))
    assert abs(r3["mu3"][0] - ref["mu3"][0]) < 1e-10 * max(1.0, abs(ref["mu3"][0]))


def test_higher_terms_fp64_two_directions_h2_only(cuda, cdmpt_lib):
    base = syn.cubic_lattice((5, 5, 5), seed=23, beta=8.0, n=12)
    H1 = np.stack([base.H1[0], _sym(base.N, 3, 0.05)])
    p = syn.Problem("cubic5_d2", base.H0, H1, base.nocc, base.beta, base.n)
    H2 = np.stack([_sym(p.N, 4, 0.05), np.diag(np.linspace(-0.2, 0.2, p.N))])
    ref = oracle.response3(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", close=0.2, quad=0.2,
                           H2=H2)
    r2, r3 = _run(cdmpt_lib, p, "fp64", H2, None)
    _check(r2, r3, ref, 2, 1e-10)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_higher_terms_float_lattice(cuda, cdmpt_lib, precision):
    p = syn.cubic_lattice((6, 6, 6), seed=33, beta=20.0, n=14)
    H2, H3 = _sym(p.N, 5, 0.02)[None], _sym(p.N, 6, 0.01)[None]
    ref = oracle.response3(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", close=0.2, quad=0.2,
                           H2=H2, H3=H3)
    r2, r3 = _run(cdmpt_lib, p, precision, H2, H3)
    _check(r2, r3, ref, 1, 1e-5)


def test_gradient_refused_while_higher_terms_are_set(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    with cdmpt_lib.Handle(precision="fp64") as h:
        h.set_H(p.H0, p.H1)
        h.set_H_orders(_sym(p.N, 7, 0.05)[None], None)
        h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
        with pytest.raises(cdmpt_lib.CdmptError) as e:
            h.response2()
        assert e.value.status == 1
        h.set_H(p.H0, p.H1)                          # clears the higher terms
        h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
        g = h.response2()["grad"].cpu().numpy()
    ref = oracle.response2(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    assert oracle.rel_frobenius(g, ref["grad_alpha"][0]) < 1e-10
