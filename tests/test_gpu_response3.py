"""GPU tests of the third-order canonical response and Omega^(4).

cdmpt_response3 returns P3 = (1/6) d^3 P / d lambda^3 (Algorithm 1, order 3,
with H^(2) = H^(3) = 0), mu3 (Tr P3 = 0, after mu2 from an order-2 pass) and
Omega^(4) = 1/4 Tr[H1 P3] (Eq. Resp_0).

Reference: the oracle's third-order Daleckii-Krein response (kind="rec", the
function the recursion computes exactly), pinned on the CPU against Algorithm
1's order-3 recursion, finite differences of P2 and a 60-digit brute force.
Bars: relative Frobenius 1e-10 (FP64), 1e-5 (FP32 and mixed). On the lattices
the oracle takes its exact-identity branch for pairs and quadruples down to a
spread of 0.2 / beta (close = quad = 0.2); on the 6^3 lattice that moves P3 by
5e-14 against the default thresholds and cuts the oracle's time from 21 s to
3.5 s.
"""
import functools

import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def _lattice_ref(L, seed, beta, n):
    p = syn.cubic_lattice(L, seed=seed, beta=beta, n=n)
    return p, oracle.response3(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", close=0.2,
                               quad=0.2)


def _r3(pkg, p, precision, **kw):
    with pkg.Handle(precision=precision, **kw) as h:
        h.set_H(p.H0, p.H1)
        h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
        r = h.response3()
        r2 = h.response2(want_P2=False, want_grad=False)
    return {"P3": r["P3"].cpu().numpy(), "mu3": r["mu3"], "omega4": r["omega4"],
            "mu2": r2["mu2"]}


def test_p3_fp64_chain64(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    ref = oracle.response3(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    r = _r3(cdmpt_lib, p, "fp64")
    assert oracle.rel_frobenius(r["P3"][0], ref["P3"][0]) < 1e-10
    assert abs(r["mu3"][0] - ref["mu3"][0]) < 1e-9 * max(1.0, abs(ref["mu3"][0]))
    assert abs(r["mu2"][0] - ref["mu2"][0]) < 1e-9 * max(1.0, abs(ref["mu2"][0]))
    assert abs(r["omega4"][0] - ref["omega4"][0]) < 1e-10 * abs(ref["omega4"][0])
    assert abs(np.trace(r["P3"][0])) < 1e-10 * np.linalg.norm(r["P3"][0])


def test_p3_fp64_two_directions_lattice(cuda, cdmpt_lib):
    """D = 2 directions (x dipole and a random symmetric field) on a disordered 5^3 lattice."""
    base = syn.cubic_lattice((5, 5, 5), seed=23, beta=8.0, n=12)
    rng = np.random.default_rng(5)
    A = rng.standard_normal((base.N, base.N)) * 0.05
    H1 = np.stack([base.H1[0], 0.5 * (A + A.T)])
    p = syn.Problem("cubic5_d2", base.H0, H1, base.nocc, base.beta, base.n)
    ref = oracle.response3(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", close=0.2, quad=0.2)
    r = _r3(cdmpt_lib, p, "fp64")
    for d in range(2):
        assert oracle.rel_frobenius(r["P3"][d], ref["P3"][d]) < 1e-10
        assert abs(r["omega4"][d] - ref["omega4"][d]) < 1e-9 * abs(ref["omega4"][d])


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_p3_float_lattice_216(cuda, cdmpt_lib, precision):
    p, ref = _lattice_ref((6, 6, 6), 33, 20.0, 14)
    r = _r3(cdmpt_lib, p, precision)
    assert oracle.rel_frobenius(r["P3"][0], ref["P3"][0]) < 1e-5
    assert abs(r["omega4"][0] - ref["omega4"][0]) < 1e-5 * abs(ref["omega4"][0])


def test_p3_grand_canonical_fp64(cuda, cdmpt_lib):
    """Fixed mu: mu1 = mu2 = mu3 = 0 and P3 equals the grand-canonical closed form."""
    p = syn.workload("chain64")
    mu = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")["mu"] + 0.05
    ref = oracle.response3(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", canonical=False, mu=mu)
    r = _r3(cdmpt_lib, p, "fp64", mu_guess=mu, grand_canonical=True)
    assert r["mu3"][0] == 0.0
    assert oracle.rel_frobenius(r["P3"][0], ref["P3"][0]) < 1e-10


def test_response3_requires_directions(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    with cdmpt_lib.Handle(precision="fp64") as h:
        with pytest.raises(cdmpt_lib.CdmptError):
            h.response3()
        h.set_H(p.H0, None)
        h.solve(p.beta, p.nocc, p.n)
        with pytest.raises(cdmpt_lib.CdmptError) as e:
            h.response3()
        assert e.value.status == 1
