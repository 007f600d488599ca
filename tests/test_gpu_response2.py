"""GPU tests of the second-order canonical response and the polarizability gradient.

cdmpt_response2 returns P2 = (1/2) d^2 P / d lambda^2 (Algorithm 1, order 2,
with H^(2) = 0), mu2 (Tr P2 = 0), Omega^(3) = 1/3 Tr[H1 P2] (Eq. Resp_0), and
d(sum_d w_d alpha_d)/dH0 = -4 sum_d w_d P2_d.

References:
- The oracle's second-order Daleckii-Krein response (kind="rec", the function
  the recursion computes exactly), itself pinned on the CPU against Algorithm
  1's order-2 recursion and finite differences.
- Central finite differences of alpha(H0 + t E) along 20 random symmetric
  directions E, alpha from the library's own FP64 solves.
Bars: relative Frobenius 1e-10 (FP64), 1e-5 (FP32 and mixed).
"""
import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


def _sym(rng, N, scale=1.0):
    A = rng.standard_normal((N, N)) * scale
    return 0.5 * (A + A.T)


def _r2(pkg, p, precision, weights=None):
    with pkg.Handle(precision=precision) as h:
        h.set_H(p.H0, p.H1)
        h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
        r = h.response2(weights=weights)
    return {"P2": r["P2"].cpu().numpy(), "mu2": r["mu2"], "omega3": r["omega3"],
            "grad": r["grad"].cpu().numpy()}


def test_p2_fp64_chain64(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    ref = oracle.response2(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    r = _r2(cdmpt_lib, p, "fp64")
    assert oracle.rel_frobenius(r["P2"][0], ref["P2"][0]) < 1e-10
    assert abs(r["mu2"][0] - ref["mu2"][0]) < 1e-9 * max(1.0, abs(ref["mu2"][0]))
    assert oracle.rel_frobenius(r["grad"], ref["grad_alpha"][0]) < 1e-10
    assert abs(r["omega3"][0] - ref["omega3"][0]) < 1e-10 * abs(ref["omega3"][0])


def test_p2_fp64_three_directions_weighted(cuda, cdmpt_lib):
    """D = 3 directions on a disordered 6^3 lattice; the gradient of sum_d w_d alpha_d."""
    base = syn.cubic_lattice((6, 6, 6), seed=21, beta=8.0, n=12)
    rng = np.random.default_rng(2)
    H1 = np.stack([base.H1[0], np.diag(rng.uniform(-1, 1, base.N)), _sym(rng, base.N, 0.05)])
    p = syn.Problem("cubic6_d3", base.H0, H1, base.nocc, base.beta, base.n)
    w = np.array([0.7, -1.3, 2.0])
    ref = oracle.response2(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    r = _r2(cdmpt_lib, p, "fp64", weights=w)
    for d in range(3):
        assert oracle.rel_frobenius(r["P2"][d], ref["P2"][d]) < 1e-10
        assert abs(r["omega3"][d] - ref["omega3"][d]) < 1e-9 * abs(ref["omega3"][d])
    g = sum(w[d] * ref["grad_alpha"][d] for d in range(3))
    assert oracle.rel_frobenius(r["grad"], g) < 1e-10


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_p2_float_lattice_512(cuda, cdmpt_lib, precision):
    p = syn.cubic_lattice((8, 8, 8), seed=31, beta=20.0, n=14)
    ref = oracle.response2(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    r = _r2(cdmpt_lib, p, precision)
    assert oracle.rel_frobenius(r["P2"][0], ref["P2"][0]) < 1e-5
    assert oracle.rel_frobenius(r["grad"], ref["grad_alpha"][0]) < 1e-5
    assert abs(r["omega3"][0] - ref["omega3"][0]) < 1e-5 * abs(ref["omega3"][0])


def test_alpha_gradient_fp64_central_differences_20_directions(cuda, cdmpt_lib):
    """<grad alpha, E> == (alpha(H0 + hE) - alpha(H0 - hE)) / 2h, 20 random symmetric E."""
    p = syn.cubic_lattice((4, 4, 4), seed=5, beta=6.0, n=12)
    g = _r2(cdmpt_lib, p, "fp64")["grad"]
    rng = np.random.default_rng(13)
    h = 1e-4
    with cdmpt_lib.Handle(precision="fp64") as hd:
        def alpha(H):
            hd.set_H(H, p.H1)
            hd.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
            return float(hd.polarizability()[0])
        errs = []
        for _ in range(20):
            E = _sym(rng, p.N, 0.1)
            fd = (alpha(p.H0 + h * E) - alpha(p.H0 - h * E)) / (2 * h)
            errs.append(abs(fd - np.sum(g * E)) / max(1e-12, abs(fd)))
    assert max(errs) < 1e-6, max(errs)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_alpha_gradient_lattice_2048(cuda, cdmpt_lib, precision):
    """The differentiation workload: 16 x 16 x 8 lattice (N = 2048), beta = 20, n = 16."""
    p = syn.workload("cubic16x16x8")
    ref = oracle.response2(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    r = _r2(cdmpt_lib, p, precision)
    assert oracle.rel_frobenius(r["grad"], ref["grad_alpha"][0]) < 1e-5


def test_polarizability_autograd(cuda, cdmpt_lib):
    """torch.autograd through Polarizability: L = sum_d c_d alpha_d + alpha_0^2."""
    import torch
    base = syn.cubic_lattice((5, 5, 5), seed=9, beta=8.0, n=12)
    rng = np.random.default_rng(8)
    H1 = np.stack([base.H1[0], np.diag(rng.uniform(-1, 1, base.N))])
    c = np.array([0.5, -2.0])
    H = torch.from_numpy(base.H0).cuda().requires_grad_(True)
    with cdmpt_lib.Handle(precision="fp64") as h:
        a = cdmpt_lib.Polarizability.apply(H, torch.from_numpy(H1).cuda(), base.beta, base.nocc,
                                           base.n, h)
        L = (a * torch.from_numpy(c).cuda()).sum() + a[0] ** 2
        L.backward()
    ref = oracle.response2(base.H0, H1, base.beta, base.nocc, n=base.n, kind="rec")
    assert np.allclose(a.detach().cpu().numpy(), ref["alpha"], rtol=1e-10, atol=0)
    w = c + np.array([2.0 * ref["alpha"][0], 0.0])
    g = sum(w[d] * ref["grad_alpha"][d] for d in range(2))
    assert oracle.rel_frobenius(H.grad.cpu().numpy(), g) < 1e-9


def test_response2_requires_a_solve_with_directions(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    with cdmpt_lib.Handle(precision="fp64") as h:
        with pytest.raises(cdmpt_lib.CdmptError):
            h.response2()
        h.set_H(p.H0, None)
        h.solve(p.beta, p.nocc, p.n)
        with pytest.raises(cdmpt_lib.CdmptError) as e:
            h.response2()
        assert e.value.status == 1
