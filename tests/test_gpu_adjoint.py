"""GPU tests of the hand-written adjoint (cdmpt_vjp_P0): d Tr[G0 P0] / d H0.

References:
- The oracle's gradient. For L = Tr[G P0] with canonical P0(H0), dL/dH0 is the
  canonical first-order response to the perturbation H1 = sym(G). The
  free-energy Hessian is symmetric (App. B: dOmega/dH0 = P0), and the oracle
  evaluates that response exactly by Daleckii-Krein.
- The forward DMPT response on the GPU, which is the tangent of the same map.
- Central finite differences of the loss along 20 random symmetric directions.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


def _sym(rng, N, scale=1.0):
    A = rng.standard_normal((N, N)) * scale
    return 0.5 * (A + A.T)


def _grad(pkg, p, G, precision, **kw):
    import torch
    with pkg.Handle(precision=precision, **kw) as h:
        h.set_H(p.H0, None)
        h.solve(p.beta, p.nocc, p.n)
        g = h.vjp_P0(torch.from_numpy(G).cuda())
    return g.cpu().numpy()


def test_adjoint_fp64_matches_oracle_and_tangent(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    rng = np.random.default_rng(7)
    G = _sym(rng, p.N)
    g = _grad(cdmpt_lib, p, G, "fp64")
    ref = oracle.solve(p.H0, G, p.beta, p.nocc, n=p.n, kind="rec")["P1"][0]
    assert oracle.rel_frobenius(g, ref) < 1e-9
    # the forward response of the library in direction G is the same matrix
    with cdmpt_lib.Handle(precision="fp64") as h:
        h.set_H(p.H0, G[None])
        r = h.solve(p.beta, p.nocc, p.n)
    assert oracle.rel_frobenius(g, r["P1"][0].cpu().numpy()) < 1e-9


def test_adjoint_fp64_central_differences_20_directions(cuda, cdmpt_lib):
    """<grad, E> == (L(H0 + hE) - L(H0 - hE)) / 2h for 20 random symmetric E, h = 1e-4."""
    import torch
    p = syn.cubic_lattice((4, 4, 4), seed=5, beta=6.0, n=12)
    rng = np.random.default_rng(11)
    G = _sym(rng, p.N)
    g = _grad(cdmpt_lib, p, G, "fp64")
    h = 1e-4
    with cdmpt_lib.Handle(precision="fp64") as hd:
        def loss(H):
            hd.set_H(H, None)
            P0 = hd.solve(p.beta, p.nocc, p.n)["P0"].cpu().numpy()
            return float(np.sum(G * P0))
        errs = []
        for _ in range(20):
            E = _sym(rng, p.N, 0.1)
            fd = (loss(p.H0 + h * E) - loss(p.H0 - h * E)) / (2 * h)
            errs.append(abs(fd - np.sum(g * E)) / max(1e-12, abs(fd)))
    assert max(errs) < 1e-6, max(errs)


def test_fp64_differentiation_workload_central_differences(cuda, cdmpt_lib):
    """The differentiation workload in FP64 (16 x 16 x 8 lattice, N = 2048, beta = 20, n = 16,
    sqrt(n) checkpoints): the gradients of the polarizability alpha = -2 Tr(P1 H1) and of the
    free energy Omega, through torch.autograd, against central differences (h = 1e-4) along
    20 random symmetric directions, and the free-energy gradient against the oracle's P0
    (dOmega/dH0 = P0, App. B)."""
    import torch
    p = syn.workload("cubic16x16x8")
    dev = torch.device("cuda")
    H0 = torch.from_numpy(p.H0).to(dev)
    H1 = torch.from_numpy(p.H1).to(dev)
    rng = np.random.default_rng(17)
    h = 1e-4
    with cdmpt_lib.Handle(precision="fp64", ckpt_stride=-1) as hd:
        X = H0.clone().requires_grad_(True)
        a = cdmpt_lib.Polarizability.apply(X, H1, p.beta, p.nocc, p.n, hd)
        a.sum().backward()
        ga = X.grad.cpu().numpy()
        Y = H0.clone().requires_grad_(True)
        om = cdmpt_lib.FreeEnergy.apply(Y, p.beta, p.nocc, p.n, hd)
        om.backward()
        gw = Y.grad.cpu().numpy()

        def alpha(H):
            hd.set_H(H, p.H1)
            hd.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
            return float(np.sum(hd.polarizability()))

        def omega(H):
            hd.set_H(H, None)
            hd.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
            return hd.free_energy(want_grad=False)["omega"]

        ea, ew = [], []
        for _ in range(20):
            E = _sym(rng, p.N, 0.05)
            fa = (alpha(p.H0 + h * E) - alpha(p.H0 - h * E)) / (2 * h)
            fw = (omega(p.H0 + h * E) - omega(p.H0 - h * E)) / (2 * h)
            ea.append(abs(fa - np.sum(ga * E)) / max(1e-12, abs(fa)))
            ew.append(abs(fw - np.sum(gw * E)) / max(1e-12, abs(fw)))
    assert max(ea) < 1e-5, max(ea)
    assert max(ew) < 1e-6, max(ew)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    assert oracle.rel_frobenius(gw, ref["P0"]) < 1e-10


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_adjoint_float_lattice_2048(cuda, cdmpt_lib, precision):
    """The differentiation workload: 16 x 16 x 8 lattice (N = 2048), beta = 20, n = 16."""
    p = syn.workload("cubic16x16x8")
    rng = np.random.default_rng(3)
    G = np.diag(rng.standard_normal(p.N)) + _sym(rng, p.N, 0.01)
    g = _grad(cdmpt_lib, p, G, precision)
    ref = oracle.solve(p.H0, G, p.beta, p.nocc, n=p.n, kind="rec")["P1"][0]
    assert oracle.rel_frobenius(g, ref) < 1e-5


def test_density_matrix_autograd(cuda, cdmpt_lib):
    """torch.autograd through DensityMatrix: L = Tr(P0 G) + ||P0||_F^2."""
    import torch
    p = syn.cubic_lattice((5, 5, 5), seed=9, beta=8.0, n=12)
    rng = np.random.default_rng(5)
    G = _sym(rng, p.N)
    H = torch.from_numpy(p.H0).cuda().requires_grad_(True)
    with cdmpt_lib.Handle(precision="fp64") as h:
        P0 = cdmpt_lib.DensityMatrix.apply(H, p.beta, p.nocc, p.n, h)
        L = (P0 * torch.from_numpy(G).cuda()).sum() + (P0 * P0).sum()
        L.backward()
    P0n = P0.detach().cpu().numpy()
    Gtot = G + 2 * P0n      # dL/dP0
    ref = oracle.solve(p.H0, Gtot, p.beta, p.nocc, n=p.n, kind="rec")["P1"][0]
    assert oracle.rel_frobenius(H.grad.cpu().numpy(), ref) < 1e-9


def test_adjoint_requires_a_solve(cuda, cdmpt_lib):
    import torch
    with cdmpt_lib.Handle(precision="fp64") as h:
        with pytest.raises(cdmpt_lib.CdmptError) as e:
            h.vjp_P0(torch.zeros((4, 4), dtype=torch.float64, device="cuda"))
        assert e.value.status == 1
