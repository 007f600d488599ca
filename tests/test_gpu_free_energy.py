"""GPU tests of the free energy Omega(H0) = Tr[P0 H0] - T_e S[P0] and its gradient.

cdmpt_free_energy evaluates Eqs. (FreeE), (SED) for the recursion's own P0
without eigenvalues (telescoped log-determinants of I - Z_0 and of the step
matrices, plus a series for atanh(Z_0) - Z_0), and dOmega/dH0 as P0 plus one
adjoint sweep. References: the oracle's free energy (eigenvalues of H0, the
n-step occupation function, the binary entropy per level) and its closed-form
gradient, pinned on the CPU by central differences; on the GPU also central
differences of the library's own FP64 Omega. Bars: 1e-10 (FP64) for Omega and
the gradient; 1e-6 for Omega and 1e-5 for the gradient in FP32 and mixed.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


def _fe(pkg, p, precision, **kw):
    with pkg.Handle(precision=precision, **kw) as h:
        h.set_H(p.H0, None)
        h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
        r = h.free_energy()
    return r["omega"], r["grad"].cpu().numpy()


def test_free_energy_fp64_chain64(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    ref = oracle.free_energy(p.H0, p.beta, p.nocc, n=p.n, kind="rec")
    om, g = _fe(cdmpt_lib, p, "fp64")
    assert abs(om - ref["omega"]) < 1e-10 * abs(ref["omega"])
    assert oracle.rel_frobenius(g, ref["grad"]) < 1e-10


@pytest.mark.parametrize("beta", [5.0, 20.0, 80.0])
def test_free_energy_fp64_lattice(cuda, cdmpt_lib, beta):
    p = syn.cubic_lattice((6, 6, 6), seed=61, beta=beta, n=14)
    ref = oracle.free_energy(p.H0, p.beta, p.nocc, n=p.n, kind="rec")
    om, g = _fe(cdmpt_lib, p, "fp64")
    assert abs(om - ref["omega"]) < 1e-10 * abs(ref["omega"])
    assert oracle.rel_frobenius(g, ref["grad"]) < 1e-10


def test_free_energy_fp64_grand_canonical(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    mu = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")["mu"] + 0.05
    ref = oracle.free_energy(p.H0, p.beta, p.nocc, n=p.n, kind="rec", canonical=False, mu=mu)
    om, g = _fe(cdmpt_lib, p, "fp64", mu_guess=mu, grand_canonical=True)
    assert abs(om - ref["omega"]) < 1e-10 * abs(ref["omega"])
    assert oracle.rel_frobenius(g, ref["grad"]) < 1e-10


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_free_energy_float_lattice_512(cuda, cdmpt_lib, precision):
    p = syn.cubic_lattice((8, 8, 8), seed=1002, beta=20.0, n=14)
    ref = oracle.free_energy(p.H0, p.beta, p.nocc, n=p.n, kind="rec")
    om, g = _fe(cdmpt_lib, p, precision)
    assert abs(om - ref["omega"]) < 1e-6 * abs(ref["omega"])
    assert oracle.rel_frobenius(g, ref["grad"]) < 1e-5


def test_free_energy_differentiation_workload_fp32_checkpointed(cuda, cdmpt_lib):
    """16 x 16 x 8 lattice (N = 2048), beta 20, n = 16, FP32 with sqrt(n) checkpoints."""
    p = syn.workload("cubic16x16x8")
    ref = oracle.free_energy(p.H0, p.beta, p.nocc, n=p.n, kind="rec")
    om, g = _fe(cdmpt_lib, p, "fp32", ckpt_stride="sqrt")
    assert abs(om - ref["omega"]) < 1e-6 * abs(ref["omega"])
    assert oracle.rel_frobenius(g, ref["grad"]) < 1e-5


def test_free_energy_gradient_central_differences_fp64(cuda, cdmpt_lib):
    """<dOmega/dH0, E> == (Omega(H0 + hE) - Omega(H0 - hE)) / 2h, 10 random symmetric E,
    Omega from the library's own FP64 free energy."""
    p = syn.cubic_lattice((4, 4, 4), seed=62, beta=6.0, n=12)
    _, g = _fe(cdmpt_lib, p, "fp64")
    rng = np.random.default_rng(17)
    h = 1e-4
    errs = []
    with cdmpt_lib.Handle(precision="fp64") as hd:
        def omega(H):
            hd.set_H(H, None)
            hd.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
            return hd.free_energy(want_grad=False)["omega"]
        for _ in range(10):
            A = rng.standard_normal((p.N, p.N)) * 0.1
            E = 0.5 * (A + A.T)
            fd = (omega(p.H0 + h * E) - omega(p.H0 - h * E)) / (2 * h)
            errs.append(abs(fd - np.sum(g * E)) / max(1e-12, abs(fd)))
    assert max(errs) < 1e-6, max(errs)


def test_free_energy_autograd(cuda, cdmpt_lib):
    """torch.autograd through FreeEnergy: L = Omega^2."""
    import torch
    p = syn.cubic_lattice((5, 5, 5), seed=63, beta=8.0, n=12)
    ref = oracle.free_energy(p.H0, p.beta, p.nocc, n=p.n, kind="rec")
    H = torch.from_numpy(p.H0).cuda().requires_grad_(True)
    with cdmpt_lib.Handle(precision="fp64") as h:
        om = cdmpt_lib.FreeEnergy.apply(H, p.beta, p.nocc, p.n, h)
        (om ** 2).backward()
    assert abs(float(om.detach()) - ref["omega"]) < 1e-10 * abs(ref["omega"])
    assert oracle.rel_frobenius(H.grad.cpu().numpy(), 2 * ref["omega"] * ref["grad"]) < 1e-9


def test_free_energy_requires_a_solve(cuda, cdmpt_lib):
    with cdmpt_lib.Handle(precision="fp64") as h:
        with pytest.raises(cdmpt_lib.CdmptError):
            h.free_energy()
