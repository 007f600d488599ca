"""GPU tests of the block-sparse screened products (opts.screen_tau; Sec. VI, Fig. 3).

Every product X Y^T of a screened solve drops the k-slice terms X_IK Y_JK^T of 128 x 32 tiles
whose Frobenius norms satisfy ||X_IK|| ||Y_JK|| <= screen_tau (a per-tile slice mask built
before each launch; the tcgen05 kernel skips the masked slices in all its roles).

References and bars:
- Decoupled chains (block-diagonal H0 and H1): every dropped term is an exact zero, so the
  screened P0 and P1 keep the exact zero pattern of the blocks and agree with the dense ones
  within the precision's bar (the two run different tile shapes, so the CG scalars differ in
  their last bits).
- The 1D chain (N = 1024, beta 10, n 12) against the oracle: at tau = 1e-8 the screened
  error stays within 1.5 x the dense error + 50 tau and within the precision's bar (the
  dense mixed-precision P1 error is near 1.4e-7, the screened one near 4.3e-7: the
  screening's own error, 12 to 30 tau, is what shows); at tau = 1e-6 and
  1e-5 the relative P1 error stays below 10 tau + 2e-6 and the alpha error below tau (the
  measured errors are 6.4 tau and 2.3 tau for P1, 0.15 tau and 0.05 tau for alpha).
- The computed slices grow linearly with N on the chain (the nearsightedness behind Fig. 3):
  doubling N multiplies the work by 1.5 to 3 (dense work grows 8x).
- The derivatives (second order, adjoint, free energy) at tau = 1e-8 against the oracle at
  the FP32 bar 1e-5.
"""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


def _solve(pkg, p, precision, tau):
    with pkg.Handle(precision=precision, screen_tau=tau) as h:
        h.set_H(p.H0, p.H1)
        r = h.solve(p.beta, p.nocc, p.n)
        st = h.stats()
        return {"P0": r["P0"].cpu().numpy(), "P1": r["P1"][0].cpu().numpy(),
                "alpha": h.polarizability()[0], "computed": st["screen_slices_computed"],
                "examined": st["screen_slices_examined"]}


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("sizes", [(128, 128, 128, 128), (100, 156, 200, 54)])
def test_screening_is_exact_on_decoupled_chains(cuda, cdmpt_lib, precision, sizes):
    """Block-diagonal chains: every screened term is an exact zero. The second block layout is
    not aligned to the 128 x 128 tiles and N = 510 is not a multiple of 4: the tiles screened to
    nothing then include partial edge tiles, whose epilogue masks the elements outside the
    matrix, next to full ones (and the transposed placement of the response's right-hand
    side).

    The screened products run on the one-SM 128 x 128 kernels (the mask's granularity), the
    dense ones with more than 128 rows on the two-SM 256 x 256 kernels. Both form every product
    element by the same accumulation, but the fused CG dot products add the same float
    partial sums in other double groupings, so the CG scalars differ in their last bits and
    the iterates in rounding. The check is therefore the exact zero pattern of the blocks in
    both solves and agreement within the precision's bar (1e-5 FP32, 1e-6 mixed)."""
    blocks = [syn.chain_1d(nb, 11 + i, 10.0, 12) for i, nb in enumerate(sizes)]
    H0 = sl.block_diag(*[b.H0 for b in blocks])
    H1 = sl.block_diag(*[b.H1[0] for b in blocks])[None]
    p = syn.Problem("four_chains", H0, H1, sum(b.nocc for b in blocks), 10.0, 12)
    dense = _solve(cdmpt_lib, p, precision, 0.0)
    scr = _solve(cdmpt_lib, p, precision, 1e-30)
    off = sl.block_diag(*[np.ones((nb, nb)) for nb in sizes]) == 0
    bar = 1e-5 if precision == "fp32" else 1e-6
    for k in ("P0", "P1"):
        assert not dense[k][off].any() and not scr[k][off].any(), k
        assert oracle.rel_frobenius(scr[k], dense[k]) < bar, k
    assert dense["examined"] == 0.0
    assert 0.0 < scr["computed"] < (0.1 if sizes[0] == 128 else 0.5) * scr["examined"]


@pytest.fixture(scope="module")
def chain1024():
    p = syn.chain_1d(1024, 1001, 10.0, 12)
    return p, oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_screening_at_1e8_keeps_the_dense_accuracy(cuda, cdmpt_lib, chain1024, precision):
    p, ref = chain1024
    dense = _solve(cdmpt_lib, p, precision, 0.0)
    scr = _solve(cdmpt_lib, p, precision, 1e-8)
    for k, r in (("P0", ref["P0"]), ("P1", ref["P1"][0])):
        e_d = oracle.rel_frobenius(dense[k], r)
        e_s = oracle.rel_frobenius(scr[k], r)
        assert e_s <= 1.5 * e_d + 50 * 1e-8, (k, e_s, e_d)
        assert e_s < (1e-5 if precision == "fp32" else 1e-6), (k, e_s)
    assert scr["computed"] < 0.05 * scr["examined"]


@pytest.mark.parametrize("tau", [1e-6, 1e-5])
def test_screening_error_follows_tau(cuda, cdmpt_lib, chain1024, tau):
    p, ref = chain1024
    scr = _solve(cdmpt_lib, p, "fp32", tau)
    assert oracle.rel_frobenius(scr["P1"], ref["P1"][0]) < 10 * tau + 2e-6
    assert abs(scr["alpha"] - ref["alpha"][0]) < tau * abs(ref["alpha"][0])


def test_screened_work_grows_linearly_on_the_chain(cuda, cdmpt_lib):
    work = [_solve(cdmpt_lib, syn.chain_1d(N, 1001, 10.0, 12), "fp32", 1e-8)["computed"]
            for N in (1024, 2048)]
    assert 1.5 <= work[1] / work[0] < 3.0, work


def test_screened_derivatives_fp32(cuda, cdmpt_lib):
    import torch
    p = syn.chain_1d(512, 1001, 10.0, 12)
    ref = oracle.response2(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    reff = oracle.free_energy(p.H0, p.beta, p.nocc, n=p.n, kind="rec")
    G = np.diag(np.linspace(-1.0, 1.0, p.N))
    refg = oracle.solve(p.H0, G, p.beta, p.nocc, n=p.n, kind="rec")["P1"][0]
    with cdmpt_lib.Handle(precision="fp32", screen_tau=1e-8) as h:
        h.set_H(p.H0, p.H1)
        h.solve(p.beta, p.nocc, p.n, want_P0=False, want_P1=False)
        r2 = h.response2()
        g = h.vjp_P0(torch.from_numpy(G).cuda()).cpu().numpy()
        fe = h.free_energy()
    assert oracle.rel_frobenius(r2["P2"][0].cpu().numpy(), ref["P2"][0]) < 1e-5
    assert oracle.rel_frobenius(r2["grad"].cpu().numpy(), ref["grad_alpha"][0]) < 1e-5
    assert oracle.rel_frobenius(g, refg) < 1e-5
    assert abs(fe["omega"] - reff["omega"]) < 1e-6 * abs(reff["omega"])
    assert oracle.rel_frobenius(fe["grad"].cpu().numpy(), reff["grad"]) < 1e-5
