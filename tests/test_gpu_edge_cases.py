"""GPU edge cases: the smallest systems, sizes one past a tile boundary, extreme
temperatures, and a batch that mixes tiny and ragged systems.

References: the FP64 oracle (recursion-exact function). Bars as elsewhere: 1e-10
(FP64), 1e-5 (FP32 and mixed). For N = 1 the canonical response vanishes
exactly (Tr P1 = P1 = 0, mu1 = the perturbation itself).
"""
import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

BAR = {"fp64": 1e-10, "fp32": 1e-5, "mixed": 1e-5}


def _tiny(N, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((N, N)) * 0.5
    H0 = 0.5 * (A + A.T)
    B = rng.standard_normal((N, N)) * 0.2
    H1 = (0.5 * (B + B.T))[None]
    return syn.Problem(f"tiny{N}", H0, H1, nocc=N / 2.0, beta=4.0, n=8)


def _run(pkg, p, precision):
    with pkg.Handle(precision=precision) as h:
        h.set_H(p.H0, p.H1)
        r = h.solve(p.beta, p.nocc, p.n)
        return {"P0": r["P0"].cpu().numpy(), "P1": r["P1"].cpu().numpy(), "mu": r["mu"],
                "mu1": r["mu1"]}


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_single_level(cuda, cdmpt_lib, precision):
    """N = 1, half occupied: mu = H0, P0 = 1/2, and the canonical response is zero with
    mu1 = H1."""
    p = syn.Problem("one", np.array([[0.3]]), np.array([[[0.7]]]), nocc=0.5, beta=4.0, n=8)
    r = _run(cdmpt_lib, p, precision)
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert abs(r["mu"] - 0.3) < tol
    assert abs(r["P0"][0, 0] - 0.5) < tol
    assert abs(r["P1"][0, 0, 0]) < tol
    assert abs(r["mu1"][0] - 0.7) < tol


@pytest.mark.parametrize("N", [2, 3, 5])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_few_levels(cuda, cdmpt_lib, N, precision):
    p = _tiny(N, 100 + N)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    r = _run(cdmpt_lib, p, precision)
    assert oracle.rel_frobenius(r["P0"], ref["P0"]) < BAR[precision]
    assert oracle.rel_frobenius(r["P1"][0], ref["P1"][0]) < 10 * BAR[precision]


@pytest.mark.parametrize("N", [129, 257])
@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_one_past_a_tile_boundary(cuda, cdmpt_lib, N, precision):
    """128-wide tcgen05 tiles with a one-row, one-column tail."""
    p = syn.chain_1d(N, seed=N, beta=10.0, n=12)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    r = _run(cdmpt_lib, p, precision)
    assert oracle.rel_frobenius(r["P0"], ref["P0"]) < BAR[precision]
    assert oracle.rel_frobenius(r["P1"][0], ref["P1"][0]) < BAR[precision]


@pytest.mark.parametrize("beta,n", [(0.05, 4), (400.0, 18)])
def test_extreme_temperatures_fp64(cuda, cdmpt_lib, beta, n):
    """Almost uniform occupation (beta 0.05, four steps) and almost a projector (beta 400)."""
    p = syn.cubic_lattice((4, 4, 4), seed=7, beta=beta, n=n)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    r = _run(cdmpt_lib, p, "fp64")
    assert oracle.rel_frobenius(r["P0"], ref["P0"]) < 1e-10
    assert oracle.rel_frobenius(r["P1"][0], ref["P1"][0]) < 1e-9


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_batch_with_tiny_and_ragged_systems(cuda, cdmpt_lib, precision):
    """Sizes 1, 3, 33, 129 and 300 in one lockstep batch."""
    sizes = [1, 3, 33, 129, 300]
    probs = []
    for i, N in enumerate(sizes):
        q = _tiny(N, 200 + i)
        q.H1 = np.concatenate([q.H1, q.H1, q.H1]) * np.array([1.0, 0.5, -1.0])[:, None, None]
        q.beta, q.n = 10.0, 12
        probs.append(q)
    bt = cdmpt_lib.Batch(sizes, 3, precision=precision)
    try:
        bt.set_H([q.H0 for q in probs], [q.H1 for q in probs], 12)
        rb = bt.solve([q.beta for q in probs], [q.nocc for q in probs], 12)
    finally:
        bt.close()
    for i, q in enumerate(probs):
        ref = oracle.solve(q.H0, q.H1, q.beta, q.nocc, n=q.n, kind="rec")
        assert oracle.rel_frobenius(rb["P0"][i].cpu().numpy(), ref["P0"]) < 1e-5, i
        for d in range(3):
            e = oracle.rel_frobenius(rb["P1"][i][d].cpu().numpy(), ref["P1"][d])
            assert e < (1e-5 if q.N > 1 else 1e-6) or np.abs(ref["P1"][d]).max() < 1e-12, (i, d, e)
