"""GPU parity of the batched solve (grouped tcgen05 launches) against the oracle.

Uneven cluster sizes (several 128 x 128 tiles with ragged tails), three dipole
directions each, FP32 with split-TF32 products: bar 1e-5 per system.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


def test_batch_clusters_match_oracle(cuda, cdmpt_lib):
    probs = syn.clusters(B=5, seed=2005, sizes=[128, 200, 333, 96, 257], n=12)
    b = cdmpt_lib.Batch([p.N for p in probs], 3)
    b.set_H([p.H0 for p in probs], [p.H1 for p in probs], 12)
    r = b.solve([p.beta for p in probs], [p.nocc for p in probs], 12)
    for i, p in enumerate(probs):
        ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
        e0 = oracle.rel_frobenius(r["P0"][i].cpu().numpy(), ref["P0"])
        assert e0 < 1e-5, (i, e0)
        assert abs(r["mu"][i] - ref["mu"]) < 1e-5
        for d in range(3):
            e1 = oracle.rel_frobenius(r["P1"][i][d].cpu().numpy(), ref["P1"][d])
            assert e1 < 1e-5, (i, d, e1)
            assert abs(r["alpha"][i, d] - ref["alpha"][d]) < 1e-4 * abs(ref["alpha"][d])
    b.close()


def test_batch_matches_single_solves(cuda, cdmpt_lib):
    """Each system of a batch equals its own single-system FP32 solve."""
    probs = syn.clusters(B=3, seed=3005, sizes=[160, 300, 130], n=12)
    b = cdmpt_lib.Batch([p.N for p in probs], 3)
    b.set_H([p.H0 for p in probs], [p.H1 for p in probs], 12)
    r = b.solve([p.beta for p in probs], [p.nocc for p in probs], 12)
    for i, p in enumerate(probs):
        with cdmpt_lib.Handle(precision="fp32") as h:
            h.set_H(p.H0, p.H1)
            s = h.solve(p.beta, p.nocc, p.n)
        assert oracle.rel_frobenius(r["P0"][i].cpu().numpy(), s["P0"].cpu().numpy()) < 1e-5
    b.close()


def test_batch_tuner_and_graph(cuda, cdmpt_lib):
    """The tile autotuner picks one of its candidates after timing both; CG iterations
    replay a CUDA graph; each fixed tile width and the graph-free path give the same
    solution (tile width and capture change no arithmetic)."""
    import os
    probs = syn.clusters(B=6, seed=4005, sizes=[128, 700, 250, 96, 513, 1100], n=12)
    args = ([p.beta for p in probs], [p.nocc for p in probs], 12)

    def run(env):
        old = {k: os.environ.get(k) for k in env}
        os.environ.update(env)
        try:
            b = cdmpt_lib.Batch([p.N for p in probs], 3)
            b.set_H([p.H0 for p in probs], [p.H1 for p in probs], 12)
            r = b.solve(*args)
            t = b.tuning()
            b.close()
        finally:
            for k, v in old.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        return r, t

    r, t = run({})
    assert t["tile_n"] in (64, 128, 256)
    assert t["ms_128"] > 0 and t["ms_64"] > 0 and t["ms_256"] > 0
    assert t["graphs"]
    for env in ({"CDMPT_BATCH_TILE": "64"}, {"CDMPT_BATCH_TILE": "128"},
                {"CDMPT_BATCH_TILE": "256"}, {"CDMPT_BATCH_GRAPH": "0"}):
        r2, t2 = run(env)
        if "CDMPT_BATCH_TILE" in env:
            assert t2["tile_n"] == int(env["CDMPT_BATCH_TILE"])
        else:
            assert not t2["graphs"]
        for i in range(len(probs)):
            assert oracle.rel_frobenius(r2["P0"][i].cpu().numpy(), r["P0"][i].cpu().numpy()) < 1e-6
            for d in range(3):
                assert oracle.rel_frobenius(r2["P1"][i][d].cpu().numpy(),
                                            r["P1"][i][d].cpu().numpy()) < 1e-5
    ref = oracle.solve(probs[5].H0, probs[5].H1, probs[5].beta, probs[5].nocc, n=12, kind="rec")
    assert oracle.rel_frobenius(r["P0"][5].cpu().numpy(), ref["P0"]) < 1e-5


def test_batch_mixed_precision_matches_oracle(cuda, cdmpt_lib):
    """CDMPT_MIXED_TF32 batches: one-pass TF32 sweeps, pair-stored trajectories refined with
    split-TF32 residuals and then Ozaki-sliced (FP64-class) residuals on the late steps,
    per-system Newton steps on mu, split-TF32 response; every system's P0, P1 (three
    directions), mu1 and alpha against the oracle at the mixed bar 1e-6 (mu1 on the scale of
    the dipole diagonal, i.e. absolute for |mu1| < 1). These clusters have levels within
    0.03 - 0.6 kT of mu, where P1 is most sensitive to the trajectory."""
    probs = syn.clusters(B=5, seed=5005, sizes=[128, 420, 333, 96, 700], n=12)
    b = cdmpt_lib.Batch([p.N for p in probs], 3, precision="mixed")
    b.set_H([p.H0 for p in probs], [p.H1 for p in probs], 12)
    r = b.solve([p.beta for p in probs], [p.nocc for p in probs], 12)
    st = b.stats()
    assert st["cg_iterations_refine"] > 0 and st["fp64_residual_passes"] > 0
    for i, p in enumerate(probs):
        ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
        e0 = oracle.rel_frobenius(r["P0"][i].cpu().numpy(), ref["P0"])
        assert e0 < 1e-6, (i, e0)
        for d in range(3):
            e1 = oracle.rel_frobenius(r["P1"][i][d].cpu().numpy(), ref["P1"][d])
            assert e1 < 1e-6, (i, d, e1)
            em = abs(float(r["mu1"][i][d]) - ref["mu1"][d]) / max(abs(ref["mu1"][d]), 1.0)
            assert em < 1e-6, (i, d, em)
            ea = abs(float(r["alpha"][i][d]) - ref["alpha"][d]) / abs(ref["alpha"][d])
            assert ea < 1e-6, (i, d, ea)
    b.close()


@pytest.mark.parametrize("precision,bar", [("mixed", 1e-6), ("fp32", 1e-5)])
def test_batch_largest_cluster_sizes(cuda, cdmpt_lib, precision, bar):
    """The top of the batched workload's size range (N_b up to 1536, the largest size the
    96-cluster draw allows) next to small ragged systems: every system's P0 and P1 (three
    directions) against the oracle at the precision's bar."""
    probs = syn.clusters(B=4, seed=7005, sizes=[1536, 1031, 777, 128], n=12)
    b = cdmpt_lib.Batch([p.N for p in probs], 3, precision=precision)
    b.set_H([p.H0 for p in probs], [p.H1 for p in probs], 12)
    r = b.solve([p.beta for p in probs], [p.nocc for p in probs], 12)
    for i, p in enumerate(probs):
        ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
        e0 = oracle.rel_frobenius(r["P0"][i].cpu().numpy(), ref["P0"])
        assert e0 < bar, (i, e0)
        for d in range(3):
            e1 = oracle.rel_frobenius(r["P1"][i][d].cpu().numpy(), ref["P1"][d])
            assert e1 < bar, (i, d, e1)
    b.close()
