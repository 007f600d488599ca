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
