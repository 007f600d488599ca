"""GPU tests of failure detection without a GPU fault.

Every mbarrier wait of the tcgen05 kernels is bounded: after its time limit the waiting thread
records a code in the library's device error word, the kernel returns (copies drained, tensor
memory freed) and the next status check reports CDMPT_ERR_TIMEOUT. cdmpt_check_bounded_wait runs
that same bounded wait, with a limit of a few milliseconds, on a barrier that nothing arrives on
and with nothing in flight, so the wait runs out by construction. The tests check the status,
that the error word is cleared, and that ordinary work afterwards still matches the oracle.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

ERR_TIMEOUT = 5


def test_bounded_wait_gives_up_with_timeout_status(cuda, cdmpt_lib):
    import time
    t0 = time.perf_counter()
    st = cdmpt_lib.check_bounded_wait(2.0)
    assert st == ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0          # the limit, not an endless wait
    assert cdmpt_lib.check_bounded_wait(1.0) == ERR_TIMEOUT   # repeatable


def test_bounded_wait_rejects_bad_limits(cuda, cdmpt_lib):
    assert cdmpt_lib.check_bounded_wait(0.0) == 1      # ERR_ARG
    assert cdmpt_lib.check_bounded_wait(5000.0) == 1


def test_solve_after_timeout_still_matches_oracle(cuda, cdmpt_lib):
    """The error word is cleared by the status check: a following tensor-core solve and the
    batch both succeed and match the oracle."""
    assert cdmpt_lib.check_bounded_wait(2.0) == ERR_TIMEOUT
    p = syn.cubic_lattice((8, 8, 8), seed=1002, beta=20.0, n=14)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    with cdmpt_lib.Handle(precision="mixed") as h:
        h.set_H(p.H0, p.H1)
        r = h.solve(p.beta, p.nocc, p.n)
    assert oracle.rel_frobenius(r["P0"].cpu().numpy(), ref["P0"]) < 1e-6
    assert oracle.rel_frobenius(r["P1"][0].cpu().numpy(), ref["P1"][0]) < 1e-6
    cl = syn.clusters(B=2, seed=7007, sizes=[130, 260], n=12)
    bt = cdmpt_lib.Batch([c.N for c in cl], 3)
    bt.set_H([c.H0 for c in cl], [c.H1 for c in cl], 12)
    rb = bt.solve([c.beta for c in cl], [c.nocc for c in cl], 12)
    bt.close()
    for i, c in enumerate(cl):
        rc = oracle.solve(c.H0, c.H1, c.beta, c.nocc, n=12, kind="rec")
        assert oracle.rel_frobenius(rb["P0"][i].cpu().numpy(), rc["P0"]) < 1e-5
