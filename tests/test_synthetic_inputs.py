"""CPU checks of the seeded synthetic inputs: the properties their docstrings promise."""
import numpy as np

import synthetic as syn


def test_inputs_are_deterministic_in_their_seed():
    a = syn.nonorthogonal_cluster(60, seed=5)
    b = syn.nonorthogonal_cluster(60, seed=5)
    c = syn.nonorthogonal_cluster(60, seed=6)
    assert np.array_equal(a.H0, b.H0) and np.array_equal(a.meta["S"], b.meta["S"])
    assert not np.array_equal(a.H0, c.H0)
    assert np.array_equal(syn.workload("chain64").H0, syn.workload("chain64").H0)


def test_nonorthogonal_cluster_overlap_and_kernel():
    """S = (1 - s0) I + s0 G with a Gaussian kernel G: symmetric, unit diagonal, eigenvalues
    >= 1 - s0; gamma positive semidefinite; F, the dipoles and gamma symmetric."""
    s0 = 0.3
    p = syn.nonorthogonal_cluster(120, seed=7, s0=s0)
    S, gamma = p.meta["S"], p.meta["gamma"]
    assert np.array_equal(S, S.T) and np.allclose(np.diag(S), 1.0)
    assert np.linalg.eigvalsh(S).min() >= 1.0 - s0 - 1e-12
    assert np.linalg.eigvalsh(gamma).min() >= -1e-12
    assert np.array_equal(p.H0, p.H0.T)
    for d in range(3):
        assert np.allclose(p.H1[d], p.H1[d].T)
    assert p.nocc == 60.0 and np.allclose(p.meta["q0"], 1.0)


def test_lattice_and_cluster_shapes():
    p = syn.cubic_lattice((4, 5, 6), seed=1)
    assert p.H0.shape == (120, 120) and p.H1.shape == (1, 120, 120)
    assert np.array_equal(p.H0, p.H0.T)
    # six nearest neighbours per site on the periodic lattice
    assert np.all(np.count_nonzero(p.H0 - np.diag(np.diag(p.H0)), axis=1) == 6)
    cl = syn.clusters(B=3, seed=11, sizes=[10, 20, 30])
    assert [q.N for q in cl] == [10, 20, 30] and all(q.D == 3 for q in cl)
