"""GPU parity of the full canonical solve (C ABI) against the FP64 oracle.

Parity reference: the oracle's recursion-exact function (kind="rec", same n).
Bars (relative Frobenius norm): 1e-10 for FP64, 1e-5 for FP32, 1e-6 for mixed
precision after refinement, on every workload (mu1 and alpha within ten times the bar).
The gap of the recursion to the exact Fermi-Dirac function is reported separately.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

BAR = {"fp64": 1e-10, "fp32": 1e-5, "mixed": 1e-6}


def _rel(a, b):
    return oracle.rel_frobenius(a, b)


def _run(pkg, prob, precision, engine="auto", device="cuda", **kw):
    with pkg.Handle(precision=precision, engine=engine, **kw) as h:
        h.set_H(prob.H0, prob.H1)
        r = h.solve(prob.beta, prob.nocc, prob.n, device=device)
        r["alpha"] = h.polarizability()
        r["stats"] = h.stats()
    r["P0"] = r["P0"].cpu().numpy()
    r["P1"] = None if r["P1"] is None else r["P1"].cpu().numpy()
    return r


def _check(r, ref, bar, D):
    e0 = _rel(r["P0"], ref["P0"])
    assert e0 < bar, f"P0 error {e0:.3e}"
    assert abs(r["mu"] - ref["mu"]) < max(bar, 1e-12) * max(1.0, abs(ref["mu"])) * 10
    for d in range(D):
        e1 = _rel(r["P1"][d], ref["P1"][d])
        assert e1 < bar, f"P1[{d}] error {e1:.3e}"
        assert abs(r["mu1"][d] - ref["mu1"][d]) < 10 * bar * max(1.0, abs(ref["mu1"][d]))
        assert abs(r["alpha"][d] - ref["alpha"][d]) < 10 * bar * abs(ref["alpha"][d])
    return e0


def test_fp64_chain64(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    r = _run(cdmpt_lib, p, "fp64")
    _check(r, ref, BAR["fp64"], p.D)
    # the recursion's own truncation gap to Fermi-Dirac is what the oracle predicts
    fd = oracle.solve(p.H0, p.H1, p.beta, p.nocc, kind="fd")
    gap_gpu = _rel(r["P0"], fd["P0"])
    gap_oracle = _rel(ref["P0"], fd["P0"])
    assert abs(gap_gpu - gap_oracle) < 1e-3 * gap_oracle + 1e-12


def test_fp64_lattice_three_directions(cuda, cdmpt_lib):
    p = syn.cubic_lattice((8, 8, 8), seed=1002, beta=20.0, n=14, directions="xyz")
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    r = _run(cdmpt_lib, p, "fp64")
    _check(r, ref, BAR["fp64"], 3)
    assert np.all(np.abs(np.trace(r["P1"], axis1=1, axis2=2)) < 1e-9)


@pytest.mark.parametrize("engine", ["3xtf32", "simt"])
def test_fp32_lattice_1000(cuda, cdmpt_lib, engine):
    p = syn.cubic_lattice((10, 10, 10), seed=1002, beta=20.0, n=14)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    r = _run(cdmpt_lib, p, "fp32", engine=engine)
    _check(r, ref, BAR["fp32"], 1)


@pytest.mark.parametrize("beta", [5.0, 20.0])
def test_mixed_lattice_1000(cuda, cdmpt_lib, beta):
    """TF32 sweeps + split-TF32 refinement of the trajectory + split-TF32 response."""
    p = syn.cubic_lattice((10, 10, 10), seed=1002, beta=beta, n=14, directions="xy")
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    r = _run(cdmpt_lib, p, "mixed")
    _check(r, ref, BAR["mixed"], 2)
    assert r["stats"]["cg_iterations_refine"] > 0 and r["stats"]["fp64_residual_passes"] > 0


@pytest.mark.parametrize("beta", [5.0, 20.0])
def test_mixed_bf16_lattice_1000(cuda, cdmpt_lib, beta):
    """BF16 occupation sweeps + split-TF32 refinement reach the mixed bar (N = 1000)."""
    p = syn.cubic_lattice((10, 10, 10), seed=7, beta=beta, n=14)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    r = _run(cdmpt_lib, p, "mixed_bf16")
    _check(r, ref, BAR["mixed"], 1)
    assert r["stats"]["cg_iterations_refine"] > 0


def test_mixed_bf16_cubic16_full_size(cuda, cdmpt_lib):
    """MIXED_BF16 on the measured workload at beta = 20 (N = 4096, n = 14)."""
    p = syn.cubic_lattice((16, 16, 16), seed=1002, beta=20.0, n=14)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", eig=_eig_cubic16())
    _check(_run(cdmpt_lib, p, "mixed_bf16"), ref, BAR["mixed"], 1)


def test_mixed_small_system(cuda, cdmpt_lib):
    """Mixed precision on a small cluster (N = 96) whose levels lie within 0.14 kT of mu, where
    P1 is most sensitive to the trajectory and to mu: FP32 with split products gives 2e-6 to
    5.5e-6 here, and a trajectory stored in FP32 left mixed precision there too. The
    pair-stored trajectory with FP64-class residuals holds every output to the mixed bar."""
    p = syn.clusters(B=1, seed=6006, sizes=[96], beta=20.0, n=12)[0]
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    _check(_run(cdmpt_lib, p, "mixed"), ref, BAR["mixed"], p.H1.shape[0])


def test_tf32_single_pass_is_coarse(cuda, cdmpt_lib):
    """One TF32 pass per product (no refinement) lands near 1e-4, far from the FP32 bar."""
    p = syn.cubic_lattice((10, 10, 10), seed=1002, beta=20.0, n=14)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    r = _run(cdmpt_lib, p, "fp32", engine="tf32", occ_tol=1e-4 * p.N)
    e0 = _rel(r["P0"], ref["P0"])
    assert 1e-7 < e0 < 5e-3


@pytest.mark.parametrize("beta", [5.0, 20.0, 80.0])
def test_fp32_cubic16_full_size(cuda, cdmpt_lib, beta):
    """The measured workload: 16^3 lattice, N = 4096, n = 14, FP32, at each temperature."""
    p = syn.cubic_lattice((16, 16, 16), seed=1002, beta=beta, n=14)
    eig = _eig_cubic16()
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", eig=eig)
    r = _run(cdmpt_lib, p, "fp32")
    _check(r, ref, BAR["fp32"], 1)


@pytest.mark.parametrize("beta", [5.0, 20.0, 80.0])
def test_fp64_cubic16_full_size(cuda, cdmpt_lib, beta):
    """FP64 on the measured lattice (16^3, N = 4096, n = 14) at each temperature against the
    1e-10 bar. The products run on the tensor cores (seven-digit Ozaki engine, the FP64
    default on sm_103), which the statistics must show."""
    p = syn.cubic_lattice((16, 16, 16), seed=1002, beta=beta, n=14)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", eig=_eig_cubic16())
    r = _run(cdmpt_lib, p, "fp64", profile=True)
    _check(r, ref, BAR["fp64"], 1)
    assert r["stats"]["engine_launches"][5] > 0 and r["stats"]["engine_launches"][1] == 0


@pytest.mark.parametrize("beta,bar", [(5.0, 1e-6), (20.0, 1e-6), (80.0, 1e-6)])
def test_mixed_cubic16_full_size(cuda, cdmpt_lib, beta, bar):
    """Mixed precision on the measured workload (N = 4096, n = 14)."""
    p = syn.cubic_lattice((16, 16, 16), seed=1002, beta=beta, n=14)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", eig=_eig_cubic16())
    r = _run(cdmpt_lib, p, "mixed")
    _check(r, ref, bar, 1)


@pytest.mark.parametrize("name,mixed_bar", [("cubic20_b20", 1e-6), ("banded8192", 1e-6)])
def test_large_mixed_and_fp32(cuda, cdmpt_lib, name, mixed_bar):
    """The large workloads: 20^3 lattice (N = 8000) and N = 8192 banded, beta = 20, n = 14.
    Mixed precision against its bar and FP32 against the FP32 bar, one oracle solve each."""
    p = syn.workload(name)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    _check(_run(cdmpt_lib, p, "mixed"), ref, mixed_bar, 1)
    _check(_run(cdmpt_lib, p, "fp32"), ref, BAR["fp32"], 1)


_EIG = {}


def _eig_cubic16():
    if "c16" not in _EIG:
        p = syn.cubic_lattice((16, 16, 16), seed=1002)
        _EIG["c16"] = np.linalg.eigh(p.H0)
    return _EIG["c16"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ragged_size_no_perturbation(cuda, cdmpt_lib, precision):
    """N = 33 (one 32-wide tile plus a 1-wide tail), D = 0: only P0 and mu."""
    p = syn.chain_1d(33, seed=4, beta=8.0, n=10)
    p.H1 = p.H1[:0]
    ref = oracle.solve(p.H0, p.H0[None], p.beta, p.nocc, n=p.n, kind="rec")
    r = _run(cdmpt_lib, p, precision)
    assert r["P1"] is None
    assert _rel(r["P0"], ref["P0"]) < BAR[precision]


def test_degenerate_clean_lattice_fp64(cuda, cdmpt_lib):
    p = syn.cubic_lattice((6, 6, 6), seed=1, onsite_sigma=0.0, bond_disorder=0.0, beta=10.0,
                          n=12)
    ref = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    r = _run(cdmpt_lib, p, "fp64")
    _check(r, ref, BAR["fp64"], 1)


def test_host_outputs_match_device_outputs(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    a = _run(cdmpt_lib, p, "fp64", device="cuda")
    b = _run(cdmpt_lib, p, "fp64", device="cpu")
    assert _rel(a["P0"], b["P0"]) < 1e-13 and _rel(a["P1"], b["P1"]) < 1e-12


def test_range_error(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    with cdmpt_lib.Handle(precision="fp64") as h:
        h.set_H(p.H0, p.H1)
        with pytest.raises(cdmpt_lib.CdmptError) as e:
            h.solve(1e4, p.nocc, 3)
        assert e.value.status == 2


def test_argument_errors(cuda, cdmpt_lib):
    p = syn.workload("chain64")
    with cdmpt_lib.Handle(precision="fp64") as h:
        with pytest.raises(cdmpt_lib.CdmptError) as e:
            h.solve(p.beta, p.nocc, p.n)        # no Hamiltonian yet
        assert e.value.status == 1
        h.set_H(p.H0, p.H1)
        for bad in ((p.beta, 0.0, p.n), (p.beta, float(p.N), p.n), (-1.0, p.nocc, p.n),
                    (p.beta, p.nocc, 0)):
            with pytest.raises(cdmpt_lib.CdmptError) as e:
                h.solve(*bad)
            assert e.value.status == 1


def test_cg_iteration_cap_reported(cuda, cdmpt_lib):
    p = syn.cubic_lattice((8, 8, 8), seed=3, beta=20.0, n=12)
    with cdmpt_lib.Handle(precision="fp64", cg_maxit=1) as h:
        h.set_H(p.H0, p.H1)
        with pytest.raises(cdmpt_lib.CdmptError) as e:
            h.solve(p.beta, p.nocc, p.n)
        assert e.value.status == 4


def test_occupation_loop_cap_reported(cuda, cdmpt_lib):
    p = syn.cubic_lattice((8, 8, 8), seed=3, beta=20.0, n=12)
    with cdmpt_lib.Handle(precision="fp64", mu_maxit=1, mu_guess=1.5) as h:
        h.set_H(p.H0, p.H1)
        with pytest.raises(cdmpt_lib.CdmptError) as e:
            h.solve(p.beta, p.nocc, p.n)
        assert e.value.status == 3


def test_stats_are_consistent(cuda, cdmpt_lib):
    p = syn.cubic_lattice((8, 8, 8), seed=1002, beta=20.0, n=14)
    r = _run(cdmpt_lib, p, "fp32", profile=True)
    st = r["stats"]
    assert st["mu_iterations"] >= 1 and st["gemm_launches"] > 0
    assert st["gemm_timed"] == st["gemm_launches"]
    assert st["gemm_ms"] > 0
    assert st["tensor_flops"] == pytest.approx(3 * st["gemm_flops"])
    assert st["occupation_error"] < 1e-7 * p.N + 1e-6
