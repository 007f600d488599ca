"""Pins for the FP64 oracle: checks against things other than the oracle itself.

Each test ties one oracle function to an independent fact: a different
algorithm (matrix exponential, Algorithm 1 with dense solves, finite
differences), an identity stated or implied by the paper, or a printed
constant. A dropped term, a wrong sign or index, or a transposed operand in
the oracle fails at least one of these.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

import oracle as o
import synthetic as syn

GOLDEN = __file__.rsplit("/", 1)[0] + "/golden"


def _rand_sym(N, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(N, N)) * scale
    return 0.5 * (A + A.T)


def _dimer_chain(N=16, t1=-1.0, t2=-0.4):
    """Gapped chain (alternating hopping), gap ~ 2|t1 - t2| at half filling."""
    H = np.zeros((N, N))
    for i in range(N - 1):
        H[i, i + 1] = H[i + 1, i] = t1 if i % 2 == 0 else t2
    x = np.arange(N) - (N - 1) / 2.0
    return H, np.diag(x)


# --------------------------------------------------------------------------
# P0 and mu: Eq. (Rec_F_1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("beta", [0.7, 3.0, 8.0])
def test_p0_fd_equals_matrix_exponential(beta):
    """Fermi-Dirac P0 from eigenvalues == [expm(beta(H - mu I)) + I]^-1 (no eigensolver)."""
    H = _rand_sym(9, 11, 0.4)
    r = o.solve(H, H, beta, 4.0, kind="fd")
    N = H.shape[0]
    E = scipy.linalg.expm(beta * (H - r["mu"] * np.eye(N)))
    P_ref = np.linalg.inv(E + np.eye(N))
    assert o.rel_frobenius(r["P0"], P_ref) < 1e-11


def test_p0_rec_equals_matrix_power_pade():
    """Recursion P0 == f_{2^n}(X0) evaluated with matrix powers and one inverse (App. A)."""
    H = _rand_sym(7, 5, 0.5)
    beta, n, mu = 4.0, 4, 0.1
    X0 = 0.5 * np.eye(7) - 2.0 ** (-(n + 2)) * beta * (H - mu * np.eye(7))
    m = 2 ** n
    Xm = np.linalg.matrix_power(X0, m)
    Ym = np.linalg.matrix_power(np.eye(7) - X0, m)
    P_ref = np.linalg.solve(Xm + Ym, Xm)
    r = o.solve(H, H, beta, 3.5, n=n, kind="rec", mu=mu)
    assert o.rel_frobenius(r["P0"], P_ref) < 1e-11


@pytest.mark.parametrize("kind,n", [("fd", None), ("rec", 12)])
def test_trace_symmetry_spectrum(kind, n):
    p = syn.workload("chain64")
    r = o.solve(p.H0, p.H1, p.beta, p.nocc, n=n, kind=kind)
    assert abs(np.trace(r["P0"]) - p.nocc) < 1e-10
    assert np.allclose(r["P0"], r["P0"].T, atol=1e-14)
    ev = np.linalg.eigvalsh(r["P0"])
    assert ev.min() > -1e-12 and ev.max() < 1 + 1e-12


# --------------------------------------------------------------------------
# first order: closed form vs the iterated map of Eq. Rec_F_2 on power series in lambda
# --------------------------------------------------------------------------

def test_closed_form_equals_series_recursion():
    """P0, P1 of kind='rec' == the first two Taylor coefficients in lambda of n applications of
    Eq. Rec_F_2's map to X_0(lambda), at the same mu, mu1."""
    p = syn.workload("chain64")
    r = o.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    (X0, X1), conds = o.series_recursion([p.H0, p.H1[0]], p.beta, [r["mu"], r["mu1"][0]], p.n)
    assert o.rel_frobenius(X0, r["P0"]) < 1e-12
    assert o.rel_frobenius(X1, r["P1"][0]) < 1e-11
    # the denominator X^2 + (I - X)^2 (the paper's T) is SPD with condition number <= 2 (Sec. II)
    assert max(conds) <= 2.0 + 1e-12 and min(conds) >= 1.0


def test_canonical_newton_fixed_point():
    """Newton steps of Eq. NewtRaphs with P_mu = beta P(I-P) reach the closed-form mu, mu1."""
    H0, H1 = _dimer_chain(24)
    beta, nocc, n = 6.0, 12.0, 8
    r = o.solve(H0, H1, beta, nocc, n=n, kind="rec")
    P0, P1, mu, mu1, it = o.canonical_newton(H0, H1, beta, nocc, n, mu0=0.3)
    assert abs(mu - r["mu"]) < 1e-11
    assert abs(mu1 - r["mu1"][0]) < 1e-9
    assert o.rel_frobenius(P1, r["P1"][0]) < 1e-10


def test_composition_rule_scalars():
    """f_{m n} = f_m o f_n (App. A) and n steps of f_2 == the tanh/atanh closed form."""
    x = np.linspace(0.02, 0.98, 41)
    for m, k in ((2, 3), (3, 2), (2, 2)):
        assert np.allclose(o.pade_f(o.pade_f(x, k), m), o.pade_f(x, m * k), rtol=1e-12, atol=1e-15)
    beta, n, mu = 10.0, 5, 0.0
    eps = np.linspace(-2.0, 2.0, 33)
    x0 = 0.5 - beta * (eps - mu) / 2.0 ** (n + 2)
    y = x0.copy()
    for _ in range(n):
        y = o.pade_f(y, 2)
    assert np.allclose(o.occupation(eps, mu, beta, n), y, rtol=1e-13, atol=1e-15)


def test_truncation_gap_follows_effective_exponent():
    """g_n(t) = FD(t + t^3/(12 4^n) + O(t^5/4^2n)): the linear X0 stretches the exponent."""
    beta, n = 20.0, 8
    eps = np.linspace(-1.0, 1.0, 51)
    t = beta * eps
    g = o.occupation(eps, 0.0, beta, n)
    f_plain = o.occupation(eps, 0.0, beta, None)
    t_eff = t + t ** 3 / (12.0 * 4.0 ** n)
    f_eff = 0.5 * (1.0 - np.tanh(0.5 * t_eff))
    gap = np.max(np.abs(g - f_plain))
    assert gap > 1e-6
    assert np.max(np.abs(g - f_eff)) < 1e-3 * gap


# --------------------------------------------------------------------------
# P1, mu1: canonical response (Eqs. P_resp, H_prt, NewtRaphs)
# --------------------------------------------------------------------------

def _canonical_P0(H0, H1, lam, beta, nocc, n, kind):
    return o.solve(H0 + lam * H1, H1, beta, nocc, n=n, kind=kind)


@pytest.mark.parametrize("kind,n", [("fd", None), ("rec", 10)])
def test_p1_equals_five_point_finite_difference(kind, n):
    """P1 == dP0/dlambda of P0(H0 + lambda H1) with mu(lambda) re-fitted (5-point stencil)."""
    H0 = _rand_sym(10, 3)
    H1 = np.diag(np.arange(10) - 4.5)
    beta, nocc, h = 2.0, 5.0, 1e-3
    r = o.solve(H0, H1, beta, nocc, n=n, kind=kind)
    P = {k: _canonical_P0(H0, H1, k * h, beta, nocc, n, kind)["P0"] for k in (-2, -1, 1, 2)}
    fd = (P[-2] - 8 * P[-1] + 8 * P[1] - P[2]) / (12 * h)
    assert o.rel_frobenius(r["P1"][0], fd) < 1e-8
    mus = {k: _canonical_P0(H0, H1, k * h, beta, nocc, n, kind)["mu"] for k in (-2, -1, 1, 2)}
    dmu = (mus[-2] - 8 * mus[-1] + 8 * mus[1] - mus[2]) / (12 * h)
    assert abs(r["mu1"][0] - dmu) < 1e-8 * max(1.0, abs(dmu))


def test_p1_traceless_symmetric_and_shift_invariant():
    p = syn.workload("chain64")
    r = o.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    P1 = r["P1"][0]
    assert abs(np.trace(P1)) < 1e-10 * np.abs(P1).max() * p.N
    assert np.allclose(P1, P1.T, atol=1e-13 * np.abs(P1).max())
    r2 = o.solve(p.H0, p.H1 + 3.7 * np.eye(p.N), p.beta, p.nocc, n=p.n, kind="rec")
    assert o.rel_frobenius(r2["P1"][0], P1) < 1e-12
    # alpha = -2 Tr(P1 H1) is unchanged by the shift since Tr P1 = 0
    assert abs(r2["alpha"][0] - r["alpha"][0]) < 1e-9 * abs(r["alpha"][0])


def test_alpha_positive_and_canonical_below_grand_canonical():
    p = syn.workload("chain64")
    c = o.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    g = o.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", canonical=False)
    assert c["alpha"][0] > 0
    assert c["alpha"][0] <= g["alpha"][0] + 1e-9


def test_Q_equals_dP0_dmu():
    """Q returned by the oracle == central difference of P0 in mu (rec kind, exact at finite n)."""
    H0 = _rand_sym(8, 21)
    beta, n, mu, h = 3.0, 6, 0.2, 1e-4
    r = o.solve(H0, H0, beta, 4.0, n=n, kind="rec", mu=mu)
    Pp = o.solve(H0, H0, beta, 4.0, n=n, kind="rec", mu=mu + h)["P0"]
    Pm = o.solve(H0, H0, beta, 4.0, n=n, kind="rec", mu=mu - h)["P0"]
    assert o.rel_frobenius(r["Q"], (Pp - Pm) / (2 * h)) < 1e-7


def test_zero_temperature_limit():
    """beta -> infinity on a gapped chain: P0 idempotent and P1 = P0 P1 + P1 P0."""
    H0, H1 = _dimer_chain(16)
    r = o.solve(H0, H1, 400.0, 8.0, kind="fd")
    P0, P1 = r["P0"], r["P1"][0]
    assert np.abs(P0 @ P0 - P0).max() < 1e-12
    assert o.rel_frobenius(P0 @ P1 + P1 @ P0, P1) < 1e-10


def test_degenerate_levels_are_finite():
    """Clean periodic lattice (highly degenerate spectrum): divided differences stay exact."""
    p = syn.cubic_lattice((4, 4, 4), seed=7, onsite_sigma=0.0, bond_disorder=0.0, beta=5.0, n=10)
    r = o.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    assert np.all(np.isfinite(r["P1"]))
    h = 1e-4
    Pp = o.solve(p.H0 + h * p.H1[0], p.H1, p.beta, p.nocc, n=p.n, kind="rec")["P0"]
    Pm = o.solve(p.H0 - h * p.H1[0], p.H1, p.beta, p.nocc, n=p.n, kind="rec")["P0"]
    assert o.rel_frobenius(r["P1"][0], (Pp - Pm) / (2 * h)) < 1e-6


# --------------------------------------------------------------------------
# free energy: Eqs. (FreeE), (SED), (Resp_0), (EntDer)
# --------------------------------------------------------------------------

def _omega(H0, H1, lam, beta, nocc):
    return o.solve(H0 + lam * H1, H1, beta, nocc, kind="fd")["omega"]


def test_n_plus_one_rule_first_and_second_order():
    """Omega^(1) = Tr[H1 P0] and Omega^(2) = 1/2 Tr[H1 P1] (Eq. Resp_0, H^(2) = 0)."""
    H0 = _rand_sym(10, 8)
    H1 = _rand_sym(10, 9, 0.3)
    beta, nocc, h = 3.0, 4.0, 1e-3
    r = o.solve(H0, H1, beta, nocc, kind="fd")
    w = {k: _omega(H0, H1, k * h, beta, nocc) for k in (-2, -1, 0, 1, 2)}
    d1 = (w[-2] - 8 * w[-1] + 8 * w[1] - w[2]) / (12 * h)
    d2 = (-w[-2] + 16 * w[-1] - 30 * w[0] + 16 * w[1] - w[2]) / (12 * h * h)
    assert abs(d1 - np.sum(H1 * r["P0"])) < 1e-9
    omega2 = 0.5 * np.sum(H1 * r["P1"][0])
    assert abs(0.5 * d2 - omega2) < 1e-5 * abs(omega2)


def test_free_energy_gradient_is_P0():
    """dOmega/dH0 along any symmetric direction E is Tr[P0 E] (App. B, canonical)."""
    H0 = _rand_sym(9, 31)
    beta, nocc, h = 5.0, 3.0, 1e-4
    r = o.solve(H0, H0, beta, nocc, kind="fd")
    for s in range(3):
        E = _rand_sym(9, 100 + s)
        d = (_omega(H0, E, h, beta, nocc) - _omega(H0, E, -h, beta, nocc)) / (2 * h)
        assert abs(d - np.sum(r["P0"] * E)) < 1e-7


def test_entropy_derivative_identity():
    """Eq. (EntDer): ln(P (I-P)^-1) = -beta (H - mu I) for the Fermi-Dirac P0."""
    H0 = _rand_sym(8, 41)
    beta = 2.5
    r = o.solve(H0, H0, beta, 3.0, kind="fd")
    P = r["P0"]
    L = scipy.linalg.logm(P @ np.linalg.inv(np.eye(8) - P)).real
    assert o.rel_frobenius(L, -beta * (H0 - r["mu"] * np.eye(8))) < 1e-9


# --------------------------------------------------------------------------
# Table 1 constants (Eq. S_Approx, exponent i; see the readings)
# --------------------------------------------------------------------------

def _golden_tab1():
    rows = {}
    for line in open(f"{GOLDEN}/tab1_entropy_coefficients.txt"):
        if line.startswith("#") or not line.strip():
            continue
        m, i, a, b = line.split()
        rows.setdefault(int(m), []).append((int(a), Fraction(b)))
    return rows


def test_table1_coefficients_match_golden():
    gold = _golden_tab1()
    coef = o.entropy_coefficients()
    for m, lst in gold.items():
        for (a, b), c in zip(lst, coef[m]):
            assert abs(c - (a * math.log(2) + float(b))) < 1e-13


def test_table1_coefficients_match_entropy_at_half():
    """s_m(x) = -sum_i c_i (x(x-1))^i matches s(x) = -x ln x - (1-x) ln(1-x) and its even
    derivatives at x = 1/2 up to order 2(m-1): the construction stated in Table 1's caption."""
    sp = pytest.importorskip("sympy")
    x = sp.symbols("x")
    s = -x * sp.log(x) - (1 - x) * sp.log(1 - x)
    for m, lst in _golden_tab1().items():
        c = [a * sp.log(2) + sp.Rational(b.numerator, b.denominator) for a, b in lst]
        sm = -sum(ci * (x * (x - 1)) ** (i + 1) for i, ci in enumerate(c))
        for k in range(0, 2 * m - 1, 2):
            lhs = sp.diff(sm, x, k).subs(x, sp.Rational(1, 2))
            rhs = sp.diff(s, x, k).subs(x, sp.Rational(1, 2))
            assert sp.simplify(lhs - rhs) == 0, (m, k)


def test_chain64_golden_regression():
    """The oracle still reproduces the stored chain64 values written by make_golden.py."""
    import json
    g = json.load(open(f"{GOLDEN}/chain64_oracle.json"))
    p = syn.workload("chain64")
    for kind, n in (("rec", p.n), ("fd", None)):
        r = o.solve(p.H0, p.H1, p.beta, p.nocc, n=n, kind=kind)
        ref = g[kind]
        assert abs(r["mu"] - ref["mu"]) < 1e-12
        assert abs(r["mu1"][0] - ref["mu1"]) < 1e-10 * max(1, abs(ref["mu1"]))
        assert abs(r["alpha"][0] - ref["alpha"]) < 1e-10 * abs(ref["alpha"])
        assert np.allclose(np.diag(r["P0"])[:8], ref["P0_diag_head"], rtol=0, atol=1e-12)


def test_pins_catch_planted_mistakes(monkeypatch):
    """Plant typical slips in the oracle (CPU only) and check a pin notices each one."""
    H0 = _rand_sym(10, 3)
    H1 = np.diag(np.arange(10) - 4.5)
    beta, nocc, h = 2.0, 5.0, 1e-3

    def fd_error():
        r = o.solve(H0, H1, beta, nocc, kind="fd")
        P = {k: o.solve(H0 + k * h * H1, H1, beta, nocc, kind="fd")["P0"] for k in (-2, -1, 1, 2)}
        fd = (P[-2] - 8 * P[-1] + 8 * P[1] - P[2]) / (12 * h)
        return o.rel_frobenius(r["P1"][0], fd)

    assert fd_error() < 1e-8
    real_dd = o.dmpt_oracle.divided_differences
    # wrong sign of the divided differences
    monkeypatch.setattr(o.dmpt_oracle, "divided_differences", lambda *a, **k: -real_dd(*a, **k))
    assert fd_error() > 1e-3
    # dropped off-diagonal (only the diagonal f' kept)
    monkeypatch.setattr(o.dmpt_oracle, "divided_differences",
                        lambda *a, **k: np.diag(np.diag(real_dd(*a, **k))))
    assert fd_error() > 1e-3
    monkeypatch.setattr(o.dmpt_oracle, "divided_differences", real_dd)
    # wrong temperature scaling in the occupation (beta/2 slip)
    real_occ = o.dmpt_oracle.occupation
    monkeypatch.setattr(o.dmpt_oracle, "occupation",
                        lambda e, mu, b, n=None: real_occ(e, mu, 0.5 * b, n))
    assert fd_error() > 1e-3


# --------------------------------------------------------------------------
# P2: second-order canonical response (Algorithm 1, order 2) and the
# polarizability gradient d alpha / d H0 = -4 P2
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind,n", [("fd", None), ("rec", 10)])
def test_second_derivative_closed_form(kind, n):
    """f'' against central differences of f' (both kinds)."""
    e = np.linspace(-3.0, 3.0, 41)
    mu, beta, h = 0.3, 2.5, 1e-5
    d2 = o.occupation_second_derivative(e, mu, beta, n)
    fd = (o.occupation_derivative(e + h, mu, beta, n) -
          o.occupation_derivative(e - h, mu, beta, n)) / (2 * h)
    assert np.max(np.abs(d2 - fd)) < 1e-8 * np.max(np.abs(d2))


def test_second_divided_difference_quadrature_matches_quotient():
    """Hermite-Genocchi quadrature == (f[a,b] - f[b,c]) / (a - c) where both are accurate."""
    rng = np.random.default_rng(4)
    beta, mu, n = 3.0, 0.1, 10
    a = rng.uniform(-1, 1, 200)
    spread = rng.uniform(1.0, 2.0, 200) / beta
    c = a + spread
    b = a + rng.uniform(0, 1, 200) * spread
    q = o.second_dd_quadrature(a, b, c, mu, beta, n)
    occ = lambda x: o.occupation(x, mu, beta, n)
    fab = (occ(a) - occ(b)) / (a - b)
    fbc = (occ(b) - occ(c)) / (b - c)
    quot = (fab - fbc) / (a - c)
    assert np.max(np.abs(q - quot)) < 1e-9 * np.max(np.abs(q))


@pytest.mark.parametrize("kind,n", [("fd", None), ("rec", 10)])
def test_p2_equals_finite_difference_of_p1(kind, n):
    """2 P2 == dP1/dlambda of the canonical P1(H0 + lambda H1) (5-point stencil)."""
    H0 = _rand_sym(12, 8)
    H1 = np.diag(np.arange(12) - 5.5) * 0.3
    beta, nocc, h = 2.0, 6.0, 1e-3
    r = o.response2(H0, H1, beta, nocc, n=n, kind=kind)
    P1 = {k: o.solve(H0 + k * h * H1, H1, beta, nocc, n=n, kind=kind)["P1"][0]
          for k in (-2, -1, 1, 2)}
    fd = (P1[-2] - 8 * P1[-1] + 8 * P1[1] - P1[2]) / (12 * h)
    assert o.rel_frobenius(2.0 * r["P2"][0], fd) < 1e-8
    assert abs(np.trace(r["P2"][0])) < 1e-12 * np.linalg.norm(r["P2"][0])
    assert np.abs(r["P2"][0] - r["P2"][0].T).max() < 1e-12 * np.abs(r["P2"][0]).max()


def test_p2_equals_series_recursion_second_order():
    """The closed form == the lambda^2 coefficient of the iterated map (chain64), and the
    oracle's mu2 makes its trace vanish (the canonical condition)."""
    p = syn.workload("chain64")
    r = o.response2(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    (X0, X1, X2), _ = o.series_recursion([p.H0, p.H1[0], 0], p.beta,
                                         [r["mu"], r["mu1"][0], r["mu2"][0]], p.n)
    assert o.rel_frobenius(X1, r["P1"][0]) < 1e-10
    assert o.rel_frobenius(X2, r["P2"][0]) < 1e-10
    assert abs(np.trace(X2)) < 1e-10 * np.linalg.norm(X2)


def test_p2_degenerate_clean_lattice():
    """Exactly degenerate levels (clean periodic lattice): the close-pair path against the
    lambda^2 coefficient of the iterated map."""
    p = syn.cubic_lattice((4, 4, 4), seed=1, beta=6.0, n=12, onsite_sigma=0.0,
                          bond_disorder=0.0)
    r = o.response2(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    (_, _, X2), _ = o.series_recursion([p.H0, p.H1[0], 0], p.beta,
                                       [r["mu"], r["mu1"][0], r["mu2"][0]], p.n)
    assert o.rel_frobenius(X2, r["P2"][0]) < 1e-10


@pytest.mark.parametrize("kind,n", [("fd", None), ("rec", 10)])
def test_alpha_gradient_equals_finite_differences(kind, n):
    """<grad alpha, E> == d alpha(H0 + t E)/dt (5-point) for random symmetric E."""
    H0 = _rand_sym(12, 9)
    H1 = np.diag(np.arange(12) - 5.5) * 0.3
    beta, nocc, h = 2.0, 6.0, 1e-3
    g = o.response2(H0, H1, beta, nocc, n=n, kind=kind)["grad_alpha"][0]
    for seed in range(3):
        E = _rand_sym(12, 100 + seed)
        al = {k: o.solve(H0 + k * h * E, H1, beta, nocc, n=n, kind=kind)["alpha"][0]
              for k in (-2, -1, 1, 2)}
        fd = (al[-2] - 8 * al[-1] + 8 * al[1] - al[2]) / (12 * h)
        assert abs(np.sum(g * E) - fd) < 1e-7 * max(1.0, abs(fd))


def test_second_order_pins_catch_planted_mistakes(monkeypatch):
    """Plant slips in the second-order oracle (CPU) and check the pins notice them."""
    H0 = _rand_sym(12, 8)
    H1 = np.diag(np.arange(12) - 5.5) * 0.3
    beta, nocc, h = 2.0, 6.0, 1e-3
    P1 = {k: o.solve(H0 + k * h * H1, H1, beta, nocc, kind="fd")["P1"][0] for k in (-2, -1, 1, 2)}
    fd = (P1[-2] - 8 * P1[-1] + 8 * P1[1] - P1[2]) / (12 * h)

    def err(**kw):
        return o.rel_frobenius(2.0 * o.response2(H0, H1, beta, nocc, kind="fd", **kw)["P2"][0], fd)

    assert err() < 1e-8
    assert err(close=100.0) < 1e-8          # every pair through the explicit sums
    real = o.dmpt_oracle.occupation_second_derivative
    # wrong sign of f'' (seen through the quadrature of clustered triples)
    monkeypatch.setattr(o.dmpt_oracle, "occupation_second_derivative",
                        lambda *a, **k: -real(*a, **k))
    assert err(close=100.0) > 1e-3
    monkeypatch.setattr(o.dmpt_oracle, "occupation_second_derivative", real)
    # mu1 left out of the second order (ht = h instead of h - mu1 I)
    real_solve = o.dmpt_oracle.solve

    def no_mu1(*a, **k):
        r = real_solve(*a, **k)
        r["mu1"] = np.zeros_like(r["mu1"])
        return r
    monkeypatch.setattr(o.dmpt_oracle, "solve", no_mu1)
    assert err() > 1e-3


def test_grand_canonical_orders_match_series_recursion():
    """Fixed mu (the grand-canonical scheme beside Algorithm 1): P0, P1 and P2 of the closed
    forms equal the coefficients of the iterated map with mu1 = mu2 = 0, chain64."""
    p = syn.workload("chain64")
    mu = o.solve(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")["mu"] + 0.05
    r = o.response2(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec", canonical=False, mu=mu)
    assert r["mu1"][0] == 0.0 and r["mu2"][0] == 0.0
    (X0, X1, X2), _ = o.series_recursion([p.H0, p.H1[0], 0], p.beta, [mu, 0.0, 0.0], p.n)
    assert o.rel_frobenius(X0, r["P0"]) < 1e-12
    assert o.rel_frobenius(X1, r["P1"][0]) < 1e-10
    assert o.rel_frobenius(X2, r["P2"][0]) < 1e-10
    assert abs(np.trace(X1)) > 1e-3     # no canonical constraint: Tr P1 != 0


def test_n_plus_one_rule_third_order():
    """Omega^(3) = 1/3 Tr[H1 P2] (Eq. Resp_0, H^(k >= 2) = 0) against the third derivative of
    the canonical free energy Omega(lambda) / 6 (six-point central differences)."""
    H0 = _rand_sym(10, 8)
    H1 = _rand_sym(10, 9, 0.3)
    beta, nocc, h = 3.0, 4.0, 1e-2
    om3 = o.response2(H0, H1, beta, nocc, kind="fd")["omega3"][0]
    w = {k: _omega(H0, H1, k * h, beta, nocc) for k in (-3, -2, -1, 1, 2, 3)}
    d3 = (-w[3] + 8 * w[2] - 13 * w[1] + 13 * w[-1] - 8 * w[-2] + w[-3]) / (8 * h ** 3)
    assert abs(d3 / 6.0 - om3) < 1e-6 * abs(om3)


# --------------------------------------------------------------------------
# P3: third-order canonical response (Algorithm 1, order 3) and Omega^(4)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind,n", [("fd", None), ("rec", 8)])
def test_third_derivative_closed_form(kind, n):
    """f''' against central differences of the closed-form f''."""
    e = np.linspace(-1.5, 1.5, 41)
    beta, mu, h = 4.0, 0.2, 1e-5
    d3 = o.occupation_third_derivative(e, mu, beta, n)
    fd = (o.occupation_second_derivative(e + h, mu, beta, n)
          - o.occupation_second_derivative(e - h, mu, beta, n)) / (2 * h)
    assert np.max(np.abs(d3 - fd)) < 1e-7 * np.max(np.abs(d3))


def test_third_divided_difference_quadrature():
    """The Hermite-Genocchi quadrature of f[a, b, c, d] equals the recursive quotient of
    well-separated points, and f'''/6 when the four points coincide."""
    beta, mu, n = 2.0, 0.1, 10
    pts = np.array([-0.3, -0.05, 0.2, 0.45])        # spread 0.75 / beta-scale 1.5
    fq = o.third_dd_quadrature(*pts, mu, beta, n)

    def f(x):
        return o.occupation(np.array(x), mu, beta, n)

    def dd(xs):
        if len(xs) == 1:
            return float(f(xs[0]))
        return (dd(xs[1:]) - dd(xs[:-1])) / (xs[-1] - xs[0])
    assert abs(fq - dd(list(pts))) < 1e-9 * abs(fq)
    x = 0.37
    assert abs(o.third_dd_quadrature(x, x, x, x, mu, beta, n)
               - o.occupation_third_derivative(x, mu, beta, n) / 6.0) < 1e-14


def test_p3_equals_series_recursion_third_order():
    """The closed form == the lambda^3 coefficient of the iterated map (chain64), and the
    oracle's mu3 makes its trace vanish (the canonical condition)."""
    p = syn.workload("chain64")
    r = o.response3(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    X, _ = o.series_recursion([p.H0, p.H1[0], 0, 0], p.beta,
                              [r["mu"], r["mu1"][0], r["mu2"][0], r["mu3"][0]], p.n)
    assert o.rel_frobenius(X[2], r["P2"][0]) < 1e-10
    assert o.rel_frobenius(X[3], r["P3"][0]) < 1e-10
    assert abs(np.trace(X[3])) < 1e-10 * np.linalg.norm(X[3])


def test_p3_degenerate_clean_lattice():
    """Exactly degenerate levels (clean 4 x 4 x 2 lattice): explicit sums and quadrature agree
    with the iterated map."""
    p = syn.cubic_lattice((4, 4, 2), seed=0, beta=5.0, n=10, onsite_sigma=0.0, bond_disorder=0.0)
    r = o.response3(p.H0, p.H1, p.beta, p.nocc, n=p.n, kind="rec")
    X, _ = o.series_recursion([p.H0, p.H1[0], 0, 0], p.beta,
                              [r["mu"], r["mu1"][0], r["mu2"][0], r["mu3"][0]], p.n)
    assert o.rel_frobenius(X[3], r["P3"][0]) < 1e-9


@pytest.mark.parametrize("kind,n", [("fd", None), ("rec", 10)])
def test_p3_equals_finite_difference_of_p2(kind, n):
    """3 P3 = d P2 / dt along H0 + t H1 (the canonical expansion re-centred at t)."""
    H0 = _rand_sym(20, 31, 0.4)
    H1 = _rand_sym(20, 32, 0.1) + np.diag(np.arange(20) - 9.5) * 0.05
    beta, nocc, h = 5.0, 10.0, 1e-4
    r = o.response3(H0, H1, beta, nocc, n=n, kind=kind)
    P2 = {k: o.response2(H0 + k * h * H1, H1, beta, nocc, n=n, kind=kind)["P2"][0]
          for k in (-2, -1, 1, 2)}
    fd = (P2[-2] - 8 * P2[-1] + 8 * P2[1] - P2[2]) / (12 * h)
    assert o.rel_frobenius(r["P3"][0], fd / 3.0) < 1e-7


def test_p3_and_mu_series_against_high_precision_brute_force():
    """Brute force at 60 digits (mpmath): P(lambda) = g_n(H0 + lambda H1 - mu(lambda) I) with
    mu(lambda) from Tr P = N_occ, by eigendecomposition at lambda = 0, +-h, +-2h, +-3h;
    Taylor coefficients of P and mu from central differences. Pins P3, mu1, mu2 and mu3."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    N, beta, nocc, n = 5, 3.0, 2.0, 6
    H0 = _rand_sym(N, 41)
    H1 = _rand_sym(N, 42, 0.5)
    r = o.response3(H0, H1, beta, nocc, n=n, kind="rec")
    B = mp.mpf(beta)
    m2 = mp.mpf(2) ** n
    c = B / mp.mpf(2) ** (n + 1)

    def g(e, mu):
        return (1 + mp.tanh(m2 * mp.atanh(-c * (e - mu)))) / 2

    def at(lam):
        A = mp.matrix(H0.tolist()) + lam * mp.matrix(H1.tolist())
        E, Q = mp.eigsy(A)
        mu = mp.findroot(lambda u: sum(g(E[i], u) for i in range(N)) - nocc, mp.mpf(r["mu"]))
        P = Q * mp.diag([g(E[i], mu) for i in range(N)]) * Q.T
        return P, mu

    h = mp.mpf("1e-12")
    vals = {k: at(k * h) for k in (-2, -1, 0, 1, 2)}
    P = {k: v[0] for k, v in vals.items()}
    mu = {k: v[1] for k, v in vals.items()}
    c3 = (P[2] - 2 * P[1] + 2 * P[-1] - P[-2]) / (12 * h ** 3)
    mu1 = (mu[1] - mu[-1]) / (2 * h)
    mu2 = (mu[1] - 2 * mu[0] + mu[-1]) / (2 * h ** 2)
    mu3 = (mu[2] - 2 * mu[1] + 2 * mu[-1] - mu[-2]) / (12 * h ** 3)
    P3 = np.array([[float(c3[i, j]) for j in range(N)] for i in range(N)])
    assert o.rel_frobenius(r["P3"][0], P3) < 1e-10
    assert abs(float(mu1) - r["mu1"][0]) < 1e-12
    assert abs(float(mu2) - r["mu2"][0]) < 1e-11 * max(1.0, abs(r["mu2"][0]))
    assert abs(float(mu3) - r["mu3"][0]) < 1e-10 * max(1.0, abs(r["mu3"][0]))


def test_n_plus_one_rule_fourth_order():
    """Omega^(4) = 1/4 Tr[H1 P3] (Eq. Resp_0, H^(k >= 2) = 0) against the fourth derivative of
    the canonical free energy Omega(lambda) / 24 (seven-point central differences)."""
    H0 = _rand_sym(10, 8)
    H1 = _rand_sym(10, 9, 0.3)
    beta, nocc, h = 3.0, 4.0, 2e-2
    om4 = o.response3(H0, H1, beta, nocc, kind="fd")["omega4"][0]
    w = {k: _omega(H0, H1, k * h, beta, nocc) for k in (-3, -2, -1, 0, 1, 2, 3)}
    d4 = (-w[3] + 12 * w[2] - 39 * w[1] + 56 * w[0] - 39 * w[-1] + 12 * w[-2] - w[-3]) / (
        6 * h ** 4)
    assert abs(d4 / 24.0 - om4) < 1e-4 * abs(om4)


def test_third_order_pins_catch_planted_mistakes(monkeypatch):
    """Plant slips in the third-order oracle (CPU) and check the pins notice them."""
    H0 = _rand_sym(24, 3, 0.4)
    H1 = _rand_sym(24, 4, 0.1) + np.diag(np.arange(24) - 11.5) * 0.1
    beta, nocc, n = 6.0, 12.0, 10
    X3 = None

    def err(**kw):
        nonlocal X3
        r = o.response3(H0, H1, beta, nocc, n=n, kind="rec", **kw)
        if X3 is None:   # the iterated map at the unplanted oracle's shifts
            X3 = o.series_recursion([H0, H1, 0, 0], beta,
                                    [r["mu"], r["mu1"][0], r["mu2"][0], r["mu3"][0]], n)[0][3]
        return o.rel_frobenius(r["P3"][0], X3)

    assert err() < 1e-10
    assert err(close=100.0) < 1e-10
    real3 = o.dmpt_oracle.occupation_third_derivative
    # wrong sign of f''' (seen through the quadrature of clustered quadruples)
    monkeypatch.setattr(o.dmpt_oracle, "occupation_third_derivative",
                        lambda *a, **k: -real3(*a, **k))
    assert err(close=100.0) > 1e-3
    monkeypatch.setattr(o.dmpt_oracle, "occupation_third_derivative", real3)
    # mu2 cross terms dropped (mu2 taken as zero inside the third order)
    real2 = o.dmpt_oracle.response2

    def no_mu2(*a, **k):
        r = real2(*a, **k)
        r["mu2"] = np.zeros_like(r["mu2"])
        return r
    monkeypatch.setattr(o.dmpt_oracle, "response2", no_mu2)
    assert err() > 1e-3


# --------------------------------------------------------------------------
# the free energy as a loss of H0 (Eqs. FreeE, SED)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind,n,canonical", [("fd", None, True), ("rec", 8, True),
                                              ("rec", 8, False)])
def test_free_energy_gradient_central_differences(kind, n, canonical):
    """<dOmega/dH0, E> == (Omega(H0 + hE) - Omega(H0 - hE)) / 2h along random symmetric E
    (canonical: mu re-found at every point; grand canonical: mu held)."""
    H0 = _rand_sym(14, 51, 0.5)
    beta, nocc, h = 4.0, 6.0, 1e-5
    r = o.free_energy(H0, beta, nocc, n=n, kind=kind)
    mu = None if canonical else r["mu"]
    g = o.free_energy(H0, beta, nocc, n=n, kind=kind, canonical=canonical, mu=mu)["grad"]
    for seed in range(5):
        E = _rand_sym(14, 100 + seed, 1.0)
        wp = o.free_energy(H0 + h * E, beta, nocc, n=n, kind=kind, mu=mu)["omega"]
        wm = o.free_energy(H0 - h * E, beta, nocc, n=n, kind=kind, mu=mu)["omega"]
        fd = (wp - wm) / (2 * h)
        assert abs(fd - np.sum(g * E)) < 1e-7 * max(1.0, abs(fd))


def test_free_energy_fermi_dirac_gradient_is_P0_and_grand_potential_identity():
    """Fermi-Dirac: the canonical gradient is P0 (the entropy term cancels the response,
    Eq. EntDer), and Omega = mu N_occ + (1/beta) sum_i ln(1 - f_i)."""
    H0 = _rand_sym(16, 52, 0.5)
    beta, nocc = 6.0, 7.0
    r = o.free_energy(H0, beta, nocc, kind="fd")
    assert o.rel_frobenius(r["grad"], r["P0"]) < 1e-13
    eps = np.linalg.eigvalsh(H0)
    ln_1mf = -np.logaddexp(0.0, -beta * (eps - r["mu"]))     # ln(1 - f), no cancellation
    assert abs(r["omega"] - (r["mu"] * nocc + np.sum(ln_1mf) / beta)) < 1e-13 * abs(r["omega"])


def test_free_energy_of_recursion_equals_telescoped_log_determinants():
    """For P = X_n of n recursion steps, 1 - x_{k+1} = (1 - x_k)^2 / T_k with
    T_k = x_k^2 + (1 - x_k)^2, so ln det(I - P) = 2^n ln det(I - X_0) -
    sum_k 2^(n-1-k) ln det T_k. With ln(P (I - P)^-1) = 2^(n+1) atanh(Z_0) this gives
    Omega = mu Tr P + (1/beta) ln det(I - P) + (2^(n+1)/beta) Tr[P (atanh Z_0 - Z_0)],
    checked here with dense slogdet along Algorithm 1's own iterates."""
    H0 = _rand_sym(20, 53, 0.5)
    beta, nocc, n = 10.0, 9.0, 8
    r = o.free_energy(H0, beta, nocc, n=n, kind="rec")
    mu = r["mu"]
    N = H0.shape[0]
    I = np.eye(N)
    X = 0.5 * I - beta / 2.0 ** (n + 2) * (H0 - mu * I)
    Z0 = 2 * X - I
    logdet = 2.0 ** n * np.linalg.slogdet(I - X)[1]
    for k in range(n):
        T = X @ X + (I - X) @ (I - X)
        logdet -= 2.0 ** (n - 1 - k) * np.linalg.slogdet(T)[1]
        X = np.linalg.solve(T, X @ X)
    w, U = np.linalg.eigh(Z0)
    R = (U * (np.arctanh(w) - w)) @ U.T
    omega = mu * np.trace(X) + logdet / beta + 2.0 ** (n + 1) / beta * np.trace(X @ R)
    assert abs(omega - r["omega"]) < 1e-11 * abs(r["omega"])


# --------------------------------------------------------------------------
# non-orthogonal basis (Sec. IV, Eq. Fermi_D)
# --------------------------------------------------------------------------

def _nonorth_case(N=40, seed=71):
    p = syn.nonorthogonal_cluster(N, seed=seed, beta=6.0, n=10)
    return p.H0, p.H1[0], p.meta["S"], p.beta, p.nocc, p.n


def test_nonorthogonal_D_equals_generalized_eigenproblem():
    """D from the Cholesky route == C f(e) C^T from LAPACK's generalized symmetric
    eigensolver (F C = S C e, C^T S C = I), and Tr[D S] = N_occ, Tr[D1 S] = 0."""
    import scipy.linalg
    F, h1, S, beta, nocc, n = _nonorth_case()
    r = o.solve_nonorthogonal(F, h1, S, beta, nocc, n=n)
    e, C = scipy.linalg.eigh(F, S)
    D = (C * o.occupation(e, r["mu"], beta, n)) @ C.T
    assert o.rel_frobenius(r["D0"], D) < 1e-12
    assert abs(np.trace(r["D0"] @ S) - nocc) < 1e-10
    assert abs(np.trace(r["D1"][0] @ S)) < 1e-10


def test_nonorthogonal_response_is_covariant_under_a_change_of_basis():
    """With F' = B^T F B, S' = B^T S B, h1' = B^T h1 B for an invertible B: D' = B^-1 D B^-T,
    D1' likewise, mu, mu1 and alpha unchanged, and d alpha / dF' = B^-1 (d alpha / dF) B^-T."""
    F, h1, S, beta, nocc, n = _nonorth_case()
    rng = np.random.default_rng(5)
    B = np.eye(F.shape[0]) + 0.2 * rng.standard_normal(F.shape)
    Bi = np.linalg.inv(B)
    r = o.solve_nonorthogonal(F, h1, S, beta, nocc, n=n, order=2)
    q = o.solve_nonorthogonal(B.T @ F @ B, B.T @ h1 @ B, B.T @ S @ B, beta, nocc, n=n, order=2)
    assert o.rel_frobenius(q["D0"], Bi @ r["D0"] @ Bi.T) < 1e-10
    assert o.rel_frobenius(q["D1"][0], Bi @ r["D1"][0] @ Bi.T) < 1e-9
    assert o.rel_frobenius(q["grad_alpha"][0], Bi @ r["grad_alpha"][0] @ Bi.T) < 1e-9
    assert abs(q["alpha"][0] - r["alpha"][0]) < 1e-10 * abs(r["alpha"][0])
    assert abs(q["mu1"][0] - r["mu1"][0]) < 1e-10


def test_nonorthogonal_D1_and_alpha_gradient_equal_finite_differences():
    """D1 = dD/dlambda along F + lambda h1 (canonical), and <d alpha/dF, E> by central
    differences of alpha(F + hE) along a random symmetric E."""
    F, h1, S, beta, nocc, n = _nonorth_case(30, 72)
    h = 1e-4
    r = o.solve_nonorthogonal(F, h1, S, beta, nocc, n=n, order=2)
    D = {k: o.solve_nonorthogonal(F + k * h * h1, h1, S, beta, nocc, n=n)["D0"]
         for k in (-2, -1, 1, 2)}
    fd = (D[-2] - 8 * D[-1] + 8 * D[1] - D[2]) / (12 * h)
    assert o.rel_frobenius(r["D1"][0], fd) < 1e-8
    E = _rand_sym(F.shape[0], 73, 0.5)
    ap = o.solve_nonorthogonal(F + h * E, h1, S, beta, nocc, n=n)["alpha"][0]
    am = o.solve_nonorthogonal(F - h * E, h1, S, beta, nocc, n=n)["alpha"][0]
    assert abs((ap - am) / (2 * h) - np.sum(r["grad_alpha"][0] * E)) < 1e-6 * abs(ap)


# --------------------------------------------------------------------------
# self-consistent charge layer (Sec. IV, Eqs. FirstOrderPRT, Resp_Omega)
# --------------------------------------------------------------------------

def _scc_case(N=24, seed=81):
    p = syn.nonorthogonal_cluster(N, seed=seed, beta=4.0, n=10)
    return p.H0, p.H1[0], p.meta["S"], p.meta["gamma"], p.meta["q0"], p.beta, p.nocc, p.n


def test_scc_without_coupling_equals_non_self_consistent_solve():
    hc, h1, S, gamma, q0, beta, nocc, n = _scc_case()
    r = o.scc_solve(hc, h1, S, 0.0 * gamma, q0, beta, nocc, n=n)
    q = o.solve_nonorthogonal(hc, h1, S, beta, nocc, n=n)
    assert o.rel_frobenius(r["D0"], q["D0"]) < 1e-12
    assert o.rel_frobenius(r["D1"][0], q["D1"][0]) < 1e-10


@pytest.mark.parametrize("kind,n", [("fd", None), ("rec", 10)])
def test_scc_D1_equals_finite_difference_of_self_consistent_D(kind, n):
    """D1 = dD/dlambda of the self-consistent solution of h + lambda h1."""
    hc, h1, S, gamma, q0, beta, nocc, _ = _scc_case()
    h = 1e-4
    r = o.scc_solve(hc, h1, S, gamma, q0, beta, nocc, n=n, kind=kind)
    D = {k: o.scc_solve(hc + k * h * h1, h1, S, gamma, q0, beta, nocc, n=n, kind=kind)["D0"]
         for k in (-2, -1, 1, 2)}
    fd = (D[-2] - 8 * D[-1] + 8 * D[1] - D[2]) / (12 * h)
    assert o.rel_frobenius(r["D1"][0], fd) < 1e-7


def test_scc_free_energy_response_rule():
    """Eq. Resp_Omega at self-consistency (Fermi-Dirac, where the functional is variational):
    Omega_SCF^(1) = 2 Tr[h1 D0] = dOmega_SCF/dlambda and Omega_SCF^(2) = Tr[h1 D1] =
    (1/2) d^2 Omega_SCF / dlambda^2, by five-point differences of the free energy."""
    hc, h1, S, gamma, q0, beta, nocc, _ = _scc_case()
    h = 1e-3
    r = o.scc_solve(hc, h1, S, gamma, q0, beta, nocc, kind="fd")
    w = {k: o.scc_solve(hc + k * h * h1, h1, S, gamma, q0, beta, nocc, kind="fd")["omega"]
         for k in (-2, -1, 0, 1, 2)}
    d1 = (w[-2] - 8 * w[-1] + 8 * w[1] - w[2]) / (12 * h)
    d2 = (-w[-2] + 16 * w[-1] - 30 * w[0] + 16 * w[1] - w[2]) / (12 * h * h)
    assert abs(d1 - r["omega1"][0]) < 1e-8 * max(1.0, abs(d1))
    assert abs(0.5 * d2 - r["omega2"][0]) < 1e-5 * abs(r["omega2"][0])


def test_table2_pattern_low_temperature_needs_enough_steps():
    """Tab. 2's qualitative pattern, on a gapped tight-binding chain instead of H2O: at low
    temperature the occupation loop (Newton with P_mu = beta P (I - P), Eq. NewtRaphs) does not
    converge with too few recursion steps (beta = 1000: M = 4 and 6 fail, M >= 8 converge),
    while at high temperature every M converges. With M too small X_0 lies far outside
    [0, 1], where x^2 / (x^2 + (1 - x)^2) sends distant levels towards 1/2, so the occupation
    is wrong. The library refuses such (beta, n) with ERR_RANGE before they are run."""
    H0, H1 = _dimer_chain(24)
    H1 = H1 * 0.05
    for M in (4, 6):
        with pytest.raises(RuntimeError):
            o.canonical_newton(H0, H1, 1000.0, 12.0, M, mu0=0.3, maxit=100)
    for M in (8, 12, 16):
        o.canonical_newton(H0, H1, 1000.0, 12.0, M, mu0=0.3, maxit=100)
    for M in (4, 6, 8):
        o.canonical_newton(H0, H1, 10.0, 12.0, M, mu0=0.3, maxit=100)


# --------------------------------------------------------------------------
# higher perturbation terms H(lambda) = H0 + lambda H1 + lambda^2 H2 + lambda^3 H3
# (Eq. H_prt; Algorithm 1's X_0^(i) with H^(i) for i = 1..3)
# --------------------------------------------------------------------------

def _higher_case(N=18, seed=91):
    H0 = _rand_sym(N, seed, 0.4)
    H1 = _rand_sym(N, seed + 1, 0.1) + np.diag(np.arange(N) - (N - 1) / 2) * 0.05
    return H0, H1, _rand_sym(N, seed + 2, 0.05), _rand_sym(N, seed + 3, 0.03)


def test_higher_terms_match_series_recursion():
    """With H2 and H3 the closed forms equal the lambda^2 and lambda^3 coefficients of the
    iterated map for H0 + lambda H1 + lambda^2 H2 + lambda^3 H3, whose traces vanish at the
    oracle's mu2 and mu3."""
    H0, H1, H2, H3 = _higher_case()
    beta, nocc, n = 5.0, 9.0, 10
    r = o.response3(H0, H1[None], beta, nocc, n=n, H2=H2[None], H3=H3[None])
    X, _ = o.series_recursion([H0, H1, H2, H3], beta,
                              [r["mu"], r["mu1"][0], r["mu2"][0], r["mu3"][0]], n)
    assert o.rel_frobenius(X[2], r["P2"][0]) < 1e-10
    assert o.rel_frobenius(X[3], r["P3"][0]) < 1e-10
    assert abs(np.trace(X[2])) < 1e-11 and abs(np.trace(X[3])) < 1e-11


def test_higher_terms_against_high_precision_brute_force():
    """60-digit brute force of the canonical P(lambda) for H(lambda) = H0 + lambda H1 +
    lambda^2 H2 + lambda^3 H3: P2, P3, mu2 and mu3 by central differences."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    N, beta, nocc, n = 5, 3.0, 2.0, 6
    H0, H1, H2, H3 = (_rand_sym(N, 61), _rand_sym(N, 62, 0.5), _rand_sym(N, 63, 0.3),
                      _rand_sym(N, 64, 0.2))
    r = o.response3(H0, H1[None], beta, nocc, n=n, H2=H2[None], H3=H3[None])
    m2 = mp.mpf(2) ** n
    c = mp.mpf(beta) / mp.mpf(2) ** (n + 1)

    def g(e, mu):
        return (1 + mp.tanh(m2 * mp.atanh(-c * (e - mu)))) / 2

    def at(lam):
        A = (mp.matrix(H0.tolist()) + lam * mp.matrix(H1.tolist())
             + lam ** 2 * mp.matrix(H2.tolist()) + lam ** 3 * mp.matrix(H3.tolist()))
        E, Q = mp.eigsy(A)
        mu = mp.findroot(lambda u: sum(g(E[i], u) for i in range(N)) - nocc, mp.mpf(r["mu"]))
        return Q * mp.diag([g(E[i], mu) for i in range(N)]) * Q.T, mu

    h = mp.mpf("1e-12")
    vals = {k: at(k * h) for k in (-2, -1, 0, 1, 2)}
    P = {k: v[0] for k, v in vals.items()}
    mu = {k: v[1] for k, v in vals.items()}
    c2 = (P[1] - 2 * P[0] + P[-1]) / (2 * h ** 2)
    c3 = (P[2] - 2 * P[1] + 2 * P[-1] - P[-2]) / (12 * h ** 3)
    to_np = lambda M: np.array([[float(M[i, j]) for j in range(N)] for i in range(N)])
    assert o.rel_frobenius(r["P2"][0], to_np(c2)) < 1e-10
    assert o.rel_frobenius(r["P3"][0], to_np(c3)) < 1e-10
    assert abs(float((mu[1] - 2 * mu[0] + mu[-1]) / (2 * h ** 2)) - r["mu2"][0]) < 1e-10
    assert abs(float((mu[2] - 2 * mu[1] + 2 * mu[-1] - mu[-2]) / (12 * h ** 3))
               - r["mu3"][0]) < 1e-10


def test_n_plus_one_rule_with_higher_perturbation_terms():
    """Eq. Resp_0 in general: Omega^(3) = (1/3)(Tr[H1 P2] + 2 Tr[H2 P1]) and
    Omega^(4) = (1/4)(Tr[H1 P3] + 2 Tr[H2 P2] + 3 Tr[H3 P1]), against the third and fourth
    derivatives of the canonical free energy of H(lambda) (Fermi-Dirac)."""
    H0, H1, H2, H3 = _higher_case(10, 8)
    beta, nocc, h = 3.0, 4.0, 2e-2
    r = o.response3(H0, H1[None], beta, nocc, kind="fd", H2=H2[None], H3=H3[None])

    def omega(lam):
        H = H0 + lam * H1 + lam ** 2 * H2 + lam ** 3 * H3
        return o.solve(H, H1, beta, nocc, kind="fd")["omega"]
    w = {k: omega(k * h) for k in (-3, -2, -1, 0, 1, 2, 3)}
    d3 = (-w[3] + 8 * w[2] - 13 * w[1] + 13 * w[-1] - 8 * w[-2] + w[-3]) / (8 * h ** 3)
    d4 = (-w[3] + 12 * w[2] - 39 * w[1] + 56 * w[0] - 39 * w[-1] + 12 * w[-2] - w[-3]) / (
        6 * h ** 4)
    assert abs(d3 / 6.0 - r["omega3"][0]) < 1e-5 * abs(r["omega3"][0])
    assert abs(d4 / 24.0 - r["omega4"][0]) < 1e-3 * abs(r["omega4"][0])


@pytest.mark.parametrize("kind,n", [("fd", None), ("rec", 10)])
def test_scc_D2_equals_finite_difference_of_self_consistent_D(kind, n):
    """D2 = (1/2) d^2 D / d lambda^2 of the self-consistent solution of h + lambda h1."""
    hc, h1, S, gamma, q0, beta, nocc, _ = _scc_case()
    h = 1e-3
    r = o.scc_solve(hc, h1, S, gamma, q0, beta, nocc, n=n, kind=kind, order=2)
    D = {k: o.scc_solve(hc + k * h * h1, h1, S, gamma, q0, beta, nocc, n=n, kind=kind)["D0"]
         for k in (-2, -1, 0, 1, 2)}
    fd = (-D[-2] + 16 * D[-1] - 30 * D[0] + 16 * D[1] - D[2]) / (12 * h * h)
    assert o.rel_frobenius(r["D2"][0], 0.5 * fd) < 1e-6


def test_scc_free_energy_third_order_rule():
    """Eq. Resp_Omega at m = 3: Omega_SCF^(3) = (2/3) Tr[h1 D2] = (1/6) d^3 Omega_SCF /
    dlambda^3 at self-consistency (Fermi-Dirac), six-point differences of the free energy."""
    hc, h1, S, gamma, q0, beta, nocc, _ = _scc_case()
    h = 1e-2
    r = o.scc_solve(hc, h1, S, gamma, q0, beta, nocc, kind="fd", order=2)
    w = {k: o.scc_solve(hc + k * h * h1, h1, S, gamma, q0, beta, nocc, kind="fd")["omega"]
         for k in (-3, -2, -1, 1, 2, 3)}
    d3 = (-w[3] + 8 * w[2] - 13 * w[1] + 13 * w[-1] - 8 * w[-2] + w[-3]) / (8 * h ** 3)
    assert abs(d3 / 6.0 - r["omega3"][0]) < 1e-4 * abs(r["omega3"][0])
