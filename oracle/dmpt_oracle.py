"""FP64 CPU oracle for canonical density matrix perturbation theory.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this module:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it. It shares no code with the CUDA library.

What it computes (Niklasson, Rubensson, Rudberg, Cawkwell, "Canonical density
matrix perturbation theory"):

* P0, the finite-temperature density matrix of an orthogonal Hamiltonian H0,
  Eq. (Rec_F_1): P0 = [exp(beta (H0 - mu I)) + I]^-1, with mu fixed by the
  canonical condition Tr P0 = N_occ (Sec. II, text after Eq. Rec_F_2).
* P1, its first-order canonical response to H(lambda) = H0 + lambda H1
  (Eqs. P_resp, H_prt), with the first-order chemical potential mu1 chosen so
  that Tr P1 = 0 (Sec. II, condition after Eq. P_resp).
* The free energy Omega = Tr[P H] - T_e S[P] (Eqs. FreeE, SED, k_B = 1) and
  the polarizability alpha = -2 Tr[P1 H1], i.e. -4 Omega^(2) by the n+1 rule
  (Eq. Resp_0 with H^(2) = 0).

Two reference functions are provided, both evaluated exactly in the
eigenbasis of H0 (LAPACK ``dsyevd`` via ``numpy.linalg.eigh``):

* ``kind="fd"``: the Fermi-Dirac function itself, Eq. (Rec_F_1).
* ``kind="rec"``: the function that the recursion of Eq. (Rec_F_2) applies
  exactly after M steps. Appendix A shows the M-fold composition of
  f_2(x) = x^2 / (x^2 + (1-x)^2) equals f_{2^M}(x) = x^(2^M) / (x^(2^M) +
  (1-x)^(2^M)). With x = 1/2 + z/2 this is 1/2 [1 + tanh(2^M atanh z)], and
  X0 of Eq. (Rec_F_2) gives z0 = -beta (eps - mu) / 2^(M+1).

The response uses the Daleckii-Krein divided-difference formula: in the
eigenbasis, (P1)_ij = f[eps_i, eps_j] (h_ij - mu1 delta_ij) with h = V^T H1 V,
and mu1 = sum_i f'_i h_ii / sum_i f'_i from Tr P1 = 0.

Higher orders use the higher Daleckii-Krein formulas: the second order
(``response2``) sums third divided differences f[e_i, e_k, e_j], the third
order (``response3``) fourth divided differences f[e_i, e_k, e_l, e_j], with
the canonical shifts mu2 and mu3 from Tr P2 = Tr P3 = 0 (Algorithm 1), and
the free-energy terms Omega^(3) = Tr[H1 P2]/3 and Omega^(4) = Tr[H1 P3]/4 of
Eq. (Resp_0).

``series_recursion`` evaluates the recursion of Eq. (Rec_F_2) itself on
truncated power series in lambda (every product and inverse in the ring of
matrix polynomials), so its Taylor coefficients are the response orders of
Eq. (P_resp) computed without eigenvalues; ``canonical_newton`` adds the
Newton steps of Eq. (NewtRaphs) on mu and mu1. They pin the closed forms above
against the iteration of the map.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np

LN2 = math.log(2.0)


# ----------------------------------------------------------------------------
# scalar building blocks
# ----------------------------------------------------------------------------

def logcosh(x):
    """log cosh(x) without overflow."""
    a = np.abs(x)
    return a + np.log1p(np.exp(-2.0 * a)) - LN2


def log_sinhc(y):
    """log(sinh(y)/y) for real y (even function, 0 at y = 0)."""
    a = np.abs(np.asarray(y, dtype=np.float64))
    out = np.empty_like(a)
    small = a < 1e-2
    s = a[small]
    # series of log(sinh(y)/y) = y^2/6 - y^4/180 + y^6/2835
    out[small] = s * s / 6.0 - s ** 4 / 180.0 + s ** 6 / 2835.0
    b = a[~small]
    out[~small] = b + np.log1p(-np.exp(-2.0 * b)) - LN2 - np.log(b)
    return out


def atanhc(w):
    """atanh(w)/w for |w| < 1 (1 at w = 0)."""
    w = np.asarray(w, dtype=np.float64)
    out = np.empty_like(w)
    small = np.abs(w) < 1e-3
    s = w[small]
    out[small] = 1.0 + s * s / 3.0 + s ** 4 / 5.0
    b = w[~small]
    out[~small] = np.arctanh(b) / b
    return out


def z0_of(eps, mu, beta, n):
    """z0 = 2 x0 - 1 = -beta (eps - mu) / 2^(n+1), from X0 of Eq. (Rec_F_2)."""
    return -beta * (np.asarray(eps) - mu) / 2.0 ** (n + 1)


# ----------------------------------------------------------------------------
# occupation functions (eigenvalue -> occupation)
# ----------------------------------------------------------------------------

def occupation(eps, mu, beta, n: Optional[int] = None):
    """Occupation of levels eps.

    n is None: Fermi-Dirac 1/(exp(beta (eps - mu)) + 1), Eq. (Rec_F_1).
    n given:   the closed form of n steps of Eq. (Rec_F_2) (Appendix A),
               1/2 [1 + tanh(2^n atanh z0)].
    """
    eps = np.asarray(eps, dtype=np.float64)
    if n is None:
        return 0.5 * (1.0 - np.tanh(0.5 * beta * (eps - mu)))
    z0 = z0_of(eps, mu, beta, n)
    if np.any(np.abs(z0) >= 1.0):
        raise ValueError("|z0| >= 1: beta * spread too large for this number of steps")
    return 0.5 * (1.0 + np.tanh(2.0 ** n * np.arctanh(z0)))


def occupation_derivative(eps, mu, beta, n: Optional[int] = None):
    """d occupation / d eps.

    Fermi-Dirac: -beta f (1 - f). Recursion (n steps): -beta g (1 - g) / (1 - z0^2),
    the chain rule through atanh of the closed form.
    """
    f = occupation(eps, mu, beta, n)
    d = -beta * f * (1.0 - f)
    if n is not None:
        z0 = z0_of(eps, mu, beta, n)
        d = d / (1.0 - z0 * z0)
    return d


def divided_differences(eps, mu, beta, n: Optional[int] = None):
    """Matrix F_ij = (f(e_i) - f(e_j)) / (e_i - e_j), with F_ii = f'(e_i).

    Evaluated in closed form, never as a raw quotient, so that degenerate and
    nearly degenerate levels are exact:

    * Fermi-Dirac, x = beta (e - mu)/2:  tanh(x_a) - tanh(x_b) =
      sinh(x_a - x_b) / (cosh x_a cosh x_b), hence
      F = -(beta/4) sinhc(y) sech(x_a) sech(x_b),  y = beta (a - b)/2.
    * Recursion, u = 2^n atanh(z):  with w = (z_a - z_b)/(1 - z_a z_b),
      u_a - u_b = 2^n atanh(w), hence
      F = -(beta/4) sinhc(u_a - u_b) atanhc(w) / (1 - z_a z_b) sech(u_a) sech(u_b).
    """
    e = np.asarray(eps, dtype=np.float64)
    a = e[:, None]
    b = e[None, :]
    if n is None:
        xa = 0.5 * beta * (a - mu)
        xb = 0.5 * beta * (b - mu)
        y = 0.5 * beta * (a - b)
        logv = log_sinhc(y) - logcosh(xa) - logcosh(xb)
        return -0.25 * beta * np.exp(logv)
    za = z0_of(a, mu, beta, n)
    zb = z0_of(b, mu, beta, n)
    ua = 2.0 ** n * np.arctanh(za)
    ub = 2.0 ** n * np.arctanh(zb)
    den = 1.0 - za * zb
    w = (za - zb) / den
    du = 2.0 ** n * np.arctanh(w)
    logv = log_sinhc(du) - logcosh(ua) - logcosh(ub)
    return -0.25 * beta * atanhc(w) / den * np.exp(logv)


# ----------------------------------------------------------------------------
# chemical potential
# ----------------------------------------------------------------------------

def mu_bracket(eps, beta, n: Optional[int] = None):
    lo, hi = float(np.min(eps)), float(np.max(eps))
    if n is None:
        pad = 40.0 / beta
    else:
        # keep |z0| < 1 over the whole spectrum for every mu in the bracket
        room = 2.0 ** (n + 1) / beta - (hi - lo)
        if room <= 0:
            raise ValueError("beta * spectral width exceeds 2^(n+1): X0 leaves [0, 1]")
        pad = min(40.0 / beta, 0.49 * room)
    return lo - pad, hi + pad


def find_mu(eps, nocc, beta, n: Optional[int] = None, iters: int = 200):
    """mu with sum_i occupation(e_i) = nocc, by bisection (Tr P0 rises with mu)."""
    lo, hi = mu_bracket(eps, beta, n)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        if np.sum(occupation(eps, mid, beta, n)) > nocc:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


# ----------------------------------------------------------------------------
# free energy, Eqs. (FreeE), (SED)
# ----------------------------------------------------------------------------

def free_energy_levels(eps, occ, beta):
    """Omega = sum_i occ_i eps_i + (1/beta) sum_i [occ ln occ + (1-occ) ln(1-occ)]."""
    occ = np.asarray(occ, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = np.where(occ > 0, occ * np.log(np.where(occ > 0, occ, 1.0)), 0.0)
        t2 = np.where(occ < 1, (1 - occ) * np.log1p(-np.where(occ < 1, occ, 0.0)), 0.0)
    return float(np.sum(occ * eps) + (t1 + t2).sum() / beta)


# ----------------------------------------------------------------------------
# full reference solve
# ----------------------------------------------------------------------------

def solve(H0, H1, beta, nocc, n: Optional[int] = None, kind: str = "rec",
          canonical: bool = True, mu: Optional[float] = None, eig=None):
    """Exact P0, P1, mu, mu1, alpha and Omega.

    H0: (N, N) symmetric. H1: (D, N, N) or (N, N) symmetric; P1 is always
    returned as (D, N, N). kind "rec" uses
    the n-step recursion function (requires n), "fd" the Fermi-Dirac function.
    canonical=False keeps mu1 = 0 (grand-canonical response). mu may be given
    to skip the occupation search. eig = (eps, V) reuses an eigendecomposition
    of H0 computed by ``numpy.linalg.eigh``.
    """
    H0 = np.asarray(H0, dtype=np.float64)
    H1 = np.asarray(H1, dtype=np.float64)
    if H1.ndim == 2:
        H1 = H1[None]
    nn = n if kind == "rec" else None
    if kind == "rec" and n is None:
        raise ValueError("kind='rec' needs n")
    eps, V = np.linalg.eigh(H0) if eig is None else eig
    if mu is None:
        mu = find_mu(eps, nocc, beta, nn)
    occ = occupation(eps, mu, beta, nn)
    P0 = (V * occ) @ V.T
    F = divided_differences(eps, mu, beta, nn)
    fprime = np.diag(F).copy()
    P1 = np.empty_like(H1)
    mu1 = np.zeros(H1.shape[0])
    alpha = np.zeros(H1.shape[0])
    for d in range(H1.shape[0]):
        h = V.T @ H1[d] @ V
        if canonical:
            mu1[d] = float(np.dot(fprime, np.diag(h)) / np.sum(fprime))
        he = h - mu1[d] * np.eye(h.shape[0])
        P1[d] = V @ (F * he) @ V.T
        alpha[d] = -2.0 * float(np.sum(P1[d] * H1[d]))
    # Q = dP0/dmu (exact for the chosen function): V diag(-f') V^T
    Q = (V * (-fprime)) @ V.T
    out = dict(P0=P0, P1=P1, mu=float(mu), mu1=mu1, alpha=alpha, eps=eps, occ=occ,
               Q=Q, omega=free_energy_levels(eps, occ, beta))
    return out


def rel_frobenius(A, B):
    """||A - B||_F / ||B||_F (the error measure used for every parity check)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    nb = np.linalg.norm(B)
    return float(np.linalg.norm(A - B) / (nb if nb > 0 else 1.0))


# ----------------------------------------------------------------------------
# the recursion of Eq. (Rec_F_2) on truncated power series in lambda
# ----------------------------------------------------------------------------

def _series_mul(A, B):
    """Cauchy product of two matrix power series in lambda, truncated to len(A) terms."""
    return [sum(A[i] @ B[k - i] for i in range(k + 1)) for k in range(len(A))]


def _series_inv(A):
    """Inverse of a matrix power series with invertible A[0]: B[0] = A[0]^-1 and
    A[0] B[k] = -sum_{j=1..k} A[j] B[k-j], from the coefficients of A(lambda) B(lambda) = I."""
    B = [np.linalg.inv(A[0])]
    for k in range(1, len(A)):
        B.append(-np.linalg.solve(A[0], sum(A[j] @ B[k - j] for j in range(1, k + 1))))
    return B


def series_recursion(Hs, beta, mus, M):
    """X_M(lambda) of Eq. (Rec_F_2) as a truncated power series in lambda.

    H(lambda) = sum_k lambda^k Hs[k] (Eq. H_prt) and mu(lambda) = sum_k lambda^k mus[k];
    X_0(lambda) = I/2 - 2^-(M+2) beta (H(lambda) - mu(lambda) I), then M applications of the
    map X -> X^2 [X^2 + (I - X)^2]^-1, every product and inverse taken in the ring of matrix
    polynomials in lambda truncated after lambda^m, m = len(Hs) - 1. Coefficient k of X_M is
    the k-th order density matrix response P^(k) of Eq. (P_resp) at the given mu^(k). This is
    a direct evaluation of the Taylor coefficients of the map, independent of how Algorithm 1
    arranges them. Hs[k] or mus[k] may be 0 (zero term).

    Returns (list of the m + 1 coefficients of X_M, spectral condition numbers of the
    order-0 denominator X^2 + (I - X)^2 at each application).
    """
    H0 = np.asarray(Hs[0], dtype=np.float64)
    N = H0.shape[0]
    I = np.eye(N)
    s = 2.0 ** (-(M + 2)) * beta
    X = []
    for k, Hk in enumerate(Hs):
        Hk = np.zeros((N, N)) if (np.isscalar(Hk) and Hk == 0) else np.asarray(Hk, dtype=np.float64)
        term = -s * (Hk - float(mus[k]) * I)
        X.append(0.5 * I + term if k == 0 else term)
    conds = []
    for _ in range(M):
        X2 = _series_mul(X, X)
        IX = [I - X[0]] + [-x for x in X[1:]]
        den = [a + b for a, b in zip(X2, _series_mul(IX, IX))]
        ev = np.linalg.eigvalsh(0.5 * (den[0] + den[0].T))
        conds.append(float(ev[-1] / ev[0]))
        X = _series_mul(X2, _series_inv(den))
    return X, conds


def canonical_newton(H0, H1, beta, nocc, M, mu0=0.0, tol=1e-9, maxit=100):
    """mu and mu1 of the canonical conditions Tr P0 = N_occ and Tr P1 = 0 by Newton steps
    with the slope of Eq. (NewtRaphs), Tr P_mu = beta Tr[P0 (I - P0)] (exact only as
    M -> infinity), on the series evaluation of Eq. (Rec_F_2):
      mu  <- mu  + (N_occ - Tr P0) / Tr P_mu,   mu1 <- mu1 - Tr P1 / Tr P_mu,
    until |Tr P0 - N_occ| + |Tr P1| <= tol. Returns (P0, P1, mu, mu1, iterations); raises
    RuntimeError when maxit steps do not get there.
    """
    mu, mu1 = float(mu0), 0.0
    for it in range(maxit):
        X, _ = series_recursion([H0, H1], beta, [mu, mu1], M)
        P0, P1 = X[0], X[1]
        tr0, tr1 = np.trace(P0), np.trace(P1)
        if abs(tr0 - nocc) + abs(tr1) <= tol:
            return P0, P1, mu, mu1, it
        slope = beta * np.trace(P0 @ (np.eye(P0.shape[0]) - P0))
        mu = mu + (nocc - tr0) / slope
        mu1 = mu1 - tr1 / slope
    raise RuntimeError("canonical Newton iteration did not converge")


def pade_f(x, m):
    """f_m(x) = x^m / (x^m + (1 - x)^m), Appendix A."""
    return x ** m / (x ** m + (1.0 - x) ** m)


def entropy_coefficients():
    """Table 1 (Eq. S_Approx) coefficients c_i(m) for m = 1, 2, 4, as printed."""
    return {
        1: [4 * LN2],
        2: [8 * LN2 - 2, 16 * LN2 - 8],
        4: [16 * LN2 - 34 / 5, 96 * LN2 - 844 / 15, 256 * LN2 - 2336 / 15, 256 * LN2 - 2368 / 15],
    }


# ----------------------------------------------------------------------------
# second order: P2 = (1/2) d^2 P / d lambda^2 (Algorithm 1, order 2, with
# H^(2) = 0) and the polarizability gradient d alpha / d H0 = -4 P2
# ----------------------------------------------------------------------------

def occupation_second_derivative(eps, mu, beta, n: Optional[int] = None):
    """d^2 occupation / d eps^2.

    Fermi-Dirac, x = beta (e - mu)/2, t = tanh x:  (beta^2/4) t (1 - t^2).
    Recursion (n steps), z = z0(e), T = tanh(2^n atanh z), s = beta / 2^(n+1):
    2^n s^2 (1 - T^2) (z - 2^n T) / (1 - z^2)^2 (the derivative of
    -beta/4 (1 - T^2) / (1 - z^2) through the closed form).
    """
    eps = np.asarray(eps, dtype=np.float64)
    if n is None:
        t = np.tanh(0.5 * beta * (eps - mu))
        return 0.25 * beta * beta * t * (1.0 - t * t)
    z = z0_of(eps, mu, beta, n)
    m = 2.0 ** n
    t = np.tanh(m * np.arctanh(z))
    s = beta / 2.0 ** (n + 1)
    return m * s * s * (1.0 - t * t) * (z - m * t) / (1.0 - z * z) ** 2


_GL_X, _GL_W = np.polynomial.legendre.leggauss(8)
_GL_X = 0.5 * (_GL_X + 1.0)
_GL_W = 0.5 * _GL_W


def second_dd_quadrature(a, b, c, mu, beta, n: Optional[int] = None):
    """f[a, b, c] as the Hermite-Genocchi integral of f'' over the 2-simplex,
    a + t1 (b - a) + t2 (c - a), t1, t2 >= 0, t1 + t2 <= 1, after the collapse
    t1 = x, t2 = (1 - x) y (Jacobian 1 - x), with an 8 x 8 Gauss-Legendre rule.
    Exact to rounding when beta * spread <= 1 (the nearest poles of f lie
    pi / beta off the real axis)."""
    a = np.asarray(a, dtype=np.float64)[..., None, None]
    b = np.asarray(b, dtype=np.float64)[..., None, None]
    c = np.asarray(c, dtype=np.float64)[..., None, None]
    x = _GL_X[:, None]
    y = _GL_X[None, :]
    pts = a + x * (b - a) + (1.0 - x) * y * (c - a)
    w = _GL_W[:, None] * _GL_W[None, :] * (1.0 - x)
    return np.sum(occupation_second_derivative(pts, mu, beta, n) * w, axis=(-2, -1))


def _second_dd_for_pairs(I, J, eps, F, mu, beta, n, quad):
    """f[e_i, e_k, e_j] for the pairs (i, j) = (I[p], J[p]) and every k: (len(I), N).

    f[x, y, z] = (f[x, y] - f[y, z]) / (x - z) is taken across the widest of the
    three pairs; triples whose whole spread is within quad / beta (where that
    quotient would cancel) use the quadrature instead.
    """
    a = eps[I][:, None]
    c = eps[J][:, None]
    b = eps[None, :]
    fac = F[I, J][:, None]                     # f[a, c]
    fab = F[I, :]                              # f[a, b]
    fcb = F[J, :]                              # f[c, b]
    dab = a - b
    dcb = c - b
    spread = np.maximum(np.maximum(np.abs(dab), np.abs(dcb)), np.abs(a - c))
    out = np.empty(dab.shape)
    use_ab = np.abs(dab) >= np.abs(dcb)        # widest pair (a, b): middle c
    with np.errstate(divide="ignore", invalid="ignore"):
        v_ab = (fac - fcb) / dab               # f[a, c, b]
        v_cb = (fac - fab) / dcb               # f[c, a, b]
    out[:] = np.where(use_ab, v_ab, v_cb)
    near = spread * beta <= quad
    if np.any(near):
        pi, kk = np.nonzero(near)
        out[pi, kk] = second_dd_quadrature(eps[I[pi]], eps[kk], eps[J[pi]], mu, beta, n)
    return out


def _dk2_matrix(ht, eps, F, mu, beta, n, close, quad, batch, b=None):
    """S_ij = sum_k f[e_i, e_k, e_j] ht_ik b_kj (b = ht if None), the second-order
    Daleckii-Krein sum.

    For pairs with beta |e_i - e_j| > close it is the exact identity
    [(F o ht) b - ht (F o b)]_ij / (e_i - e_j); closer pairs are summed
    explicitly with ``_second_dd_for_pairs``.
    """
    if b is None:
        b = ht
    diff = eps[:, None] - eps[None, :]
    ci, cj = np.nonzero(np.abs(diff) * beta <= close)
    with np.errstate(divide="ignore", invalid="ignore"):
        S = ((F * ht) @ b - ht @ (F * b)) / diff
    for s0 in range(0, ci.shape[0], batch):
        I = ci[s0:s0 + batch]
        J = cj[s0:s0 + batch]
        F3 = _second_dd_for_pairs(I, J, eps, F, mu, beta, n, quad)
        S[I, J] = np.sum(F3 * ht[I, :] * b[:, J].T, axis=1)
    return S


def response2(H0, H1, beta, nocc, n: Optional[int] = None, kind: str = "rec", eig=None,
              close: float = 1.0, quad: float = 1.0, batch: int = 1024, canonical: bool = True,
              mu: Optional[float] = None, H2=None):
    """Second-order canonical response P2 = (1/2) d^2 P / d lambda^2 of P(H0 + lambda H1).

    Second-order Daleckii-Krein formula in the eigenbasis of H0, with
    ht = h - mu1 I (h = V^T H1 V, mu1 the first-order canonical shift):
      (P2)_ij = sum_k f[e_i, e_k, e_j] ht_ik ht_kj - mu2 f'_i delta_ij,
    and mu2 = sum_i (P2)_ii|_{mu2=0} / sum_i f'_i from Tr P2 = 0 (the second-
    order canonical condition of Algorithm 1). For pairs with beta |e_i - e_j|
    > close the sum over k is the exact identity
      [(F o ht) ht - ht (F o ht)]_ij / (e_i - e_j),
    F the first divided differences; closer pairs are summed explicitly, with
    the quadrature for triples of spread <= quad / beta.
    Returns the first-order results of ``solve`` plus P2 (D, N, N), mu2 (D,),
    grad_alpha = -4 P2 (d alpha_d / d H0, by the symmetry of the third
    derivatives of the canonical free energy, whose gradient is P0) and
    omega3 (D,) = (1/3) Tr[H1 P2], the third-order free-energy term of
    Eq. (Resp_0) (the n+1 rule: P^(2) suffices for Omega^(3)).
    canonical=False keeps mu fixed (given by ``mu``, else found from nocc):
    mu1 = mu2 = 0, the grand-canonical response.
    H2 (D, N, N), optional: a second-order term of the perturbation, H(lambda) = H0 +
    lambda H1 + lambda^2 H2 (Eq. H_prt); it adds sum f[e_i, e_j] (h2)_ij, and Omega^(3)
    becomes (1/3)(Tr[H1 P2] + 2 Tr[H2 P1]) (Eq. Resp_0). grad_alpha is the gradient of
    alpha = -2 Tr[P1 H1] and does not involve H2.
    """
    H0 = np.asarray(H0, dtype=np.float64)
    H1 = np.asarray(H1, dtype=np.float64)
    if H1.ndim == 2:
        H1 = H1[None]
    nn = n if kind == "rec" else None
    eps, V = np.linalg.eigh(H0) if eig is None else eig
    base = solve(H0, H1, beta, nocc, n, kind, canonical=canonical, mu=mu, eig=(eps, V))
    mu = base["mu"]
    F = divided_differences(eps, mu, beta, nn)
    fp = np.diag(F).copy()
    N = eps.shape[0]
    P2 = np.empty_like(H1)
    mu2 = np.zeros(H1.shape[0])
    grad = np.empty_like(H1)
    for d in range(H1.shape[0]):
        ht = V.T @ H1[d] @ V - base["mu1"][d] * np.eye(N)
        S = _dk2_matrix(ht, eps, F, mu, beta, nn, close, quad, batch)
        # d alpha / d H0 = -4 P2 of H1 alone (mu2 from Tr = 0 for that part)
        m0 = float(np.trace(S) / np.sum(fp)) if canonical else 0.0
        grad[d] = -4.0 * V @ (S - m0 * np.diag(fp)) @ V.T
        if H2 is not None:
            S = S + F * (V.T @ H2[d] @ V)
        mu2[d] = float(np.trace(S) / np.sum(fp)) if canonical else 0.0
        P2[d] = V @ (S - mu2[d] * np.diag(fp)) @ V.T
    out = dict(base)
    # Eq. (Resp_0): Omega^(3) = (1/3)(Tr[H1 P2] + 2 Tr[H2 P1] + 3 Tr[H3 P0]), H3 = 0 here
    omega3 = np.array([(np.sum(H1[d] * P2[d])
                        + (2.0 * np.sum(H2[d] * base["P1"][d]) if H2 is not None else 0.0)) / 3.0
                       for d in range(H1.shape[0])])
    out.update(P2=P2, mu2=mu2, grad_alpha=grad, omega3=omega3)
    return out


# ----------------------------------------------------------------------------
# third order: P3 = (1/6) d^3 P / d lambda^3 (Algorithm 1, order 3, with
# H^(2) = H^(3) = 0) and Omega^(4) = (1/4) Tr[H1 P3] (Eq. Resp_0)
# ----------------------------------------------------------------------------

def occupation_third_derivative(eps, mu, beta, n: Optional[int] = None):
    """d^3 occupation / d eps^3.

    Fermi-Dirac, x = beta (e - mu)/2, t = tanh x: (beta^3/8) (1 - t^2)(1 - 3 t^2).
    Recursion (n steps): g = (1 + tanh u)/2 with u = 2^n atanh z(e), z linear in e
    with slope -c (c = beta / 2^(n+1)). With t = tanh u, S = 1 - t^2 and
    u' = -2^n c / (1 - z^2), u'' = 2^(n+1) c^2 z / (1 - z^2)^2,
    u''' = -2^(n+1) c^3 (1 + 3 z^2) / (1 - z^2)^3, the chain rule gives
    g''' = S/2 [u''' - 6 t u' u'' + (6 t^2 - 2) u'^3].
    """
    eps = np.asarray(eps, dtype=np.float64)
    if n is None:
        t = np.tanh(0.5 * beta * (eps - mu))
        return beta ** 3 / 8.0 * (1.0 - t * t) * (1.0 - 3.0 * t * t)
    z = z0_of(eps, mu, beta, n)
    m = 2.0 ** n
    c = beta / 2.0 ** (n + 1)
    t = np.tanh(m * np.arctanh(z))
    S = 1.0 - t * t
    q = 1.0 - z * z
    u1 = -m * c / q
    u2 = 2.0 * m * c * c * z / q ** 2
    u3 = -2.0 * m * c ** 3 * (1.0 + 3.0 * z * z) / q ** 3
    return 0.5 * S * (u3 - 6.0 * t * u1 * u2 + (6.0 * t * t - 2.0) * u1 ** 3)


def third_dd_quadrature(a, b, c, d, mu, beta, n: Optional[int] = None):
    """f[a, b, c, d] as the Hermite-Genocchi integral of f''' over the 3-simplex,
    a + t1 (b - a) + t2 (c - a) + t3 (d - a), after the collapse t1 = x,
    t2 = (1 - x) y, t3 = (1 - x)(1 - y) z (Jacobian (1 - x)^2 (1 - y)), with an
    8 x 8 x 8 Gauss-Legendre rule. For clustered points (beta * spread <= 1)."""
    a = np.asarray(a, dtype=np.float64)[..., None, None, None]
    b = np.asarray(b, dtype=np.float64)[..., None, None, None]
    c = np.asarray(c, dtype=np.float64)[..., None, None, None]
    d = np.asarray(d, dtype=np.float64)[..., None, None, None]
    x = _GL_X[:, None, None]
    y = _GL_X[None, :, None]
    z = _GL_X[None, None, :]
    t1 = x
    t2 = (1.0 - x) * y
    t3 = (1.0 - x) * (1.0 - y) * z
    pts = a + t1 * (b - a) + t2 * (c - a) + t3 * (d - a)
    w = (_GL_W[:, None, None] * _GL_W[None, :, None] * _GL_W[None, None, :]
         * (1.0 - x) ** 2 * (1.0 - y))
    return np.sum(occupation_third_derivative(pts, mu, beta, n) * w, axis=(-3, -2, -1))


def _dd3_idx(p, q, r, eps, F, mu, beta, n, quad):
    """f[e_p, e_q, e_r] for broadcastable index arrays p, q, r.

    The quotient f[x, y, z] = (f[y, z] - f[x, y]) / (z - x) is taken across the
    widest of the three pairs (any order of the points gives the same value);
    triples whose spread is within quad / beta use ``second_dd_quadrature``.
    """
    p, q, r = np.broadcast_arrays(np.asarray(p), np.asarray(q), np.asarray(r))
    ep, eq, er = eps[p], eps[q], eps[r]
    dpq, dqr, dpr = np.abs(ep - eq), np.abs(eq - er), np.abs(ep - er)
    with np.errstate(divide="ignore", invalid="ignore"):
        v_pr = (F[q, r] - F[p, q]) / (er - ep)      # outer p, r; middle q
        v_pq = (F[r, q] - F[p, r]) / (eq - ep)      # outer p, q; middle r
        v_qr = (F[p, r] - F[q, p]) / (er - eq)      # outer q, r; middle p
    out = np.where((dpr >= dpq) & (dpr >= dqr), v_pr, np.where(dpq >= dqr, v_pq, v_qr))
    spread = np.maximum(np.maximum(dpq, dqr), dpr)
    near = spread * beta <= quad
    if np.any(near):
        out = np.array(out, dtype=np.float64)
        out[near] = second_dd_quadrature(ep[near], eq[near], er[near], mu, beta, n)
    return out


def _dd4_idx(i, k, l, j, eps, F, mu, beta, n, quad):
    """f[e_i, e_k, e_l, e_j] for broadcastable index arrays.

    With (s, t) the widest pair of the four points and (u, v) the other two,
    f = (f[u, v, t] - f[s, u, v]) / (e_t - e_s); quadruples whose spread is
    within quad / beta use ``third_dd_quadrature``.
    """
    idx = np.broadcast_arrays(np.asarray(i), np.asarray(k), np.asarray(l), np.asarray(j))
    e = [eps[x] for x in idx]
    pairs = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    dist = np.stack([np.abs(e[a] - e[b]) for a, b in pairs])
    widest = np.argmax(dist, axis=0)
    spread = np.max(dist, axis=0)
    out = np.zeros(idx[0].shape)
    for w, (a, b) in enumerate(pairs):
        sel = widest == w
        if not np.any(sel):
            continue
        u, v = [x for x in range(4) if x not in (a, b)]
        sa, sb, su, sv = idx[a][sel], idx[b][sel], idx[u][sel], idx[v][sel]
        with np.errstate(divide="ignore", invalid="ignore"):
            out[sel] = ((_dd3_idx(su, sv, sb, eps, F, mu, beta, n, quad)
                         - _dd3_idx(sa, su, sv, eps, F, mu, beta, n, quad))
                        / (eps[sb] - eps[sa]))
    near = spread * beta <= quad
    if np.any(near):
        out[near] = third_dd_quadrature(e[0][near], e[1][near], e[2][near], e[3][near],
                                        mu, beta, n)
    return out


def response3(H0, H1, beta, nocc, n: Optional[int] = None, kind: str = "rec", eig=None,
              close: float = 1.0, quad: float = 1.0, batch: int = 1024, canonical: bool = True,
              mu: Optional[float] = None, H2=None, H3=None):
    """Third-order canonical response P3 = (1/6) d^3 P / d lambda^3 of P(H0 + lambda H1).

    P(lambda) = f(H0 + lambda ht - lambda^2 mu2 I - lambda^3 mu3 I) with ht = H1 -
    mu1 I, so in the eigenbasis of H0 (g = V^T H1 V - mu1 I) the third-order
    Daleckii-Krein expansion reads
      (P3)_ij = sum_kl f[e_i, e_k, e_l, e_j] g_ik g_kl g_lj
                - mu2 (f[e_i, e_i, e_j] + f[e_i, e_j, e_j]) g_ij - mu3 f'_i delta_ij,
    with mu2 the second-order shift and mu3 = sum_i (P3)_ii|_{mu3=0} / sum_i f'_i
    from Tr P3 = 0 (the third-order canonical condition of Algorithm 1). For
    pairs with beta |e_i - e_j| > close the double sum is the exact identity
      [S2 g - g S2]_ij / (e_i - e_j),  S2_il = sum_k f[e_i, e_k, e_l] g_ik g_kl;
    closer pairs are summed explicitly over (k, l). Omega^(4) = (1/4) Tr[H1 P3]
    (Eq. Resp_0 with H^(1) = H1 only). Returns the results of ``response2`` plus
    P3 (D, N, N), mu3 (D,) and omega4 (D,). canonical=False: mu fixed, mu1 =
    mu2 = mu3 = 0.
    H2, H3 (D, N, N), optional: higher terms of the perturbation, H(lambda) = H0 +
    lambda H1 + lambda^2 H2 + lambda^3 H3 (Eq. H_prt). With h2 = V^T H2 V and h3 =
    V^T H3 V the mu2 cross term becomes sum_k f[e_i, e_k, e_j] (g_ik g2_kj + g2_ik g_kj)
    with g2 = h2 - mu2 I, the first-order term f[e_i, e_j] (h3)_ij is added, and
    Omega^(4) = (1/4)(Tr[H1 P3] + 2 Tr[H2 P2] + 3 Tr[H3 P1]) (Eq. Resp_0).
    """
    H0 = np.asarray(H0, dtype=np.float64)
    H1 = np.asarray(H1, dtype=np.float64)
    if H1.ndim == 2:
        H1 = H1[None]
    nn = n if kind == "rec" else None
    eps, V = np.linalg.eigh(H0) if eig is None else eig
    base = response2(H0, H1, beta, nocc, n, kind, eig=(eps, V), close=close, quad=quad,
                     batch=batch, canonical=canonical, mu=mu, H2=H2)
    mu = base["mu"]
    F = divided_differences(eps, mu, beta, nn)
    fp = np.diag(F).copy()
    N = eps.shape[0]
    diff = eps[:, None] - eps[None, :]
    ci, cj = np.nonzero(np.abs(diff) * beta <= close)
    ii, jj = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    # f[e_i, e_i, e_j] + f[e_i, e_j, e_j], the coefficient of the mu2 cross terms
    f_iij = (_dd3_idx(ii, ii, jj, eps, F, mu, beta, nn, quad)
             + _dd3_idx(ii, jj, jj, eps, F, mu, beta, nn, quad))
    kk, ll = ii, jj
    P3 = np.empty_like(H1)
    mu3 = np.zeros(H1.shape[0])
    for d in range(H1.shape[0]):
        g = V.T @ H1[d] @ V - base["mu1"][d] * np.eye(N)
        S2 = _dk2_matrix(g, eps, F, mu, beta, nn, close, quad, batch)
        with np.errstate(divide="ignore", invalid="ignore"):
            S = (S2 @ g - g @ S2) / diff
        for p in range(ci.shape[0]):
            i, j = ci[p], cj[p]
            f4 = _dd4_idx(i, kk, ll, j, eps, F, mu, beta, nn, quad)
            S[i, j] = np.sum(f4 * g[i, :][:, None] * g * g[:, j][None, :])
        S = S - base["mu2"][d] * f_iij * g
        if H2 is not None:
            h2 = V.T @ H2[d] @ V
            S = (S + _dk2_matrix(g, eps, F, mu, beta, nn, close, quad, batch, b=h2)
                 + _dk2_matrix(h2, eps, F, mu, beta, nn, close, quad, batch, b=g))
        if H3 is not None:
            S = S + F * (V.T @ H3[d] @ V)
        mu3[d] = float(np.trace(S) / np.sum(fp)) if canonical else 0.0
        P3[d] = V @ (S - mu3[d] * np.diag(fp)) @ V.T
    out = dict(base)
    if H3 is not None:   # Omega^(3) gains 3 Tr[H3 P0] / 3 (Eq. Resp_0)
        out["omega3"] = out["omega3"] + np.array([np.sum(H3[d] * base["P0"])
                                                  for d in range(H1.shape[0])])
    omega4 = np.array([(np.sum(H1[d] * P3[d])
                        + (2.0 * np.sum(H2[d] * base["P2"][d]) if H2 is not None else 0.0)
                        + (3.0 * np.sum(H3[d] * base["P1"][d]) if H3 is not None else 0.0)) / 4.0
                       for d in range(H1.shape[0])])
    out.update(P3=P3, mu3=mu3, omega4=omega4)
    return out


# ----------------------------------------------------------------------------
# the free energy Omega = Tr[P H0] - T_e S[P] (Eqs. FreeE, SED) as a loss of H0
# ----------------------------------------------------------------------------

def free_energy(H0, beta, nocc, n: Optional[int] = None, kind: str = "rec",
                canonical: bool = True, mu: Optional[float] = None, eig=None):
    """Omega(H0) = Tr[P H0] - (1/beta) S[P] at P = f(H0) and its gradient dOmega/dH0.

    P is the occupation function applied to H0 (the recursion's own function
    for kind="rec"). With u = ln(f / (1 - f)) per level (u = -beta (e - mu) for
    Fermi-Dirac, u = 2^(n+1) atanh z0 for the recursion), dOmega/dP = H0 +
    (1/beta) ln(P (I - P)^-1) has eigenvalues G_i = e_i + u_i / beta, and the
    chain rule through the canonical first-order response (Sec. II) gives
      dOmega/dH0 = V diag(f_i + f'_i (G_i - Gbar)) V^T,
    Gbar = sum_i f'_i G_i / sum_i f'_i (canonical; Gbar = 0 at fixed mu). For
    Fermi-Dirac G_i = mu, so the canonical gradient is P0 itself.
    Returns dict(omega, grad, mu, P0).
    """
    H0 = np.asarray(H0, dtype=np.float64)
    nn = n if kind == "rec" else None
    eps, V = np.linalg.eigh(H0) if eig is None else eig
    if mu is None:
        mu = find_mu(eps, nocc, beta, nn)
    occ = occupation(eps, mu, beta, nn)
    fp = occupation_derivative(eps, mu, beta, nn)
    if nn is None:
        u = -beta * (eps - mu)
    else:
        u = 2.0 ** (nn + 1) * np.arctanh(z0_of(eps, mu, beta, nn))
    G = eps + u / beta
    gbar = float(np.sum(fp * G) / np.sum(fp)) if canonical else 0.0
    grad = (V * (occ + fp * (G - gbar))) @ V.T
    return dict(omega=free_energy_levels(eps, occ, beta), grad=grad, mu=float(mu),
                P0=(V * occ) @ V.T)


# ----------------------------------------------------------------------------
# non-orthogonal basis (Sec. IV, Eq. Fermi_D): D = Z f(Z^T F Z) Z^T with Z^T S Z = I
# ----------------------------------------------------------------------------

def cholesky_factor(S):
    """Inverse Cholesky factor: Linv = L^-1 with S = L L^T, so Z = Linv^T satisfies
    Z^T S Z = I. (A different inverse factor than the Loewdin S^(-1/2) the library uses;
    D and every derivative mapped back to the non-orthogonal basis do not depend on the
    choice.)"""
    import scipy.linalg
    L = np.linalg.cholesky(np.asarray(S, dtype=np.float64))
    return scipy.linalg.solve_triangular(L, np.eye(L.shape[0]), lower=True)


def to_orthogonal(X, Linv):
    """X_perp = Z^T X Z = Linv X Linv^T (Hamiltonian-like matrices, Eq. Fermi_D)."""
    return Linv @ X @ Linv.T


def from_orthogonal(P, Linv):
    """D = Z P Z^T = Linv^T P Linv (density-like matrices and gradients with respect to F:
    F_perp = Z^T F Z gives dL/dF = Z (dL/dF_perp) Z^T)."""
    return Linv.T @ P @ Linv


def solve_nonorthogonal(F, h1, S, beta, nocc, n: Optional[int] = None, kind: str = "rec",
                        order: int = 1, canonical: bool = True, mu: Optional[float] = None):
    """Canonical DMPT in a non-orthogonal basis (Eq. Fermi_D with the perturbation h1 of
    Eq. FirstOrderPRT, no self-consistency): the orthogonal oracle applied to
    F_perp = Z^T F Z and h1_perp = Z^T h1 Z, results mapped back. Returns D0, D1 (D, N, N),
    mu, mu1, alpha (basis independent), omega, and for order >= 2 also D2, mu2 and
    grad_alpha = d alpha / dF (D, N, N); free-energy gradient dOmega/dF as grad_omega."""
    h1 = np.asarray(h1, dtype=np.float64)
    if h1.ndim == 2:
        h1 = h1[None]
    Linv = cholesky_factor(S)
    Fp = to_orthogonal(F, Linv)
    h1p = np.stack([to_orthogonal(h1[d], Linv) for d in range(h1.shape[0])])
    if order >= 2:
        r = response2(Fp, h1p, beta, nocc, n, kind, canonical=canonical, mu=mu)
    else:
        r = solve(Fp, h1p, beta, nocc, n, kind, canonical=canonical, mu=mu)
    fe = free_energy(Fp, beta, nocc, n, kind, canonical=canonical, mu=r["mu"] if not canonical
                     else None)
    out = dict(mu=r["mu"], mu1=r["mu1"], alpha=r["alpha"], omega=r["omega"], Linv=Linv,
               D0=from_orthogonal(r["P0"], Linv),
               D1=np.stack([from_orthogonal(p, Linv) for p in r["P1"]]),
               grad_omega=from_orthogonal(fe["grad"], Linv))
    if order >= 2:
        out.update(mu2=r["mu2"], D2=np.stack([from_orthogonal(p, Linv) for p in r["P2"]]),
                   grad_alpha=np.stack([from_orthogonal(g, Linv) for g in r["grad_alpha"]]))
    return out


# ----------------------------------------------------------------------------
# self-consistent charge layer (Sec. IV with a synthetic G(D)): F = h + G(D),
# G_ij = S_ij (V_i + V_j) / 2, V = gamma dq, dq_i = 2 (D S)_ii - q0_i
# ----------------------------------------------------------------------------

def scc_fock(hcore, S, gamma, dq):
    V = gamma @ dq
    return hcore + 0.5 * S * (V[:, None] + V[None, :])


def scc_charges(D, S, q0):
    return 2.0 * np.sum(D * S, axis=1) - q0


def scc_solve(hcore, h1, S, gamma, q0, beta, nocc, n: Optional[int] = None, kind: str = "rec",
              tol: float = 1e-13, maxit: int = 2000, mix: float = 0.3, order: int = 1):
    """Self-consistent canonical solve and its coupled-perturbed response.

    SCF: plain fixed-point iteration on the charges with linear mixing, each step the
    non-orthogonal solve of F(dq) (eigenvalues of the Cholesky-orthogonalised F). CPSCF:
    the response charges satisfy the linear system (I - K) dq1 = b, where b are the charges
    of R(h1) and column j of K the charges of R(G(e_j)), R the canonical first-order
    response of the converged solve; it is solved directly (LAPACK), then
    D1 = R(h1 + G(dq1)). Omega_SCF^(m) = (2/m) Tr[h1 D^(m-1)] (Eq. Resp_Omega).
    The free energy Omega_SCF = 2 Tr[h D] + 1/2 dq^T gamma dq - 2 T_e S[D_perp] (Eq.
    FreeE_tot for this model) is returned as omega.
    order=2 adds the second-order self-consistent response D2 = (1/2) d^2 D / d lambda^2:
    the canonical order-2 response to F^(1) = h1 + G(D1) and F^(2) = G(D2), a linear fixed
    point in its charges, (I - K) dq2 = b2 with the same K, and Omega_SCF^(3) =
    (2/3) Tr[h1 D2] (Eq. Resp_Omega).
    """
    h1 = np.asarray(h1, dtype=np.float64)
    if h1.ndim == 2:
        h1 = h1[None]
    nn = n if kind == "rec" else None
    N = hcore.shape[0]
    Linv = cholesky_factor(S)
    x = np.zeros(N)
    for it in range(maxit):
        F = scc_fock(hcore, S, gamma, x)
        eps, V = np.linalg.eigh(to_orthogonal(F, Linv))
        mu = find_mu(eps, nocc, beta, nn)
        occ = occupation(eps, mu, beta, nn)
        D = from_orthogonal((V * occ) @ V.T, Linv)
        y = scc_charges(D, S, q0)
        if np.max(np.abs(y - x)) < tol:
            break
        x = x + mix * (y - x)
    else:
        raise RuntimeError("oracle SCF did not converge")
    Fdd = divided_differences(eps, mu, beta, nn)
    fp = np.diag(Fdd)

    def response(dF):
        """Canonical first-order response of D to dF (non-orthogonal), with its mu1."""
        h = V.T @ to_orthogonal(dF, Linv) @ V
        m1 = float(np.dot(fp, np.diag(h)) / np.sum(fp))
        P1 = V @ (Fdd * (h - m1 * np.eye(N))) @ V.T
        return from_orthogonal(P1, Linv), m1

    K = np.empty((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        K[:, j] = scc_charges(response(scc_fock(np.zeros((N, N)), S, gamma, e))[0], S,
                              np.zeros(N))
    D1 = np.empty_like(h1)
    D2 = np.empty_like(h1)
    mu1 = np.zeros(h1.shape[0])
    mu2 = np.zeros(h1.shape[0])
    for d in range(h1.shape[0]):
        b = scc_charges(response(h1[d])[0], S, np.zeros(N))
        dq1 = np.linalg.solve(np.eye(N) - K, b)
        F1 = scc_fock(h1[d], S, gamma, dq1)
        D1[d], mu1[d] = response(F1)
        if order >= 2:
            # second order: sum_k f[e_i, e_k, e_j] g_ik g_kj of g = F1 in the eigenbasis (mu1
            # shift included), then the first-order response to F2 = G(dq2)
            g = V.T @ to_orthogonal(F1, Linv) @ V - mu1[d] * np.eye(N)
            S2 = _dk2_matrix(g, eps, Fdd, mu, beta, nn, 1.0, 1.0, 1024)
            m2 = float(np.trace(S2) / np.sum(fp))
            D2a = from_orthogonal(V @ (S2 - m2 * np.diag(fp)) @ V.T, Linv)
            dq2 = np.linalg.solve(np.eye(N) - K, scc_charges(D2a, S, np.zeros(N)))
            D2b, m2b = response(scc_fock(np.zeros((N, N)), S, gamma, dq2))
            D2[d] = D2a + D2b
            mu2[d] = m2 + m2b
    ent = -np.sum(np.where(occ > 0, occ * np.log(np.where(occ > 0, occ, 1.0)), 0.0)
                  + np.where(occ < 1, (1 - occ) * np.log1p(-np.where(occ < 1, occ, 0.0)), 0.0))
    omega = 2.0 * np.sum(hcore * D) + 0.5 * x @ gamma @ x - 2.0 * ent / beta
    out = dict(D0=D, D1=D1, mu=float(mu), mu1=mu1, dq=y, iters=it + 1,
               omega1=np.array([2.0 * np.sum(h1[d] * D) for d in range(h1.shape[0])]),
               omega2=np.array([np.sum(h1[d] * D1[d]) for d in range(h1.shape[0])]),
               omega=float(omega))
    if order >= 2:
        out.update(D2=D2, mu2=mu2,
                   omega3=np.array([2.0 / 3.0 * np.sum(h1[d] * D2[d])
                                    for d in range(h1.shape[0])]))
    return out
