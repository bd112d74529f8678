"""Pins for the CPU oracle (no GPU).

Each test checks the oracle against something other than itself: closed
forms (Boys function, Gaussian geminal, overlap), brute-force quadrature in
two dimensions, permutational and translational symmetry, and
finite-difference centre derivatives.  References are to arXiv:1412.5070.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as O
from paper_1412_5070_gb300 import molecules as M

P0 = M.P0


def boys(n, T):
    """Boys function F_n(T) = int_0^1 t^{2n} e^{-T t^2} dt (textbook definition)."""
    if T < 1e-12:
        return 1.0 / (2 * n + 1)
    a = n + 0.5
    return special.gamma(a) * special.gammainc(a, T) / (2.0 * T ** a)


# ------------------------------------------------------------------ radial --

@pytest.mark.parametrize("xi,D", [(0.7, 0.3), (2.0, 3.0), (0.05, 10.0), (50.0, 0.01), (50.0, 5.0),
                                  (1.3, 0.0), (10.0, 1.3)])
def test_radial_coulomb_is_boys(xi, D):
    """k = 1/r: the basic integral of Eq. bfinal reduces to the Boys function,
    hat g_n = 2 (-2 xi)^n F_n(xi D^2)."""
    g = O.radial(O.test_kernel(O.K_COULOMB), 3, xi, D, 12)
    T = xi * D * D
    ref = np.array([2 * (-2 * xi) ** n * boys(n, T) for n in range(13)])
    np.testing.assert_allclose(g, ref, rtol=2e-13, atol=0)


@pytest.mark.parametrize("gam", [0.3, 1.0, 4.0])
@pytest.mark.parametrize("xi,D", [(0.5, 0.0), (0.5, 1.7), (3.0, 2.2), (20.0, 0.4)])
def test_radial_gaussian_closed_form(gam, xi, D):
    """k = exp(-gam r^2): B is a Gaussian in D with exponent w = xi gam/(xi+gam),
    so hat g_n = (-2w)^n hat g_0 with hat g_0 = sqrt(pi/xi) xi^{3/2} ... written out:
    hat g_0 = (pi/(xi+gam))^{3/2} * xi^{3/2} / pi^{3/2} * 2 sqrt(pi) / sqrt(xi) ... (see below)."""
    # (ss|k|ss)/(K_ab K_cd) = (pi/(p+q))^{3/2} (pi/(xi+gam))^{3/2} e^{-w D^2}; and
    # (ss|k|ss)/(K_ab K_cd) = sqrt(pi^5/(p+q))/(pq) hat g_0 with pq/(p+q) = xi, so
    # hat g_0 = (pi/(p+q))^{3/2} (pi/(xi+gam))^{3/2} e^{-wD^2} pq / sqrt(pi^5/(p+q))
    #         = pi^{1/2} xi (xi+gam)^{-3/2} e^{-wD^2}.
    w = xi * gam / (xi + gam)
    g = O.radial(O.test_kernel(O.K_GAUSS, gam), 3, xi, D, 10)
    g0 = math.sqrt(math.pi) * xi * (xi + gam) ** -1.5 * math.exp(-w * D * D)
    ref = np.array([(-2 * w) ** n * g0 for n in range(11)])
    np.testing.assert_allclose(g, ref, rtol=2e-13, atol=0)


@pytest.mark.parametrize("xi,D", [(200.0, 7.0), (20.0, 30.0), (200.0, 15.0), (3.0, 60.0)])
def test_radial_coulomb_is_boys_large_T(xi, D):
    """k = 1/r at T = xi D^2 from 9800 to 45000 and orders up to 14: the
    integration-by-parts form of the oracle against the Boys function."""
    g = O.radial(O.test_kernel(O.K_COULOMB), 3, xi, D, 14)
    T = xi * D * D
    ref = np.array([2 * (-2 * xi) ** n * boys(n, T) for n in range(15)])
    np.testing.assert_allclose(g, ref, rtol=2e-13, atol=0)


@pytest.mark.parametrize("gam", [0.3, 4.0])
@pytest.mark.parametrize("xi,D", [(200.0, 5.0), (80.0, 9.0), (3000.0, 1.5)])
def test_radial_gaussian_closed_form_large_T(gam, xi, D):
    """k = exp(-gam r^2) at T from 2000 to 6750, orders up to 14:
    hat g_n = (-2w)^n sqrt(pi) xi (xi+gam)^{-3/2} e^{-w D^2}, w = xi gam/(xi+gam)."""
    w = xi * gam / (xi + gam)
    g = O.radial(O.test_kernel(O.K_GAUSS, gam), 3, xi, D, 14)
    g0 = math.sqrt(math.pi) * xi * (xi + gam) ** -1.5 * math.exp(-w * D * D)
    ref = np.array([(-2 * w) ** n * g0 for n in range(15)])
    np.testing.assert_allclose(g, ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("xi,D", [(50.0, 6.0), (400.0, 4.0), (2.0, 40.0)])
def test_radial_linear_kernel_large_T(xi, D):
    """k = r: up to terms of order e^{-T}, hat g_0 = sqrt(pi/xi) (D + 1/(2 xi D)),
    so hat g_n = sqrt(pi/xi) [(-1)^{n-1} (2n-3)!! D^{1-2n} + (-1)^n (2n-1)!! D^{-1-2n}/(2 xi)]
    for n >= 1 (D_Q D = 1/D, D_Q^n (1/D) = (-1)^n (2n-1)!! / D^{2n+1})."""
    g = O.radial(O.test_kernel(O.K_R), 3, xi, D, 14)

    def dfact(k):
        return 1.0 if k <= 0 else float(np.prod(np.arange(k, 0, -2)))

    s = math.sqrt(math.pi / xi)
    ref = [s * (D + 1 / (2 * xi * D))]
    for n in range(1, 15):
        ref.append(s * ((-1) ** (n - 1) * dfact(2 * n - 3) * D ** (1 - 2 * n)
                        + (-1) ** n * dfact(2 * n - 1) * D ** (-1 - 2 * n) / (2 * xi)))
    np.testing.assert_allclose(g, np.array(ref), rtol=1e-13, atol=0)


@pytest.mark.parametrize("cls", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("xi,D", [(100.0, 3.2), (10.0, 11.0), (400.0, 1.8)])
def test_radial_ibp_form_agrees_with_hermite_form(cls, xi, D):
    """Near T = 1000, where the separated-exponential form is still accurate,
    the integration-by-parts form (derivatives of x k(x) by Taylor jets) must
    agree with it for every order up to 14."""
    K = O.factor_kernel(P0)
    a = O.radial_mode(K, cls, xi, D, 14, 1)
    b = O.radial_mode(K, cls, xi, D, 14, 2)
    scale = np.maximum(np.abs(a), np.abs(b))
    assert np.all(np.abs(a - b) <= 1e-13 * scale + 1e-300), (a, b)


@pytest.mark.parametrize("cls", [2, 3, 4, 6])
@pytest.mark.parametrize("xi,D", [(0.3, 13.0), (2.0, 2.9), (8.0, 1.5), (0.9, 5.0)])
def test_radial_two_forms_agree(cls, xi, D):
    """The oracle evaluates D_Q^n of the bracket of Eq. bfinal in two forms
    (Bessel form and separated exponentials); they must agree wherever both
    are accurate (around the switch T = 16)."""
    K = O.factor_kernel(P0)
    a = O.radial_mode(K, cls, xi, D, 10, 0)
    b = O.radial_mode(K, cls, xi, D, 10, 1)
    scale = np.maximum(np.abs(a), np.abs(b))
    assert np.all(np.abs(a - b) <= 1e-13 * scale + 1e-300), (a, b)


# ---------------------------------------------------------- decaying factors --
# Closed form for any kernel written as terms c r^a e^{b r - g r^2}, in
# arbitrary precision (mpmath): each term of hat g_0 is
#   c e^{-xi D^2} [S(a+1, b + 2 xi D, g + xi) - S(a+1, b - 2 xi D, g + xi)] / D
# (the Gaussian bracket of Eq. bfinal completed into e^{+-2 xi D r}), with
# S(alpha, beta, gamma) of Eq. sila summed from its power series in beta by
# parity into Kummer functions, an identity for either sign of beta, and
# D_Q^n = 2^n d^n/ds^n in s = D^2 by numerical differentiation.

def _mp_S(mp, alpha, beta, gam):
    z = beta * beta / (4 * gam)
    return 0.5 * gam ** (-(alpha + 1) / 2) * (
        mp.gamma((alpha + 1) / 2) * mp.hyp1f1((alpha + 1) / 2, 0.5, z)
        + beta / mp.sqrt(gam) * mp.gamma((alpha + 2) / 2) * mp.hyp1f1((alpha + 2) / 2, 1.5, z))


def _mp_rs12_terms(mp, f):
    """Eq. rs12 with the damping of Eq. ttdamp written out,
    S_n(x) = 1 - e^{-x} sum_{k<=n} x^k/k!, x = mu r^2."""
    c0, rho, B, mu = (mp.mpf(f[k]) for k in ("c0", "rho", "B", "mu"))
    t = [(mp.mpf(1), 0, 0, mu), (mp.mpf(0.5), 1, 0, mu), (c0, rho, B, 0)]
    for k in range(f["n"] + 1):
        t.append((-c0 * mu ** k / mp.factorial(k), rho + 2 * k, B, mu))
    return t


def _mp_hat_g(mp, terms, xi, D, nmax):
    xi = mp.mpf(xi)

    def g0(s):
        d = mp.sqrt(s)
        acc = 0
        for c, a, b, g in terms:
            acc += c * (_mp_S(mp, a + 1, b + 2 * xi * d, g + xi) - _mp_S(mp, a + 1, b - 2 * xi * d, g + xi))
        return acc * mp.exp(-xi * s) / d

    s0 = mp.mpf(D) ** 2
    return np.array([float(2 ** n * mp.diff(g0, s0, n)) for n in range(nmax + 1)])


NEG_B = [dict(c0=0.5, rho=-0.5, B=-0.8, mu=1.0, n=0), dict(c0=1.0, rho=0.0, B=-1.3, mu=1.5, n=1)]


@pytest.mark.parametrize("fi", [0, 1])
@pytest.mark.parametrize("cls", [2, 3])
@pytest.mark.parametrize("xi,D", [(0.5, 1.2), (2.0, 0.7), (0.1, 3.0), (8.0, 0.4)])
def test_radial_decaying_factor_closed_form(fi, cls, xi, D):
    """B < 0 in Eq. rs12 (the long-range part decays): the oracle's hat g_n,
    n <= 6, for k3 = f and k2 = f/r against the closed form above."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    f = NEG_B[fi]
    terms = _mp_rs12_terms(mp, f)
    if cls == 2:
        terms = [(c, a - 1, b, g) for c, a, b, g in terms]
    ref = _mp_hat_g(mp, terms, xi, D, 6)
    got = O.radial(O.factor_kernel(f), cls, xi, D, 6)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("om", [0.7, 1.5])
@pytest.mark.parametrize("xi,D", [(0.5, 1.2), (3.0, 2.0), (0.05, 6.0)])
def test_radial_slater_kernel_closed_form(om, xi, D):
    """k = e^{-om r}, the Ten-no factor: the oracle's hat g_n, n <= 6,
    against the closed form above (one term, b = -om)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    ref = _mp_hat_g(mp, [(mp.mpf(1), 0, -mp.mpf(om), 0)], xi, D, 6)
    got = O.radial(O.test_kernel(O.K_SLATER, om), 3, xi, D, 6)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


def _mp_kernel_terms(cls, t):
    """Kernel of class cls (Eqs. k2, k3, k4, I6_ with f' = f) from a factor's
    terms (c, a, b, g), written out: f/r, f, f f', f_r f'_r."""
    def d(u):
        out = []
        for c, a, b, g in u:
            out += [(c * a, a - 1, b, g), (c * b, a, b, g), (-2 * g * c, a + 1, b, g)]
        return [x for x in out if x[0] != 0]

    def prod(u, v):
        return [(c1 * c2, a1 + a2, b1 + b2, g1 + g2) for c1, a1, b1, g1 in u for c2, a2, b2, g2 in v]

    return {2: [(c, a - 1, b, g) for c, a, b, g in t], 3: t, 4: prod(t, t), 6: prod(d(t), d(t))}[cls]


@pytest.mark.parametrize("name,terms", [("Ten-no", [(1.0, 0, -1.2, 0)]),
                                        ("Gaussians", [(0.3, 0, 0, 0.2), (0.25, 0, 0, 1.1), (0.2, 0, 0, 4.0)])])
@pytest.mark.parametrize("cls", [2, 3, 4, 6])
@pytest.mark.parametrize("xi,D", [(0.5, 1.2), (3.0, 2.0)])
def test_radial_term_list_factor_closed_form(name, terms, cls, xi, D):
    """The oracle's term-list kernels (factors given as c r^a e^{b r - g r^2})
    against the closed form above, hat g_n for n <= 6."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    kt = [(mp.mpf(c), a, mp.mpf(b), mp.mpf(g)) for c, a, b, g in _mp_kernel_terms(cls, terms)]
    ref = _mp_hat_g(mp, kt, xi, D, 6)
    got = O.radial(O.factor_kernel_terms(terms), cls, xi, D, 6)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


def _mp_rs12_kernel(mp, f, cls):
    """Eq. rs12 pointwise in arbitrary precision, the damping S_n of Eq. ttdamp
    as the regularized lower incomplete gamma P(n+1, x) (no cancellation at
    small r), f_r from dS_n/dx = e^{-x} x^n/n!; k2, k3, k4, k6 with f' = f."""
    c0, rho, B, mu, n = mp.mpf(f["c0"]), mp.mpf(f["rho"]), mp.mpf(f["B"]), mp.mpf(f["mu"]), f["n"]

    def val(r):
        x = mu * r * r
        return (1 + r / 2) * mp.exp(-x) + c0 * mp.gammainc(n + 1, 0, x, regularized=True) * r ** rho * mp.exp(B * r)

    def der(r):
        x = mu * r * r
        S = mp.gammainc(n + 1, 0, x, regularized=True)
        dS = mp.exp(-x) * x ** n / mp.factorial(n) * 2 * mu * r
        pw = r ** rho * mp.exp(B * r)
        return (mp.mpf(0.5) - 2 * mu * r * (1 + r / 2)) * mp.exp(-x) + c0 * (dS * pw + S * pw * (rho / r + B))

    return {2: lambda r: val(r) / r, 3: val, 4: lambda r: val(r) ** 2, 6: lambda r: der(r) ** 2}[cls]


@pytest.mark.parametrize("rho,n,cls,xi,D", [(-1.0, 0, 6, 0.5, 1.2), (-2.5, 1, 2, 3.0, 0.6), (-2.5, 1, 4, 0.5, 1.2)])
def test_radial_singular_factor_quadrature(rho, n, cls, xi, D):
    """rho <= -1 in Eq. rs12: the damped kernel is integrable, its terms are
    not (lowest powers of x^2 k: -2 for I6 with rho = -1, -3/2 and -3 for I2
    and I4 with rho = -5/2).  The oracle's hat g_n (n <= 2) against 30-digit
    quadrature of the kernel of Eq. bfinal, D_Q^n by differentiation in D^2."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    f = dict(P0, rho=rho, n=n)
    k = _mp_rs12_kernel(mp, f, cls)
    x = mp.mpf(xi)

    def g0(s):
        dd = mp.sqrt(s)
        fn = lambda r: k(r) * r * (mp.exp(-x * (r - dd) ** 2) - mp.exp(-x * (r + dd) ** 2)) / dd
        return mp.quad(fn, [0, dd / 2, dd, dd + 8 / mp.sqrt(x), mp.inf])

    ref = np.array([float(2 ** m * mp.diff(g0, mp.mpf(D) ** 2, m)) for m in range(3)])
    got = O.radial(O.factor_kernel(f), cls, xi, D, 2)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


def test_jhat_switch_continuity():
    """e^{-z} j_m(z) from the series and from the closed forms meet at the switch."""
    N = 10
    z0 = 40 + 2 * N
    lo = O.jhat(z0 * (1 - 1e-12), N)
    hi = O.jhat(z0 * (1 + 1e-12), N)
    # the two evaluation points differ by 2e-12 in z; a wrong branch would differ by far more
    np.testing.assert_allclose(lo, hi, rtol=1e-10)
    # spot values against the elementary closed forms
    z = 2.5
    np.testing.assert_allclose(O.jhat(z, 1)[0], math.exp(-z) * math.sinh(z) / z, rtol=1e-15)
    j1 = (math.cosh(z) / z - math.sinh(z) / z ** 2) / z
    np.testing.assert_allclose(O.jhat(z, 1)[1], math.exp(-z) * j1, rtol=1e-14)


# ----------------------------------------------------- kernels (pointwise) --

def f_rs(r, c0, rho, B, mu, n):
    """Eq. rs12 with Eq. ttdamp, written independently for the tests."""
    x = mu * r * r
    Sn = 1.0 - math.exp(-x) * sum(x ** k / math.factorial(k) for k in range(n + 1))
    return (1 + r / 2) * math.exp(-mu * r * r) + Sn * c0 * r ** rho * math.exp(B * r)


@pytest.mark.parametrize("r", [0.05, 0.4, 1.0, 2.7, 6.0])
def test_kernel_derivative_by_finite_differences(r):
    """k6 = f_r f'_r (Eq. I6_): the oracle's f_r agrees with a finite-difference
    derivative of Eq. rs12."""
    h = 1e-5 * max(r, 0.1)
    f = lambda x: f_rs(x, **P0)
    fr = (f(r - 2 * h) - 8 * f(r - h) + 8 * f(r + h) - f(r + 2 * h)) / (12 * h)
    K = O.factor_kernel(P0)
    np.testing.assert_allclose(O.kernel_value(K, 6, r), fr * fr, rtol=1e-9)
    np.testing.assert_allclose(O.kernel_value(K, 3, r), f(r), rtol=1e-14)
    np.testing.assert_allclose(O.kernel_value(K, 2, r), f(r) / r, rtol=1e-14)
    np.testing.assert_allclose(O.kernel_value(K, 4, r), f(r) ** 2, rtol=1e-14)


def test_kernel_cusp_values():
    """f(0) = 1 and f_r(0) = 1/2 for the default parameters (cusp condition).
    With rho = -1/2 the damped long-range term adds O(r^{3/2}) to f and
    O(r^{1/2}) to f_r, hence the tolerances at r = 1e-12."""
    K = O.factor_kernel(P0)
    assert abs(O.kernel_value(K, 3, 1e-12) - 1.0) < 1e-11
    assert abs(O.kernel_value(K, 6, 1e-12) - 0.25) < 2e-6


# ----------------------------------------------------- s-type brute force --

def brute_ss(kfun, a, A, b, B_, c, C, d, D_):
    """(ss|k|ss) by two-dimensional quadrature of
    K_ab K_cd (pi/(p+q))^{3/2} int d^3s k(s) exp(-xi |s - R|^2)
    over s in [0, inf) and cos(theta) in [-1, 1] (Gauss-Legendre, 128 nodes)."""
    A, B_, C, D_ = map(np.asarray, (A, B_, C, D_))
    p, q = a + b, c + d
    P = (a * A + b * B_) / p
    Q = (c * C + d * D_) / q
    Kab = math.exp(-a * b / p * np.dot(A - B_, A - B_))
    Kcd = math.exp(-c * d / q * np.dot(C - D_, C - D_))
    xi = p * q / (p + q)
    R = float(np.linalg.norm(P - Q))
    xc, wc = np.polynomial.legendre.leggauss(128)

    def inner(s):
        return 2 * math.pi * s * s * kfun(s) * float(np.dot(wc, np.exp(-xi * (s * s + R * R - 2 * s * R * xc))))

    top = R + 3.0 + 14.0 / math.sqrt(xi)
    pts = sorted({0.0, 0.5, 1.0, 2.0, max(R - 4 / math.sqrt(xi), 0.0), R, R + 4 / math.sqrt(xi), top})
    tot = 0.0
    for lo, hi in zip(pts[:-1], pts[1:]):
        if hi > lo:
            val, _ = integrate.quad(inner, lo, hi, epsabs=0, epsrel=2e-14, limit=400)
            tot += val
    return Kab * Kcd * (math.pi / (p + q)) ** 1.5 * tot


def fr_rs(r, c0, rho, B, mu, n):
    h = 1e-6 * max(r, 1e-3)
    return (f_rs(r + h, c0, rho, B, mu, n) - f_rs(r - h, c0, rho, B, mu, n)) / (2 * h)


SS_CASES = [
    (0.9, (0, 0, 0), 0.3, (0, 0, 0), 2.7, (0, 0, 5.6), 0.1, (0, 0, 5.6)),
    (0.1, (0, 0, 0), 0.1, (0, 0, 5.6), 0.3, (0, 0, 0), 0.9, (0, 0, 0)),
    (1.7, (0.3, -0.2, 0.1), 0.6, (1.1, 0.4, -0.5), 0.25, (-0.7, 1.3, 0.9), 3.0, (0.2, 0.1, 2.4)),
]


@pytest.mark.parametrize("case", SS_CASES)
@pytest.mark.parametrize("cls", [2, 3, 4])
def test_ss_brute_force(case, cls):
    """s-type quartets against 2-D brute-force quadrature (pins the prefactor
    of Eq. bfinal and the kernels of Eqs. k2-k4)."""
    a, A, b, B_, c, C, d, D_ = case
    f = lambda s: f_rs(s, **P0)
    kf = {2: lambda s: f(s) / s, 3: f, 4: lambda s: f(s) ** 2}[cls]
    ref = brute_ss(kf, a, A, b, B_, c, C, d, D_)
    got = O.prim_block(O.factor_kernel(P0), cls, [0, 0, 0, 0], [a, b, c, d], [A, B_, C, D_])[0, 0, 0, 0]
    assert abs(got - ref) <= 1e-10 * abs(ref), (got, ref)


@pytest.mark.parametrize("case", SS_CASES[:2])
def test_ss_brute_force_k6(case):
    """I6 kernel f_r^2 (Eq. I6_) against brute force with a finite-difference f_r."""
    a, A, b, B_, c, C, d, D_ = case
    kf = lambda s: fr_rs(s, **P0) ** 2
    ref = brute_ss(kf, a, A, b, B_, c, C, d, D_)
    got = O.prim_block(O.factor_kernel(P0), 6, [0, 0, 0, 0], [a, b, c, d], [A, B_, C, D_])[0, 0, 0, 0]
    assert abs(got - ref) <= 1e-8 * abs(ref), (got, ref)


# ------------------------------------- separable kernels: full angular momentum --

def cart(l):
    return [(i, j, l - i - j) for i in range(l, -1, -1) for j in range(l - i, -1, -1)]


def geminal_block_ref(ls, ex, cen, gam):
    """(ab|exp(-gam r12^2)|cd) for Cartesian GTOs by a product of 2-D
    Gauss-Hermite quadratures, one per Cartesian direction (the kernel is
    separable).  gam = 0 gives the overlap product S_ab S_cd."""
    a, b, c, d = ex
    p, q = a + b, c + d
    t, w = np.polynomial.hermite.hermgauss(60)
    blocks = []
    comps = [cart(l) for l in ls]
    out = np.zeros([len(x) for x in comps])
    cen = np.asarray(cen, dtype=float).reshape(4, 3)
    per_dim = []
    for k in range(3):
        A, B_, C, D_ = cen[:, k]
        P = (a * A + b * B_) / p
        Q = (c * C + d * D_) / q
        Kab = math.exp(-a * b / p * (A - B_) ** 2)
        Kcd = math.exp(-c * d / q * (C - D_) ** 2)
        x1 = P + t / math.sqrt(p)
        x2 = Q + t / math.sqrt(q)
        X1, X2 = np.meshgrid(x1, x2, indexing="ij")
        W = np.outer(w, w) / math.sqrt(p * q) * Kab * Kcd * np.exp(-gam * (X1 - X2) ** 2)
        tab = {}
        for ia in range(ls[0] + 1):
            for ib in range(ls[1] + 1):
                for ic in range(ls[2] + 1):
                    for id_ in range(ls[3] + 1):
                        tab[(ia, ib, ic, id_)] = float(np.sum(W * (X1 - A) ** ia * (X1 - B_) ** ib *
                                                              (X2 - C) ** ic * (X2 - D_) ** id_))
        per_dim.append(tab)
    for i0, ca in enumerate(comps[0]):
        for i1, cb in enumerate(comps[1]):
            for i2, cc in enumerate(comps[2]):
                for i3, cd in enumerate(comps[3]):
                    v = 1.0
                    for k in range(3):
                        v *= per_dim[k][(ca[k], cb[k], cc[k], cd[k])]
                    out[i0, i1, i2, i3] = v
    return out


GEOM = [(0.3, -0.2, 0.1), (1.1, 0.4, -0.5), (-0.7, 1.3, 0.9), (0.2, 0.1, 1.4)]


@pytest.mark.parametrize("ls", [(0, 0, 0, 0), (1, 0, 0, 0), (1, 1, 0, 0), (1, 0, 1, 0), (2, 1, 1, 0),
                                (2, 2, 1, 1), (3, 1, 2, 0), (3, 3, 0, 0), (2, 2, 2, 2)])
@pytest.mark.parametrize("gam", [0.0, 0.8])
def test_separable_kernels_all_l(ls, gam):
    """k = 1 (overlap product) and k = exp(-gam r12^2) (Gaussian geminal) for
    Cartesian shells up to f: pins the E coefficients (Eq. AB), the Hermite
    recursion for R (Eq. ri), the contraction of Eq. ii and the component
    order, independently of the McMurchie-Davidson machinery."""
    ex = [1.3, 0.7, 0.9, 2.1]
    kern = O.test_kernel(O.K_ONE) if gam == 0.0 else O.test_kernel(O.K_GAUSS, gam)
    got = O.prim_block(kern, 3, list(ls), ex, GEOM)
    ref = geminal_block_ref(ls, ex, GEOM, gam)
    scale = np.max(np.abs(ref))
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-12 * scale)


# --------------------------------------------------- symmetry / invariance --

def test_permutational_symmetry():
    """8-fold symmetry of I1-I4 and I6 (real orbitals, symmetric kernel)."""
    ex = [1.3, 0.7, 0.9, 2.1]
    ls = [2, 1, 1, 0]
    K = O.factor_kernel(P0)
    for cls in (1, 2, 3, 4, 6):
        base = O.prim_block(K, cls, ls, ex, GEOM)
        # a <-> b
        sw = O.prim_block(K, cls, [ls[1], ls[0], ls[2], ls[3]], [ex[1], ex[0], ex[2], ex[3]],
                          [GEOM[1], GEOM[0], GEOM[2], GEOM[3]])
        np.testing.assert_allclose(sw.transpose(1, 0, 2, 3), base, rtol=1e-12, atol=1e-14)
        # bra <-> ket
        bk = O.prim_block(K, cls, [ls[2], ls[3], ls[0], ls[1]], [ex[2], ex[3], ex[0], ex[1]],
                          [GEOM[2], GEOM[3], GEOM[0], GEOM[1]])
        np.testing.assert_allclose(bk.transpose(2, 3, 0, 1), base, rtol=1e-12, atol=1e-14)


def test_i5_symmetries():
    """I5 is antisymmetric under a <-> b (Eq. I5_) and symmetric under c <-> d."""
    ex = [1.3, 0.7, 0.9, 2.1]
    ls = [1, 1, 1, 0]
    K = O.factor_kernel(P0)
    base = O.prim_block(K, 5, ls, ex, GEOM)
    sw = O.prim_block(K, 5, [ls[1], ls[0], ls[2], ls[3]], [ex[1], ex[0], ex[2], ex[3]],
                      [GEOM[1], GEOM[0], GEOM[2], GEOM[3]])
    np.testing.assert_allclose(sw.transpose(1, 0, 2, 3), -base, rtol=1e-11, atol=1e-14)
    cd = O.prim_block(K, 5, [ls[0], ls[1], ls[3], ls[2]], [ex[0], ex[1], ex[3], ex[2]],
                      [GEOM[0], GEOM[1], GEOM[3], GEOM[2]])
    np.testing.assert_allclose(cd.transpose(0, 1, 3, 2), base, rtol=1e-11, atol=1e-14)


def test_translation_invariance():
    ex = [1.3, 0.7, 0.9, 2.1]
    ls = [1, 1, 0, 1]
    K = O.factor_kernel(P0)
    shift = np.array([0.37, -1.1, 2.3])
    for cls in (2, 5, 6):
        a = O.prim_block(K, cls, ls, ex, GEOM)
        b = O.prim_block(K, cls, ls, ex, [np.asarray(g) + shift for g in GEOM])
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-13 * np.max(np.abs(a)))


# --------------------------------------------------- finite differences --

def test_centre_derivative_raises_angular_momentum():
    """d/dA_x [x_A^i e^{-a r_A^2}] = 2a x_A^{i+1} e - i x_A^{i-1} e ties the
    l+1 components to derivatives of the l components (checked for p <- s and
    d <- p, every class)."""
    ex = [1.1, 0.8, 0.6, 1.9]
    K = O.factor_kernel(P0)
    h = 1e-3
    for cls in (1, 2, 3, 4, 6):
        for l_lo in (0, 1):
            ls_lo = [l_lo, 1, 0, 1]
            ls_hi = [l_lo + 1, 1, 0, 1]
            hi = O.prim_block(K, cls, ls_hi, ex, GEOM)
            comps_lo, comps_hi = cart(l_lo), cart(l_lo + 1)
            for k in range(3):
                def blk(dx):
                    g = [np.array(x, dtype=float) for x in GEOM]
                    g[0][k] += dx
                    return O.prim_block(K, cls, ls_lo, ex, g)
                deriv = (blk(-2 * h) - 8 * blk(-h) + 8 * blk(h) - blk(2 * h)) / (12 * h)
                lower = O.prim_block(K, cls, [max(l_lo - 1, 0), 1, 0, 1], ex, GEOM) if l_lo > 0 else None
                for i_lo, c in enumerate(comps_lo):
                    up = list(c)
                    up[k] += 1
                    i_hi = comps_hi.index(tuple(up))
                    rhs = deriv[i_lo].copy()
                    if c[k] > 0:
                        dn = list(c)
                        dn[k] -= 1
                        rhs += c[k] * lower[cart(l_lo - 1).index(tuple(dn))]
                    rhs /= 2 * ex[0]
                    scale = np.max(np.abs(hi)) + 1e-300
                    np.testing.assert_allclose(hi[i_hi], rhs, rtol=0, atol=2e-9 * scale)


def test_i5_equals_laplacian_difference_of_i3():
    """Eq. I5_: I5 = 1/2 (lap_A - lap_B) I3, with the Laplacians taken by
    finite differences of I3 in the centres A and B."""
    ex = [1.1, 0.8, 0.6, 1.9]
    ls = [1, 0, 1, 0]
    K = O.factor_kernel(P0)
    h = 2e-3

    def i3(dA, dB):
        g = [np.array(x, dtype=float) for x in GEOM]
        g[0] += dA
        g[1] += dB
        return O.prim_block(K, 3, ls, ex, g)

    base = i3(np.zeros(3), np.zeros(3))
    lapA = np.zeros_like(base)
    lapB = np.zeros_like(base)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        for which, acc in ((0, lapA), (1, lapB)):
            f = lambda s: i3(s * e, 0 * e) if which == 0 else i3(0 * e, s * e)
            acc += (-f(2) + 16 * f(1) - 30 * base + 16 * f(-1) - f(-2)) / (12 * h * h)
    ref = 0.5 * (lapA - lapB)
    got = O.prim_block(K, 5, ls, ex, GEOM)
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-7 * np.max(np.abs(ref)))


def test_i5_vanishes_for_constant_factor():
    """[f, T1] = 0 for constant f, so I5 = 0 (Eq. I5)."""
    ex = [1.1, 0.8, 0.6, 1.9]
    got = O.prim_block(O.test_kernel(O.K_ONE), 5, [2, 1, 1, 0], ex, GEOM)
    ref_scale = np.max(np.abs(O.prim_block(O.test_kernel(O.K_ONE), 3, [2, 1, 1, 0], ex, GEOM)))
    assert np.max(np.abs(got)) <= 1e-13 * ref_scale * max(ex) ** 2


def test_coulomb_ss_closed_form():
    """I1 for s functions: 2 pi^{5/2} / (p q sqrt(p+q)) K_ab K_cd F_0(T)."""
    a, b, c, d = 0.9, 0.3, 2.7, 0.1
    A, B_, C, D_ = map(np.array, [(0, 0, 0), (0, 0, 0), (0, 0, 5.6), (0, 0, 5.6)])
    p, q = a + b, c + d
    T = p * q / (p + q) * 5.6 ** 2
    ref = 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * boys(0, T)
    got = O.prim_block(O.factor_kernel(P0), 1, [0, 0, 0, 0], [a, b, c, d], [A, B_, C, D_])[0, 0, 0, 0]
    assert abs(got - ref) <= 1e-14 * ref


def test_contracted_blocks_sum_primitives():
    """Contracted blocks are the coefficient-weighted sums of primitive blocks."""
    basis = M.twelve_atom_spd(2)
    q = np.array([[5, 3, 1, 0]], dtype=np.int32)
    K = O.factor_kernel(P0)
    out, off = O.shell_blocks(K, 3, basis, q)
    po = basis.prim_off
    ls = [int(basis.l[s]) for s in q[0]]
    acc = 0
    for i0 in range(3):
        for i1 in range(3):
            for i2 in range(3):
                for i3 in range(3):
                    idx = [po[q[0][0]] + i0, po[q[0][1]] + i1, po[q[0][2]] + i2, po[q[0][3]] + i3]
                    co = np.prod([basis.coefs[i] for i in idx])
                    acc = acc + co * O.prim_block(K, 3, ls, [basis.exps[i] for i in idx],
                                                  [basis.centers[s] for s in q[0]])
    np.testing.assert_allclose(out.reshape(acc.shape), acc, rtol=1e-13, atol=0)


# --------------------------------------------------- term magnitude block --

@pytest.mark.parametrize("cls", [1, 3, 5, 6])
def test_term_magnitude_bounds_block(cls):
    """The magnitude block (absolute-value evaluation of the sum of Eq. ii)
    bounds every element: |I| <= M (triangle inequality), and M is unchanged
    when the sign of a contraction coefficient flips."""
    basis = M.twelve_atom_spd(2)
    q = np.array([[5, 3, 1, 0], [7, 7, 2, 1], [11, 4, 9, 6]], dtype=np.int32)
    K = O.factor_kernel(P0)
    out, off, mag = O.shell_blocks(K, cls, basis, q, with_mag=True)
    assert np.all(mag >= np.abs(out) * (1 - 1e-14))
    assert np.all(mag[out != 0] > 0)
    flipped = M.Basis(**{**basis.__dict__, "coefs": -basis.coefs})
    out2, _, mag2 = O.shell_blocks(K, cls, flipped, q, with_mag=True)
    np.testing.assert_allclose(mag2, mag, rtol=1e-14)
    np.testing.assert_allclose(out2, out, rtol=1e-14)   # four coefficients: sign cancels


def test_term_magnitude_single_term():
    """An (ss|ss) primitive block has one term, so M = |I|; with cancelling
    contraction coefficients M is the sum of the primitive magnitudes while I
    shrinks."""
    K = O.factor_kernel(P0)
    basis = M.Basis(name="ss", centers=np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.4]]), l=np.array([0, 0]),
                    nprim=np.array([2, 1]), exps=np.array([1.2, 1.19, 0.8]), coefs=np.array([1.0, -1.0, 1.0]))
    q = np.array([[0, 0, 1, 1], [1, 1, 1, 1]], dtype=np.int32)
    out, off, mag = O.shell_blocks(K, 3, basis, q, with_mag=True)
    assert mag[1] == pytest.approx(abs(out[1]), rel=1e-15)
    assert abs(out[0]) < 0.05 * mag[0]


# --------------------------------------------------------- Hobson cross-check --

def _laplacian_power(t, u, v, k):
    """Delta^k of x^t y^u z^v as {(i, j, l): coefficient} (exact integers)."""
    poly = {(t, u, v): 1}
    for _ in range(k):
        nxt = {}
        for (i, j, l), c in poly.items():
            for d, e in ((0, i), (1, j), (2, l)):
                if e >= 2:
                    key = [i, j, l]
                    key[d] -= 2
                    nxt[tuple(key)] = nxt.get(tuple(key), 0) + c * e * (e - 1)
        poly = {key: c for key, c in nxt.items() if c}
    return poly


def hermite_r_hobson(X, g, L):
    """R_tuv = d^t/dX^t d^u/dY^u d^v/dZ^v B(|X|) by Hobson's theorem (the
    spherical route of App. A): for a monomial m of degree n,
    m(grad) B = sum_k (Delta^k m)(X) / (2^k k!) g_{n-k}, g_j = (r^-1 d/dr)^j B."""
    R = {}
    for t in range(L + 1):
        for u in range(L + 1 - t):
            for v in range(L + 1 - t - u):
                n = t + u + v
                s = 0.0
                for k in range(n // 2 + 1):
                    lap = sum(c * X[0] ** i * X[1] ** j * X[2] ** l
                              for (i, j, l), c in _laplacian_power(t, u, v, k).items())
                    s += lap / (2.0 ** k * math.factorial(k)) * g[n - k]
                R[(t, u, v)] = s
    return R


def hermite_r_recursion(X, g, L):
    """R by the Cartesian recursion R^(n)_{t+1,u,v} = t R^(n+1)_{t-1,u,v} + X R^(n+1)_{tuv}."""
    R = {(n, 0, 0, 0): g[n] for n in range(L + 1)}
    for tot in range(1, L + 1):
        for n in range(L - tot, -1, -1):
            for t in range(tot, -1, -1):
                for u in range(tot - t, -1, -1):
                    v = tot - t - u
                    if t > 0:
                        val = X[0] * R[(n + 1, t - 1, u, v)] + ((t - 1) * R[(n + 1, t - 2, u, v)] if t > 1 else 0.0)
                    elif u > 0:
                        val = X[1] * R[(n + 1, t, u - 1, v)] + ((u - 1) * R[(n + 1, t, u - 2, v)] if u > 1 else 0.0)
                    else:
                        val = X[2] * R[(n + 1, t, u, v - 1)] + ((v - 1) * R[(n + 1, t, u, v - 2)] if v > 1 else 0.0)
                    R[(n, t, u, v)] = val
    return {(t, u, v): R[(0, t, u, v)] for (n, t, u, v) in R if n == 0}


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_hermite_recursion_matches_hobson(seed):
    """The Cartesian recursion for R_tuv (used by the oracle and the kernels)
    against Hobson's theorem, for arbitrary radial derivatives g_n and
    separations, up to L = 14."""
    rng = np.random.default_rng(seed)
    X = rng.normal(size=3) * [0.7, 1.3, 0.4][seed % 3]
    g = rng.normal(size=15)
    L = 14
    a = hermite_r_recursion(X, g, L)
    b = hermite_r_hobson(X, g, L)
    keys = sorted(b)
    va, vb = np.array([a[k] for k in keys]), np.array([b[k] for k in keys])
    np.testing.assert_allclose(va, vb, rtol=1e-11, atol=1e-13 * np.max(np.abs(vb)))


def _e_direct(a, b, A, B, i, j):
    """E_t^{ij}: x_A^i x_B^j e^{-a x_A^2 - b x_B^2} = sum_t E_t Lambda_t(x; p, P),
    Lambda_t = (d/dP)^t e^{-p x_P^2}, by binomial expansion about P and
    x_P^k = sum_t c_kt Lambda_t (Hermite inversion) -- written from the definition."""
    p = a + b
    P = (a * A + b * B) / p
    K = math.exp(-a * b / p * (A - B) ** 2)
    mono = np.zeros(i + j + 1)   # coefficients of x_P^k in x_A^i x_B^j
    for r in range(i + 1):
        for s in range(j + 1):
            mono[r + s] += math.comb(i, r) * math.comb(j, s) * (P - A) ** (i - r) * (P - B) ** (j - s)
    # x_P^k e^{-p x_P^2} = sum_t c_kt (d/dP)^t e^{-p x_P^2}: from x e^{-p x^2} = (1/2p) d/dP e^{-p x^2}
    # and the product rule, c_{k+1,t} = c_{k,t-1}/(2p) + (t+1) c_{k,t+1}
    n = i + j
    c = np.zeros((n + 1, n + 2))
    c[0, 0] = 1.0
    for k in range(n):
        for t in range(k + 2):
            c[k + 1, t] = (c[k, t - 1] / (2 * p) if t > 0 else 0.0) + (t + 1) * c[k, t + 1]
    return K * np.array([sum(mono[k] * c[k, t] for k in range(n + 1)) for t in range(n + 1)])


def test_prim_block_through_hobson():
    """A (p p|p d) primitive block of I3 assembled here from the oracle's radial
    derivatives, Hobson's R, direct-expansion E and Eq. ii equals the oracle's."""
    K = O.factor_kernel(P0)
    ls = [1, 1, 1, 2]
    ex = [0.9, 0.35, 1.4, 0.6]
    cen = [np.array(c) for c in ([0.0, 0.0, 0.0], [0.4, -1.1, 0.7], [1.8, 0.3, -0.5], [1.2, 1.0, 0.2])]
    p, q = ex[0] + ex[1], ex[2] + ex[3]
    P = (ex[0] * cen[0] + ex[1] * cen[1]) / p
    Q = (ex[2] * cen[2] + ex[3] * cen[3]) / q
    X = Q - P
    xi, D = p * q / (p + q), float(np.linalg.norm(X))
    L = sum(ls)
    g = math.pi ** 2.5 / (math.sqrt(p + q) * p * q) * O.radial(K, 3, xi, D, L)
    R = hermite_r_hobson(X, g, L)
    cart = lambda l: [(i, j, l - i - j) for i in range(l, -1, -1) for j in range(l - i, -1, -1)]
    out = []
    for ca in cart(ls[0]):
        for cb in cart(ls[1]):
            for cc in cart(ls[2]):
                for cd in cart(ls[3]):
                    Eab = [_e_direct(ex[0], ex[1], cen[0][k], cen[1][k], ca[k], cb[k]) for k in range(3)]
                    Ecd = [_e_direct(ex[2], ex[3], cen[2][k], cen[3][k], cc[k], cd[k]) for k in range(3)]
                    s = 0.0
                    for t, et in enumerate(Eab[0]):
                        for u, eu in enumerate(Eab[1]):
                            for v, ev in enumerate(Eab[2]):
                                for t2, ft in enumerate(Ecd[0]):
                                    for u2, fu in enumerate(Ecd[1]):
                                        for v2, fv in enumerate(Ecd[2]):
                                            s += (-1) ** (t + u + v) * et * eu * ev * ft * fu * fv * \
                                                 R[(t + t2, u + u2, v + v2)]
                    out.append(s)
    ref = O.prim_block(K, 3, ls, ex, cen).ravel()
    np.testing.assert_allclose(np.array(out), ref, rtol=1e-11, atol=1e-13 * np.max(np.abs(ref)))


def _rs12_as_terms(f):
    """Eq. rs12 with Eq. ttdamp expanded: (1 + r/2) e^{-mu r^2} + c0 r^rho e^{Br}
    - c0 sum_{k<=n} mu^k/k! r^{rho+2k} e^{Br - mu r^2}."""
    t = [(1.0, 0.0, 0.0, f["mu"]), (0.5, 1.0, 0.0, f["mu"]), (f["c0"], f["rho"], f["B"], 0.0)]
    for k in range(f["n"] + 1):
        t.append((-f["c0"] * f["mu"] ** k / math.factorial(k), f["rho"] + 2 * k, f["B"], f["mu"]))
    return t


@pytest.mark.parametrize("f", [P0, dict(P0, B=-0.8), dict(P0, rho=0.0, n=1)])
@pytest.mark.parametrize("cls", [2, 3, 4, 6])
def test_term_list_mode_matches_rs12_mode(f, cls):
    """The oracle's two factor modes (Eq. rs12 pointwise with its damping, and
    the same factor as a term list) agree where the expanded terms do not
    cancel badly near r = 0 (n = 0, or rho >= 0)."""
    a = O.radial(O.factor_kernel(f), cls, 0.7, 1.3, 8)
    b = O.radial(O.factor_kernel_terms(_rs12_as_terms(f)), cls, 0.7, 1.3, 8)
    np.testing.assert_allclose(b, a, rtol=1e-12, atol=0)
