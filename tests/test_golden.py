"""Values the paper prints, as golden fixtures (no GPU).

tests/golden/omega_fits_appD.txt holds the coefficients of the piecewise fits
of omega_0(x) and omega_1(x) that arXiv:1412.5070 prints in App. D, Tables 1-4
(functional form Eq. ffit, 3 < x < 50, at least 13 significant digits),
omega_k(x) = int_0^inf z^k log(z) e^{-x z - z^2} dz.  Integration by parts of
the finite-part integral gives

    FP int_0^inf z^-1 e^{-y z - z^2} dz = y omega_0(y) + 2 omega_1(y) + C,

C a constant fixed by the finite-part convention.  For the kernel
k(r) = r^-3 (e^{-y1 r} - e^{-y2 r}), integrable although each of its terms is
not, the basic integral's hat g_0 at xi = 1, D = 0 (Eq. bfinal: 4 int x^2 k(x)
e^{-x^2} dx) is therefore

    4 [y1 omega_0(y1) + 2 omega_1(y1) - y2 omega_0(y2) - 2 omega_1(y2)],

with C cancelled: a value built from the paper's printed numbers alone.  The
oracle integrates the kernel pointwise; the library takes each term as a
finite part (b < 0, lowest power -1).  Both are checked against it.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

from test_aux_host import host_aux_terms, lib  # noqa: F401  (lib is a fixture)

HERE = os.path.dirname(os.path.abspath(__file__))
PAIRS = [(4.0, 7.5), (12.0, 30.0), (3.5, 45.0), (6.0, 15.0)]


def _fits():
    fits = {}
    with open(os.path.join(HERE, "golden", "omega_fits_appD.txt")) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            fn, lo, hi, k, c, d = line.split()
            fits.setdefault((fn, float(lo), float(hi)), []).append((int(k), float(c), float(d)))
    return fits


FITS = _fits()


def omega(k, x):
    """omega_k(x) from the paper's fit for the interval holding x."""
    for (fn, lo, hi), co in FITS.items():
        if fn == "omega%d" % k and lo < x < hi:
            return sum(c / x ** j for j, c, _ in co) + np.log(x) * sum(d / x ** j for j, _, d in co)
    raise ValueError(x)


def paper_value(y1, y2):
    return 4.0 * (y1 * omega(0, y1) + 2.0 * omega(1, y1) - y2 * omega(0, y2) - 2.0 * omega(1, y2))


def test_fixture_covers_the_tables():
    """Four intervals, each with omega_0 and omega_1 (7+6, 7+7, 6+6, 5+6 coefficients)."""
    assert sorted({(lo, hi) for _, lo, hi in FITS}) == [(3, 5), (5, 10), (10, 20), (20, 50)]
    n = {key: len(v) for key, v in FITS.items()}
    assert n[("omega0", 3, 5)] == 7 and n[("omega1", 3, 5)] == 6 and n[("omega0", 20, 50)] == 5


@pytest.mark.parametrize("x", [3.5, 4.5, 6.0, 9.0, 12.0, 18.0, 25.0, 45.0])
def test_paper_fits_reproduce_their_definition(x):
    """The transcribed fits against 30-digit quadrature of omega_k's definition
    (checks the fixture and the reading of Table 4; the paper states 13 digits)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for k in (0, 1):
        ref = float(mp.quad(lambda z: z ** k * mp.log(z) * mp.exp(-mp.mpf(x) * z - z * z), [0, 1 / mp.mpf(x), 1, mp.inf]))
        assert abs(omega(k, x) - ref) <= 1e-12 * abs(ref), (k, x)


@pytest.mark.parametrize("y1,y2", PAIRS)
def test_oracle_against_paper_omega(y1, y2):
    t = [(1.0, -3.0, -y1, 0.0), (-1.0, -3.0, -y2, 0.0)]
    got = O.radial(O.factor_kernel_terms(t), 3, 1.0, 0.0, 0)[0]
    ref = paper_value(y1, y2)
    assert abs(got - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("y1,y2", PAIRS)
def test_library_finite_parts_against_paper_omega(lib, y1, y2):  # noqa: F811
    t = [(1.0, -3.0, -y1, 0.0), (-1.0, -3.0, -y2, 0.0)]
    rc, got = host_aux_terms(lib, t, t, 3, [(1.0, 0.0)], 0)
    assert rc == 0
    ref = paper_value(y1, y2)
    assert abs(got[0, 0] - ref) <= 1e-12 * abs(ref)


# The worked example of Sec. 3.3: the finite part of S(-2, beta, 0), beta < 0,
# is -beta [gamma_E + log(-beta) - 1].  For sum_i c_i x^-2 e^{b_i x} with
# sum c_i = sum c_i b_i = 0 (the integral is then proper) the constants cancel:
#   int_0^inf x^-2 sum_i c_i e^{b_i x} dx = -sum_i c_i b_i log(-b_i).
EXAMPLES = [([(1.0, -1.0), (-2.0, -2.0), (1.0, -3.0)], 3 * np.log(3) - 4 * np.log(2)),
            ([(2.0, -1.0), (-3.0, -2.0), (1.0, -4.0)], 2 * np.log(2))]


@pytest.mark.parametrize("terms,value", EXAMPLES)
def test_library_x2_finite_parts_against_paper_example(lib, terms, value):  # noqa: F811
    """k3 = r^-4 sum_i c_i e^{b_i r}: three families of lowest power -2 with
    different b, each taken as its own finite part (two subtracted Taylor
    terms).  hat g_0 / (4 xi) at D = 0 tends to the integral above as xi -> 0;
    the library's values at xi = 1e-6 and 2e-6, extrapolated to xi = 0 (the
    xi-dependence is smooth), match the paper's example to 1e-10."""
    assert abs(sum(c for c, _ in terms)) < 1e-15 and abs(sum(c * b for c, b in terms)) < 1e-15
    t = [(c, -4.0, b, 0.0) for c, b in terms]
    vals = []
    for xi in (1e-6, 2e-6):
        rc, got = host_aux_terms(lib, t, t, 3, [(xi, 0.0)], 0)
        assert rc == 0
        vals.append(got[0, 0] / (4.0 * xi))
    assert abs(2.0 * vals[0] - vals[1] - value) <= 1e-10 * abs(value)


def omega_small_x(k, x, terms=120):
    """omega_k(x) from the small-x expansion of App. D, term-by-term integration
    of e^{-x z}, with the factor 1/4 that int z^k log z e^{-z^2} dz =
    Gamma((k+1)/2) psi((k+1)/2) / 4 carries (reading: the printed expansions
    lack it and are 4 omega_k)."""
    from scipy import special
    s = 0.0
    for j in range(terms):
        a = (j + 1) / 2.0 if k == 0 else j / 2.0 + 1.0
        s += (-x) ** j / math.factorial(j) * special.gamma(a) * special.digamma(a)
    return 0.25 * s


@pytest.mark.parametrize("y1,y2", [(0.5, 1.5), (1.0, 2.5), (0.3, 3.0)])
def test_series_finite_parts_against_paper_omega_expansion(lib, y1, y2):  # noqa: F811
    """b > 0: k = r^-3 (e^{y1 r} - e^{y2 r}); its two alpha = -1 families go
    through the library's series route (the closed series for S(-1), b >= 0).
    By parts, FP int z^-1 e^{y z - z^2} dz = -y omega_0(-y) + 2 omega_1(-y) + C,
    with omega_k at negative argument from App. D's small-x expansion.  The
    library and the oracle match it to 1e-12."""
    ref = 4.0 * ((-y1 * omega_small_x(0, -y1) + 2 * omega_small_x(1, -y1))
                 - (-y2 * omega_small_x(0, -y2) + 2 * omega_small_x(1, -y2)))
    t = [(1.0, -3.0, y1, 0.0), (-1.0, -3.0, y2, 0.0)]
    rc, got = host_aux_terms(lib, t, t, 3, [(1.0, 0.0)], 0)
    assert rc == 0
    assert abs(got[0, 0] - ref) <= 1e-12 * abs(ref)
    orc = O.radial(O.factor_kernel_terms(t), 3, 1.0, 0.0, 0)[0]
    assert abs(orc - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("x", [0.5, 2.0, -1.0])
def test_small_x_expansion_reading(x):
    """Reading of App. D's small-x expansions: with the factor 1/4 they give
    omega_k (30-digit quadrature of its definition)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for k in (0, 1):
        ref = float(mp.quad(lambda z: z ** k * mp.log(z) * mp.exp(-mp.mpf(x) * z - z * z), [0, 1, mp.inf]))
        assert abs(omega_small_x(k, x) - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("x", [0.1, 0.5, 3.0, 7.0])   # x = 2 is where the two arguments coincide
def test_T0_closed_form_reading(x):
    """Reading of Eq. t0 (not used by the library, which never forms T_s):
    T_0^{+-}(x) = int_0^inf e^{+-t - x t^2} dt = sqrt(pi/(4x)) e^{1/(4x)}
    [1 +- erf(1/(2 sqrt x))] by completing the square, against quadrature;
    the printed argument 1/(sqrt(2) x) does not reproduce it."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    xx = mp.mpf(x)
    for sgn in (1, -1):
        ref = mp.quad(lambda t: mp.exp(sgn * t - xx * t * t), [0, 1, mp.inf])
        derived = mp.sqrt(mp.pi / (4 * xx)) * mp.exp(1 / (4 * xx)) * (1 + sgn * mp.erf(1 / (2 * mp.sqrt(xx))))
        printed = mp.sqrt(mp.pi / (4 * xx)) * mp.exp(1 / (4 * xx)) * (1 + sgn * mp.erf(1 / (mp.sqrt(2) * xx)))
        assert abs(derived - ref) <= mp.mpf(10) ** -25 * abs(ref)
        assert abs(printed - ref) > 1e-3 * abs(ref)
