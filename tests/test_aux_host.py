"""The library's auxiliary-function stage compiled for the CPU (tests/aux_host.cpp
builds paper_1412_5070_gb300/csrc/aux.cuh as plain C++ with the library's own
table code) against the oracle, without a GPU.

On the GPU the same functions run inside the kernels; these tests check the
arithmetic of the stage, including the Gauss-Legendre branch for families
with b < 0 (a factor that decays, B < 0 in Eq. rs12), on the grid of the GPU
aux test and up to the highest order, 14.  The GPU tests repeat the
comparison through the C ABI.
"""
import ctypes
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from oracle import oracle as O
from paper_1412_5070_gb300 import molecules as M

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1412_5070_gb300", "csrc")
SRC = [os.path.join(HERE, "aux_host.cpp"), os.path.join(CSRC, "termlist.cpp")]
DEPS = SRC + [os.path.join(CSRC, f) for f in ("aux.cuh", "auxtab.h", "termlist.h")]
LIB = os.path.join(HERE, "_build", "libauxhost.so")

XI_D_GRID = [(xi, D) for xi in (0.025, 0.1, 0.5, 2.0, 10.0, 50.0) for D in (0.0, 0.05, 0.3, 1.0, 2.5, 5.0, 7.0,
                                                                            10.0, 20.0)]
FACTORS = {
    "P0": M.P0,
    "B<0 rho=-1/2": dict(c0=0.5, rho=-0.5, B=-0.8, mu=1.0, n=0),
    "B<0 rho=0 n=1": dict(c0=1.0, rho=0.0, B=-1.3, mu=1.5, n=1),
    "B<0 rho=-1 n=2": dict(c0=0.7, rho=-1.0, B=-4.0, mu=0.8, n=2),
}


@pytest.fixture(scope="module")
def lib():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not os.path.exists(LIB) or any(os.path.getmtime(d) > os.path.getmtime(LIB) for d in DEPS):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.run([gxx, "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, *SRC], check=True)
        os.replace(tmp, LIB)
    L = ctypes.CDLL(LIB)
    dp = ctypes.POINTER(ctypes.c_double)
    L.aux_host_eval.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int64, dp, dp, ctypes.c_int, dp]
    L.aux_host_eval.restype = ctypes.c_int
    L.aux_host_eval_terms.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, dp, dp,
                                      ctypes.c_int, dp]
    L.aux_host_eval_terms.restype = ctypes.c_int
    ip = ctypes.POINTER(ctypes.c_int)
    L.aux_host_jhat.argtypes = [ctypes.c_double, ctypes.c_int, dp]
    L.aux_host_kummer.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double, ip]
    L.aux_host_kummer.restype = ctypes.c_double
    L.aux_host_s_minus1.argtypes = [ctypes.c_double, ctypes.c_double, ip]
    L.aux_host_s_minus1.restype = ctypes.c_double
    L.aux_host_exp_rem.argtypes = [ctypes.c_double, ctypes.c_int]
    L.aux_host_exp_rem.restype = ctypes.c_double
    L.aux_host_gauss_legendre.argtypes = [dp, dp]
    L.aux_host_jhat_start.argtypes = [ctypes.c_double, ctypes.c_double, ip]
    L.aux_host_jhat_start.restype = ctypes.c_double
    return L


def host_aux(lib, f, fp, cls, pts, nmax):
    dp = ctypes.POINTER(ctypes.c_double)
    fa = np.array([f["c0"], f["rho"], f["B"], f["mu"], f["n"]], dtype=np.float64)
    fb = np.array([fp["c0"], fp["rho"], fp["B"], fp["mu"], fp["n"]], dtype=np.float64)
    xi = np.ascontiguousarray([p[0] for p in pts], dtype=np.float64)
    D = np.ascontiguousarray([p[1] for p in pts], dtype=np.float64)
    out = np.zeros(len(pts) * (nmax + 1))
    rc = lib.aux_host_eval(fa.ctypes.data_as(dp), fb.ctypes.data_as(dp), cls, len(pts), xi.ctypes.data_as(dp),
                           D.ctypes.data_as(dp), nmax, out.ctypes.data_as(dp))
    return rc, out.reshape(len(pts), nmax + 1)


def host_aux_terms(lib, t, tp, cls, pts, nmax):
    dp = ctypes.POINTER(ctypes.c_double)
    a = np.ascontiguousarray(t, dtype=np.float64).ravel()
    b = np.ascontiguousarray(tp, dtype=np.float64).ravel()
    xi = np.ascontiguousarray([p[0] for p in pts], dtype=np.float64)
    D = np.ascontiguousarray([p[1] for p in pts], dtype=np.float64)
    out = np.zeros(len(pts) * (nmax + 1))
    rc = lib.aux_host_eval_terms(a.ctypes.data_as(dp), len(t), b.ctypes.data_as(dp), len(tp), cls, len(pts),
                                 xi.ctypes.data_as(dp), D.ctypes.data_as(dp), nmax, out.ctypes.data_as(dp))
    return rc, out.reshape(len(pts), nmax + 1)


def worst_relative(got, kern, cls, pts, nmax):
    # the oracle's calls release the GIL: one point per thread
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        refs = list(ex.map(lambda p: O.radial(kern, cls, p[0], p[1], nmax), pts))
    return max(float(np.max(np.abs(got[i] - ref) / np.abs(ref))) for i, ref in enumerate(refs))


@pytest.mark.parametrize("name", list(FACTORS))
@pytest.mark.parametrize("cls", [1, 2, 3, 4, 6])
def test_aux_stage_on_cpu_against_oracle(lib, name, cls):
    """hat g_n, n <= 10, on the (xi, D) grid of the GPU aux test: relative error
    below 1e-8 (I6 at large xi is limited by cancellation between its
    families, for either sign of B), below 1e-10 for the other classes."""
    f = FACTORS[name]
    if cls == 1 and name != "P0":
        pytest.skip("I1 does not depend on the factor")
    rc, got = host_aux(lib, f, f, cls, XI_D_GRID, 10)
    assert rc == 0
    worst = worst_relative(got, O.factor_kernel(f), cls, XI_D_GRID, 10)
    assert worst < (1e-8 if cls == 6 else 1e-10), worst


SINGULAR = {   # kernels whose lowest power of x^2 k is below -1
    "I6 rho=-1 (x^-2)": (dict(M.P0, rho=-1.0), 6),
    "I6 rho=-1 n=1 (x^-2)": (dict(M.P0, rho=-1.0, n=1), 6),
    "I2 rho=-5/2 n=1 (x^-3/2)": (dict(M.P0, rho=-2.5, n=1), 2),
    "I4 rho=-5/2 n=1 (x^-3)": (dict(M.P0, rho=-2.5, n=1), 4),
    "I6 rho=-5/2 n=1 (x^-5)": (dict(M.P0, rho=-2.5, n=1), 6),
    "I6 rho=-5/4 (x^-5/2)": (dict(M.P0, rho=-1.25), 6),
    "I6 rho=-1 B=-4 n=2 (x^-2)": (dict(c0=0.7, rho=-1.0, B=-4.0, mu=0.8, n=2), 6),
}


@pytest.mark.parametrize("name", list(SINGULAR))
def test_singular_families(lib, name):
    """The damped long range of Eq. rs12 with rho <= -1: its families of the
    same b are evaluated together, their singular terms cancelled in a base
    polynomial.  Relative error of hat g_n (n <= 10) below 1e-10 for xi <= 2
    and below 1e-8 up to xi = 50."""
    f, cls = SINGULAR[name]
    for pts, tol in (([p for p in XI_D_GRID if p[0] <= 2.0], 1e-10), ([p for p in XI_D_GRID if p[0] > 2.0], 1e-8)):
        rc, got = host_aux(lib, f, f, cls, pts, 10)
        assert rc == 0
        assert worst_relative(got, O.factor_kernel(f), cls, pts, 10) < tol


def test_unsupported_singular_kernels_are_refused(lib):
    """A lowest power below -1 that is neither an integer nor a half-integer
    (I6 with rho = -1.3) is refused, and so is a kernel whose singular terms
    do not cancel (I6 of r^-3 (1 - e^{-0.7 r^2}), whose f_r^2 ~ r^-4)."""
    assert host_aux(lib, dict(M.P0, rho=-1.3), dict(M.P0, rho=-1.3), 6, XI_D_GRID[:2], 4)[0] == -3
    damped = [(1.0, -3, 0, 0), (-1.0, -3, 0, 0.7)]
    assert host_aux_terms(lib, damped, damped, 6, XI_D_GRID[:2], 4)[0] == -3


@pytest.mark.parametrize("name", ["P0", "B<0 rho=-1/2", "B<0 rho=-1 n=2"])
@pytest.mark.parametrize("cls", [2, 3, 4])
def test_aux_stage_on_cpu_highest_order(lib, name, cls):
    """All orders up to 14 (f-shell I5) on a coarser grid."""
    f = FACTORS[name]
    pts = XI_D_GRID[::4]
    rc, got = host_aux(lib, f, f, cls, pts, 14)
    assert rc == 0
    assert worst_relative(got, O.factor_kernel(f), cls, pts, 14) < 1e-9


def test_negative_B_with_a_general_power_is_refused(lib):
    """A family with b < 0 and a power that is neither an integer nor a
    half-integer is outside the quadrature's end-point forms: the class is
    refused (-3), while the same power with B >= 0 is served."""
    f = dict(c0=0.5, rho=-0.3, B=-0.8, mu=1.0, n=0)
    for cls in (2, 3, 4, 6):
        rc, _ = host_aux(lib, f, f, cls, XI_D_GRID[:3], 4)
        assert rc == -3
    rc, _ = host_aux(lib, dict(f, B=0.8), dict(f, B=0.8), 3, XI_D_GRID[:3], 4)
    assert rc == 0
    rc, _ = host_aux(lib, f, f, 1, XI_D_GRID[:3], 4)   # I1 does not use the factor
    assert rc == 0


@pytest.mark.parametrize("pair", [(dict(c0=0.5, rho=-0.5, B=-0.8, mu=1.0, n=0), dict(c0=0.3, rho=0.5, B=0.4, mu=0.7, n=0)),
                                  (M.P0, dict(c0=0.3, rho=0.5, B=-1.2, mu=0.7, n=0))])
def test_factor_pair_with_negative_B(lib, pair):
    """f' != f with B < 0 in one and B > 0 in the other (either way round):
    the product families of I4 and I6 have b of either sign."""
    f, fp = pair
    for cls in (4, 6):
        rc, got = host_aux(lib, f, fp, cls, XI_D_GRID[1::3], 8)
        assert rc == 0
        assert worst_relative(got, O.factor_kernel(f, fp), cls, XI_D_GRID[1::3], 8) < 1e-8


# factors given as terms (c, a, b, g): c r^a exp(b r - g r^2)
TERM_SETS = {
    "Ten-no exp(-1.2 r)": [(1.0, 0, -1.2, 0)],
    "three Gaussians": [(0.3, 0, 0, 0.2), (0.25, 0, 0, 1.1), (0.2, 0, 0, 4.0)],
    "Ten-no + Gaussian + r exp": [(-1 / 1.2, 0, -1.2, 0), (0.1, 0, 0, 0.5), (0.05, 1, -0.7, 0.3)],
    "r exp(-r)": [(1.0, 1, -1.0, 0)],
    "half-integer powers": [(0.4, -0.5, -0.9, 0), (0.2, 0.5, 0.0, 0.8)],
}


@pytest.mark.parametrize("name", list(TERM_SETS))
@pytest.mark.parametrize("cls", [2, 3, 4, 6])
def test_term_list_factors_on_cpu_against_oracle(lib, name, cls):
    """Factors given as term lists (the Ten-no factor, Gaussian geminals,
    mixtures): hat g_n up to order 14 against the oracle's term-list kernel."""
    t = TERM_SETS[name]
    pts = XI_D_GRID[::2]
    rc, got = host_aux_terms(lib, t, t, cls, pts, 14)
    if name == "half-integer powers" and cls == 6:
        assert rc == -3   # f_r^2 ~ r^-3: x^2 k has an x^-1 term that nothing cancels
        return
    assert rc == 0
    assert worst_relative(got, O.factor_kernel_terms(t), cls, pts, 14) < 1e-11


def test_term_list_pair(lib):
    """f' != f as term lists (Ten-no and Gaussians) for I4 and I6."""
    t, tp = TERM_SETS["Ten-no exp(-1.2 r)"], TERM_SETS["three Gaussians"]
    for cls in (4, 6):
        rc, got = host_aux_terms(lib, t, tp, cls, XI_D_GRID[1::3], 10)
        assert rc == 0
        assert worst_relative(got, O.factor_kernel_terms(t, tp), cls, XI_D_GRID[1::3], 10) < 1e-11


def test_term_list_domain(lib):
    """r^-3 diverges in every class and is refused; r^-3 (1 - e^{-0.7 r^2})
    has integrable I2, I3 and I4 kernels (singular terms cancelling between
    its families) and is served there, while its I6 kernel, f_r^2 ~ r^-4,
    diverges and is refused."""
    bare = [(1.0, -3, 0, 0)]
    damped = [(1.0, -3, 0, 0), (-1.0, -3, 0, 0.7)]
    for cls in (2, 3, 4, 6):
        assert host_aux_terms(lib, bare, bare, cls, XI_D_GRID[:2], 4)[0] == -3
        assert host_aux_terms(lib, damped, damped, cls, XI_D_GRID[:2], 4)[0] == (0 if cls != 6 else -3)


@pytest.mark.parametrize("cls", [2, 3])
def test_cancelling_terms_against_quadrature(lib, cls):
    """k3 = r^-3 (1 - e^{-0.7 r^2}) (two finite-part families, lowest power -1)
    and k2 = k3/r (a group, lowest power -2), against 30-digit quadrature of
    the kernel itself (written with expm1, so without the cancellation),
    hat g_n for n <= 3."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    damped = [(1.0, -3, 0, 0), (-1.0, -3, 0, 0.7)]
    pts = [(0.5, 1.2), (2.0, 0.7)]
    rc, got = host_aux_terms(lib, damped, damped, cls, pts, 3)
    assert rc == 0

    def k(r):
        return -mp.expm1(-mp.mpf("0.7") * r * r) / r ** (3 if cls == 3 else 4)

    for i, (x, d) in enumerate(pts):
        x = mp.mpf(x)

        def g0(s):
            dd = mp.sqrt(s)
            f = lambda r: k(r) * r * (mp.exp(-x * (r - dd) ** 2) - mp.exp(-x * (r + dd) ** 2)) / dd
            return mp.quad(f, [0, dd, dd + 10 / mp.sqrt(x), mp.inf])

        ref = np.array([float(2 ** n * mp.diff(g0, mp.mpf(d) ** 2, n)) for n in range(4)])
        np.testing.assert_allclose(got[i], ref, rtol=1e-11, atol=0)


def test_gpu_factor_sets_domain_matches_library(lib):
    """The GPU factor tests decide from a rule which classes each parameter set
    leaves out; the library's own class tables (here on the CPU) must agree."""
    tg = pytest.importorskip("test_gpu_factors")
    for name, (f, fp) in tg.SETS.items():
        fpp = fp if fp is not None else f
        for cls in (2, 3, 4, 5, 6):
            rc, _ = host_aux(lib, f, fpp, cls, XI_D_GRID[:1], 2)
            assert (rc == 0) == tg.supported(f, fpp, cls), (name, cls, rc)
    for name, t in tg.TERM_SETS.items():
        for cls in (2, 3, 4, 5, 6):
            assert host_aux_terms(lib, t, t, cls, XI_D_GRID[:1], 2)[0] == 0, (name, cls)


def _random_regular_terms(rng):
    n = int(rng.integers(1, 4))
    return [(float(rng.uniform(0.2, 1.0) * rng.choice([-1, 1])), float(rng.choice([0.0, 0.5, 1.0, 2.0])),
             float(rng.uniform(-2.0, 1.0)), float(rng.choice([0.0, rng.uniform(0.1, 2.0)]))) for _ in range(n)]


@pytest.mark.parametrize("seed", range(10))
def test_random_term_lists_on_cpu_against_oracle(lib, seed):
    """Seeded random factors of 1-3 terms (powers 0..2, b of either sign, with
    and without a Gaussian) through every branch of the stage: hat g_n (n <= 10)
    against the oracle, relative to |g_n| plus 1e-2 of the point's natural scale
    (2 xi)^n max_m |g_m|/(2 xi)^m, for random coefficients can make one g_n
    small by cancellation."""
    rng = np.random.default_rng(seed)
    t = _random_regular_terms(rng)
    pts = XI_D_GRID[::2]
    K = O.factor_kernel_terms(t)
    for cls in (2, 3, 4, 6):
        rc, got = host_aux_terms(lib, t, t, cls, pts, 10)
        assert rc == 0
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            refs = list(ex.map(lambda p: O.radial(K, cls, p[0], p[1], 10), pts))
        for i, (x, d) in enumerate(pts):
            sc = (2.0 * x) ** np.arange(11)
            nat = np.max(np.abs(refs[i]) / sc) * sc
            err = np.abs(got[i] - refs[i]) / (np.abs(refs[i]) + 1e-2 * nat)
            assert err.max() < 1e-9, (cls, x, d, float(err.max()))


def test_family_limits(lib):
    """At most MAXFAM = 24 families per kernel: a six-Gaussian geminal fits
    every class, a seven-Gaussian one only I2 and I3 (I4 and I6 have a family
    per pair sum of exponents); a family polynomial longer than 48 terms
    refuses the whole factor."""
    six = [(0.5 / (i + 1), 0, 0, 0.2 * 2.5 ** i) for i in range(6)]
    seven = [(0.5 / (i + 1), 0, 0, 0.2 * 2.5 ** i) for i in range(7)]
    for cls in (2, 3, 4, 6):
        assert host_aux_terms(lib, six, six, cls, XI_D_GRID[:1], 2)[0] == 0
        assert host_aux_terms(lib, seven, seven, cls, XI_D_GRID[:1], 2)[0] == (0 if cls in (2, 3) else -3)
    long_poly = [(1.0 / (j + 1), float(j), 0.0, 1.0) for j in range(0, 60, 2)]
    assert host_aux_terms(lib, long_poly, long_poly, 3, XI_D_GRID[:1], 2)[0] == -3



# ---------------------------------------------------------------- single device functions --

@pytest.mark.parametrize("z", [0.0, 1e-3, 0.7, 5.0, 31.9, 45.0, 200.0])
def test_jhat_against_definition(lib, z):
    """e^{-z} j_m(z), j_m = (z^-1 d/dz)^m (sinh z / z), m <= 14: the series /
    closed-form switch of jhat_all against 40-digit arithmetic of the
    definition (differentiation of sinh z / z in z^2/2)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    out = np.zeros(15)
    lib.aux_host_jhat(z, 14, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    for m in range(15):
        # j_m(z) = sum_k 2^m (k+m)!/(k! (2k+2m+1)!) z^{2k}
        zz = mp.mpf(z)
        ref = mp.nsum(lambda k: 2 ** m * mp.factorial(k + m) / (mp.factorial(k) * mp.factorial(2 * k + 2 * m + 1))
                      * zz ** (2 * k), [0, mp.inf]) * mp.exp(-zz)
        assert abs(out[m] - ref) <= 1e-13 * abs(ref), (m, out[m], ref)


@pytest.mark.parametrize("a,ib,z", [(0.25, 0, 0.0), (0.75, 1, 0.3), (1.5, 0, 4.0), (0.25, 1, 20.0), (3.0, 0, 36.0)])
def test_kummer_m_against_mpmath(lib, a, ib, z):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    bad = ctypes.c_int(0)
    got = lib.aux_host_kummer(a, ib, z, ctypes.byref(bad))
    ref = mp.hyp1f1(a, 0.5 if ib == 0 else 1.5, z)
    assert bad.value == 0 and abs(got - ref) <= 1e-14 * abs(ref)


@pytest.mark.parametrize("b,gam", [(0.0, 1.0), (0.5, 0.3), (1.0, 2.5), (2.0, 0.05), (1.0, 0.01)])
def test_s_minus1_against_finite_part_quadrature(lib, b, gam):
    """The closed series for S(-1, b, gamma), b >= 0, against its definition
    in the drop-log(eps) convention: int_0^inf (e^{bx} - 1) e^{-gamma x^2} / x dx
    + (-gamma_E - log gamma)/2."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    bad = ctypes.c_int(0)
    got = lib.aux_host_s_minus1(b, gam, ctypes.byref(bad))
    bb, gg = mp.mpf(b), mp.mpf(gam)
    ref = mp.quad(lambda x: mp.expm1(bb * x) * mp.exp(-gg * x * x) / x, [0, 1, mp.inf]) - (mp.euler + mp.log(gg)) / 2
    assert bad.value == 0 and abs(got - ref) <= 1e-13 * max(abs(ref), 1.0)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 5])
def test_exp_rem_against_mpmath(lib, k):
    """R_k(y) = e^{-y} - sum_{i<k} (-y)^i / i! on both sides of its series /
    direct switch at y = 1."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for y in (0.0, 1e-8, 0.2, 0.999, 1.0, 3.0):
        yy = mp.mpf(y)
        # the remainder's own series: no cancellation even where it is ~y^k
        ref = mp.nsum(lambda i: (-yy) ** int(i) / mp.factorial(int(i)), [k, mp.inf]) if y > 0 else (1 if k == 0 else 0)
        got = lib.aux_host_exp_rem(y, k)
        assert abs(got - ref) <= 1e-14 * abs(ref) + (0 if ref != 0 else 1e-300), (k, y, got, ref)


def test_gauss_legendre_nodes(lib):
    """The 16-point rule integrates x^j exactly for j <= 31 on [-1, 1]."""
    dp = ctypes.POINTER(ctypes.c_double)
    x, w = np.zeros(16), np.zeros(16)
    lib.aux_host_gauss_legendre(x.ctypes.data_as(dp), w.ctypes.data_as(dp))
    assert np.all(np.diff(x) > 0) and abs(w.sum() - 2.0) < 1e-14
    for j in range(32):
        exact = 0.0 if j % 2 else 2.0 / (j + 1)
        assert abs(np.dot(w, x ** j) - exact) < 1e-14



@pytest.mark.parametrize("alpha", [-0.5, 0.0, 0.5, 1.5, 3.0])
@pytest.mark.parametrize("y", [0.0, 0.4, 2.0, 6.0, 11.5])
def test_jhat_start_against_definition(lib, alpha, y):
    """Start values of the S recursion (Kummer form, Eq. msmallz for beta >= 0):
    J_alpha(y) / Gamma((alpha+1)/2) against 30-digit quadrature."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    bad = ctypes.c_int(0)
    got = lib.aux_host_jhat_start(alpha, y, ctypes.byref(bad))
    a, yy = mp.mpf(alpha), mp.mpf(y)
    ref = mp.quad(lambda t: t ** a * mp.exp(yy * t - t * t), [0, 1, yy / 2 + 1, mp.inf]) / mp.gamma((a + 1) / 2)
    assert bad.value == 0 and abs(got - ref) <= 1e-14 * abs(ref), (got, ref)


@pytest.mark.parametrize("name", ["P0", "B<0 rho=-1/2", "B<0 rho=0 n=1"])
def test_random_points_wide_range(lib, name):
    """60 seeded random (xi, D) with xi log-uniform in [0.01, 2000] and D in
    [0, 30] (a tenth at D = 0), orders <= 12, against the oracle relative to
    |g_n| plus 1e-3 of the point's natural scale; I6 with B > 0 is limited by
    its finite-part families at xi ~ 1000 (7e-9 there)."""
    f = FACTORS[name]
    rng = np.random.default_rng(123)
    n = 60
    xi = np.exp(rng.uniform(np.log(0.01), np.log(2000.0), n))
    D = rng.uniform(0.0, 30.0, n) * rng.choice([0.0, 1.0], n, p=[0.1, 0.9])
    pts = list(zip(xi, D))
    K = O.factor_kernel(f)
    for cls in (2, 3, 4, 6):
        rc, got = host_aux(lib, f, f, cls, pts, 12)
        assert rc == 0
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            refs = list(ex.map(lambda p: O.radial(K, cls, p[0], p[1], 12), pts))
        tol = 2e-8 if cls == 6 else 1e-9
        for i, (x, d) in enumerate(pts):
            sc = (2.0 * x) ** np.arange(13)
            nat = np.max(np.abs(refs[i]) / sc) * sc
            err = np.abs(got[i] - refs[i]) / (np.abs(refs[i]) + 1e-3 * nat)
            assert err.max() < tol, (cls, x, d, float(err.max()))


@pytest.mark.parametrize("cls", [1, 2, 3, 4])
def test_gaussian_families_from_the_kummer_table(lib, cls):
    """A Gaussian geminal's kernels have only b = 0 families, which the stage
    takes from its table of e^{-x} M(a, l + 3/2, x) (x = xi^2 D^2 / gamma,
    grid step 1/2, 14 Taylor terms) wherever x < 100.  Points at the largest
    Taylor step (x half-way between grid points) and at the table's end
    (x = 99.75), orders up to 14, against the oracle."""
    gam = 0.7
    t = [(1.0, 0, 0, gam)]
    g = {1: 0.0, 2: gam, 3: gam, 4: 2 * gam}[cls]          # the family's Gaussian exponent
    pts = []
    for xi in (0.3, 2.0, 15.0):
        for x in (0.25, 10.25, 49.75, 99.75):
            pts.append((xi, float(np.sqrt(x * (g + xi)) / xi)))
    rc, got = host_aux_terms(lib, t, t, cls, pts, 14)
    assert rc == 0
    assert worst_relative(got, O.factor_kernel_terms(t), cls, pts, 14) < 1e-12   # measured: 2.6e-13 at worst


@pytest.mark.parametrize("cls", [2, 3, 4, 6])
def test_series_start_values_from_the_y_table(lib, cls):
    """The series families with b > 0 take their start values J_as, J_as+1
    (and, for the finite-part family of I6, the S(-1) series) from a table in
    y = b / sqrt(g + xi) by Taylor steps from the nearest grid point (step
    1/16).  For every such family of the default factor, xi is chosen so that
    y sits half-way between grid points (the largest step), from y = 0.28 to
    19.03, where the series serves the high orders (z = y^2/4 at D = 0, and a
    small D); orders up to 14 against the oracle."""
    f = M.P0
    b_g = {2: [(0.5, 0.0), (0.5, 1.0)], 3: [(0.5, 0.0), (0.5, 1.0)],
           4: [(0.5, 1.0), (0.5, 2.0), (1.0, 0.0), (1.0, 1.0), (1.0, 2.0)],
           6: [(0.5, 1.0), (0.5, 2.0), (1.0, 0.0), (1.0, 1.0), (1.0, 2.0)]}[cls]
    pts = []
    for b, g in b_g:
        for i in (4, 40, 100, 200, 304):
            y = (i + 0.5) / 16.0
            xi = (b / y) ** 2 - g
            if xi <= 1e-3:
                continue
            pts += [(xi, 0.0), (xi, 0.02 / np.sqrt(xi))]
    rc, got = host_aux(lib, f, f, cls, pts, 14)
    assert rc == 0
    # measured: 2.3e-13 at worst (I2-I4), 6e-11 for I6 (its families cancel at order 14)
    assert worst_relative(got, O.factor_kernel(f), cls, pts, 14) < (2e-10 if cls == 6 else 1e-12)


@pytest.mark.parametrize("cls", [1, 2, 3, 4, 6])
def test_short_peak_rule_at_its_threshold(lib, cls):
    """Far from r = 0 (z >= 60 + 12 l) orders l <= 3 take the 10-node
    Gauss-Hermite rule about the peak instead of 16 nodes.  For every family
    of the default factor, points just past the switch of each order 0..3
    (z = 60.01 + 12 l at xi = 1), orders up to 14, against the oracle:
    orders 0..3 relative to themselves, all orders against the natural scale
    max(|g_n|, (2 xi)^n |g_0|) (far from r = 0 the high orders are sums over
    the families that cancel to far below that scale)."""
    f = M.P0
    fam = {1: [(0.0, 0.0)], 2: [(0.0, 1.0), (0.5, 0.0), (0.5, 1.0)], 3: [(0.0, 1.0), (0.5, 0.0), (0.5, 1.0)],
           4: [(0.0, 2.0), (0.5, 1.0), (0.5, 2.0), (1.0, 0.0), (1.0, 1.0), (1.0, 2.0)],
           6: [(0.0, 2.0), (0.5, 1.0), (0.5, 2.0), (1.0, 0.0), (1.0, 1.0), (1.0, 2.0)]}[cls]
    xi = 1.0
    pts = []
    for b, g in fam:
        for l in range(4):
            z = 60.01 + 12.0 * l
            pts.append((xi, (np.sqrt(4.0 * z * (g + xi)) - b) / (2.0 * xi)))
    rc, got = host_aux(lib, f, f, cls, pts, 14)
    assert rc == 0
    kern = O.factor_kernel(f)
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        refs = list(ex.map(lambda p: O.radial(kern, cls, p[0], p[1], 14), pts))
    low = max(float(np.max(np.abs(got[i][:4] - r[:4]) / np.abs(r[:4]))) for i, r in enumerate(refs))
    nat = max(float(np.max(np.abs(got[i] - r) / np.maximum(np.abs(r), (2 * xi) ** np.arange(15) * abs(r[0]))))
              for i, r in enumerate(refs))
    assert low < 1e-14 and nat < 1e-14, (low, nat)   # measured: 7.8e-16 and 7.4e-16 at worst
