"""Python access to the CPU oracle (``f12_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use this module.
The product library never imports it and shares no code with it.

The oracle evaluates the plain definitions of the six integral classes of
arXiv:1412.5070 (Sec. 2.1, Eqs. I1-I6; kernels Eqs. k1-k6; correlation factor
Eq. rs12 with Eq. ttdamp) in binary128; see the header of ``f12_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "f12_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libf12oracle.so")
_lock = threading.Lock()
_lib = None


class OrkKernel(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_int),
        ("c0", ctypes.c_double), ("rho", ctypes.c_double), ("B", ctypes.c_double), ("mu", ctypes.c_double),
        ("n", ctypes.c_int),
        ("c0p", ctypes.c_double), ("rhop", ctypes.c_double), ("Bp", ctypes.c_double), ("mup", ctypes.c_double),
        ("np", ctypes.c_int),
        ("gam", ctypes.c_double),
        ("nt", ctypes.c_int), ("ntp", ctypes.c_int),
        ("t", (ctypes.c_double * 4) * 16), ("tp", (ctypes.c_double * 4) * 16),
    ]


# plain test kernels (id field of OrkKernel)
K_ONE, K_GAUSS, K_R, K_COULOMB, K_SLATER = 10, 11, 12, 13, 14
K_TERMS = 20        # factor pair given as term lists
MAX_TERMS = 16


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libf12oracle.so`` (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    libs = ["-lm"]
    if platform.machine() in ("x86_64", "AMD64", "i686"):
        libs.append("-lquadmath")
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC] + libs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.ork_radial.argtypes = [ctypes.POINTER(OrkKernel), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, dp]
            L.ork_radial.restype = ctypes.c_int
            L.ork_radial_mode.argtypes = [ctypes.POINTER(OrkKernel), ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, ctypes.c_int, dp]
            L.ork_radial_mode.restype = ctypes.c_int
            L.ork_prim_block.argtypes = [ctypes.POINTER(OrkKernel), ctypes.c_int, ip, dp, dp, dp]
            L.ork_prim_block.restype = ctypes.c_int
            L.ork_shell_blocks.argtypes = [ctypes.POINTER(OrkKernel), ctypes.c_int, dp, ip, ip, ip, dp, dp,
                                           ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int64), dp, dp, ctypes.c_int]
            L.ork_shell_blocks.restype = ctypes.c_int64
            L.ork_jhat.argtypes = [ctypes.c_double, ctypes.c_int, dp]
            L.ork_jhat.restype = ctypes.c_int
            L.ork_kernel_value.argtypes = [ctypes.POINTER(OrkKernel), ctypes.c_int, ctypes.c_double]
            L.ork_kernel_value.restype = ctypes.c_double
            L.ork_mantissa_bits.argtypes = []
            L.ork_mantissa_bits.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def factor_kernel(f, fprime=None) -> OrkKernel:
    """Kernel record for the range-separated factor pair (Eq. rs12).

    ``f`` and ``fprime`` are mappings with keys c0, rho, B, mu, n; ``fprime``
    defaults to ``f``.
    """
    fp = f if fprime is None else fprime
    return OrkKernel(0, f["c0"], f["rho"], f["B"], f["mu"], int(f["n"]),
                     fp["c0"], fp["rho"], fp["B"], fp["mu"], int(fp["n"]), 0.0)


def factor_kernel_terms(terms, terms_prime=None) -> OrkKernel:
    """Kernel record for a factor pair given as sums of terms c r^a e^{b r - g r^2}.

    ``terms`` and ``terms_prime`` are sequences of (c, a, b, g) (at most 16
    each); ``terms_prime`` defaults to ``terms``.  The classes' kernels are
    formed from them as for the range-separated factor (Eqs. k1-k6, I6_).
    """
    tp = terms if terms_prime is None else terms_prime
    if not (0 < len(terms) <= MAX_TERMS and 0 < len(tp) <= MAX_TERMS):
        raise ValueError("1 to %d terms per factor" % MAX_TERMS)
    k = OrkKernel(K_TERMS, 0.0, 0.0, 0.0, 1.0, 0, 0.0, 0.0, 0.0, 1.0, 0, 0.0)
    k.nt, k.ntp = len(terms), len(tp)
    for i, row in enumerate(terms):
        for j in range(4):
            k.t[i][j] = float(row[j])
    for i, row in enumerate(tp):
        for j in range(4):
            k.tp[i][j] = float(row[j])
    return k


def test_kernel(kid: int, gam: float = 0.0) -> OrkKernel:
    return OrkKernel(kid, 0.0, 0.0, 0.0, 1.0, 0, 0.0, 0.0, 0.0, 1.0, 0, gam)


def radial(kern: OrkKernel, cls: int, xi: float, D: float, nmax: int) -> np.ndarray:
    """hat g_n(xi, D) for n = 0..nmax.  g_n = sqrt(pi^5/(p+q))/(p q) * hat g_n."""
    out = np.zeros(nmax + 1)
    rc = lib().ork_radial(ctypes.byref(kern), cls, float(xi), float(D), nmax, _dp(out))
    if rc:
        raise RuntimeError("oracle radial quadrature failed (%d)" % rc)
    return out


def radial_mode(kern: OrkKernel, cls: int, xi: float, D: float, nmax: int, mode: int) -> np.ndarray:
    """As :func:`radial` with the integrand form forced (0 Bessel, 1 separated
    exponentials, 2 derivatives on x k(x) for very large T)."""
    out = np.zeros(nmax + 1)
    rc = lib().ork_radial_mode(ctypes.byref(kern), cls, float(xi), float(D), nmax, int(mode), _dp(out))
    if rc:
        raise RuntimeError("oracle radial quadrature failed (%d)" % rc)
    return out


def jhat(z: float, N: int) -> np.ndarray:
    out = np.zeros(N + 1)
    lib().ork_jhat(float(z), N, _dp(out))
    return out


def kernel_value(kern: OrkKernel, cls: int, r: float) -> float:
    return lib().ork_kernel_value(ctypes.byref(kern), cls, float(r))


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def prim_block(kern: OrkKernel, cls: int, ls, exps, centers) -> np.ndarray:
    """Block [a][b][c][d] of one primitive quartet (unnormalised Cartesian GTOs)."""
    ls = np.ascontiguousarray(ls, dtype=np.int32)
    exps = np.ascontiguousarray(exps, dtype=np.float64)
    centers = np.ascontiguousarray(centers, dtype=np.float64).reshape(4, 3)
    shape = tuple(ncart(int(l)) for l in ls)
    out = np.zeros(int(np.prod(shape)))
    rc = lib().ork_prim_block(ctypes.byref(kern), cls, _ip(ls), _dp(exps), _dp(centers), _dp(out))
    if rc:
        raise RuntimeError("oracle primitive block failed (%d)" % rc)
    return out.reshape(shape)


def shell_blocks(kern: OrkKernel, cls: int, basis, quartets, offsets=None, nthreads: int = 0,
                 with_mag: bool = False):
    """Contracted blocks for a list of shell quartets.

    ``basis`` has arrays centers[nshell,3], l[nshell], nprim[nshell],
    exps[total], coefs[total] (attribute or key access).  Returns
    (out, offsets) with each block stored row-major [a][b][c][d]; with
    ``with_mag`` also the magnitude of the terms each element sums,
    (out, offsets, mag).
    """
    get = (lambda k: basis[k]) if isinstance(basis, dict) else (lambda k: getattr(basis, k))
    centers = np.ascontiguousarray(get("centers"), dtype=np.float64)
    l = np.ascontiguousarray(get("l"), dtype=np.int32)
    nprim = np.ascontiguousarray(get("nprim"), dtype=np.int32)
    prim_off = np.ascontiguousarray(np.concatenate([[0], np.cumsum(nprim)[:-1]]), dtype=np.int32)
    exps = np.ascontiguousarray(get("exps"), dtype=np.float64)
    coefs = np.ascontiguousarray(get("coefs"), dtype=np.float64)
    q = np.ascontiguousarray(quartets, dtype=np.int32).reshape(-1, 4)
    sizes = np.array([ncart(l[a]) * ncart(l[b]) * ncart(l[c]) * ncart(l[d]) for a, b, c, d in q], dtype=np.int64)
    if offsets is None:
        offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    total = int(offsets[-1] + sizes[-1]) if len(q) else 0
    out = np.zeros(max(total, 1))
    mag = np.zeros(max(total, 1)) if with_mag else None
    nbad = lib().ork_shell_blocks(ctypes.byref(kern), cls, _dp(centers), _ip(l), _ip(nprim), _ip(prim_off),
                                  _dp(exps), _dp(coefs), len(q),
                                  q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out),
                                  _dp(mag) if with_mag else None, nthreads)
    if nbad:
        raise RuntimeError("oracle quadrature did not converge for %d primitive quartets" % nbad)
    if with_mag:
        return out[:total], offsets, mag[:total]
    return out[:total], offsets
