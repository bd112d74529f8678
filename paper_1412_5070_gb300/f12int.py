"""Thin Python binding of the C ABI in include/f12int.h.

Argument marshalling only: every step of the integral path runs in the CUDA
library ``_build/libf12int.so``.  PyTorch supplies device memory and
streams (tensors' ``data_ptr()`` and ``torch.cuda.Stream.cuda_stream``).
The functions carry the C names; a nonzero status raises F12IntError.
Importing this module does not need a GPU; loading the library does need
the library to have been built (``paper_1412_5070_gb300.build``) and fails
loudly otherwise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

F12INT_I1, F12INT_I2, F12INT_I3, F12INT_I4, F12INT_I5, F12INT_I6 = 1, 2, 3, 4, 5, 6
OK, EINVAL, ENOMEM, EDOMAIN, ENOTREADY, ETIMEOUT, ECUDA, EDEVICE = 0, -1, -2, -3, -4, -5, -6, -7
STATUS = {0: "F12INT_OK", -1: "F12INT_EINVAL", -2: "F12INT_ENOMEM", -3: "F12INT_EDOMAIN",
          -4: "F12INT_ENOTREADY", -5: "F12INT_ETIMEOUT", -6: "F12INT_ECUDA", -7: "F12INT_EDEVICE"}

# every entry point declared in include/f12int.h
EXPORTS = ("f12int_create", "f12int_destroy", "f12int_set_basis", "f12int_set_factor", "f12int_set_factor_terms",
           "f12int_kernel_radial_terms", "f12int_factor_classes", "f12int_factor_classes_terms", "f12int_screen",
           "f12int_compute_class", "f12int_compute_class_mixed", "f12int_compute_class_static", "f12int_aux", "f12int_launch_count",
           "f12int_device_status", "f12int_set_timing", "f12int_kernel_stats", "f12int_kernel_radial",
           "f12int_submit", "f12int_poll", "f12int_batch_limits", "f12int_batch_autotune", "f12int_batch_stats",
           "f12int_set_fp32_below", "f12int_pair_bounds", "f12int_quartet_estimates",
           "f12int_measure_peak", "f12int_host_stats", "f12int_set_series_cap", "f12int_strerror")


class F12IntError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.f12int_strerror(status).decode() if _lib is not None else STATUS.get(status, "?")
        super().__init__("%s failed: %s (%s)" % (where, STATUS.get(status, status), msg))


class Factor(ctypes.Structure):
    _fields_ = [("c0", ctypes.c_double), ("rho", ctypes.c_double), ("B", ctypes.c_double),
                ("mu", ctypes.c_double), ("n", ctypes.c_int)]

    @classmethod
    def of(cls, d):
        return cls(float(d["c0"]), float(d["rho"]), float(d["B"]), float(d["mu"]), int(d["n"]))


class Term(ctypes.Structure):
    """c r^a exp(b r - g r^2)."""
    _fields_ = [("c", ctypes.c_double), ("a", ctypes.c_double), ("b", ctypes.c_double), ("g", ctypes.c_double)]


def _terms(rows):
    rows = [tuple(float(v) for v in r) for r in rows]
    arr = (Term * max(len(rows), 1))(*[Term(*r) for r in rows])
    return arr, len(rows)


class Request(ctypes.Structure):
    _fields_ = [("n_quartets", ctypes.c_int64), ("quartets", ctypes.POINTER(ctypes.c_int32)),
                ("class_mask", ctypes.c_uint32), ("precision", ctypes.c_int), ("schwarz_thresh", ctypes.c_double),
                ("out_dev", ctypes.c_void_p), ("offsets", ctypes.POINTER(ctypes.c_int64))]


_lib = None
_vp, _dp, _ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)


def library_path() -> str:
    return _build.LIB


def load():
    """Load the compiled library; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError("CUDA library %s is missing: run paper_1412_5070_gb300.build.build() first" % path)
    L = ctypes.CDLL(path)
    L.f12int_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t, _vp]
    L.f12int_destroy.argtypes = [_vp]
    L.f12int_set_basis.argtypes = [_vp, ctypes.c_int, _dp, _ip, _ip, _dp, _dp, _ip]
    L.f12int_set_factor.argtypes = [_vp, ctypes.POINTER(Factor), ctypes.POINTER(Factor)]
    L.f12int_set_factor_terms.argtypes = [_vp, ctypes.POINTER(Term), ctypes.c_int, ctypes.POINTER(Term), ctypes.c_int]
    L.f12int_kernel_radial_terms.argtypes = [ctypes.c_int, ctypes.POINTER(Term), ctypes.c_int, ctypes.POINTER(Term),
                                             ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp]
    L.f12int_factor_classes.argtypes = [ctypes.POINTER(Factor), ctypes.POINTER(Factor), _ip]
    L.f12int_factor_classes_terms.argtypes = [ctypes.POINTER(Term), ctypes.c_int, ctypes.POINTER(Term), ctypes.c_int,
                                              _ip]
    L.f12int_screen.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                ctypes.POINTER(ctypes.c_int32), ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    L.f12int_compute_class.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int64, _vp, _vp, _vp]
    L.f12int_compute_class_mixed.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int64, _vp, _vp,
                                             ctypes.c_double, _vp]
    L.f12int_compute_class_static.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int64, _vp, _vp, _vp]
    L.f12int_aux.argtypes = [_vp, ctypes.c_int, ctypes.c_int64, _vp, _vp, ctypes.c_int, _vp, _vp]
    L.f12int_launch_count.argtypes = [_vp]
    L.f12int_launch_count.restype = ctypes.c_int64
    L.f12int_device_status.argtypes = [_vp]
    L.f12int_set_timing.argtypes = [_vp, ctypes.c_int]
    L.f12int_kernel_radial.argtypes = [ctypes.c_int, ctypes.POINTER(Factor), ctypes.POINTER(Factor), ctypes.c_int,
                                       ctypes.c_double, _dp]
    L.f12int_kernel_stats.argtypes = [_vp, ctypes.c_int, _dp]
    L.f12int_submit.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    L.f12int_poll.argtypes = [_vp, ctypes.c_uint64, ctypes.c_int64, _ip]
    L.f12int_batch_limits.argtypes = [_vp, ctypes.c_int64, ctypes.c_int64]
    L.f12int_batch_stats.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
    L.f12int_set_fp32_below.argtypes = [_vp, ctypes.c_double]
    L.f12int_pair_bounds.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _dp]
    L.f12int_quartet_estimates.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.c_int64, _dp]
    L.f12int_batch_autotune.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64,
                                        ctypes.c_uint32, _dp]
    L.f12int_measure_peak.argtypes = [ctypes.c_int, ctypes.c_int, _dp]
    L.f12int_host_stats.argtypes = [_vp, ctypes.c_int, _dp]
    L.f12int_set_series_cap.argtypes = [_vp, ctypes.c_int]
    L.f12int_strerror.argtypes = [ctypes.c_int]
    L.f12int_strerror.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("f12int_launch_count", "f12int_strerror"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, where: str):
    if rc != 0:
        raise F12IntError(rc, where)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _ptr(t):
    """Device pointer of a torch tensor (must be contiguous and on CUDA)."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def f12int_strerror(status: int) -> str:
    return load().f12int_strerror(int(status)).decode()


def f12int_create(device: int = 0, hbm_budget_bytes: int = 0, stream=None):
    L = load()
    h = _vp()
    _check(L.f12int_create(ctypes.byref(h), int(device), int(hbm_budget_bytes), _stream_ptr(stream)),
           "f12int_create")
    return h


def f12int_destroy(ctx) -> None:
    _check(load().f12int_destroy(ctx), "f12int_destroy")


def f12int_set_basis(ctx, basis) -> int:
    c = np.ascontiguousarray(basis.centers, dtype=np.float64)
    l = np.ascontiguousarray(basis.l, dtype=np.int32)
    npr = np.ascontiguousarray(basis.nprim, dtype=np.int32)
    e = np.ascontiguousarray(basis.exps, dtype=np.float64)
    co = np.ascontiguousarray(basis.coefs, dtype=np.float64)
    bid = ctypes.c_int(-1)
    _check(load().f12int_set_basis(ctx, len(l), c.ctypes.data_as(_dp), l.ctypes.data_as(_ip),
                                   npr.ctypes.data_as(_ip), e.ctypes.data_as(_dp), co.ctypes.data_as(_dp),
                                   ctypes.byref(bid)), "f12int_set_basis")
    return bid.value


def f12int_set_factor(ctx, f, fprime=None) -> None:
    F = Factor.of(f)
    Fp = Factor.of(fprime) if fprime is not None else None
    _check(load().f12int_set_factor(ctx, ctypes.byref(F), ctypes.byref(Fp) if Fp is not None else None),
           "f12int_set_factor")


def f12int_set_factor_terms(ctx, terms, terms_prime=None) -> None:
    """Factors as sums of terms: ``terms`` (and ``terms_prime``, default the
    same) are sequences of (c, a, b, g) for c r^a exp(b r - g r^2)."""
    t, n = _terms(terms)
    if terms_prime is None:
        _check(load().f12int_set_factor_terms(ctx, t, n, None, 0), "f12int_set_factor_terms")
    else:
        tp, npr = _terms(terms_prime)
        _check(load().f12int_set_factor_terms(ctx, t, n, tp, npr), "f12int_set_factor_terms")


def f12int_screen(ctx, basis_id: int, cls: int, thresh: float, cap: int = 0) -> np.ndarray:
    """Canonical quartets surviving the Schwarz-type screen (host int32 [n, 4])."""
    L = load()
    n = ctypes.c_int64(0)
    _check(L.f12int_screen(ctx, int(basis_id), int(cls), float(thresh), None, 0, ctypes.byref(n)), "f12int_screen")
    out = np.zeros((max(n.value, 1), 4), dtype=np.int32)
    _check(L.f12int_screen(ctx, int(basis_id), int(cls), float(thresh),
                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n.value, ctypes.byref(n)),
           "f12int_screen")
    return out[: n.value]


def f12int_compute_class(ctx, basis_id: int, cls: int, quartets_dev, out_dev, offsets_dev, stream=None) -> None:
    n = quartets_dev.numel() // 4
    _check(load().f12int_compute_class(ctx, int(basis_id), int(cls), _ptr(quartets_dev), n, _ptr(out_dev),
                                       _ptr(offsets_dev), _stream_ptr(stream)), "f12int_compute_class")


def f12int_compute_class_mixed(ctx, basis_id: int, cls: int, quartets_dev, out_dev, offsets_dev, fp32_below: float,
                               stream=None) -> None:
    """As f12int_compute_class, with the Hermite recursion and contraction in
    FP32 for quartets whose shell-pair bound product is below fp32_below."""
    n = quartets_dev.numel() // 4
    _check(load().f12int_compute_class_mixed(ctx, int(basis_id), int(cls), _ptr(quartets_dev), n, _ptr(out_dev),
                                             _ptr(offsets_dev), float(fp32_below), _stream_ptr(stream)),
           "f12int_compute_class_mixed")


def f12int_compute_class_static(ctx, basis_id: int, cls: int, quartets_dev, out_dev, offsets_dev,
                                stream=None) -> None:
    """As f12int_compute_class, for callers that cannot allocate device memory
    during the call: the library's scratch comes from one fixed device array
    per GPU (64 MiB, shared by every call on that GPU, so calls must not
    overlap on the device).  The first call on a device resolves that array's
    address and should happen before any stream capture."""
    n = quartets_dev.numel() // 4
    _check(load().f12int_compute_class_static(ctx, int(basis_id), int(cls), _ptr(quartets_dev), n, _ptr(out_dev),
                                              _ptr(offsets_dev), _stream_ptr(stream)),
           "f12int_compute_class_static")


def f12int_aux(ctx, cls: int, xi_dev, D_dev, nmax: int, out_dev, stream=None) -> None:
    _check(load().f12int_aux(ctx, int(cls), xi_dev.numel(), _ptr(xi_dev), _ptr(D_dev), int(nmax), _ptr(out_dev),
                             _stream_ptr(stream)), "f12int_aux")


def f12int_launch_count(ctx) -> int:
    return int(load().f12int_launch_count(ctx))


def f12int_kernel_radial(cls: int, f, l: int, x: float, fprime=None) -> float:
    """x^{2l+2} (D_r^l k)(x) from the host-side term lists (no GPU needed)."""
    F = Factor.of(f)
    Fp = Factor.of(fprime) if fprime is not None else None
    v = ctypes.c_double(0.0)
    _check(load().f12int_kernel_radial(int(cls), ctypes.byref(F), ctypes.byref(Fp) if Fp is not None else None,
                                       int(l), float(x), ctypes.byref(v)), "f12int_kernel_radial")
    return v.value


def f12int_factor_classes(f, fprime=None) -> dict:
    """{class: 0 left out / 1 served / 3 served, with the quadrature launch}
    for an Eq. rs12 factor pair (no GPU needed)."""
    F = Factor.of(f)
    Fp = Factor.of(fprime) if fprime is not None else None
    flags = (ctypes.c_int * 7)()
    _check(load().f12int_factor_classes(ctypes.byref(F), ctypes.byref(Fp) if Fp is not None else None, flags),
           "f12int_factor_classes")
    return {c: flags[c] for c in range(1, 7)}


def f12int_factor_classes_terms(terms, terms_prime=None) -> dict:
    """f12int_factor_classes for factors given as terms."""
    t, n = _terms(terms)
    flags = (ctypes.c_int * 7)()
    if terms_prime is None:
        rc = load().f12int_factor_classes_terms(t, n, None, 0, flags)
    else:
        tp, npr = _terms(terms_prime)
        rc = load().f12int_factor_classes_terms(t, n, tp, npr, flags)
    _check(rc, "f12int_factor_classes_terms")
    return {c: flags[c] for c in range(1, 7)}


def f12int_kernel_radial_terms(cls: int, terms, l: int, x: float, terms_prime=None) -> float:
    """f12int_kernel_radial for factors given as terms (no GPU needed)."""
    t, n = _terms(terms)
    v = ctypes.c_double(0.0)
    if terms_prime is None:
        rc = load().f12int_kernel_radial_terms(int(cls), t, n, None, 0, int(l), float(x), ctypes.byref(v))
    else:
        tp, npr = _terms(terms_prime)
        rc = load().f12int_kernel_radial_terms(int(cls), t, n, tp, npr, int(l), float(x), ctypes.byref(v))
    _check(rc, "f12int_kernel_radial_terms")
    return v.value


def f12int_set_timing(ctx, on: bool) -> None:
    _check(load().f12int_set_timing(ctx, 1 if on else 0), "f12int_set_timing")


def f12int_kernel_stats(ctx, reset: bool = False) -> dict:
    s = (ctypes.c_double * 6)()
    _check(load().f12int_kernel_stats(ctx, 1 if reset else 0, s), "f12int_kernel_stats")
    return {"aux_ms": s[0], "aux_launches": int(s[1]), "contract_ms": s[2], "contract_launches": int(s[3]),
            "aux_flops": s[4], "contract_flops": s[5]}


def f12int_device_status(ctx) -> None:
    _check(load().f12int_device_status(ctx), "f12int_device_status")


def f12int_submit(ctx, basis_id: int, quartets, classes, out_dev, offsets, schwarz_thresh: float = 0.0,
                  precision: int = 0) -> int:
    """Queue the blocks of ``classes`` (iterable of 1..6) over the host quartet
    list ``quartets`` [n, 4] into the CUDA tensor ``out_dev``; ``offsets`` is a
    host int64 array [len(classes), n] (rows in increasing class order).
    Returns the ticket."""
    q = np.ascontiguousarray(quartets, dtype=np.int32).reshape(-1, 4)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    mask = 0
    for c in classes:
        mask |= 1 << (int(c) - 1)
    req = Request(len(q), q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), mask, int(precision),
                  float(schwarz_thresh), _ptr(out_dev), off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    t = ctypes.c_uint64(0)
    _check(load().f12int_submit(ctx, int(basis_id), ctypes.byref(req), ctypes.byref(t)), "f12int_submit")
    return t.value


def f12int_poll(ctx, ticket: int, timeout_us: int = 0) -> bool:
    """True once the request has finished (its status is checked: a failed
    request raises F12IntError); False while it is queued or running (the
    library's F12INT_ETIMEOUT of a wait that ran out)."""
    done = ctypes.c_int(0)
    rc = load().f12int_poll(ctx, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(done))
    if rc == ETIMEOUT and not done.value:
        return False
    _check(rc, "f12int_poll")
    return bool(done.value)


def f12int_poll_status(ctx, ticket: int, timeout_us: int = 0):
    """(status, done) exactly as the C call returns them."""
    done = ctypes.c_int(0)
    rc = load().f12int_poll(ctx, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(done))
    return rc, bool(done.value)


def f12int_batch_limits(ctx, max_quartets: int, max_items: int) -> None:
    _check(load().f12int_batch_limits(ctx, int(max_quartets), int(max_items)), "f12int_batch_limits")


def f12int_batch_stats(ctx) -> dict:
    s = (ctypes.c_int64 * 3)()
    _check(load().f12int_batch_stats(ctx, s), "f12int_batch_stats")
    return {"batches": int(s[0]), "requests_done": int(s[1]), "pending": int(s[2])}


def f12int_batch_autotune(ctx, basis_id: int, quartets, classes) -> dict:
    """Measure and keep the fastest batch schedule of each class on the host
    sample ``quartets`` [n, 4]; returns {class: (task target, grid divisor,
    seconds)}."""
    q = np.ascontiguousarray(quartets, dtype=np.int32).reshape(-1, 4)
    mask = 0
    for c in classes:
        mask |= 1 << (int(c) - 1)
    rep = (ctypes.c_double * 18)()
    _check(load().f12int_batch_autotune(ctx, int(basis_id), q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                        len(q), mask, rep), "f12int_batch_autotune")
    return {int(c): (rep[3 * (c - 1)], int(rep[3 * (c - 1) + 1]), rep[3 * (c - 1) + 2]) for c in classes}


def f12int_set_fp32_below(ctx, bound: float) -> None:
    _check(load().f12int_set_fp32_below(ctx, float(bound)), "f12int_set_fp32_below")


def f12int_pair_bounds(ctx, basis_id: int, cls: int, nshell: int) -> np.ndarray:
    """Shell-pair bounds sqrt(max |(ab|k|ab)|) of class cls, [nshell, nshell]."""
    out = np.zeros((nshell, nshell))
    _check(load().f12int_pair_bounds(ctx, int(basis_id), int(cls), out.ctypes.data_as(_dp)), "f12int_pair_bounds")
    return out


def f12int_quartet_estimates(ctx, basis_id: int, cls: int, quartets) -> np.ndarray:
    """The screening estimate of f12int_screen for each host quartet [n, 4]."""
    q = np.ascontiguousarray(quartets, dtype=np.int32).reshape(-1, 4)
    out = np.zeros(len(q))
    _check(load().f12int_quartet_estimates(ctx, int(basis_id), int(cls),
                                           q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(q),
                                           out.ctypes.data_as(_dp)), "f12int_quartet_estimates")
    return out


PEAK_KINDS = {"fp64_fma": 0, "fp64_mma_m8n8k4": 1, "fp64_mma_m16n8k4": 2, "fp64_mma_m16n8k16": 3, "fp32_fma": 4}


def f12int_measure_peak(device: int, kind) -> float:
    """Measured peak of one instruction kind on a device, TFLOP/s (kind: a key
    of PEAK_KINDS or its number)."""
    k = PEAK_KINDS[kind] if isinstance(kind, str) else int(kind)
    v = ctypes.c_double(0.0)
    _check(load().f12int_measure_peak(int(device), k, ctypes.byref(v)), "f12int_measure_peak")
    return v.value


def f12int_host_stats(ctx, reset: bool = False) -> dict:
    """Host planning time of f12int_compute_class calls: {"plan_ms", "calls"}."""
    st = (ctypes.c_double * 2)()
    _check(load().f12int_host_stats(ctx, 1 if reset else 0, st), "f12int_host_stats")
    return {"plan_ms": st[0], "calls": int(st[1])}


def f12int_set_series_cap(ctx, kmax: int) -> None:
    """Cap on the auxiliary series length (0 restores the default); a series
    that reaches it sets the device status word (F12INT_EDEVICE)."""
    _check(load().f12int_set_series_cap(ctx, int(kmax)), "f12int_set_series_cap")
