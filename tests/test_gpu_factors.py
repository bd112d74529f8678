"""Parity of the CUDA path with the oracle for other parameter sets of the
correlation factor (Eq. rs12, Eq. ttdamp), which reach other branches of
the auxiliary stage: an integer power (rho = -1, finite parts of integer
alpha), a negative half-integer power with n = 1 damping, the B = 0 limit,
no long-range term (c0 = 0), f' different from f (I4, I6), and B < 0 (a
decaying long-range part, whose families go to the Gauss-Legendre branch
and a second evaluation launch)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_1412_5070_gb300 import build as B
from paper_1412_5070_gb300 import f12int as F
from paper_1412_5070_gb300 import molecules as M

from test_gpu_parity import close, report

P0 = M.P0
SETS = {
    "P1 rho=-1": (dict(P0, rho=-1.0), None),
    "P2 rho=-2.5 n=1": (dict(P0, rho=-2.5, n=1), None),
    "P3 rho=0 B=0": (dict(P0, rho=0.0, B=0.0), None),
    "P4 f'!=f": (P0, dict(c0=0.3, rho=-0.3, B=0.3, mu=0.7, n=0)),
    "P5 c0=0": (dict(P0, c0=0.0), None),
    "N1 B<0": (dict(P0, B=-0.8), None),
    "N2 rho=0 B<0 n=1": (dict(c0=1.0, rho=0.0, B=-1.3, mu=1.5, n=1), None),
    "N3 f' B<0": (P0, dict(c0=0.3, rho=0.5, B=-1.2, mu=0.7, n=0)),
    "N4 rho=-0.3 B<0": (dict(P0, rho=-0.3, B=-0.8), None),
}
DECAYING = dict(c0=0.5, rho=-0.5, B=-0.8, mu=1.0, n=0)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def lowest_power(f, fp, cls):
    """Lowest power of x^2 k(x) among the kernel's long-range terms: rho + 2
    (k3), rho + 1 (k2), rho + rho' + 2 (k4), rho + rho' (k6)."""
    return {2: f["rho"] + 1, 3: f["rho"] + 2, 5: f["rho"] + 2,
            4: (f["rho"] if f["c0"] else 0) + (fp["rho"] if fp["c0"] else 0) + 2,
            6: (f["rho"] - 1 if f["c0"] else 0) + (fp["rho"] - 1 if fp["c0"] else 0) + 2}[cls]


def supported(f, fp, cls):
    """The auxiliary stage serves a lowest power of x^2 k(x) (lowest_power())
    below -1 when it is an integer or a half-integer (the damping of Eq. rs12
    makes the singular terms cancel)."""
    if f["c0"] == 0 and fp["c0"] == 0:
        return True
    # a term group with b < 0 must have an integer or half-integer power
    # (the end-point forms of the Gauss-Legendre branch)
    groups = []
    if f["c0"]:
        groups.append((f["B"], f["rho"]))
    if cls in (4, 6):
        if fp["c0"]:
            groups.append((fp["B"], fp["rho"]))
        if f["c0"] and fp["c0"]:
            groups.append((f["B"] + fp["B"], f["rho"] + fp["rho"]))
    if any(b < 0 and abs(2 * a - round(2 * a)) > 1e-9 for b, a in groups):
        return False
    low = lowest_power(f, fp, cls)
    return not (low < -1 and abs(2 * low - round(2 * low)) > 1e-9)


@pytest.mark.parametrize("name", list(SETS))
@pytest.mark.parametrize("cls", [2, 3, 4, 5, 6])
def test_factor_sets_two_centre(dev, name, cls):
    f, fp = SETS[name]
    fpp = fp if fp is not None else f
    ctx = F.f12int_create(0, 0, None)
    if not supported(f, fpp, cls):
        try:
            F.f12int_set_factor(ctx, f, fp)   # accepted: the class alone is left out
            basis = M.two_centre_sp()
            bid = F.f12int_set_basis(ctx, basis)
            q = M.canonical_quartets(basis, cls)[:4]
            off = M.block_offsets(basis, q)
            out = torch.zeros(int(off[-1]), dtype=torch.float64, device="cuda")
            with pytest.raises(F.F12IntError) as e:
                F.f12int_compute_class(ctx, bid, cls, torch.from_numpy(q).cuda(), out,
                                       torch.from_numpy(off[:-1].copy()).cuda())
            assert e.value.status == -3
        finally:
            F.f12int_destroy(ctx)
        return
    try:
        F.f12int_set_factor(ctx, f, fp)
        basis = M.two_centre_sp()
        bid = F.f12int_set_basis(ctx, basis)
        q = M.canonical_quartets(basis, cls)[3::12]
        off = M.block_offsets(basis, q)
        out = torch.full((int(off[-1]),), float("nan"), dtype=torch.float64, device="cuda")
        F.f12int_compute_class(ctx, bid, cls, torch.from_numpy(q).cuda(), out,
                               torch.from_numpy(off[:-1].copy()).cuda())
        torch.cuda.synchronize()
        F.f12int_device_status(ctx)
        got = out.cpu().numpy()
    finally:
        F.f12int_destroy(ctx)
    ref, _, mag = O.shell_blocks(O.factor_kernel(f, fp), cls, basis, q, with_mag=True)
    assert not np.isnan(got).any()
    if (f["c0"] or fpp["c0"]) and lowest_power(f, fpp, cls) < -1:
        # singular families evaluated as groups: hat g_n to 1e-10 on the CPU
        # for xi <= 2; 1e-9 here leaves room for the GPU's rounding (with the
        # term-magnitude allowance of the parity tests)
        big = np.abs(ref) > 1e-12
        tol = np.maximum(1e-9 * np.abs(ref[big]), 32 * 2.0 ** -53 * mag[big])
        assert np.all(np.abs(got[big] - ref[big]) <= tol)
        assert np.all(np.abs(got[~big] - ref[~big]) <= 1e-12)
        return
    bad = close(got, ref, mag)
    assert not bad.any(), report(got, ref, mag, bad)


XI_D_GRID = [(xi, D) for xi in (0.025, 0.1, 0.5, 2.0, 10.0, 50.0) for D in (0.0, 0.05, 0.3, 1.0, 2.5, 5.0, 7.0,
                                                                            10.0, 20.0)]


@pytest.mark.parametrize("cls", [2, 3, 4, 6])
def test_aux_stage_decaying_factor(dev, cls):
    """hat g_n (n <= 10) of a factor with B < 0 through the C ABI against the
    oracle, on the grid of the aux-stage parity test."""
    nmax = 10
    ctx = F.f12int_create(0, 0, None)
    try:
        F.f12int_set_factor(ctx, DECAYING)
        xi = torch.tensor([p[0] for p in XI_D_GRID], dtype=torch.float64, device="cuda")
        D = torch.tensor([p[1] for p in XI_D_GRID], dtype=torch.float64, device="cuda")
        out = torch.zeros(len(XI_D_GRID) * (nmax + 1), dtype=torch.float64, device="cuda")
        F.f12int_aux(ctx, cls, xi, D, nmax, out)
        torch.cuda.synchronize()
        F.f12int_device_status(ctx)
        got = out.cpu().numpy().reshape(len(XI_D_GRID), nmax + 1)
    finally:
        F.f12int_destroy(ctx)
    K = O.factor_kernel(DECAYING)
    worst = 0.0
    for i, (x, d) in enumerate(XI_D_GRID):
        ref = O.radial(K, cls, x, d, nmax)
        worst = max(worst, float(np.max(np.abs(got[i] - ref) / np.abs(ref))))
    print("class %d worst relative error of hat g_n (B < 0): %.3g" % (cls, worst))
    assert worst < 1e-8


@pytest.mark.parametrize("cls", [3, 5, 6])
def test_decaying_factor_f_shells(dev, cls):
    """f-shell quartets (radial orders up to 12, 14 for I5) with B < 0."""
    from test_gpu_parity import f_shell_molecule
    basis = f_shell_molecule()
    q = M.canonical_quartets(basis, cls)
    q = q[np.any(basis.l[q] == 3, axis=1)][::15 if cls == 5 else 9]
    ctx = F.f12int_create(0, 0, None)
    try:
        F.f12int_set_factor(ctx, DECAYING)
        bid = F.f12int_set_basis(ctx, basis)
        off = M.block_offsets(basis, q)
        out = torch.full((int(off[-1]),), float("nan"), dtype=torch.float64, device="cuda")
        F.f12int_compute_class(ctx, bid, cls, torch.from_numpy(q).cuda(), out, torch.from_numpy(off[:-1].copy()).cuda())
        torch.cuda.synchronize()
        F.f12int_device_status(ctx)
        got = out.cpu().numpy()
    finally:
        F.f12int_destroy(ctx)
    ref, _, mag = O.shell_blocks(O.factor_kernel(DECAYING), cls, basis, q, with_mag=True)
    bad = close(got, ref, mag)
    assert not np.isnan(got).any()
    assert not bad.any(), report(got, ref, mag, bad)


def test_decaying_factor_batch_equals_per_call(dev):
    """The batch engine's captured graph carries the second evaluation launch
    when the factor has b < 0 families: its blocks equal the per-call path's
    (both FP64) to 1e-13."""
    basis = M.twelve_atom_spd(2)
    ctx = F.f12int_create(0, 0, None)
    try:
        F.f12int_set_factor(ctx, DECAYING)
        F.f12int_batch_limits(ctx, 1 << 16, 1 << 21)
        bid = F.f12int_set_basis(ctx, basis)
        q = M.canonical_quartets(basis, 3)
        q = q[np.random.default_rng(3).choice(len(q), size=300, replace=False)]
        classes = (2, 3, 5, 6)
        sizes = np.diff(M.block_offsets(basis, q))
        off = np.stack([k * int(sizes.sum()) + np.concatenate([[0], np.cumsum(sizes)[:-1]])
                        for k in range(len(classes))]).astype(np.int64)
        out = torch.full((len(classes) * int(sizes.sum()),), float("nan"), dtype=torch.float64, device="cuda")
        t = F.f12int_submit(ctx, bid, q, classes, out, off)
        t0 = time.time()
        while not F.f12int_poll(ctx, t, 1000):
            assert time.time() - t0 < 120.0, "request did not finish"
        got_all = out.cpu().numpy()
        for k, cls in enumerate(classes):
            o = M.block_offsets(basis, q)
            ref = torch.full((int(o[-1]),), float("nan"), dtype=torch.float64, device="cuda")
            F.f12int_compute_class(ctx, bid, cls, torch.from_numpy(q).cuda(), ref,
                                   torch.from_numpy(o[:-1].copy()).cuda())
            torch.cuda.synchronize()
            ref = ref.cpu().numpy()
            got = got_all[off[k, 0]:off[k, 0] + len(ref)]
            tol = 1e-13 * np.abs(ref) + 1e-15 * np.max(np.abs(ref))
            assert np.all(np.abs(got - ref) <= tol), (cls, float(np.max(np.abs(got - ref) - tol)))
    finally:
        F.f12int_destroy(ctx)


TERM_SETS = {
    "Ten-no exp(-1.2 r)": [(1.0, 0, -1.2, 0)],
    "three Gaussians": [(0.3, 0, 0, 0.2), (0.25, 0, 0, 1.1), (0.2, 0, 0, 4.0)],
    "Ten-no + Gaussian + r exp": [(-1 / 1.2, 0, -1.2, 0), (0.1, 0, 0, 0.5), (0.05, 1, -0.7, 0.3)],
}


@pytest.mark.parametrize("name", list(TERM_SETS))
@pytest.mark.parametrize("cls", [2, 3, 4, 5, 6])
def test_term_list_factors_two_centre(dev, name, cls):
    """Factors given as term lists (f12int_set_factor_terms): the Ten-no
    factor, a Gaussian geminal and a mixture, on the two-centre s/p basis."""
    t = TERM_SETS[name]
    ctx = F.f12int_create(0, 0, None)
    try:
        F.f12int_set_factor_terms(ctx, t)
        basis = M.two_centre_sp()
        bid = F.f12int_set_basis(ctx, basis)
        q = M.canonical_quartets(basis, cls)[5::12]
        off = M.block_offsets(basis, q)
        out = torch.full((int(off[-1]),), float("nan"), dtype=torch.float64, device="cuda")
        F.f12int_compute_class(ctx, bid, cls, torch.from_numpy(q).cuda(), out,
                               torch.from_numpy(off[:-1].copy()).cuda())
        torch.cuda.synchronize()
        F.f12int_device_status(ctx)
        got = out.cpu().numpy()
    finally:
        F.f12int_destroy(ctx)
    ref, _, mag = O.shell_blocks(O.factor_kernel_terms(t), cls, basis, q, with_mag=True)
    bad = close(got, ref, mag)
    assert not np.isnan(got).any()
    assert not bad.any(), report(got, ref, mag, bad)
