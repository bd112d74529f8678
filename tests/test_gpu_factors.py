"""Parity of the CUDA path with the oracle for other parameter sets of the
correlation factor (Eq. rs12, Eq. ttdamp), which reach other branches of
the auxiliary stage: an integer power (rho = -1, finite parts of integer
alpha), a negative half-integer power with n = 1 damping, the B = 0 limit,
no long-range term (c0 = 0), and f' different from f (I4, I6)."""
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
}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def supported(f, fp, cls):
    """The auxiliary stage evaluates S(alpha) for alpha > -1 and the alpha = -1
    finite part; the lowest power of x^2 k(x) among the kernel's long-range
    terms is rho + 2 (k3), rho + 1 (k2), rho + rho' + 2 (k4), rho + rho' (k6)."""
    if f["c0"] == 0 and fp["c0"] == 0:
        return True
    low = {2: f["rho"] + 1, 3: f["rho"] + 2, 5: f["rho"] + 2,
           4: (f["rho"] if f["c0"] else 0) + (fp["rho"] if fp["c0"] else 0) + 2,
           6: (f["rho"] - 1 if f["c0"] else 0) + (fp["rho"] - 1 if fp["c0"] else 0) + 2}[cls]
    return low > -1 or low == -1


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
    bad = close(got, ref, mag)
    assert not np.isnan(got).any()
    assert not bad.any(), report(got, ref, mag, bad)
