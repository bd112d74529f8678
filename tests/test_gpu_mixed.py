"""Mixed precision (FP32 Hermite recursion and contraction for small-bound
quartets) against the oracle and the FP64 path.

Bar: absolute error <= 1e-10 on every element of the quartets that take the
FP32 path; the FP64 quartets of a mixed call are bitwise those of the plain
FP64 call (and so meet the FP64 bar).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_1412_5070_gb300 import build as B
from paper_1412_5070_gb300 import f12int as F
from paper_1412_5070_gb300 import molecules as M

FP32_BELOW = 1e-5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    c = F.f12int_create(0, 0, None)
    F.f12int_set_factor(c, M.P0)
    yield c
    F.f12int_destroy(c)


def run(ctx, bid, cls, basis, q, fp32_below):
    q = np.ascontiguousarray(q, dtype=np.int32)
    off = M.block_offsets(basis, q)
    out = torch.full((int(off[-1]),), float("nan"), dtype=torch.float64, device="cuda")
    dq, doff = torch.from_numpy(q).cuda(), torch.from_numpy(off[:-1].copy()).cuda()
    if fp32_below > 0:
        F.f12int_compute_class_mixed(ctx, bid, cls, dq, out, doff, fp32_below)
    else:
        F.f12int_compute_class(ctx, bid, cls, dq, out, doff)
    torch.cuda.synchronize()
    F.f12int_device_status(ctx)
    return out.cpu().numpy(), off


def bounds(ctx, bid, cls, basis, q):
    """Screening estimates of the quartets (the FP32 decision's quantity)."""
    return F.f12int_quartet_estimates(ctx, bid, cls, q)


@pytest.mark.parametrize("cls", [1, 2, 3, 4, 5, 6])
def test_mixed_against_oracle(ctx, cls):
    """12-atom s/p/d molecule: quartets on both sides of the FP32 bound;
    every element within 1e-10 of the oracle, FP64-side blocks unchanged."""
    basis = M.twelve_atom_spd(2)
    bid = F.f12int_set_basis(ctx, basis)
    q = M.canonical_quartets(basis, cls)
    rng = np.random.default_rng(90 + cls)
    q = q[np.sort(rng.choice(len(q), size=240, replace=False))]
    lo = bounds(ctx, bid, cls, basis, q)
    assert (lo < FP32_BELOW).sum() >= 30 and (lo >= FP32_BELOW).sum() >= 10
    got, off = run(ctx, bid, cls, basis, q, FP32_BELOW)
    full, _ = run(ctx, bid, cls, basis, q, 0.0)
    ref, _ = O.shell_blocks(O.factor_kernel(M.P0), cls, basis, q)
    f32 = np.zeros(len(got), dtype=bool)
    for i in np.nonzero(lo < FP32_BELOW)[0]:
        f32[off[i]:off[i + 1]] = True
    err = np.abs(got - ref)[f32]
    print("class %d: FP32-side max abs error %.3g (FP64 path on the same elements %.3g)" % (
        cls, err.max(), np.abs(full - ref)[f32].max()))
    assert err.max() <= 1e-10
    assert np.array_equal(got[~f32], full[~f32])


def test_mixed_request(ctx):
    """precision = 1 through f12int_submit gives the blocks of the mixed call."""
    basis = M.twelve_atom_spd(2)
    bid = F.f12int_set_basis(ctx, basis)
    q = M.canonical_quartets(basis, 3)[::997]
    F.f12int_set_fp32_below(ctx, FP32_BELOW)
    off = M.block_offsets(basis, q)
    out = torch.full((int(off[-1]),), float("nan"), dtype=torch.float64, device="cuda")
    t = F.f12int_submit(ctx, bid, q, (3,), out, off[:-1][None, :], precision=1)
    while not F.f12int_poll(ctx, t, 1000):
        pass
    direct = torch.full_like(out, float("nan"))
    F.f12int_compute_class_mixed(ctx, bid, 3, torch.from_numpy(np.ascontiguousarray(q)).cuda(), direct,
                                 torch.from_numpy(off[:-1].copy()).cuda(), FP32_BELOW)
    torch.cuda.synchronize()
    tol = 1e-13 * torch.abs(direct) + 1e-15 * torch.max(torch.abs(direct))
    assert bool(torch.all(torch.abs(out - direct) <= tol))
