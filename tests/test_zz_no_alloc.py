"""The static-scratch entry point (no device allocation during the call).

f12int_compute_class_static serves callers that cannot allocate device
memory while they run (an application that reserves all device memory up
front for its own pool, or a service in which the device-wide
synchronisation of an allocation would stall other streams).  Its blocks
must equal those of f12int_compute_class, on consecutive calls that reuse
the same fixed device array.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_5070_gb300 import build as B
from paper_1412_5070_gb300 import f12int as F
from paper_1412_5070_gb300 import molecules as M

RTOL, SMALL = 1e-10, 1e-12


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    c = F.f12int_create(0, 0, None)
    F.f12int_set_factor(c, M.P0)
    yield c
    F.f12int_destroy(c)


def within_tolerance(got, ref):
    big = np.abs(ref) > SMALL
    ok_big = np.all(np.abs(got[big] - ref[big]) <= RTOL * np.abs(ref[big]))
    ok_small = np.all(np.abs(got[~big] - ref[~big]) <= SMALL)
    return bool(ok_big and ok_small)


@pytest.mark.parametrize("cls", [1, 3, 5, 6])
def test_static_scratch_matches_allocating_path(ctx, cls):
    basis = M.twelve_atom_spd(2)
    bid = F.f12int_set_basis(ctx, basis)
    q = M.canonical_quartets(basis, cls)
    rng = np.random.default_rng(100 + cls)
    sel = np.ascontiguousarray(q[np.sort(rng.choice(len(q), size=3000, replace=False))])
    off = M.block_offsets(basis, sel)
    dq = torch.from_numpy(sel).cuda()
    doff = torch.from_numpy(off[:-1].copy()).cuda()
    ref = torch.full((int(off[-1]),), float("nan"), dtype=torch.float64, device="cuda")
    F.f12int_compute_class(ctx, bid, cls, dq, ref, doff)
    torch.cuda.synchronize()
    ref_h = ref.cpu().numpy()
    assert not np.isnan(ref_h).any()
    for _ in range(2):  # two calls in a row share the one static array
        out = torch.full_like(ref, float("nan"))
        F.f12int_compute_class_static(ctx, bid, cls, dq, out, doff)
        torch.cuda.synchronize()
        F.f12int_device_status(ctx)
        got = out.cpu().numpy()
        assert not np.isnan(got).any()
        assert within_tolerance(got, ref_h)


def test_static_scratch_rejects_oversized_lists(ctx):
    basis = M.two_centre_sp()
    bid = F.f12int_set_basis(ctx, basis)
    n = 3_000_000
    dq = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    doff = torch.zeros(n, dtype=torch.int64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(F.F12IntError) as e:
        F.f12int_compute_class_static(ctx, bid, 3, dq, out, doff)
    assert e.value.status == -1
