"""The static-scratch entry point (no device allocation during the call).

f12int_compute_class_static serves callers that cannot allocate device
memory while they run (an application that reserves all device memory up
front for its own pool, or a service in which the device-wide
synchronisation of an allocation would stall other streams).  Its blocks
must match those of f12int_compute_class on consecutive calls that reuse the
same fixed device array, and a call must leave the device's free memory as
it found it.  This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_5070_gb300 import build as B
from paper_1412_5070_gb300 import f12int as F
from paper_1412_5070_gb300 import molecules as M

RTOL, SMALL = 1e-10, 1e-12
B_NEGATIVE = dict(c0=0.5, rho=-0.5, B=-0.8, mu=1.0, n=0)   # decaying long range: the quadrature launch


def make_ctx(factor):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    c = F.f12int_create(0, 0, None)
    F.f12int_set_factor(c, factor)
    return c


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx(M.P0)
    yield c
    F.f12int_destroy(c)


@pytest.fixture(scope="module")
def ctx_neg():
    c = make_ctx(B_NEGATIVE)
    yield c
    F.f12int_destroy(c)


def within_tolerance(got, ref):
    big = np.abs(ref) > SMALL
    ok_big = np.all(np.abs(got[big] - ref[big]) <= RTOL * np.abs(ref[big]))
    ok_small = np.all(np.abs(got[~big] - ref[~big]) <= SMALL)
    return bool(ok_big and ok_small)


def check_class(c, basis, cls, nsel, seed):
    """Static calls before and after the allocating path has built its
    primitive screen: within tolerance before, bitwise after, on two calls in
    a row, with the device's free memory unchanged by a static call."""
    bid = F.f12int_set_basis(c, basis)
    q = M.canonical_quartets(basis, cls)
    rng = np.random.default_rng(seed)
    sel = np.ascontiguousarray(q[np.sort(rng.choice(len(q), size=min(nsel, len(q)), replace=False))])
    off = M.block_offsets(basis, sel)
    dq = torch.from_numpy(sel).cuda()
    doff = torch.from_numpy(off[:-1].copy()).cuda()
    # first: no primitive-screen table exists yet for this (basis, class)
    early = torch.full((int(off[-1]),), float("nan"), dtype=torch.float64, device="cuda")
    F.f12int_compute_class_static(c, bid, cls, dq, early, doff)
    torch.cuda.synchronize()
    F.f12int_device_status(c)
    ref = torch.full_like(early, float("nan"))
    F.f12int_compute_class(c, bid, cls, dq, ref, doff)
    torch.cuda.synchronize()
    ref_h = ref.cpu().numpy()
    assert not np.isnan(ref_h).any()
    early_h = early.cpu().numpy()
    assert not np.isnan(early_h).any()
    assert within_tolerance(early_h, ref_h)
    outs = [torch.full_like(ref, float("nan")) for _ in range(2)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for out in outs:   # two calls in a row share the one static array
        F.f12int_compute_class_static(c, bid, cls, dq, out, doff)
        torch.cuda.synchronize()
        F.f12int_device_status(c)
    assert torch.cuda.mem_get_info()[0] == free0
    for out in outs:
        got = out.cpu().numpy()
        assert not np.isnan(got).any()
        assert within_tolerance(got, ref_h)
        assert np.array_equal(got, ref_h)


@pytest.mark.parametrize("cls", [1, 2, 3, 4, 5, 6])
def test_static_scratch_matches_allocating_path(ctx, cls):
    check_class(ctx, M.twelve_atom_spd(2), cls, 3000, 100 + cls)


@pytest.mark.parametrize("cls", [3, 6])
def test_static_scratch_quadrature_launch(ctx_neg, cls):
    """B < 0: families with b < 0 go through the second (quadrature)
    evaluation launch, which the static path queues as well."""
    assert F.f12int_factor_classes(B_NEGATIVE)[cls] == 3
    check_class(ctx_neg, M.twelve_atom_spd(2), cls, 600, 200 + cls)


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
