"""Failure handling of the library, with no GPU fault: every failure here is
made on the host (a budget too small, a request larger than one batch, a wait
that runs out) or by a bounded device-side check (a series length cap that
sets the status word), and each must come back as the documented status with
the context still usable afterwards."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_5070_gb300 import build as B
from paper_1412_5070_gb300 import f12int as F
from paper_1412_5070_gb300 import molecules as M


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    return F


def compute(ctx, bid, cls, basis, q):
    q = np.ascontiguousarray(q, dtype=np.int32)
    off = M.block_offsets(basis, q)
    out = torch.full((int(off[-1]),), float("nan"), dtype=torch.float64, device="cuda")
    F.f12int_compute_class(ctx, bid, cls, torch.from_numpy(q).cuda(), out, torch.from_numpy(off[:-1].copy()).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_budget_too_small_is_enomem_and_the_context_recovers(lib):
    basis = M.twelve_atom_spd(2)
    ctx = F.f12int_create(0, 256 << 20, None)   # 256 MiB
    try:
        F.f12int_set_factor(ctx, M.P0)
        bid = F.f12int_set_basis(ctx, basis)
        q = M.canonical_quartets(basis, 3)
        with pytest.raises(F.F12IntError) as e:
            compute(ctx, bid, 3, basis, q)   # the whole list needs far more scratch than the budget
        assert e.value.status == F.ENOMEM
        small = q[::20000]
        got = compute(ctx, bid, 3, basis, small)   # a small list still fits
        assert not np.isnan(got).any()
        F.f12int_device_status(ctx)
    finally:
        F.f12int_destroy(ctx)
    # the same small list on an unlimited context: the same blocks
    ctx = F.f12int_create(0, 0, None)
    try:
        F.f12int_set_factor(ctx, M.P0)
        bid = F.f12int_set_basis(ctx, basis)
        assert np.array_equal(compute(ctx, bid, 3, basis, q[::20000]), got)
    finally:
        F.f12int_destroy(ctx)


def test_request_larger_than_one_batch_is_refused(lib):
    basis = M.twelve_atom_spd(2)
    ctx = F.f12int_create(0, 0, None)
    try:
        F.f12int_set_factor(ctx, M.P0)
        F.f12int_batch_limits(ctx, 1000, 1 << 22)
        bid = F.f12int_set_basis(ctx, basis)
        q = M.canonical_quartets(basis, 3)[:5000]
        off = M.block_offsets(basis, q)
        out = torch.empty(int(off[-1]), dtype=torch.float64, device="cuda")
        with pytest.raises(F.F12IntError) as e:
            F.f12int_submit(ctx, bid, q, (3,), out, off[None, :-1])
        assert e.value.status == F.ENOMEM
        # a request that fits is still served
        t = F.f12int_submit(ctx, bid, q[:800], (3,), out, off[None, :800])
        while not F.f12int_poll(ctx, t, 100000):
            pass
        torch.cuda.synchronize()
        assert not np.isnan(out[:int(off[800])].cpu().numpy()).any()
    finally:
        F.f12int_destroy(ctx)


def test_poll_of_a_running_request_times_out(lib):
    """A bounded wait on a request that cannot be done yet returns
    F12INT_ETIMEOUT with done = 0, and the ticket stays valid."""
    basis = M.twelve_atom_spd(2)
    ctx = F.f12int_create(0, 0, None)
    try:
        F.f12int_set_factor(ctx, M.P0)
        bid = F.f12int_set_basis(ctx, basis)
        q = M.canonical_quartets(basis, 5)[:100000]   # I5: about 0.2 s of work
        off = M.block_offsets(basis, q)
        out = torch.empty(int(off[-1]), dtype=torch.float64, device="cuda")
        warm = F.f12int_submit(ctx, bid, q[:10], (5,), out, off[None, :10])   # bounds, buffers, graph
        while not F.f12int_poll(ctx, warm, 100000):
            pass
        t = F.f12int_submit(ctx, bid, q, (5,), out, off[None, :-1])
        rc, done = F.f12int_poll_status(ctx, t, 1000)   # 1 ms
        assert (rc, done) == (F.ETIMEOUT, False)
        rc, done = F.f12int_poll_status(ctx, t, 0)       # a query does not time out
        assert rc == F.OK
        while not done:
            rc, done = F.f12int_poll_status(ctx, t, 200000)
            assert rc in (F.OK, F.ETIMEOUT)
        assert rc == F.OK
        rc, _ = F.f12int_poll_status(ctx, t, 0)          # reported once, then unknown
        assert rc == F.EINVAL
    finally:
        F.f12int_destroy(ctx)


def test_series_cap_sets_the_status_word(lib):
    """A series that reaches its length cap sets the device status word: the
    plain path reports F12INT_EDEVICE through f12int_device_status, a request
    through f12int_poll; restoring the cap restores the results."""
    basis = M.twelve_atom_spd(2)
    ctx = F.f12int_create(0, 0, None)
    try:
        F.f12int_set_factor(ctx, M.P0)
        bid = F.f12int_set_basis(ctx, basis)
        q = M.canonical_quartets(basis, 3)[::997]
        ref = compute(ctx, bid, 3, basis, q)
        F.f12int_device_status(ctx)
        F.f12int_set_series_cap(ctx, 2)
        compute(ctx, bid, 3, basis, q)
        with pytest.raises(F.F12IntError) as e:
            F.f12int_device_status(ctx)
        assert e.value.status == F.EDEVICE
        F.f12int_device_status(ctx)   # read and cleared
        off = M.block_offsets(basis, q)
        out = torch.empty(int(off[-1]), dtype=torch.float64, device="cuda")
        t = F.f12int_submit(ctx, bid, q, (3,), out, off[None, :-1])
        with pytest.raises(F.F12IntError) as e:
            while not F.f12int_poll(ctx, t, 100000):
                pass
        assert e.value.status == F.EDEVICE
        F.f12int_set_series_cap(ctx, 0)
        F.f12int_device_status(ctx)
        assert np.array_equal(compute(ctx, bid, 3, basis, q), ref)
        F.f12int_device_status(ctx)
    finally:
        F.f12int_destroy(ctx)
