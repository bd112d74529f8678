"""Batched requests (f12int_submit / f12int_poll) on the GPU.

The batch path runs the kernels of f12int_compute_class from one captured
graph over the merged lists of many requests; these tests compare it with
the per-call path and with the oracle, and check that a request's blocks do
not depend on what else is in its batch.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_1412_5070_gb300 import build as B
from paper_1412_5070_gb300 import f12int as F
from paper_1412_5070_gb300 import molecules as M

from test_gpu_parity import close, f_shell_molecule, report


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    c = F.f12int_create(0, 0, None)
    F.f12int_set_factor(c, M.P0)
    F.f12int_batch_limits(c, 1 << 17, 1 << 22)
    yield c
    F.f12int_destroy(c)


def layout(basis, quartets, classes):
    """Offsets [len(classes), n] of consecutive blocks, class after class."""
    sizes = np.array([np.prod([(basis.l[s] + 1) * (basis.l[s] + 2) // 2 for s in q]) for q in quartets],
                     dtype=np.int64)
    off = np.zeros((len(classes), len(quartets)), dtype=np.int64)
    base = 0
    for k in range(len(classes)):
        off[k] = base + np.concatenate([[0], np.cumsum(sizes)[:-1]])
        base += int(sizes.sum())
    return off, base


def wait(ctx, tickets, limit_s=120.0):
    t0 = time.time()
    left = list(tickets)
    while left:
        left = [t for t in left if not F.f12int_poll(ctx, t, 1000)]
        assert time.time() - t0 < limit_s, "requests did not finish"


def per_call(ctx, bid, cls, quartets, basis):
    q = np.ascontiguousarray(quartets, dtype=np.int32)
    off = M.block_offsets(basis, q)
    out = torch.full((int(off[-1]),), float("nan"), dtype=torch.float64, device="cuda")
    F.f12int_compute_class(ctx, bid, cls, torch.from_numpy(q).cuda(), out, torch.from_numpy(off[:-1].copy()).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def sample(basis, cls, k, seed):
    q = M.canonical_quartets(basis, cls)
    rng = np.random.default_rng(seed)
    return q[np.sort(rng.choice(len(q), size=min(k, len(q)), replace=False))]


def test_batch_matches_per_call_and_oracle(ctx):
    """Requests on two bases with different class masks, all in flight at
    once: every block equals the per-call path's to 1e-13 (both FP64; their
    contraction may split the work over warps differently) and a subset
    matches the oracle to the parity tolerance."""
    bases = [M.two_centre_sp(), M.twelve_atom_spd(2)]
    bids = [F.f12int_set_basis(ctx, b) for b in bases]
    plan = [(0, (1, 3, 5)), (1, (2, 4, 6)), (1, (1, 5)), (0, (6,)), (1, (3,))]
    reqs = []
    for i, (bi, classes) in enumerate(plan):
        q = sample(bases[bi], classes[0], 300, 70 + i)
        off, tot = layout(bases[bi], q, classes)
        out = torch.full((tot,), float("nan"), dtype=torch.float64, device="cuda")
        t = F.f12int_submit(ctx, bids[bi], q, classes, out, off)
        reqs.append((bi, classes, q, off, out, t))
    wait(ctx, [r[-1] for r in reqs])
    for bi, classes, q, off, out, _ in reqs:
        got_all = out.cpu().numpy()
        assert not np.isnan(got_all).any()
        for k, cls in enumerate(classes):
            n = int(M.block_offsets(bases[bi], q)[-1])
            got = got_all[off[k, 0]:off[k, 0] + n]
            ref = per_call(ctx, bids[bi], cls, q, bases[bi])
            tol = 1e-13 * np.abs(ref) + 1e-15 * np.max(np.abs(ref))
            assert np.all(np.abs(got - ref) <= tol), (cls, np.max(np.abs(got - ref) - tol))
            sub = q[:12]
            o_ref, _, mag = O.shell_blocks(O.factor_kernel(M.P0), cls, bases[bi], sub, with_mag=True)
            bad = close(got[:len(o_ref)], o_ref, mag)
            assert not bad.any(), report(got[:len(o_ref)], o_ref, mag, bad)


def test_alone_equals_in_mix(ctx):
    """A request's blocks are bitwise the same whether it runs alone or in a
    batch with other requests of other molecules and classes."""
    b1, b2 = M.twelve_atom_spd(2), M.random_molecule(1001, 3, 12.0, 1.8, (2, 1, 1, 1), (1, 3), (0.03, 200.0))
    i1, i2 = F.f12int_set_basis(ctx, b1), F.f12int_set_basis(ctx, b2)
    q = sample(b1, 2, 400, 5)
    off, tot = layout(b1, q, (2, 5))
    alone = torch.zeros(tot, dtype=torch.float64, device="cuda")
    wait(ctx, [F.f12int_submit(ctx, i1, q, (2, 5), alone, off)])
    mixed = torch.zeros(tot, dtype=torch.float64, device="cuda")
    others = []
    for j, (bid, bas, classes) in enumerate([(i2, b2, (1, 2, 3, 4, 5, 6)), (i1, b1, (2,)), (i2, b2, (5,))]):
        qq = sample(bas, classes[0], 250, 40 + j)
        oo, tt = layout(bas, qq, classes)
        buf = torch.zeros(tt, dtype=torch.float64, device="cuda")
        others.append((buf, F.f12int_submit(ctx, bid, qq, classes, buf, oo)))
        if j == 1:
            mine = F.f12int_submit(ctx, i1, q, (2, 5), mixed, off)
    wait(ctx, [t for _, t in others] + [mine])
    assert torch.equal(alone, mixed)


def test_screened_quartets_are_zero(ctx):
    """With a threshold, quartets below it get zero blocks and the others are
    the unscreened results."""
    basis = M.twelve_atom_spd(2)
    bid = F.f12int_set_basis(ctx, basis)
    q = sample(basis, 3, 600, 9)
    off, tot = layout(basis, q, (3,))
    full = torch.full((tot,), float("nan"), dtype=torch.float64, device="cuda")
    scr = torch.full((tot,), float("nan"), dtype=torch.float64, device="cuda")
    wait(ctx, [F.f12int_submit(ctx, bid, q, (3,), full, off),
               F.f12int_submit(ctx, bid, q, (3,), scr, off, schwarz_thresh=1e-6)])
    keep = {tuple(x) for x in F.f12int_screen(ctx, bid, 3, 1e-6)}
    keep |= {(c, d, a, b) for a, b, c, d in keep}
    full, scr = full.cpu().numpy(), scr.cpu().numpy()
    sizes = np.diff(np.append(off[0], tot))
    nzero = 0
    for i, quart in enumerate(q):
        a = slice(off[0, i], off[0, i] + sizes[i])
        if tuple(quart) in keep:
            assert np.array_equal(scr[a], full[a])
        else:
            assert np.all(scr[a] == 0.0)
            nzero += 1
    assert 0 < nzero < len(q)


@pytest.mark.parametrize("cls", [3, 5, 6])
def test_f_shells_in_batch(ctx, cls):
    """f-shell quartets (including the ket-split (ff|ff) contraction of I5)
    through the batch path against the oracle."""
    basis = f_shell_molecule()
    bid = F.f12int_set_basis(ctx, basis)
    q = M.canonical_quartets(basis, cls)
    q = q[np.any(basis.l[q] == 3, axis=1)][:: 7 if cls == 5 else 5]
    off, tot = layout(basis, q, (cls,))
    out = torch.full((tot,), float("nan"), dtype=torch.float64, device="cuda")
    wait(ctx, [F.f12int_submit(ctx, bid, q, (cls,), out, off)])
    got = out.cpu().numpy()
    ref, _, mag = O.shell_blocks(O.factor_kernel(M.P0), cls, basis, q, with_mag=True)
    bad = close(got, ref, mag)
    assert not np.isnan(got).any()
    assert not bad.any(), report(got, ref, mag, bad)


def test_ticket_semantics(ctx):
    """poll with no wait returns at once; a finished ticket is reported once;
    unknown tickets and bad requests are rejected."""
    basis = M.two_centre_sp()
    bid = F.f12int_set_basis(ctx, basis)
    q = M.canonical_quartets(basis, 1)[:50]
    off, tot = layout(basis, q, (1,))
    out = torch.zeros(tot, dtype=torch.float64, device="cuda")
    t = F.f12int_submit(ctx, bid, q, (1,), out, off)
    t0 = time.time()
    F.f12int_poll(ctx, t, 0)
    assert time.time() - t0 < 0.05
    wait(ctx, [t])
    with pytest.raises(F.F12IntError):
        F.f12int_poll(ctx, t, 0)
    with pytest.raises(F.F12IntError):
        F.f12int_poll(ctx, 10 ** 12, 0)
    with pytest.raises(F.F12IntError):
        F.f12int_submit(ctx, bid, q, (), out, off)
    bad = q.copy()
    bad[0, 0] = 999
    with pytest.raises(F.F12IntError):
        F.f12int_submit(ctx, bid, bad, (1,), out, off)
    stats = F.f12int_batch_stats(ctx)
    assert stats["batches"] >= 1 and stats["pending"] == 0


def test_autotune_keeps_results(ctx):
    """The autotuner picks one of its candidate schedules per class, and the
    blocks computed under the chosen schedule still match the per-call path."""
    basis = M.twelve_atom_spd(2)
    bid = F.f12int_set_basis(ctx, basis)
    q = sample(basis, 3, 500, 11)
    rep = F.f12int_batch_autotune(ctx, bid, q, (3, 5))
    for c in (3, 5):
        target, div, sec = rep[c]
        assert target in (5e7 / 8, 5e7 * 0.3, 5e7, 5e7 * 4) and div in (1, 2) and sec > 0
    for c in (3, 5):
        off, tot = layout(basis, q, (c,))
        out = torch.full((tot,), float("nan"), dtype=torch.float64, device="cuda")
        wait(ctx, [F.f12int_submit(ctx, bid, q, (c,), out, off)])
        ref = per_call(ctx, bid, c, q, basis)
        got = out.cpu().numpy()
        tol = 1e-13 * np.abs(ref) + 1e-15 * np.max(np.abs(ref))
        assert np.all(np.abs(got - ref) <= tol)
