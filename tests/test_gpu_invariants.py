"""Invariants of the GPU blocks that need no oracle, on many more quartets
of the 12-atom s/p/d molecule than the oracle can afford: permutational
symmetry (8-fold for I1-I4 and I6; I5 antisymmetric in a <-> b and
symmetric in c <-> d) and invariance under a translation of every centre.

I5 quartets with a = b are left out here: their blocks are antisymmetric
matrices in the bra components whose elements are differences of the
(i, j) and (j, i) primitive-pair contributions, exact zeros up to rounding
of much larger terms; the oracle parity tests cover them with the
term-magnitude bound that such cancellation needs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_5070_gb300 import build as B
from paper_1412_5070_gb300 import f12int as F
from paper_1412_5070_gb300 import molecules as M


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    ctx = F.f12int_create(0, 0, None)
    F.f12int_set_factor(ctx, M.P0)
    basis = M.twelve_atom_spd(2)
    bid = F.f12int_set_basis(ctx, basis)
    yield ctx, bid, basis
    F.f12int_destroy(ctx)


def blocks(ctx, bid, basis, cls, q):
    q = np.ascontiguousarray(q, dtype=np.int32)
    off = M.block_offsets(basis, q)
    out = torch.full((int(off[-1]),), float("nan"), dtype=torch.float64, device="cuda")
    F.f12int_compute_class(ctx, bid, cls, torch.from_numpy(q).cuda(), out, torch.from_numpy(off[:-1].copy()).cuda())
    torch.cuda.synchronize()
    F.f12int_device_status(ctx)
    o = out.cpu().numpy()
    nc = (basis.l + 1) * (basis.l + 2) // 2
    return [o[off[i]:off[i + 1]].reshape(nc[q[i, 0]], nc[q[i, 1]], nc[q[i, 2]], nc[q[i, 3]]) for i in range(len(q))]


def agree(x, y, scale):
    return np.all(np.abs(x - y) <= 1e-11 * np.maximum(np.abs(x), np.abs(y)) + 1e-13 * scale)


def sample(basis, cls, n, seed):
    q = M.canonical_quartets(basis, cls)
    if cls == 5:
        q = q[q[:, 0] != q[:, 1]]
    rng = np.random.default_rng(seed)
    return q[np.sort(rng.choice(len(q), size=n, replace=False))]


@pytest.mark.parametrize("cls", [1, 2, 3, 4, 5, 6])
def test_permutational_symmetry(setup, cls):
    ctx, bid, basis = setup
    q = sample(basis, cls, 600, 200 + cls)
    base = blocks(ctx, bid, basis, cls, q)
    sw_ab = blocks(ctx, bid, basis, cls, q[:, [1, 0, 2, 3]])
    sw_cd = blocks(ctx, bid, basis, cls, q[:, [0, 1, 3, 2]])
    sign = -1.0 if cls == 5 else 1.0
    for i in range(len(q)):
        s = np.max(np.abs(base[i]))
        assert agree(sw_ab[i].transpose(1, 0, 2, 3), sign * base[i], s), (cls, q[i])
        assert agree(sw_cd[i].transpose(0, 1, 3, 2), base[i], s), (cls, q[i])
    if cls != 5:
        sw_bk = blocks(ctx, bid, basis, cls, q[:, [2, 3, 0, 1]])
        for i in range(len(q)):
            assert agree(sw_bk[i].transpose(2, 3, 0, 1), base[i], np.max(np.abs(base[i]))), (cls, q[i])


@pytest.mark.parametrize("cls", [1, 3, 5, 6])
def test_translation_invariance(setup, cls):
    ctx, bid, basis = setup
    moved = M.Basis(**{**basis.__dict__, "centers": basis.centers + np.array([1.3, -2.7, 0.9])})
    bid2 = F.f12int_set_basis(ctx, moved)
    q = sample(basis, cls, 600, 300 + cls)
    a = blocks(ctx, bid, basis, cls, q)
    b = blocks(ctx, bid2, moved, cls, q)
    for i in range(len(q)):
        assert agree(a[i], b[i], np.max(np.abs(a[i]))), (cls, q[i])
