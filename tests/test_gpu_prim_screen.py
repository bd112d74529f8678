"""The primitive-quartet screen under kernels that grow with distance.

With B > 0 in Eq. rs12 the kernels k4 = f f' and k6 = f_r f'_r grow like
e^{2Br}, so a primitive quartet whose short-range Schwarz product is tiny can
still matter when its two charge distributions lie far apart.  On a 40-atom
molecule in a 16 bohr cube (4s3p2d1f per atom, 1-6 primitives, exponents
log-uniform in [0.03, 200]), far-separated s/p quartets (pair midpoints 8 bohr or more apart) are
computed with the primitive screen and without it (the static entry point before any screen
table exists evaluates every primitive quartet); the two must agree to the
FP64 bar, and the smallest significant ones (largest element just above
1e-12) are also checked against the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_1412_5070_gb300 import build as B
from paper_1412_5070_gb300 import f12int as F
from paper_1412_5070_gb300 import molecules as M

RTOL, SMALL = 1e-10, 1e-12


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    c = F.f12int_create(0, 0, None)
    F.f12int_set_factor(c, M.P0)
    basis = M.random_molecule(77, 40, 16.0, 1.8, (4, 3, 2, 1), (1, 6), (0.03, 200.0), name="40-atom spdf")
    yield c, basis
    F.f12int_destroy(c)


def far_quartets(basis, rmin, n, seed):
    """Seeded quartets (ab|cd) of s/p shells from the molecule's significant
    shell pairs (overlap measure above 1e-10, so that a pair of two atoms
    with tight exponents gives small integrals), the two pairs' atom midpoints
    at least rmin apart."""
    rng = np.random.default_rng(seed)
    pairs = M.significant_pairs(basis, 1e-10)
    pairs = pairs[(basis.l[pairs[:, 0]] <= 1) & (basis.l[pairs[:, 1]] <= 1)]
    mid = 0.5 * (basis.centers[pairs[:, 0]] + basis.centers[pairs[:, 1]])
    i = rng.integers(0, len(pairs), size=20 * n)
    j = rng.integers(0, len(pairs), size=20 * n)
    far = np.linalg.norm(mid[i] - mid[j], axis=1) >= rmin
    i, j = i[far][:n], j[far][:n]
    return np.ascontiguousarray(np.concatenate([pairs[i], pairs[j]], axis=1).astype(np.int32))


def blocks(fn, ctx, bid, cls, basis, q):
    off = M.block_offsets(basis, q)
    out = torch.full((int(off[-1]),), float("nan"), dtype=torch.float64, device="cuda")
    fn(ctx, bid, cls, torch.from_numpy(q).cuda(), out, torch.from_numpy(off[:-1].copy()).cuda())
    torch.cuda.synchronize()
    F.f12int_device_status(ctx)
    return out.cpu().numpy(), off


def outside(got, ref):
    big = np.abs(ref) > SMALL
    return np.where(big, np.abs(got - ref) > RTOL * np.abs(ref), np.abs(got - ref) > SMALL)


@pytest.mark.parametrize("cls", [4, 6])
def test_growing_kernel_far_quartets_screened(setup, cls):
    ctx, basis = setup
    bid_screen = F.f12int_set_basis(ctx, basis)   # compute_class: primitive screen on
    bid_all = F.f12int_set_basis(ctx, basis)      # static entry point only: no screen table is ever built
    q = far_quartets(basis, 8.0, 200000, 300 + cls)
    est = F.f12int_quartet_estimates(ctx, bid_screen, cls, q)
    q = np.ascontiguousarray(q[est >= 1e-14][:60000])
    screened, off = blocks(F.f12int_compute_class, ctx, bid_screen, cls, basis, q)
    every, _ = blocks(F.f12int_compute_class_static, ctx, bid_all, cls, basis, q)
    assert not np.isnan(screened).any() and not np.isnan(every).any()
    bad = outside(screened, every)
    qmax = np.maximum.reduceat(np.abs(every), off[:-1])
    print("I%d: %d far quartets (R >= 8 bohr), %d elements above 1e-12, largest |I| %.3g; "
          "screened vs every primitive quartet: max rel diff %.3g, %d elements outside the bar" % (
              cls, len(q), int((np.abs(every) > SMALL).sum()), qmax.max(),
              float(np.max(np.abs(screened - every)[np.abs(every) > SMALL] / np.abs(every)[np.abs(every) > SMALL])),
              int(bad.sum())))
    assert not bad.any()
    # the oracle on the smallest significant ones with few primitive quartets
    npq = np.prod(basis.nprim[q], axis=1)
    cand = np.nonzero((qmax > SMALL) & (qmax < 1e-9) & (npq <= 256))[0]
    print("I%d: %d far quartets with largest |I| in (1e-12, 1e-9)" % (cls, len(cand)))
    assert len(cand) >= 4, "no far quartet just above 1e-12"
    pick = cand[np.argsort(qmax[cand])[:8]]
    sel = np.ascontiguousarray(q[pick])
    got, _ = blocks(F.f12int_compute_class, ctx, bid_screen, cls, basis, sel)
    ref, _ = O.shell_blocks(O.factor_kernel(M.P0), cls, basis, sel)
    print("I%d oracle check of %d quartets, largest |I| from %.3g to %.3g" % (
        cls, len(sel), qmax[pick].min(), qmax[pick].max()))
    bad = outside(got, ref)
    assert not bad.any(), (got[bad][:5], ref[bad][:5])
