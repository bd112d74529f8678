"""The screening estimate against the integrals it discards (12-atom s/p/d
molecule): quartets whose estimate is below a threshold must be at most 10
times the threshold (the largest are also checked with the oracle), and the
estimate is exact Schwarz for I1."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_1412_5070_gb300 import build as B
from paper_1412_5070_gb300 import f12int as F
from paper_1412_5070_gb300 import molecules as M

THRESH = 1e-12


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    c = F.f12int_create(0, 0, None)
    F.f12int_set_factor(c, M.P0)
    basis = M.twelve_atom_spd(2)
    bid = F.f12int_set_basis(c, basis)
    yield c, bid, basis
    F.f12int_destroy(c)


@pytest.mark.parametrize("cls", [1, 2, 3, 4, 5, 6])
def test_discarded_quartets_are_below_ten_times_threshold(setup, cls):
    ctx, bid, basis = setup
    a, b = np.tril_indices(basis.nshell)
    rng = np.random.default_rng(60 + cls)
    i = rng.integers(0, len(a), size=300000)
    j = rng.integers(0, len(a), size=300000)
    q = np.stack([a[i], b[i], a[j], b[j]], axis=1).astype(np.int32)
    est = F.f12int_quartet_estimates(ctx, bid, cls, q)
    worst = []
    for lo, hi in ((1e-14, THRESH), (0.0, 1e-14)):
        sel = q[(est >= lo) & (est < hi)][:15000]
        if len(sel) == 0:
            continue
        off = M.block_offsets(basis, sel)
        out = torch.zeros(int(off[-1]), dtype=torch.float64, device="cuda")
        F.f12int_compute_class(ctx, bid, cls, torch.from_numpy(sel).cuda(), out,
                               torch.from_numpy(off[:-1].copy()).cuda())
        torch.cuda.synchronize()
        qmax = np.maximum.reduceat(out.abs().cpu().numpy(), off[:-1])
        k = np.argsort(qmax)[-3:]
        worst.extend((float(qmax[x]), sel[x]) for x in k)
        print("I%d estimate in [%.0e, %.0e): %d quartets, max |I| %.3g" % (cls, lo, hi, len(sel), qmax.max()))
        assert qmax.max() <= 10 * THRESH
    # the largest discarded ones, from the oracle
    worst.sort(key=lambda t: -t[0])
    top = np.array([w[1] for w in worst[:3]], dtype=np.int32)
    ref, _ = O.shell_blocks(O.factor_kernel(M.P0), cls, basis, top)
    assert np.abs(ref).max() <= 10 * THRESH


def test_i1_estimate_is_schwarz(setup):
    """For the positive-definite 1/r kernel the estimate is the plain
    Schwarz product (no growth, no safety factor)."""
    ctx, bid, basis = setup
    pb = F.f12int_pair_bounds(ctx, bid, 1, basis.nshell)
    q = M.canonical_quartets(basis, 1)[::5000]
    est = F.f12int_quartet_estimates(ctx, bid, 1, q)
    np.testing.assert_array_equal(est, pb[q[:, 0], q[:, 1]] * pb[q[:, 2], q[:, 3]])
