"""Parity at the benchmark's full size, in its launch configuration (needs a GPU).

The 12-atom 3s2p1d workload of bench.py: per class the whole screened quartet
list (Schwarz 1e-12) in one f12int_compute_class call on a side stream, as
the benchmark launches it; then a seeded sample of its blocks, with the first
and the last block of the list, is compared element by element with the
oracle under the tolerance of the parity tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_1412_5070_gb300 import build as B
from paper_1412_5070_gb300 import f12int as F
from paper_1412_5070_gb300 import molecules as M

from test_gpu_parity import close, report

SAMPLE = 14


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    stream = torch.cuda.Stream()
    ctx = F.f12int_create(0, 0, stream)
    F.f12int_set_factor(ctx, M.P0)
    basis = M.twelve_atom_spd(2)
    bid = F.f12int_set_basis(ctx, basis)
    yield ctx, bid, basis, stream
    F.f12int_destroy(ctx)


@pytest.mark.parametrize("cls", [1, 2, 3, 4, 5, 6])
def test_full_list_sampled_blocks(setup, cls):
    ctx, bid, basis, stream = setup
    q = F.f12int_screen(ctx, bid, cls, 1e-12)
    assert len(q) > 100000
    off = M.block_offsets(basis, q)
    out = torch.full((int(off[-1]),), float("nan"), dtype=torch.float64, device="cuda")
    F.f12int_compute_class(ctx, bid, cls, torch.from_numpy(np.ascontiguousarray(q)).cuda(), out,
                           torch.from_numpy(off[:-1].copy()).cuda(), stream)
    stream.synchronize()
    F.f12int_device_status(ctx)
    rng = np.random.default_rng(100 + cls)
    idx = np.unique(np.concatenate([[0, len(q) - 1], rng.choice(len(q), SAMPLE, replace=False)]))
    host = out.cpu().numpy()
    del out
    got = np.concatenate([host[off[i]:off[i + 1]] for i in idx])
    assert not np.isnan(host).any()
    ref, _, mag = O.shell_blocks(O.factor_kernel(M.P0), cls, basis, q[idx], with_mag=True)
    bad = close(got, ref, mag)
    assert not bad.any(), report(got, ref, mag, bad)
