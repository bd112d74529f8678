"""Host-side checks that need no GPU: the C ABI library loads and exports
every entry point its header declares; the term lists it generates match
the kernels of arXiv:1412.5070 (Eqs. k1-k6, rs12, ttdamp) as evaluated by
the oracle; factor validation; the weak-scaling shard logic on two gloo
ranks."""
import math
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_1412_5070_gb300 import build as B
from paper_1412_5070_gb300 import f12int as F
from paper_1412_5070_gb300 import molecules as M
from paper_1412_5070_gb300 import sharding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return F.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "f12int.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(f12int_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_entry_point(lib):
    names = declared_functions()
    assert "f12int_compute_class" in names and "f12int_compute_class_static" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(F.EXPORTS)


def test_strerror_without_gpu(lib):
    assert F.f12int_strerror(0) == "ok"
    assert "factor" in F.f12int_strerror(-3)
    assert F.f12int_strerror(12345) == "unknown status"


def test_create_reports_missing_gpu(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(F.F12IntError) as e:
        F.f12int_create(0, 0, None)
    assert e.value.status in (-1, -6)


DECAYING = dict(c0=0.5, rho=-0.5, B=-0.8, mu=1.0, n=0)


@pytest.mark.parametrize("f", [M.P0, DECAYING], ids=["P0", "B<0"])
@pytest.mark.parametrize("cls", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("x", [0.03, 0.4, 1.1, 2.7, 6.5])
def test_term_lists_reproduce_the_kernels(lib, f, cls, x):
    """l = 0: x^2 k(x) from the generated families equals x^2 k(x) from the
    oracle's pointwise kernel (separation of the damping, Eq. hj00eps), for a
    growing (B > 0) and a decaying (B < 0) long-range part."""
    got = F.f12int_kernel_radial(cls, f, 0, x)
    ref = x * x * O.kernel_value(O.factor_kernel(f), cls, x)
    assert abs(got - ref) <= 1e-13 * abs(ref) + 1e-15


@pytest.mark.parametrize("cls", [2, 3, 4, 6])
@pytest.mark.parametrize("x", [0.6, 1.3, 3.0])
def test_radial_derivative_of_term_lists(lib, cls, x):
    """l = 1, 2: x^{2l+2} D_r^l k with D_r = x^-1 d/dx, against finite
    differences of the oracle's kernel values."""
    K = O.factor_kernel(M.P0)
    k = lambda r: O.kernel_value(K, cls, r)
    h = 1e-3 * x

    def d1(fun, r):
        return (fun(r - 2 * h) - 8 * fun(r - h) + 8 * fun(r + h) - fun(r + 2 * h)) / (12 * h)

    dr1 = lambda r: d1(k, r) / r
    v1 = x ** 4 * dr1(x)
    v2 = x ** 6 * d1(dr1, x) / x
    assert abs(F.f12int_kernel_radial(cls, M.P0, 1, x) - v1) <= 1e-8 * max(abs(v1), 1e-3)
    assert abs(F.f12int_kernel_radial(cls, M.P0, 2, x) - v2) <= 1e-6 * max(abs(v2), 1e-3)


def test_factor_pair_with_different_parameters(lib):
    """f' != f (Eq. I4, Eq. I6_): the product term lists still reproduce f f'
    and f_r f'_r pointwise."""
    fp = dict(c0=0.3, rho=-0.3, B=0.3, mu=0.7, n=0)
    K = O.factor_kernel(M.P0, fp)
    for cls in (4, 6):
        for x in (0.2, 1.0, 3.3):
            got = F.f12int_kernel_radial(cls, M.P0, 0, x, fprime=fp)
            ref = x * x * O.kernel_value(K, cls, x)
            assert abs(got - ref) <= 1e-13 * abs(ref) + 1e-15


@pytest.mark.parametrize("bad", [dict(c0=0.5, rho=-0.5, B=0.5, mu=0.0, n=0),
                                 dict(c0=0.5, rho=-2.5, B=0.5, mu=1.0, n=0),
                                 dict(c0=-0.5, rho=-0.5, B=0.5, mu=1.0, n=0),
                                 dict(c0=0.5, rho=-0.5, B=0.5, mu=1.0, n=21),
                                 dict(c0=float("nan"), rho=-0.5, B=0.5, mu=1.0, n=0)])
def test_factor_domain_checks(lib, bad):
    """mu > 0 and rho + 2n + 2 > 0 (Sec. 3.1); c0 >= 0, 0 <= n <= 20 and
    finite values are what the library supports (B of either sign)."""
    with pytest.raises(F.F12IntError) as e:
        F.f12int_kernel_radial(3, bad, 0, 1.0)
    assert e.value.status == -3


TENNO = [(1.0, 0, -1.2, 0)]
GAUSSIANS = [(0.3, 0, 0, 0.2), (0.25, 0, 0, 1.1), (0.2, 0, 0, 4.0)]


@pytest.mark.parametrize("terms", [TENNO, GAUSSIANS], ids=["Ten-no", "Gaussians"])
@pytest.mark.parametrize("cls", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("x", [0.05, 0.9, 3.0])
def test_term_list_factors_reproduce_the_kernels(lib, terms, cls, x):
    """Factors given as terms: x^2 k(x) from the library's term lists equals
    the oracle's pointwise kernel of the same factor."""
    got = F.f12int_kernel_radial_terms(cls, terms, 0, x)
    ref = x * x * O.kernel_value(O.factor_kernel_terms(terms), cls, x)
    assert abs(got - ref) <= 1e-13 * abs(ref) + 1e-15


def test_term_list_pair_and_domain(lib):
    """f' != f as term lists; g < 0, non-finite values, an empty or all-zero
    list, and more than 64 terms are refused."""
    x = 1.3
    got = F.f12int_kernel_radial_terms(6, TENNO, 0, x, terms_prime=GAUSSIANS)
    ref = x * x * O.kernel_value(O.factor_kernel_terms(TENNO, GAUSSIANS), 6, x)
    assert abs(got - ref) <= 1e-13 * abs(ref)
    for bad, status in (([(1.0, 0, 0, -0.5)], -3), ([(float("inf"), 0, 0, 1.0)], -3), ([], -1),
                        ([(1.0, 0, 0, 1.0), (-1.0, 0, 0, 1.0)], -3), ([(1.0, 0, 0, 1.0)] * 65, -1)):
        with pytest.raises(F.F12IntError) as e:
            F.f12int_kernel_radial_terms(3, bad, 0, 1.0)
        assert e.value.status == status


def test_shard_partitions_every_list():
    lst = np.arange(103 * 4).reshape(103, 4)
    parts = [sharding.shard(lst, r, 3) for r in range(3)]
    joined = np.concatenate(parts)
    assert len(joined) == len(lst)
    assert sorted(map(tuple, joined)) == sorted(map(tuple, lst))
    with pytest.raises(ValueError):
        sharding.shard(lst, 3, 3)


def _gloo_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    basis = M.two_centre_sp()
    full = M.canonical_quartets(basis, 3)
    mine = sharding.shard(full, rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine.tolist())
    mx = sharding.max_over_ranks(1.5 + rank)
    if rank == 0:
        union = sorted(tuple(x) for part in got for x in part)
        q.put((union == sorted(map(tuple, full.tolist())), sum(len(p) for p in got) == len(full), mx))
    dist.destroy_process_group()


def test_two_rank_gloo_weak_scaling_split():
    """Two gloo ranks: the shards are disjoint and cover the list; the
    step-time reduction takes the maximum over ranks."""
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_gloo_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    covered, sizes_ok, mx = q.get(timeout=10)
    assert covered and sizes_ok and mx == 2.5


def _random_terms(rng):
    n = int(rng.integers(1, 5))
    return [(float(rng.uniform(-1, 1)), float(rng.choice([-1.0, -0.5, 0.0, 0.5, 1.0, 2.0])),
             float(rng.uniform(-2.0, 1.0)), float(rng.choice([0.0, rng.uniform(0.1, 2.0)]))) for _ in range(n)]


@pytest.mark.parametrize("seed", range(12))
def test_random_term_lists_against_the_oracle_kernel(lib, seed):
    """Seeded random factors of 1-4 terms: the library's term algebra (products,
    derivatives, families, D_r) against the oracle's pointwise kernels; order 0
    directly, orders 1 and 2 through finite differences of the oracle."""
    rng = np.random.default_rng(seed)
    t, tp = _random_terms(rng), _random_terms(rng)
    K = O.factor_kernel_terms(t, tp)
    for cls in (2, 3, 4, 6):
        for x in (0.35, 1.1, 2.4):
            got = F.f12int_kernel_radial_terms(cls, t, 0, x, terms_prime=tp)
            ref = x * x * O.kernel_value(K, cls, x)
            assert abs(got - ref) <= 1e-12 * abs(ref) + 1e-14, (cls, x)
            k = lambda r: O.kernel_value(K, cls, r)
            h = 1e-3 * x

            def d1(fun, r):
                return (fun(r - 2 * h) - 8 * fun(r - h) + 8 * fun(r + h) - fun(r + 2 * h)) / (12 * h)

            dr1 = lambda r: d1(k, r) / r
            v1 = x ** 4 * dr1(x)
            v2 = x ** 6 * d1(dr1, x) / x
            g1 = F.f12int_kernel_radial_terms(cls, t, 1, x, terms_prime=tp)
            g2 = F.f12int_kernel_radial_terms(cls, t, 2, x, terms_prime=tp)
            scale = max(abs(ref), abs(v1), abs(v2), 1e-3)
            assert abs(g1 - v1) <= 1e-8 * scale, (cls, x, g1, v1)
            assert abs(g2 - v2) <= 1e-6 * scale, (cls, x, g2, v2)


def test_factor_classes_query(lib):
    """The host-only class query: P0 is served everywhere without the
    quadrature launch; B < 0 needs it in the F12 classes; rho = -5/2 needs it
    for its singular classes I2, I4, I6; rho = -1.3 leaves I6 out (a general
    power below -1); r^-3 leaves every F12 class out; seven Gaussians overflow
    the family table in I4 and I6."""
    assert F.f12int_factor_classes(M.P0) == {c: 1 for c in range(1, 7)}
    assert F.f12int_factor_classes(dict(M.P0, B=-0.8)) == {1: 1, 2: 3, 3: 3, 4: 3, 5: 3, 6: 3}
    assert F.f12int_factor_classes(dict(M.P0, rho=-2.5, n=1)) == {1: 1, 2: 3, 3: 1, 4: 3, 5: 1, 6: 3}
    assert F.f12int_factor_classes(dict(M.P0, rho=-1.3))[6] == 0
    assert F.f12int_factor_classes_terms([(1.0, -3, 0, 0)]) == {1: 1, 2: 0, 3: 0, 4: 0, 5: 0, 6: 0}
    seven = [(0.5 / (i + 1), 0, 0, 0.2 * 2.5 ** i) for i in range(7)]
    assert F.f12int_factor_classes_terms(seven) == {1: 1, 2: 1, 3: 1, 4: 0, 5: 1, 6: 0}
    with pytest.raises(F.F12IntError):
        F.f12int_factor_classes(dict(M.P0, mu=0.0))


def test_factor_classes_query_matches_gpu_test_rule(lib):
    """The GPU factor tests decide from their own rule which classes each
    parameter set leaves out; the library's query must agree."""
    tg = pytest.importorskip("test_gpu_factors")
    for name, (f, fp) in tg.SETS.items():
        flags = F.f12int_factor_classes(f, fp)
        fpp = fp if fp is not None else f
        for cls in (2, 3, 4, 5, 6):
            assert (flags[cls] != 0) == tg.supported(f, fpp, cls), (name, cls)


def test_bench_traffic_scaling():
    """The roofline's traffic of the auxiliary kernel: the captured DRAM
    bytes per primitive quartet and class, times the step's primitive
    quartets per class, over the step's launches of the kernel."""
    import bench
    assert sorted(bench.AUX_DRAM_BYTES_PER_PRIM_QUARTET) == [1, 2, 3, 4, 5, 6]
    npq = {1: 1000, 3: 2000}
    want = (bench.AUX_DRAM_BYTES_PER_PRIM_QUARTET[1] * 1000 + bench.AUX_DRAM_BYTES_PER_PRIM_QUARTET[3] * 2000) / 4
    assert abs(bench.aux_traffic_per_launch(npq, 4) - want) <= 1e-9 * want
    assert bench.aux_traffic_per_launch(npq, 0) is None


def _cart(l):
    return [(i, j, l - i - j) for i in range(l, -1, -1) for j in range(l - i, -1, -1)]


def test_ket_term_count_order_visits_every_entry_once():
    """The general contraction's ket step takes its (bra Hermite index, ket
    component) entries in order of the component's term count: a task builds
    kord (the components by increasing count, then the class starts at
    KORD_CLS) and lane r of the flat loop maps to (bi, j) through the class
    it falls in.  Replayed here for every (lc, ld), ket-range split and bra
    order the kernel serves: each entry is visited exactly once and the
    indexes stay inside kord's 116 entries."""
    KORD_CLS, KORD_SIZE = 100, 116
    nh = lambda L: (L + 1) * (L + 2) * (L + 3) // 6
    for lc in range(4):
        for ld in range(4):
            nd = len(_cart(ld))
            ncd_all = len(_cart(lc)) * nd
            for nsplit in range(1, ncd_all + 1):
                jc = (ncd_all + nsplit - 1) // nsplit
                if (ncd_all + jc - 1) // jc != nsplit:
                    continue
                for split in range(nsplit):
                    j0 = split * jc
                    ncd = min(jc, ncd_all - j0)
                    off = [0]
                    for j in range(ncd):
                        ec, ed = _cart(lc)[(j0 + j) // nd], _cart(ld)[(j0 + j) % nd]
                        off.append(off[-1] + (ec[0] + ed[0] + 1) * (ec[1] + ed[1] + 1) * (ec[2] + ed[2] + 1))
                    kord = [None] * KORD_SIZE
                    nc, pos = 0, 0
                    while pos < ncd:
                        prev = off[kord[pos - 1] + 1] - off[kord[pos - 1]] if nc else 0
                        ln = min(off[j + 1] - off[j] for j in range(ncd) if off[j + 1] - off[j] > prev)
                        kord[KORD_CLS + nc] = pos
                        for j in range(ncd):
                            if off[j + 1] - off[j] == ln:
                                kord[pos] = j
                                pos += 1
                        nc += 1
                    kord[KORD_CLS + nc] = ncd
                    assert KORD_CLS + nc < KORD_SIZE
                    for lb_ext in range(0, 9):
                        nhB = nh(lb_ext)
                        seen = set()
                        for lane in range(32):
                            c = 0
                            for r in range(lane, nhB * ncd, 32):
                                while r >= nhB * kord[KORD_CLS + c + 1]:
                                    c += 1
                                c0, n_c = kord[KORD_CLS + c], kord[KORD_CLS + c + 1] - kord[KORD_CLS + c]
                                rr = r - nhB * c0
                                bi = rr // n_c
                                j = kord[c0 + rr - bi * n_c]
                                assert 0 <= bi < nhB and 0 <= j < ncd
                                seen.add((bi, j))
                        assert len(seen) == nhB * ncd
