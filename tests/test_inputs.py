"""The seeded input generators (no GPU): molecules, canonical quartet lists,
block offsets and the batching, serving and mixed-precision samplers, each
checked against a direct enumeration or the property its docstring states."""
import itertools

import numpy as np
import pytest

from paper_1412_5070_gb300 import molecules as M


def ncart(l):
    return (l + 1) * (l + 2) // 2


def test_random_molecule_is_seeded_and_respects_its_recipe():
    a = M.random_molecule(7, 9, 10.0, 1.8, (2, 1, 1, 1), (1, 4), (0.05, 80.0))
    b = M.random_molecule(7, 9, 10.0, 1.8, (2, 1, 1, 1), (1, 4), (0.05, 80.0))
    for f in ("centers", "l", "nprim", "exps", "coefs", "atom_of_shell"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert a.nshell == 9 * 5
    assert list(a.l[:5]) == [0, 0, 1, 2, 3]
    pos = a.centers[::5]
    d = np.linalg.norm(pos[:, None] - pos[None], axis=-1) + np.eye(9) * 99
    assert d.min() >= 1.8 and pos.min() >= 0.0 and pos.max() <= 10.0
    assert a.nprim.min() >= 1 and a.nprim.max() <= 4 and a.exps.size == a.nprim.sum()
    assert a.exps.min() >= 0.05 and a.exps.max() <= 80.0
    assert a.coefs.min() >= 0.1 and a.coefs.max() <= 1.0
    for s in range(a.nshell):
        e = a.exps[a.prim_off[s]:a.prim_off[s] + a.nprim[s]]
        assert np.all(np.diff(e) <= 0.0)
    assert a.nfunc() == sum(ncart(int(l)) for l in a.l)
    c = M.random_molecule(8, 9, 10.0, 1.8, (2, 1, 1, 1), (1, 4), (0.05, 80.0))
    assert not np.array_equal(a.centers, c.centers)


@pytest.mark.parametrize("cls", [1, 2, 3, 4, 5, 6])
def test_canonical_quartets_enumerate_each_orbit_once(cls):
    """The 8-fold classes list one quartet per orbit of the index symmetries
    a<->b, c<->d, (ab)<->(cd); I5 (antisymmetric in a<->b, no bra-ket symmetry)
    lists one per orbit of a<->b, c<->d. Checked against brute force."""
    basis = M.two_centre_sp()
    n = basis.nshell
    q = M.canonical_quartets(basis, cls)
    assert q.dtype == np.int32 and q.shape[1] == 4
    assert len({tuple(x) for x in q}) == len(q)

    def orbit(t):
        a, b, c, d = t
        s = {(a, b, c, d), (b, a, c, d), (a, b, d, c), (b, a, d, c)}
        if cls != 5:
            s |= {(c, d, a, b) for a, b, c, d in s}
        return frozenset(s)

    orbits = {orbit(t) for t in itertools.product(range(n), repeat=4)}
    assert len(orbits) == len(q)
    assert {orbit(tuple(x)) for x in q} == orbits
    npair = n * (n + 1) // 2
    assert len(q) == (npair * npair if cls == 5 else npair * (npair + 1) // 2)


def test_block_offsets_are_the_running_sum_of_block_sizes():
    basis = M.twelve_atom_spd(2)
    q = M.canonical_quartets(basis, 3)[::997]
    off = M.block_offsets(basis, q)
    assert off.dtype == np.int64 and off[0] == 0 and len(off) == len(q) + 1
    for i, (a, b, c, d) in enumerate(q):
        n = ncart(basis.l[a]) * ncart(basis.l[b]) * ncart(basis.l[c]) * ncart(basis.l[d])
        assert off[i + 1] - off[i] == n


def test_significant_pairs_match_a_loop_over_primitives():
    basis = M.c3_molecule(1003)
    for cut in (1e-2, 1e-6, 1e-12):
        got = {tuple(x) for x in M.significant_pairs(basis, cut)}
        want = set()
        for a in range(basis.nshell):
            for b in range(a + 1):
                r2 = float(np.sum((basis.centers[a] - basis.centers[b]) ** 2))
                best = 0.0
                for i in range(basis.prim_off[a], basis.prim_off[a] + basis.nprim[a]):
                    for j in range(basis.prim_off[b], basis.prim_off[b] + basis.nprim[b]):
                        ea, eb = basis.exps[i], basis.exps[j]
                        best = max(best, np.exp(-ea * eb / (ea + eb) * r2))
                if best >= cut:
                    want.add((a, b))
        assert got == want
    # every diagonal pair has overlap factor 1
    diag = {(a, a) for a in range(basis.nshell)}
    assert diag <= {tuple(x) for x in M.significant_pairs(basis, 0.5)}


def test_pair_block_is_a_full_bra_by_ket_product():
    basis = M.c3_molecule(1010)
    sig = M.significant_pairs(basis)
    q = M.pair_block(basis, 5, 7, 3)
    assert q.shape == (35, 4) and q.dtype == np.int32
    sig_set = {tuple(x) for x in sig}
    bra = q[::7, :2]
    ket = q[:7, 2:]
    for i in range(5):
        for j in range(7):
            assert tuple(q[i * 7 + j, :2]) == tuple(bra[i]) and tuple(q[i * 7 + j, 2:]) == tuple(ket[j])
    assert all(tuple(x) in sig_set for x in np.concatenate([bra, ket]))
    assert np.array_equal(q, M.pair_block(basis, 5, 7, 3, sig))


def test_batching_workload_recipe():
    wl = M.batching_workload(nmol=4, seed0=1000, block=8)
    assert len(wl) == 4
    for i, (b, q) in enumerate(wl):
        natom = int(np.random.default_rng(1000 + i).integers(2, 31))
        assert b.nshell == natom * 10
        assert q.shape == (64, 4)
        assert b.l.max() == 3 and b.nprim.min() >= 1 and b.nprim.max() <= 6


def test_serving_requests_are_a_seeded_poisson_stream():
    pool = M.serving_pool(npool=3, seed0=500)
    r1 = M.serving_requests(200, 20.0, pool, seed=5)
    r2 = M.serving_requests(200, 20.0, pool, seed=5)
    t = np.array([x[0] for x in r1])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert 0.035 < gaps.mean() < 0.065          # mean 1/rate = 0.05 s over 200 draws
    for (ta, ma, ca, qa), (tb, mb, cb, qb) in zip(r1, r2):
        assert ta == tb and ma == mb and ca == cb and np.array_equal(qa, qb)
    singles = 0
    for _, m, classes, q in r1:
        assert 0 <= m < 3
        assert classes == (2, 3, 4, 5, 6) or (len(classes) == 1 and 2 <= classes[0] <= 6)
        singles += len(classes) == 1
        n = len(q)
        assert n in {nb * nk for nb in range(8, 65) for nk in range(8, 65)}
        assert q.max() < pool[m].nshell
    assert 60 < singles < 140


def test_bound_stratified_quartets_fill_both_strata():
    rng = np.random.default_rng(0)
    ns = 30
    pb = np.exp(rng.uniform(np.log(1e-8), 0.0, size=(ns, ns)))
    pb = np.maximum(pb, pb.T)
    split, floor = 1e-5, 1e-12
    q = M.bound_stratified_quartets(pb, 101, split, floor, seed=4)
    assert q.shape == (101, 4)
    assert np.all(q[:, 0] >= q[:, 1]) and np.all(q[:, 2] >= q[:, 3])
    prod = pb[q[:, 0], q[:, 1]] * pb[q[:, 2], q[:, 3]]
    assert np.all(prod[:50] >= split)
    assert np.all((prod[50:] >= floor) & (prod[50:] < split))
    pair_index = {p: i for i, p in enumerate(zip(*np.tril_indices(ns)))}
    bra = np.array([pair_index[(a, b)] for a, b in q[:, :2]])
    ket = np.array([pair_index[(c, d)] for c, d in q[:, 2:]])
    assert np.all(bra >= ket)
    with pytest.raises(RuntimeError):
        M.bound_stratified_quartets(np.full((4, 4), 1e-3), 10, 1.0, 1e-9, seed=1)
