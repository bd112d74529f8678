"""Seeded synthetic molecules and Cartesian Gaussian basis sets.

This module only draws inputs; it holds none of the integral arithmetic.
Both the CUDA path and the CPU oracle read the arrays it returns.

Draw order (numpy ``default_rng(seed)``, PCG64):
  1. atom positions by rejection sampling against the minimum separation;
  2. for each atom, its shells in s, p, d, f order;
  3. for each shell: the primitive count (uniform integer), then the
     exponents (log-uniform, sorted in descending order), then the
     contraction coefficients (uniform).

Primitives are unnormalised (Sec. 2.1, Eq. basis of arXiv:1412.5070);
coefficients multiply them as given.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Basis:
    centers: np.ndarray          # [nshell, 3] bohr
    l: np.ndarray                # [nshell] int32
    nprim: np.ndarray            # [nshell] int32
    exps: np.ndarray             # [sum nprim]
    coefs: np.ndarray            # [sum nprim]
    atom_of_shell: np.ndarray = field(default=None)
    name: str = ""

    @property
    def nshell(self) -> int:
        return int(len(self.l))

    @property
    def prim_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.nprim)[:-1]]).astype(np.int32)

    def nfunc(self) -> int:
        return int(sum((l + 1) * (l + 2) // 2 for l in self.l))


def _place_atoms(rng, natom, box, min_sep, max_tries=100000):
    pos = []
    tries = 0
    while len(pos) < natom:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place %d atoms in a %g box" % (natom, box))
        x = rng.uniform(0.0, box, size=3)
        if all(np.linalg.norm(x - y) >= min_sep for y in pos):
            pos.append(x)
    return np.array(pos)


def random_molecule(seed, natom, box, min_sep, shells_per_l, nprim_range, exp_range, coef_range=(0.1, 1.0),
                    name=""):
    """Seeded molecule; ``shells_per_l`` = counts of s, p, d, f shells per atom."""
    rng = np.random.default_rng(seed)
    pos = _place_atoms(rng, natom, box, min_sep)
    centers, ls, nprims, exps, coefs, atoms = [], [], [], [], [], []
    lo, hi = np.log(exp_range[0]), np.log(exp_range[1])
    for ia in range(natom):
        for l, cnt in enumerate(shells_per_l):
            for _ in range(cnt):
                npr = int(rng.integers(nprim_range[0], nprim_range[1] + 1))
                e = np.sort(np.exp(rng.uniform(lo, hi, size=npr)))[::-1]
                c = rng.uniform(coef_range[0], coef_range[1], size=npr)
                centers.append(pos[ia]); ls.append(l); nprims.append(npr)
                exps.extend(e.tolist()); coefs.extend(c.tolist()); atoms.append(ia)
    return Basis(np.array(centers, dtype=np.float64), np.array(ls, dtype=np.int32),
                 np.array(nprims, dtype=np.int32), np.array(exps), np.array(coefs),
                 np.array(atoms, dtype=np.int32), name)


def two_centre_sp() -> Basis:
    """Two centres 5.6 bohr apart on z; on each, uncontracted s shells with
    exponents 0.1, 0.3, 0.9, 2.7 and p shells with exponents 0.3, 0.9
    (6 shells per centre, coefficient 1)."""
    centers, ls, exps = [], [], []
    for z in (0.0, 5.6):
        for e in (0.1, 0.3, 0.9, 2.7):
            centers.append((0.0, 0.0, z)); ls.append(0); exps.append(e)
        for e in (0.3, 0.9):
            centers.append((0.0, 0.0, z)); ls.append(1); exps.append(e)
    n = len(ls)
    return Basis(np.array(centers, dtype=np.float64), np.array(ls, dtype=np.int32), np.ones(n, dtype=np.int32),
                 np.array(exps), np.ones(n), np.array([0] * 6 + [1] * 6, dtype=np.int32), "two-centre s4p2")


def twelve_atom_spd(seed: int = 2) -> Basis:
    """12 atoms in a 12 bohr cube (minimum separation 1.8 bohr), each with
    3s2p1d contracted shells of 3 primitives, exponents log-uniform in
    [0.05, 50], coefficients uniform in [0.1, 1]."""
    return random_molecule(seed, 12, 12.0, 1.8, (3, 2, 1, 0), (3, 3), (0.05, 50.0), name="12-atom 3s2p1d")


def canonical_quartets(basis: Basis, cls: int) -> np.ndarray:
    """All canonical shell quartets: a >= b, c >= d and (ab) >= (cd) for the
    classes with 8-fold symmetry; a >= b, c >= d with every (ab), (cd)
    combination for I5 (antisymmetric in a <-> b, no bra-ket symmetry)."""
    n = basis.nshell
    pairs = [(a, b) for a in range(n) for b in range(a + 1)]
    out = []
    if cls == 5:
        for ab in pairs:
            for cd in pairs:
                out.append(ab + cd)
    else:
        for i, ab in enumerate(pairs):
            for cd in pairs[: i + 1]:
                out.append(ab + cd)
    return np.array(out, dtype=np.int32).reshape(-1, 4)


def block_offsets(basis: Basis, quartets: np.ndarray) -> np.ndarray:
    nc = (basis.l + 1) * (basis.l + 2) // 2
    q = np.asarray(quartets).reshape(-1, 4)
    sizes = nc[q[:, 0]] * nc[q[:, 1]] * nc[q[:, 2]] * nc[q[:, 3]]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


# factor parameter set used throughout: f' = f
P0 = dict(c0=0.5, rho=-0.5, B=0.5, mu=1.0, n=0)


# ------------------------------------------------------- batching and serving --

def significant_pairs(basis: Basis, cut: float = 1e-6) -> np.ndarray:
    """Shell pairs (a >= b) whose largest primitive overlap factor
    exp(-ab/(a+b) |AB|^2) is at least ``cut`` (a geometric estimate; it
    needs no integrals)."""
    shell = np.repeat(np.arange(basis.nshell), basis.nprim)
    e = basis.exps
    cen = basis.centers[shell]
    r2 = np.sum((cen[:, None, :] - cen[None, :, :]) ** 2, axis=-1)
    f = np.exp(-(e[:, None] * e[None, :] / (e[:, None] + e[None, :])) * r2)
    po = basis.prim_off
    g = np.maximum.reduceat(np.maximum.reduceat(f, po, axis=0), po, axis=1)
    a, b = np.nonzero(np.tril(g >= cut))
    return np.stack([a, b], axis=1).astype(np.int32).reshape(-1, 2)


def c3_molecule(seed: int) -> Basis:
    """Molecule of the batching workload: U{2..30} atoms (drawn first from
    the seed's generator) in a 12 bohr cube with minimum separation 1.8 bohr,
    4s3p2d1f shells per atom, U{1..6} primitives per shell, exponents
    log-uniform in [0.03, 200], coefficients uniform in [0.1, 1]."""
    natom = int(np.random.default_rng(seed).integers(2, 31))
    return random_molecule(seed, natom, 12.0, 1.8, (4, 3, 2, 1), (1, 6), (0.03, 200.0),
                           name="batch molecule %d" % seed)


def pair_block(basis: Basis, nbra: int, nket: int, seed: int, pairs=None) -> np.ndarray:
    """Shell quartets of a seeded block of nbra bra x nket ket significant
    shell pairs (drawn with replacement); ``pairs`` may pass the molecule's
    significant pairs when they are already known."""
    if pairs is None:
        pairs = significant_pairs(basis)
    rng = np.random.default_rng(seed)
    bra = pairs[rng.integers(0, len(pairs), size=nbra)]
    ket = pairs[rng.integers(0, len(pairs), size=nket)]
    return np.concatenate([np.repeat(bra, nket, axis=0), np.tile(ket, (nbra, 1))], axis=1).astype(np.int32)


def batching_workload(nmol: int = 64, seed0: int = 1000, block: int = 64):
    """(basis, quartets) of nmol molecules, seeds seed0.. : per molecule a
    block x block significant-pair block (4096 shell quartets per class for
    block = 64), the same list for every class."""
    out = []
    for i in range(nmol):
        b = c3_molecule(seed0 + i)
        out.append((b, pair_block(b, block, block, seed0 + i)))
    return out


def serving_requests(nreq: int, rate: float, pool, seed: int = 5):
    """Poisson arrival stream: (arrival time s, molecule index, classes,
    quartets) per request.  Half the requests ask for one class (uniform over
    I2..I6), half for all five; each covers a seeded block of U{8..64} bra x
    U{8..64} ket significant shell pairs of a molecule drawn uniformly from
    ``pool``."""
    rng = np.random.default_rng(seed)
    sig = [significant_pairs(b) for b in pool]
    t = 0.0
    out = []
    for k in range(nreq):
        t += rng.exponential(1.0 / rate)
        m = int(rng.integers(0, len(pool)))
        classes = (int(rng.integers(2, 7)),) if rng.random() < 0.5 else (2, 3, 4, 5, 6)
        nb, nk = int(rng.integers(8, 65)), int(rng.integers(8, 65))
        out.append((t, m, classes, pair_block(pool[m], nb, nk, int(rng.integers(0, 2 ** 31)), sig[m])))
    return out


def serving_pool(npool: int = 12, seed0: int = 500):
    """Molecules of the serving workload: U{2..60} atoms each (drawn first),
    basis as the batching workload."""
    out = []
    for i in range(npool):
        natom = int(np.random.default_rng(seed0 + i).integers(2, 61))
        out.append(random_molecule(seed0 + i, natom, 12.0 + 4.0 * (natom > 30), 1.8, (4, 3, 2, 1), (1, 6),
                                   (0.03, 200.0), name="serving molecule %d" % (seed0 + i)))
    return out


def c4_molecule(seed: int = 40) -> Basis:
    """Molecule of the mixed-precision workload: 40 atoms in a 20 bohr cube
    (minimum separation 1.8 bohr), 5s4p3d2f shells per atom, U{1..8}
    primitives per shell, exponents log-uniform in [0.02, 500], coefficients
    uniform in [0.1, 1]."""
    return random_molecule(seed, 40, 20.0, 1.8, (5, 4, 3, 2), (1, 8), (0.02, 500.0), name="40-atom 5s4p3d2f")


def bound_stratified_quartets(pair_bound: np.ndarray, n: int, split: float, floor: float, seed: int,
                              canonical_braket: bool = True) -> np.ndarray:
    """n shell quartets drawn at random from pairs (a >= b): half with bound
    product >= split, half in [floor, split); pair_bound is [nshell, nshell]."""
    ns = pair_bound.shape[0]
    a, b = np.tril_indices(ns)
    pb = pair_bound[a, b]
    keep = pb * pb.max() >= floor
    a, b, pb = a[keep], b[keep], pb[keep]
    rng = np.random.default_rng(seed)
    want = {True: n // 2, False: n - n // 2}
    got = {True: [], False: []}
    have = {True: 0, False: 0}
    for _ in range(10000):
        if have[True] >= want[True] and have[False] >= want[False]:
            break
        i = rng.integers(0, len(a), size=4 * n)
        j = rng.integers(0, len(a), size=4 * n)
        if canonical_braket:
            i, j = np.maximum(i, j), np.minimum(i, j)
        prod = pb[i] * pb[j]
        for side, sel in ((True, prod >= split), (False, (prod >= floor) & (prod < split))):
            k = np.nonzero(sel)[0][: max(0, want[side] - have[side])]
            got[side].append(np.stack([a[i[k]], b[i[k]], a[j[k]], b[j[k]]], axis=1))
            have[side] += len(k)
    else:
        raise RuntimeError("could not draw the stratified sample")
    return np.concatenate([np.concatenate(got[True]), np.concatenate(got[False])]).astype(np.int32)
