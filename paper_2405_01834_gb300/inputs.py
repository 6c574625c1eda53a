"""Seeded synthetic inputs: Gaussian shell bases, shell-quartet lists, densities.

This module is shared by the CUDA engine's tests/benchmark and by the oracle's
tests. It holds no integral arithmetic (no Boys function, no Hermite
expansion, no recursion): only random geometry, exponents, contraction
coefficients, index lists and the textbook normalisation of a primitive
Cartesian Gaussian.

Shapes follow the workloads of Asadchev & Valeev (arXiv:2405.01834): random
shells and centres that avoid screening for the per-class microbenchmarks
(Sec. 5), contracted segmented shells (Eq. 3) up to l = 6, and
molecule-like clusters for the exchange build (Sec. 6). The paper's own
molecules and basis-set files are not available, so these seeded recipes
stand in for them; each generator's docstring states its recipe.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

LMAX = 6


def ncart(l: int) -> int:
    """Number of Cartesian components of a shell of angular momentum l."""
    return (l + 1) * (l + 2) // 2


def _dfact(n: int) -> float:
    """Double factorial n!! with (-1)!! = 0!! = 1."""
    r = 1.0
    while n > 1:
        r *= n
        n -= 2
    return r


def primitive_norm(l: int, zeta: np.ndarray) -> np.ndarray:
    """Normalisation of the axis-aligned primitive x^l exp(-zeta r^2).

    N = (2 zeta / pi)^(3/4) (4 zeta)^(l/2) / sqrt((2l-1)!!).
    """
    zeta = np.asarray(zeta, dtype=np.float64)
    return (2.0 * zeta / math.pi) ** 0.75 * (4.0 * zeta) ** (l / 2.0) / math.sqrt(_dfact(2 * l - 1))


def contracted_self_overlap(l: int, zeta: np.ndarray, coef: np.ndarray) -> float:
    """<phi|phi> of the x^l component of a contracted shell (textbook Gaussian integral)."""
    z = np.add.outer(zeta, zeta)
    s = (math.pi / z) ** 1.5 * _dfact(2 * l - 1) / (2.0 * z) ** l
    return float(coef @ s @ coef)


@dataclass
class Basis:
    """A set of contracted Cartesian Gaussian shells (Eq. 3).

    Arrays have one entry per shell except exps/coefs (one per primitive).
    coefs multiply the UNNORMALISED primitives x^ax y^ay z^az exp(-zeta r^2);
    any normalisation is already folded in.
    """
    l: np.ndarray          # int32 [n_shells]
    nprim: np.ndarray      # int32 [n_shells]
    prim_off: np.ndarray   # int32 [n_shells]
    ao_off: np.ndarray     # int32 [n_shells]
    atom: np.ndarray       # int32 [n_shells]
    center: np.ndarray     # float64 [n_shells, 3], bohr
    exps: np.ndarray       # float64 [n_prims]
    coefs: np.ndarray      # float64 [n_prims]
    atoms: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))  # float64 [n_atoms, 3]

    @property
    def n_shells(self) -> int:
        return int(len(self.l))

    @property
    def nao(self) -> int:
        return int(sum(ncart(int(x)) for x in self.l))

    @property
    def n_atoms(self) -> int:
        return int(len(self.atoms))


class BasisBuilder:
    def __init__(self):
        self.l, self.nprim, self.atom, self.center, self.exps, self.coefs = [], [], [], [], [], []
        self.atoms = []

    def add_atom(self, xyz) -> int:
        self.atoms.append(np.asarray(xyz, dtype=np.float64))
        return len(self.atoms) - 1

    def add_shell(self, l: int, xyz, exps, coefs, atom: int = -1):
        exps = np.asarray(exps, dtype=np.float64)
        coefs = np.asarray(coefs, dtype=np.float64)
        assert exps.shape == coefs.shape and exps.ndim == 1 and len(exps) >= 1
        assert 0 <= l <= LMAX
        self.l.append(l)
        self.nprim.append(len(exps))
        self.atom.append(atom)
        self.center.append(np.asarray(xyz, dtype=np.float64))
        self.exps.append(exps)
        self.coefs.append(coefs)

    def build(self) -> Basis:
        l = np.array(self.l, dtype=np.int32)
        nprim = np.array(self.nprim, dtype=np.int32)
        prim_off = np.zeros(len(l), dtype=np.int32)
        if len(l) > 1:
            prim_off[1:] = np.cumsum(nprim)[:-1]
        nc = (l + 1) * (l + 2) // 2
        ao_off = np.zeros(len(l), dtype=np.int32)
        if len(l) > 1:
            ao_off[1:] = np.cumsum(nc)[:-1]
        return Basis(l=l, nprim=nprim, prim_off=prim_off, ao_off=ao_off,
                     atom=np.array(self.atom, dtype=np.int32),
                     center=np.array(self.center, dtype=np.float64).reshape(-1, 3),
                     exps=np.concatenate(self.exps) if self.exps else np.zeros(0),
                     coefs=np.concatenate(self.coefs) if self.coefs else np.zeros(0),
                     atoms=np.array(self.atoms, dtype=np.float64).reshape(-1, 3))


def _loguniform(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def random_shell(rng, bb: BasisBuilder, l: int, xyz, K: int, zlo: float, zhi: float, atom: int = -1):
    """Shell with K log-uniform exponents and coefficients uniform in [0.1, 1] x primitive norm."""
    z = _loguniform(rng, zlo, zhi, K)
    c = rng.uniform(0.1, 1.0, K) * primitive_norm(l, z)
    bb.add_shell(l, xyz, z, c, atom)


def unique_quartets(n_shells: int) -> np.ndarray:
    """All unique shell quartets (ij|kl) with i>=j, k>=l, ij>=kl (8-fold symmetry)."""
    pairs = [(i, j) for i in range(n_shells) for j in range(i + 1)]
    out = []
    for a in range(len(pairs)):
        for b in range(a + 1):
            out.append(pairs[a] + pairs[b])
    return np.array(out, dtype=np.int32).reshape(-1, 4)


# ---------------------------------------------------------------- small molecules
def small_molecule(seed: int = 1001, n_atoms: int = 6, box: float = 6.0, K: int = 3,
                   shells=(0, 1, 2), zlo: float = 0.1, zhi: float = 10.0) -> Basis:
    """Atoms uniform in a box, each with s,p,d Cartesian shells of contraction K.

    Exponents log-uniform in [zlo, zhi], coefficients uniform [0.1, 1] times the
    primitive normalisation (shells are not renormalised).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    bb = BasisBuilder()
    xyz = rng.uniform(0.0, box, (n_atoms, 3))
    for a in range(n_atoms):
        bb.add_atom(xyz[a])
        for l in shells:
            random_shell(rng, bb, l, xyz[a], K, zlo, zhi, a)
    return bb.build()


def chain(seed: int = 1006, n_atoms: int = 500, spacing: float = 3.0, jitter: float = 0.5, K: int = 3,
          shells=(0, 1, 2), zlo: float = 0.1, zhi: float = 10.0) -> Basis:
    """A long chain of atoms: atom i at (i * spacing, 0, 0) moved by a uniform jitter in [-jitter, jitter]
    on each axis, each atom with s,p,d shells of contraction K (exponents log-uniform in [zlo, zhi],
    coefficients as in small_molecule). Many AOs (10 per atom) with few significant shell pairs per shell,
    so that the density and exchange matrices are far larger than the GPU's L2 while the number of
    screened quartets stays moderate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    bb = BasisBuilder()
    for a in range(n_atoms):
        xyz = np.array([a * spacing, 0.0, 0.0]) + rng.uniform(-jitter, jitter, 3)
        bb.add_atom(xyz)
        for l in shells:
            random_shell(rng, bb, l, xyz, K, zlo, zhi, a)
    return bb.build()


# ---------------------------------------------------------------- per-class quartet grids
def class_sweep(lq, n_bra: int = 224, n_ket: int = 224, seed: int = 1002, box: float = 10.0,
                zlo: float = 0.05, zhi: float = 50.0, K=(1, 1, 1, 1)):
    """Random quartets of one class (la,lb|lc,ld): an n_bra x n_ket grid of
    independent random bra and ket shell pairs (uniform centres in a box,
    log-uniform exponents), as in the per-class microbenchmarks of Sec. 5.

    Returns (basis, quartets[n_bra*n_ket, 4]); quartet (i, k) pairs bra pair i
    with ket pair k, bra-pair index fastest.
    """
    la, lb, lc, ld = (int(x) for x in lq)
    ss = np.random.SeedSequence([seed, la, lb, lc, ld, n_bra, n_ket])
    rng = np.random.Generator(np.random.PCG64(ss))
    bb = BasisBuilder()
    for _ in range(n_bra):
        random_shell(rng, bb, la, rng.uniform(0, box, 3), K[0], zlo, zhi)
        random_shell(rng, bb, lb, rng.uniform(0, box, 3), K[1], zlo, zhi)
    for _ in range(n_ket):
        random_shell(rng, bb, lc, rng.uniform(0, box, 3), K[2], zlo, zhi)
        random_shell(rng, bb, ld, rng.uniform(0, box, 3), K[3], zlo, zhi)
    basis = bb.build()
    i = np.arange(n_bra, dtype=np.int32)
    k = np.arange(n_ket, dtype=np.int32)
    ii, kk = np.meshgrid(i, k, indexing="xy")   # bra index fastest
    ii = ii.reshape(-1); kk = kk.reshape(-1)
    q = np.stack([2 * ii, 2 * ii + 1, 2 * n_bra + 2 * kk, 2 * n_bra + 2 * kk + 1], axis=1).astype(np.int32)
    return basis, q


SWEEP_CLASSES = [(1, 1, 1, 1), (2, 2, 2, 2), (3, 3, 3, 3), (4, 4, 4, 4), (5, 5, 5, 5), (6, 6, 6, 6)]


# ---------------------------------------------------------------- clusters
def class_sweep3(lt, n_aux: int = 224, n_ket: int = 224, seed: int = 1007, box: float = 10.0,
                 zlo: float = 0.05, zhi: float = 50.0, K=(1, 1, 1)):
    """Random triplets of one 3-center class (la|lc,ld): an n_aux x n_ket grid of independent random
    auxiliary shells and orbital shell pairs (uniform centres in a box, log-uniform exponents), the
    3-center counterpart of class_sweep. Returns (aux basis, orbital basis, triplets[n_aux*n_ket, 3]),
    auxiliary index fastest."""
    la, lc, ld = (int(x) for x in lt)
    ss = np.random.SeedSequence([seed, la, lc, ld, n_aux, n_ket])
    rng = np.random.Generator(np.random.PCG64(ss))
    aux, orb = BasisBuilder(), BasisBuilder()
    for _ in range(n_aux):
        random_shell(rng, aux, la, rng.uniform(0, box, 3), K[0], zlo, zhi)
    for _ in range(n_ket):
        random_shell(rng, orb, lc, rng.uniform(0, box, 3), K[1], zlo, zhi)
        random_shell(rng, orb, ld, rng.uniform(0, box, 3), K[2], zlo, zhi)
    i = np.arange(n_aux, dtype=np.int32)
    k = np.arange(n_ket, dtype=np.int32)
    ii, kk = np.meshgrid(i, k, indexing="xy")
    t = np.stack([ii.reshape(-1), 2 * kk.reshape(-1), 2 * kk.reshape(-1) + 1], axis=1).astype(np.int32)
    return aux.build(), orb.build(), t


def cluster(rng, n_atoms: int, min_sep: float = 2.8, density_radius: float = 2.2) -> np.ndarray:
    """Seeded sequential random insertion of atoms in a sphere at >= min_sep bohr."""
    R = density_radius * n_atoms ** (1.0 / 3.0) + min_sep
    pts = []
    tries = 0
    while len(pts) < n_atoms:
        tries += 1
        if tries > 1000000:
            raise RuntimeError("cluster insertion did not converge")
        p = rng.uniform(-R, R, 3)
        if p @ p > R * R:
            continue
        if pts:
            d = np.linalg.norm(np.asarray(pts) - p, axis=1)
            if d.min() < min_sep:
                continue
        pts.append(p)
    return np.asarray(pts)


# per element kind: list of (l, n_shells, K)
HEAVY_SHELLS = [(0, 5, 6), (1, 4, 3), (2, 3, 1), (3, 2, 1), (4, 1, 1)]     # 5s4p3d2f1g
LIGHT_SHELLS = [(0, 4, 6), (1, 3, 3), (2, 2, 1), (3, 1, 1)]                 # 4s3p2d1f
AUX_SHELLS = [(l, n, 1) for l, n in enumerate((6, 5, 4, 3, 2, 2, 1))]      # s..i, K=1


def _add_element_shells(rng, bb: BasisBuilder, atom: int, xyz, recipe, zmin: float = 0.1,
                        ratio: float = 2.5, cratio: float = 3.5, renormalise: bool = False):
    """Geometric exponents: shell i of angular momentum l has primitives
    zmin * 2^l * ratio^i * cratio^k, k = 0..K-1; coefficients uniform [0.1, 1]
    times the primitive normalisation, optionally renormalised to unit
    self-overlap of the x^l component."""
    for l, n, K in recipe:
        for i in range(n):
            z = zmin * (2.0 ** l) * ratio ** i * cratio ** np.arange(K)
            c = rng.uniform(0.1, 1.0, K) * primitive_norm(l, z)
            if renormalise:
                c = c / math.sqrt(contracted_self_overlap(l, z, c))
            bb.add_shell(l, xyz, z, c, atom)


def df_cluster(seed: int = 1003, n_atoms: int = 100):
    """Density-fitting cluster: orbital basis 4s3p2d1f (K 6/3/1/1) and auxiliary basis
    s..i (K=1, even-tempered ratio 2.5) on a random cluster. Returns (aux, orb)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = cluster(rng, n_atoms)
    orb = BasisBuilder(); aux = BasisBuilder()
    for a in range(n_atoms):
        orb.add_atom(xyz[a]); aux.add_atom(xyz[a])
        _add_element_shells(rng, orb, a, xyz[a], LIGHT_SHELLS)
        _add_element_shells(rng, aux, a, xyz[a], AUX_SHELLS)
    return aux.build(), orb.build()


def molecule(seed: int, n_atoms: int, heavy_fraction: float = 0.5) -> Basis:
    """Compact cluster molecule, heavy atoms 5s4p3d2f1g and H-like 4s3p2d1f,
    shells renormalised (the molecules of the batched-exchange and gradient workloads)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = cluster(rng, n_atoms)
    heavy = rng.uniform(0, 1, n_atoms) < heavy_fraction
    bb = BasisBuilder()
    for a in range(n_atoms):
        bb.add_atom(xyz[a])
        _add_element_shells(rng, bb, a, xyz[a], HEAVY_SHELLS if heavy[a] else LIGHT_SHELLS,
                            renormalise=True)
    return bb.build()


def molecule_batch(seed: int = 1004, n_mol: int = 64, lo: int = 10, hi: int = 120):
    """Batch of uneven molecules: n_mol molecules with seeded atom counts uniform in [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = rng.integers(lo, hi + 1, n_mol)
    return [molecule(seed * 1000 + i, int(s)) for i, s in enumerate(sizes)]


def density(nao: int, seed: int, occ_fraction: float = 0.2) -> np.ndarray:
    """D = C C^T with C a random orthonormal nao x max(1, nao*occ_fraction) matrix."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nocc = max(1, int(nao * occ_fraction))
    G = rng.standard_normal((nao, nocc))
    C, _ = np.linalg.qr(G)
    return C @ C.T


def random_symmetric(n: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    M = rng.uniform(-1, 1, (n, n))
    return 0.5 * (M + M.T)


def random_quartets(basis: Basis, n: int, seed: int) -> np.ndarray:
    """n random (non-canonical) shell quartets of a basis."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, basis.n_shells, (n, 4)).astype(np.int32)
