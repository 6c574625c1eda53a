"""Oracle for the McMurchie-Davidson integral engine: plain CPU FP64 reference.

TEST INFRASTRUCTURE ONLY. The test-suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers; the product path never imports this
package. It shares no code with the CUDA engine: the C++ source
`mdx_oracle.cpp` is written directly from Sec. 2 of Asadchev & Valeev
(arXiv:2405.01834) and is compiled here with the host compiler.

Functions take numpy arrays and the `Basis` object of the seeded input module
(`paper_2405_01834_gb300.inputs`), which carries no method arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mdx_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmdx_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (OpenMP). Returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            lib.orc_boys.argtypes = [ctypes.c_int, ctypes.c_double, P, ctypes.c_int]
            lib.orc_e2c.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, P]
            lib.orc_e1c.argtypes = [ctypes.c_int, ctypes.c_double, P]
            lib.orc_rtable.argtypes = [ctypes.c_int, ctypes.c_double, P, P]
            lib.orc_eri4.argtypes = [P] * 7 + [ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int]
            lib.orc_eri3.argtypes = [P] * 13 + [ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int]
            lib.orc_eri3_sph.argtypes = [P] * 13 + [ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int]
            lib.orc_exchange.argtypes = [P] * 7 + [ctypes.c_int32, ctypes.c_int32, P, P, ctypes.c_int]
            lib.orc_exchange_rows.argtypes = [P] * 7 + [ctypes.c_int32, ctypes.c_int32, P, P, P,
                                                        ctypes.c_int32, ctypes.c_int]
            lib.orc_exchange_grad.argtypes = [P] * 8 + [ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32, P,
                                                        ctypes.c_int]
            lib.orc_solid_coefs.argtypes = [ctypes.c_int, P]
            lib.orc_eri4_sph.argtypes = [P] * 7 + [ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def boys(mmax: int, x: float, precision: int = 0) -> np.ndarray:
    """F_m(x) for m = 0..mmax (Eq. boys); precision=1 evaluates in long double."""
    F = np.zeros(mmax + 1)
    _load().orc_boys(mmax, float(x), _p(F), precision)
    return F


def e2c(la: int, lb: int, za: float, zb: float, A: float, B: float) -> np.ndarray:
    """(E)_{ij}^t along one axis as an array [la+1, lb+1, la+lb+1] (Eqs. E2rr1/E2rr2)."""
    E = np.zeros((la + 1) * (lb + 1) * (la + lb + 1))
    _load().orc_e2c(la, lb, za, zb, A, B, _p(E))
    return E.reshape(la + 1, lb + 1, la + lb + 1)


def e1c(la: int, za: float) -> np.ndarray:
    """E_a^t along one axis as an array [la+1, la+1] (Eq. E1rr)."""
    E = np.zeros((la + 1) * (la + 1))
    _load().orc_e1c(la, za, _p(E))
    return E.reshape(la + 1, la + 1)


def rtable(L: int, rho: float, PQ) -> np.ndarray:
    """[tuv]^(0) with the 2 pi^(5/2)/(...) prefactor set to 1: array [L+1]^3 (Eqs. 0m, r)."""
    PQ = np.ascontiguousarray(PQ, dtype=np.float64)
    R = np.zeros((L + 1) ** 3)
    _load().orc_rtable(L, rho, _p(PQ), _p(R))
    return R.reshape(L + 1, L + 1, L + 1)


def _basis_arrays(b):
    return (np.ascontiguousarray(b.l, dtype=np.int32), np.ascontiguousarray(b.nprim, dtype=np.int32),
            np.ascontiguousarray(b.prim_off, dtype=np.int32), np.ascontiguousarray(b.center, dtype=np.float64),
            np.ascontiguousarray(b.exps, dtype=np.float64), np.ascontiguousarray(b.coefs, dtype=np.float64))


def shellset_sizes4(basis, quartets: np.ndarray) -> np.ndarray:
    l = np.asarray(basis.l)
    q = np.asarray(quartets).reshape(-1, 4)
    nc = (l + 1) * (l + 2) // 2
    return nc[q[:, 0]] * nc[q[:, 1]] * nc[q[:, 2]] * nc[q[:, 3]]


def eri4(basis, quartets, nthreads: int = 0, precision: int = 0):
    """Contracted shellsets [ab|cd] for quartets[n][4]; returns (flat values, offsets[n+1])."""
    q = np.ascontiguousarray(np.asarray(quartets, dtype=np.int32).reshape(-1, 4))
    sizes = shellset_sizes4(basis, q).astype(np.int64)
    off = np.zeros(len(q) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    out = np.zeros(int(off[-1]))
    arrs = _basis_arrays(basis)
    _load().orc_eri4(*[_p(a) for a in arrs], _p(q), len(q), _p(out), _p(off), nthreads, precision)
    return out, off


def eri3(aux, orb, triplets, nthreads: int = 0, precision: int = 0):
    """Contracted shellsets [a|cd] for triplets[n][3] = (aux, orb, orb); returns (values, offsets)."""
    t = np.ascontiguousarray(np.asarray(triplets, dtype=np.int32).reshape(-1, 3))
    la = np.asarray(aux.l); lo = np.asarray(orb.l)
    nca = (la + 1) * (la + 2) // 2; nco = (lo + 1) * (lo + 2) // 2
    sizes = (nca[t[:, 0]] * nco[t[:, 1]] * nco[t[:, 2]]).astype(np.int64)
    off = np.zeros(len(t) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    out = np.zeros(int(off[-1]))
    a1 = _basis_arrays(aux); a2 = _basis_arrays(orb)
    _load().orc_eri3(*[_p(a) for a in a1], *[_p(a) for a in a2], _p(t), len(t), _p(out), _p(off),
                     nthreads, precision)
    return out, off


def eri3_sph(aux, orb, triplets, nthreads: int = 0, precision: int = 0):
    """[a|cd] over real solid harmonics (m = -l..l for a, c and d); returns (values, offsets).
    precision 1: the long double build (Cartesian shellsets and transform), rounded at the end."""
    t = np.ascontiguousarray(np.asarray(triplets, dtype=np.int32).reshape(-1, 3))
    la = np.asarray(aux.l); lo = np.asarray(orb.l)
    sizes = ((2 * la[t[:, 0]] + 1) * (2 * lo[t[:, 1]] + 1) * (2 * lo[t[:, 2]] + 1)).astype(np.int64)
    off = np.zeros(len(t) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    out = np.zeros(int(off[-1]))
    a1 = _basis_arrays(aux); a2 = _basis_arrays(orb)
    _load().orc_eri3_sph(*[_p(a) for a in a1], *[_p(a) for a in a2], _p(t), len(t), _p(out), _p(off),
                         nthreads, precision)
    return out, off


def exchange(basis, D: np.ndarray, row_shells=None, nthreads: int = 0) -> np.ndarray:
    """Dense K_ik = sum_jl D_jl (ij|kl) (Sec. 6).

    Full K: every unique shell quartet once, scattered over its distinct index
    permutations. row_shells: only those shells' K rows, by the direct sum over
    all (j, k, l) shells (other rows zero).
    """
    arrs = _basis_arrays(basis)
    ao_off = np.ascontiguousarray(basis.ao_off, dtype=np.int32)
    nao = int(basis.nao)
    D = np.ascontiguousarray(D, dtype=np.float64)
    assert D.shape == (nao, nao)
    K = np.zeros((nao, nao))
    if row_shells is None:
        _load().orc_exchange(*[_p(a) for a in arrs], _p(ao_off), int(basis.n_shells), nao, _p(D), _p(K), nthreads)
    else:
        rows = np.ascontiguousarray(row_shells, dtype=np.int32)
        _load().orc_exchange_rows(*[_p(a) for a in arrs], _p(ao_off), int(basis.n_shells), nao, _p(D), _p(K),
                                  _p(rows), len(rows), nthreads)
    return K


def exchange_energy(basis, D: np.ndarray, nthreads: int = 0) -> float:
    """S = sum_ik D_ik K_ik with K the dense exchange matrix (E_x = alpha S)."""
    return float(np.sum(np.asarray(D) * exchange(basis, D, nthreads=nthreads)))


def exchange_grad(basis, D: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """dS/dR per atom, S = sum_ijkl D_ik D_jl (ij|kl), D fixed: array [n_atoms, 3].
    Every ordered quartet and all four centres differentiated explicitly."""
    arrs = _basis_arrays(basis)
    ao_off = np.ascontiguousarray(basis.ao_off, dtype=np.int32)
    atom = np.ascontiguousarray(basis.atom, dtype=np.int32)
    nao = int(basis.nao)
    D = np.ascontiguousarray(D, dtype=np.float64)
    n_atoms = int(max(basis.n_atoms, int(atom.max()) + 1 if len(atom) else 0))
    g = np.zeros((n_atoms, 3))
    _load().orc_exchange_grad(*[_p(a) for a in arrs], _p(ao_off), _p(atom), int(basis.n_shells), nao, _p(D),
                              n_atoms, _p(g), nthreads)
    return g


def solid_coefs(l: int) -> np.ndarray:
    """Real solid harmonics S_lm as Cartesian polynomials: [2l+1 (m = -l..l), ncart(l)]."""
    C = np.zeros((2 * l + 1) * ncart(l))
    _load().orc_solid_coefs(l, _p(C))
    return C.reshape(2 * l + 1, ncart(l))


def eri4_sph(basis, quartets, nthreads: int = 0, precision: int = 0):
    """[ab|cd] over real solid harmonics (m = -l..l per shell); returns (values, offsets).
    precision 1: the long double build (Cartesian shellsets and transform), rounded at the end."""
    q = np.ascontiguousarray(np.asarray(quartets, dtype=np.int32).reshape(-1, 4))
    l = np.asarray(basis.l)
    ns = 2 * l + 1
    sizes = (ns[q[:, 0]] * ns[q[:, 1]] * ns[q[:, 2]] * ns[q[:, 3]]).astype(np.int64)
    off = np.zeros(len(q) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    out = np.zeros(int(off[-1]))
    arrs = _basis_arrays(basis)
    _load().orc_eri4_sph(*[_p(a) for a in arrs], _p(q), len(q), _p(out), _p(off), nthreads, precision)
    return out, off
