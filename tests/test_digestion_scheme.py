"""The engine's exchange digestion and gradient scheme, checked on the CPU as
mathematics against the definitions (Sec. 6: K_ik = sum_jl D_jl (ij|kl);
S = sum_ijkl D_ik D_jl (ij|kl)), with the oracle's integrals.

The GPU evaluates each unique shell quartet (i >= j, k >= l, ij >= kl) once
and, with the weight w = (1/2 if i = j) (1/2 if k = l) (1/2 if ij = kl),
  - adds four blocks, K_ik += w sum D_jl V, K_il += w sum D_jk V,
    K_jk += w sum D_il V, K_jl += w sum D_ik V, then forms K + K^T;
  - for the energy, adds 4 w sum G V with G = D_ik D_jl + D_il D_jk.
These tests restate that scheme in numpy and compare it with the plain sums
over all ordered quartets, so a wrong weight or a missing block fails here
without a GPU.
"""
import numpy as np

import oracle
from paper_2405_01834_gb300 import inputs


def _full_tensor(b):
    ns = b.n_shells
    nao = b.nao
    nc = [inputs.ncart(int(x)) for x in b.l]
    ao = b.ao_off
    quart = np.array([[i, j, k, l] for i in range(ns) for j in range(ns) for k in range(ns) for l in range(ns)],
                     dtype=np.int32)
    v, off = oracle.eri4(b, quart)
    full = np.zeros((nao,) * 4)
    for n, (i, j, k, l) in enumerate(quart):
        full[ao[i]:ao[i] + nc[i], ao[j]:ao[j] + nc[j], ao[k]:ao[k] + nc[k], ao[l]:ao[l] + nc[l]] = \
            v[off[n]:off[n + 1]].reshape(nc[i], nc[j], nc[k], nc[l])
    return full


def _unique(ns):
    pairs = [(i, j) for i in range(ns) for j in range(i + 1)]
    for p in range(len(pairs)):
        for q in range(p + 1):
            yield pairs[p], pairs[q], p == q


def _blocks(b):
    nc = [inputs.ncart(int(x)) for x in b.l]
    return [slice(int(o), int(o) + n) for o, n in zip(b.ao_off, nc)]


def test_unique_quartet_digestion_gives_the_exchange_matrix():
    b = inputs.small_molecule(seed=13, n_atoms=2, shells=(0, 1, 2), K=2)
    full = _full_tensor(b)
    D = inputs.density(b.nao, 4, occ_fraction=0.4)
    sl = _blocks(b)
    K = np.zeros_like(D)
    for (i, j), (k, l), same in _unique(b.n_shells):
        w = (0.5 if i == j else 1.0) * (0.5 if k == l else 1.0) * (0.5 if same else 1.0)
        V = full[sl[i], sl[j], sl[k], sl[l]]
        K[sl[i], sl[k]] += w * np.einsum("abcd,bd->ac", V, D[sl[j], sl[l]])
        K[sl[i], sl[l]] += w * np.einsum("abcd,bc->ad", V, D[sl[j], sl[k]])
        K[sl[j], sl[k]] += w * np.einsum("abcd,ad->bc", V, D[sl[i], sl[l]])
        K[sl[j], sl[l]] += w * np.einsum("abcd,ac->bd", V, D[sl[i], sl[k]])
    K = K + K.T
    ref = np.einsum("ijkl,jl->ik", full, D)
    np.testing.assert_allclose(K, ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))
    # a wrong degeneracy weight is caught
    Kbad = np.zeros_like(D)
    for (i, j), (k, l), same in _unique(b.n_shells):
        w = (0.5 if k == l else 1.0) * (0.5 if same else 1.0)   # i = j half dropped
        V = full[sl[i], sl[j], sl[k], sl[l]]
        Kbad[sl[i], sl[k]] += w * np.einsum("abcd,bd->ac", V, D[sl[j], sl[l]])
        Kbad[sl[i], sl[l]] += w * np.einsum("abcd,bc->ad", V, D[sl[j], sl[k]])
        Kbad[sl[j], sl[k]] += w * np.einsum("abcd,ad->bc", V, D[sl[i], sl[l]])
        Kbad[sl[j], sl[l]] += w * np.einsum("abcd,ac->bd", V, D[sl[i], sl[k]])
    assert np.max(np.abs(Kbad + Kbad.T - ref)) > 1e-6 * np.max(np.abs(ref))


def test_unique_quartet_energy_sum():
    """S = sum_unique 4 w sum_abcd (D_ik D_jl + D_il D_jk) (ab|cd) equals the full sum,
    and equals Tr(D K)."""
    b = inputs.small_molecule(seed=17, n_atoms=2, shells=(0, 1, 2), K=1)
    full = _full_tensor(b)
    D = inputs.density(b.nao, 6, occ_fraction=0.4)
    sl = _blocks(b)
    S = 0.0
    for (i, j), (k, l), same in _unique(b.n_shells):
        w = (0.5 if i == j else 1.0) * (0.5 if k == l else 1.0) * (0.5 if same else 1.0)
        V = full[sl[i], sl[j], sl[k], sl[l]]
        G = np.einsum("ac,bd->abcd", D[sl[i], sl[k]], D[sl[j], sl[l]]) + \
            np.einsum("ad,bc->abcd", D[sl[i], sl[l]], D[sl[j], sl[k]])
        S += 4.0 * w * float(np.sum(G * V))
    ref = float(np.einsum("ijkl,ik,jl->", full, D, D))
    assert abs(S - ref) <= 1e-13 * abs(ref)
    K = np.einsum("ijkl,jl->ik", full, D)
    assert abs(float(np.sum(D * K)) - ref) <= 1e-13 * abs(ref)
