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
import pytest

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


def _cart(l):
    return [(ax, ay, l - ax - ay) for ax in range(l, -1, -1) for ay in range(l - ax, -1, -1)]


@pytest.mark.parametrize("omit", [0, 1, 2, 3])
def test_shifted_class_gradient_scheme(omit):
    """The GPU's gradient scheme: per unique quartet and each of three of its
    shells, the class with that shell raised (l+1, coefficients 2 zeta c) and
    lowered (l-1), contracted with G = D_ik D_jl + D_il D_jk at the unshifted
    component (raised element a' feeds a' - 1_x with weight +1, lowered element
    a' feeds a' + 1_x with weight -(a'_x + 1)); the atom of the fourth shell
    (position `omit`, chosen per class on the GPU) takes minus the sum
    (translational invariance). Against the oracle's gradient, which
    differentiates all four centres explicitly."""
    b = inputs.small_molecule(seed=23, n_atoms=3, shells=(0, 1, 2), K=2)
    D = inputs.density(b.nao, 8, occ_fraction=0.4)
    ref = oracle.exchange_grad(b, D)
    ns = b.n_shells
    # extended basis: shell s, its raised partner ns + s, its lowered partner 2 ns + s (an s shell
    # gets a placeholder s shell there, never used)
    bb = inputs.BasisBuilder()
    for v in range(3):
        for s in range(ns):
            p0, n = int(b.prim_off[s]), int(b.nprim[s])
            z, c = b.exps[p0:p0 + n], b.coefs[p0:p0 + n]
            l = int(b.l[s])
            if v == 0:
                bb.add_shell(l, b.center[s], z, c)
            elif v == 1:
                bb.add_shell(l + 1, b.center[s], z, 2.0 * z * c)
            else:
                bb.add_shell(max(l - 1, 0), b.center[s], z, c)
    ext = bb.build()
    sl = _blocks(b)
    g = np.zeros((b.n_atoms, 3))
    jobs = []
    for (i, j), (k, l), same in _unique(ns):
        w = (0.5 if i == j else 1.0) * (0.5 if k == l else 1.0) * (0.5 if same else 1.0)
        for pos in range(4):
            if pos == omit:
                continue
            for sign in (1, -1):
                sh = (i, j, k, l)[pos]
                if sign < 0 and b.l[sh] == 0:
                    continue
                q = [i, j, k, l]
                q[pos] = sh + (ns if sign > 0 else 2 * ns)
                jobs.append((q, (i, j, k, l), w, pos, sign))
    vals, off = oracle.eri4(ext, np.array([j[0] for j in jobs], dtype=np.int32))
    for n, (q, (i, j, k, l), w, pos, sign) in enumerate(jobs):
        ls = [int(ext.l[x]) for x in q]
        V = vals[off[n]:off[n + 1]].reshape([inputs.ncart(x) for x in ls])
        G = np.einsum("ac,bd->abcd", D[sl[i], sl[k]], D[sl[j], sl[l]]) + \
            np.einsum("ad,bc->abcd", D[sl[i], sl[l]], D[sl[j], sl[k]])
        lorg = int(b.l[(i, j, k, l)[pos]])
        orig_index = {c: idx for idx, c in enumerate(_cart(lorg))}
        for sidx, comp in enumerate(_cart(ls[pos])):
            Vs = np.take(V, sidx, axis=pos)
            for x in range(3):
                o = list(comp)
                if sign > 0:
                    if o[x] == 0:
                        continue
                    o[x] -= 1
                    wt = 1.0
                else:
                    o[x] += 1
                    wt = -float(o[x])
                Gs = np.take(G, orig_index[tuple(o)], axis=pos)
                t = 4.0 * w * wt * float(np.sum(Vs * Gs))
                g[b.atom[(i, j, k, l)[pos]], x] += t
                g[b.atom[(i, j, k, l)[omit]], x] -= t
    np.testing.assert_allclose(g, ref, rtol=0, atol=1e-11 * np.max(np.abs(ref)))
