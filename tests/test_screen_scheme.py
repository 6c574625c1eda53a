"""Host logic of the exchange screening, on the CPU.

The screening kernel keeps the unique quartet (ij|kl) of a shell-pair list when
Q_ij Q_kl max(|D_ik|, |D_il|, |D_jk|, |D_jl|) >= tau (FP64, that product order).
To avoid testing every pair of pairs it lists each class's pairs by decreasing Q
and stops a bra pair's scan of a ket class at the first pair where
Q_ij Q_kl rowmax < tau (rowmax: the largest density-block maximum of shells i
and j), which no later pair of the class can pass. This test restates that
procedure step by step in numpy and compares its kept set with the plain rule
applied to every unordered pair of pairs, on random inputs with ties, zeros and
Schwarz factors spanning many orders of magnitude.
"""
import numpy as np
import pytest


def brute_force(pairs, Q, dmax, tau):
    kept = set()
    n = len(pairs)
    for p in range(n):
        i, j = pairs[p]
        for q in range(p + 1):
            k, l = pairs[q]
            d = max(max(dmax[i, k], dmax[i, l]), max(dmax[j, k], dmax[j, l]))
            if Q[p] * Q[q] * d >= tau:
                kept.add((max(p, q), min(p, q)))
    return kept


def kernel_scheme(pairs, Q, pclass, dmax, tau):
    """The kernel's procedure: pairs sorted by (class, decreasing Q); for bra pair p, every
    segment (class) cq <= cp, in the own segment only up to p's position; binary search of the cut."""
    n = len(pairs)
    order = sorted(range(n), key=lambda x: (pclass[x], -Q[x], x))
    pos = {p: i for i, p in enumerate(order)}
    seg_begin, seg_class = [], []
    for i, p in enumerate(order):
        if i == 0 or pclass[p] != pclass[order[i - 1]]:
            seg_begin.append(i)
            seg_class.append(pclass[p])
    seg_begin.append(n)
    rowmax = dmax.max(axis=1)
    kept, tested = set(), 0
    for p in range(n):
        i, j = pairs[p]
        dr = max(rowmax[i], rowmax[j])
        for g in range(len(seg_class)):
            cq = seg_class[g]
            if cq > pclass[p]:
                break
            b0 = seg_begin[g]
            e0 = pos[p] + 1 if cq == pclass[p] else seg_begin[g + 1]
            lo, hi = b0, e0
            while lo < hi:
                mid = lo + (hi - lo) // 2
                if Q[p] * Q[order[mid]] * dr >= tau:
                    lo = mid + 1
                else:
                    hi = mid
            for x in range(b0, lo):
                q = order[x]
                tested += 1
                k, l = pairs[q]
                d = max(max(dmax[i, k], dmax[i, l]), max(dmax[j, k], dmax[j, l]))
                if Q[p] * Q[q] * d >= tau:
                    kept.add((max(p, q), min(p, q)))
    return kept, tested


@pytest.mark.parametrize("seed", range(6))
def test_sorted_scan_keeps_exactly_the_rule(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    n_shells = int(rng.integers(3, 14))
    pairs = [(i, j) for i in range(n_shells) for j in range(i + 1)]
    m = len(pairs)
    Q = 10.0 ** rng.uniform(-9, 1, m)
    Q[rng.uniform(size=m) < 0.1] = 0.0
    ties = rng.uniform(size=m) < 0.2
    Q[ties] = Q[0]
    pclass = rng.integers(0, 4, m)
    A = 10.0 ** rng.uniform(-6, 0, (n_shells, n_shells))
    dmax = np.maximum(A, A.T)
    for tau in (0.0, 1e-12, 1e-8, 1e-4):
        ref = brute_force(pairs, Q, dmax, tau)
        got, tested = kernel_scheme(pairs, Q, pclass, dmax, tau)
        assert got == ref, (seed, tau, len(got), len(ref))
        assert tested <= m * (m + 1) // 2


def test_scan_cost_follows_the_kept_quartets():
    """With Q spread over orders of magnitude and a tight threshold, the scan tests far fewer
    pairs of pairs than the square of the pair count."""
    rng = np.random.Generator(np.random.PCG64(99))
    n_shells = 30
    pairs = [(i, j) for i in range(n_shells) for j in range(i + 1)]
    m = len(pairs)
    Q = 10.0 ** rng.uniform(-12, 0, m)
    dmax = np.ones((n_shells, n_shells))
    got, tested = kernel_scheme(pairs, Q, np.zeros(m, dtype=int), dmax, 1e-10)
    assert got == brute_force(pairs, Q, dmax, 1e-10)
    assert tested == len(got)              # with flat D every tested quartet passes
    assert tested < 0.5 * m * (m + 1) // 2   # about 35 % of all pairs of pairs are kept here
