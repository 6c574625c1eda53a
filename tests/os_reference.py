"""Independent Obara-Saika / Head-Gordon-Pople integrals, used only to pin the oracle.

Written from the recurrence relations of Obara & Saika (J. Chem. Phys. 84, 3963
(1986)) and the horizontal recurrence of Head-Gordon & Pople (J. Chem. Phys. 89,
5777 (1988)), the scheme the paper compares against in Sec. 5. It shares nothing
with the McMurchie-Davidson oracle: no Hermite expansion, no R recursion, and its
Boys function is mpmath's confluent hypergeometric function at 30 digits,
F_m(T) = 1F1(m+1/2; m+3/2; -T) / (2m+1).

Pure Python with memoisation: only for tiny inputs (a few quartets up to
[dd|dd] / [ff|ff]).
"""
from __future__ import annotations

import math
from functools import lru_cache

import mpmath

mpmath.mp.dps = 30


def boys_mp(mmax: int, T: float):
    return [float(mpmath.hyp1f1(m + 0.5, m + 1.5, -mpmath.mpf(T)) / (2 * m + 1)) for m in range(mmax + 1)]


def cart_list(l):
    return [(ax, ay, l - ax - ay) for ax in range(l, -1, -1) for ay in range(l - ax, -1, -1)]


def _prim_e0f0(za, zb, zc, zd, A, B, C, D, lmax_e, lmax_f):
    """Primitive [e0|f0]^(0) for all |e| <= lmax_e, |f| <= lmax_f (OS vertical recursion)."""
    p = za + zb
    q = zc + zd
    P = [(za * A[i] + zb * B[i]) / p for i in range(3)]
    Q = [(zc * C[i] + zd * D[i]) / q for i in range(3)]
    W = [(p * P[i] + q * Q[i]) / (p + q) for i in range(3)]
    rho = p * q / (p + q)
    AB2 = sum((A[i] - B[i]) ** 2 for i in range(3))
    CD2 = sum((C[i] - D[i]) ** 2 for i in range(3))
    PQ2 = sum((P[i] - Q[i]) ** 2 for i in range(3))
    Kab = math.exp(-za * zb / p * AB2)
    Kcd = math.exp(-zc * zd / q * CD2)
    pref = 2.0 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * Kab * Kcd
    L = lmax_e + lmax_f
    F = boys_mp(L, rho * PQ2)
    base = [pref * f for f in F]

    @lru_cache(maxsize=None)
    def v(e, f, m):
        if min(e) < 0 or min(f) < 0:
            return 0.0
        if sum(e) == 0 and sum(f) == 0:
            return base[m]
        if sum(e) > 0:
            i = next(k for k in range(3) if e[k] > 0)
            em = tuple(e[k] - (k == i) for k in range(3))
            emm = tuple(e[k] - 2 * (k == i) for k in range(3))
            fm = tuple(f[k] - (k == i) for k in range(3))
            r = (P[i] - A[i]) * v(em, f, m) + (W[i] - P[i]) * v(em, f, m + 1)
            if em[i] > 0:
                r += em[i] / (2 * p) * (v(emm, f, m) - rho / p * v(emm, f, m + 1))
            if f[i] > 0:
                r += f[i] / (2 * (p + q)) * v(em, fm, m + 1)
            return r
        i = next(k for k in range(3) if f[k] > 0)
        fm = tuple(f[k] - (k == i) for k in range(3))
        fmm = tuple(f[k] - 2 * (k == i) for k in range(3))
        r = (Q[i] - C[i]) * v(e, fm, m) + (W[i] - Q[i]) * v(e, fm, m + 1)
        if fm[i] > 0:
            r += fm[i] / (2 * q) * (v(e, fmm, m) - rho / q * v(e, fmm, m + 1))
        return r

    return v


def eri4_shellset(la, lb, lc, ld, A, B, C, D, ea, ca, eb, cb, ec, cc, ed, cd):
    """Contracted [ab|cd] as nested lists [a][b][c][d] (library Cartesian order),
    via contracted [e0|f0] followed by the horizontal recursion
    [a,b+1_i| = [a+1_i,b| + (A_i - B_i)[a,b|  (and the same in the ket)."""
    le_max, lf_max = la + lb, lc + ld
    # contracted [e0|f0] for la <= |e| <= la+lb, lc <= |f| <= lc+ld
    es = [e for l in range(la, le_max + 1) for e in cart_list(l)]
    fs = [f for l in range(lc, lf_max + 1) for f in cart_list(l)]
    acc = {(e, f): 0.0 for e in es for f in fs}
    for za, wa in zip(ea, ca):
        for zb, wb in zip(eb, cb):
            for zc, wc in zip(ec, cc):
                for zd, wd in zip(ed, cd):
                    v = _prim_e0f0(za, zb, zc, zd, A, B, C, D, le_max, lf_max)
                    w = wa * wb * wc * wd
                    for e in es:
                        for f in fs:
                            acc[(e, f)] += w * v(e, f, 0)
    AB = [A[i] - B[i] for i in range(3)]
    CD = [C[i] - D[i] for i in range(3)]

    @lru_cache(maxsize=None)
    def hrr(a, b, c, d):
        if sum(b) > 0:
            i = next(k for k in range(3) if b[k] > 0)
            bm = tuple(b[k] - (k == i) for k in range(3))
            ap = tuple(a[k] + (k == i) for k in range(3))
            return hrr(ap, bm, c, d) + AB[i] * hrr(a, bm, c, d)
        if sum(d) > 0:
            i = next(k for k in range(3) if d[k] > 0)
            dm = tuple(d[k] - (k == i) for k in range(3))
            cp = tuple(c[k] + (k == i) for k in range(3))
            return hrr(a, b, cp, dm) + CD[i] * hrr(a, b, c, dm)
        return acc[(a, c)]

    return [[[[hrr(a, b, c, d) for d in cart_list(ld)] for c in cart_list(lc)]
             for b in cart_list(lb)] for a in cart_list(la)]


def eri3_shellset(la, lc, ld, A, C, D, ea, ca, ec, cc, ed, cd):
    """Contracted [a|cd]: the 4-center result with an s function of zero exponent
    and unit coefficient in the second bra position (phi_b = 1)."""
    v = eri4_shellset(la, 0, lc, ld, A, A, C, D, ea, ca, [0.0], [1.0], ec, cc, ed, cd)
    return [[[v[a][0][c][d] for d in range(len(v[a][0][c]))] for c in range(len(v[a][0]))]
            for a in range(len(v))]
