"""Algorithmic work model of McMurchie-Davidson shellsets (the paper's Table 1).

Counts follow the Table 1 convention of Asadchev & Valeev (arXiv:2405.01834,
Sec. 2, "md-scheme" table): per primitive shellset the steps
  [0]^(m) -> [r]^(0)        R_L = (2+L)(7+L)(12+5L+L^2)/8 FLOPs (Eq. r)
  [r]^(0) -> [p|q]          Nb~ Nk~ / 2                        (Eq. pq)
  [p|q]   -> [p|ket]        2 Nb~ Nk~ N_ket                    (Eq. ket-from-hermite)
  [p|ket] -> [bra|ket]      2 N_bra Nb~ N_ket                  (Eq. bra-from-hermite)
with Nt(l) = (l+1)(l+2)(l+3)/6 Hermite functions. For contracted Cartesian
shellsets the first three steps run for every primitive quartet (K_b K_k times)
and the bra step once per bra primitive pair (ket primitives are folded into the
ket transform), with N_bra = ncart(la) ncart(lb), N_ket = ncart(lc) ncart(ld).
For 3-center [a|cd] the bra is one shell: Nb~ = Nt(la), N_bra = ncart(la).
These are the "model FLOPs" that throughput and roofline figures are quoted in.
"""
from __future__ import annotations


def nherm(l: int) -> int:
    """Nt(l): Hermite Gaussians with total index <= l."""
    return (l + 1) * (l + 2) * (l + 3) // 6


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def nsolid(l: int) -> int:
    return 2 * l + 1


def r_flops(L: int) -> float:
    """R_L of Table 1."""
    return (2 + L) * (7 + L) * (12 + 5 * L + L * L) / 8


def table1_steps(lbra: int, lket: int, nbra: int, nket: int):
    """(A_in, A_out, N_F) of the four steps of Table 1 for one primitive shellset
    with bra/ket total angular momenta lbra/lket and nbra/nket AO functions."""
    L = lbra + lket
    nb, nk = nherm(lbra), nherm(lket)
    return [
        (L + 1, nherm(L), r_flops(L)),
        (nherm(L), nb * nk, nb * nk / 2),
        (nb * nk, nb * nket, 2 * nb * nk * nket),
        (nb * nket, nbra * nket, 2 * nbra * nb * nket),
    ]


def eri4_flops(la: int, lb: int, lc: int, ld: int, Kb: int = 1, Kk: int = 1) -> float:
    """Model FLOPs of one contracted Cartesian shellset [ab|cd]."""
    Lb, Lk = la + lb, lc + ld
    Nb, Nk = ncart(la) * ncart(lb), ncart(lc) * ncart(ld)
    hb, hk = nherm(Lb), nherm(Lk)
    return Kb * Kk * (r_flops(Lb + Lk) + hb * hk / 2 + 2 * hb * hk * Nk) + Kb * 2 * Nb * hb * Nk


def eri3_flops(la: int, lc: int, ld: int, Ka: int = 1, Kk: int = 1) -> float:
    """Model FLOPs of one contracted Cartesian shellset [a|cd]."""
    Lk = lc + ld
    Na, Nk = ncart(la), ncart(lc) * ncart(ld)
    ha, hk = nherm(la), nherm(Lk)
    return Ka * Kk * (r_flops(la + Lk) + ha * hk / 2 + 2 * ha * hk * Nk) + Ka * 2 * Na * ha * Nk
