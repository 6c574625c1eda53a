"""CPU emulator of the team kernel's step programs (test infrastructure).

The team kernel is a generic interpreter: everything class-specific lives in
the programs that the host planner emits (R levels of Eq. r, the ket steps
k1/k2/k3 of Eq. ket-from-hermite, the bra steps b1/b23 of Eq.
bra-from-hermite, the column map). This module builds those programs with the
library's own planner (compiled here with the host compiler through
`planner_shim.cpp`) and executes them on one flat float64 workspace with the
semantics the kernel gives each entry, so that the CPU suite can check every
class's programs against the oracle without a GPU.

Everything else the kernel takes as input is formed here from the paper's
definitions, not from the library: primitive-pair records (zeta_p, P, the
prefactor c_a c_b exp(-zeta_a zeta_b |AB|^2 / zeta_p) and per-axis E tables
with E_00^0 = 1, Eqs. E2rr1/E2rr2 or E1rr, taken from the oracle's E routines)
and the Boys values (the oracle's F_m). The ket records carry the (-1)^t of
Eq. pq, as the kernel expects.

Within a step the kernel runs all entries in parallel; the emulator gathers
every operand before it writes, and `check_hazards` asserts that no entry of a
step reads or writes what another entry of the same step writes.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2405_01834_gb300", "csrc")
SHIM_SRC = os.path.join(HERE, "planner_shim.cpp")
BUILD = os.path.join(HERE, "_build")
SHIM_LIB = os.path.join(BUILD, "libplanner_shim.so")

SCALARS = ("la lb lc ld Kb Kk onec L Lb Lk Nb Nk hb T teams_per_cta team_doubles recb reck o_recb o_reck o_scal "
           "o_G o_R0 o_R1 o_A o_B o_X o_C1 o_OUT c1size ngroups ncols_max nb1 nb23 cache_R has_out "
           "sph nsa nsb nsc nsd ncols_s o_Xs o_C1s o_OUTs c1s hbp xg_doubles o_Rc rstride top_only").split()
STEP = np.dtype([("out", "<u2"), ("src", "<u2"), ("coef", "<u2"), ("n", "u1"), ("stride", "u1")])
B23 = np.dtype([("out", "<u2"), ("src", "<u2"), ("ey", "<u2"), ("ez", "<u2"), ("u0", "u1"), ("nu", "u1"),
                ("su", "u1"), ("v0", "u1"), ("nv", "u1"), ("sv", "u1"), ("r", "u1"), ("pad", "u1")])
GROUP = np.dtype([(n, "<i4") for n in ("k1_off", "k1_n", "k2_off", "k2_n", "k3_off", "k3_n", "ncols", "col_off",
                                       "o_B", "pad")])
REC_HEADER = 8
TWO_PI_52 = 2.0 * math.pi ** 2.5

_lock = threading.Lock()
_lib = None


def _build_shim() -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, f) for f in ("plan.cpp", "boys_table.cpp", "solid.cpp")]
    deps = [SHIM_SRC, os.path.join(CSRC, "mdx_internal.h")] + srcs
    if not os.path.exists(SHIM_LIB) or any(os.path.getmtime(d) > os.path.getmtime(SHIM_LIB) for d in deps):
        tmp = SHIM_LIB + ".tmp%d" % os.getpid()
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I", CSRC, SHIM_SRC, *srcs, "-o", tmp],
                       check=True)
        os.replace(tmp, SHIM_LIB)
    return SHIM_LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(_build_shim())
            lib.shim_build.argtypes = [ctypes.c_int] * 13 + [ctypes.c_char_p, ctypes.c_int]
            lib.shim_build.restype = ctypes.c_int
            lib.shim_scalars.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.shim_scalars.restype = ctypes.c_int
            lib.shim_array.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64]
            lib.shim_array.restype = ctypes.c_int64
            lib.shim_rprog.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64]
            lib.shim_rprog.restype = ctypes.c_int64
            lib.shim_sizes.argtypes = [ctypes.c_void_p]
            lib.shim_boys.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
            lib.shim_boys.restype = ctypes.c_int64
            lib.shim_solid.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64]
            lib.shim_solid.restype = ctypes.c_int64
            lib.shim_exec_fma.argtypes = []
            lib.shim_exec_fma.restype = ctypes.c_double
            sizes = np.zeros(4, dtype=np.int32)
            lib.shim_sizes(sizes.ctypes.data)
            assert (sizes[0], sizes[1], sizes[2], sizes[3]) == (STEP.itemsize, B23.itemsize, GROUP.itemsize,
                                                                REC_HEADER), sizes
            _lib = lib
    return _lib


def _array(lib, fn, which, dtype):
    nbytes = fn(which, None, 0)
    buf = np.zeros(max(nbytes, 0), dtype=np.uint8)
    if nbytes > 0:
        fn(which, buf.ctypes.data, nbytes)
    return buf.view(dtype)


@dataclass
class Plan:
    s: dict
    groups: np.ndarray
    kprog: np.ndarray
    b1: np.ndarray
    b23: np.ndarray
    colmap: np.ndarray
    rprog: np.ndarray
    roff: np.ndarray
    exec_fma: float = 0.0   # FP64 FMAs per shellset as the planner reports them


class PlanError(RuntimeError):
    pass


def plan(la, lb, lc, ld, Kb=1, Kk=1, onec=False, store=False, T=0, budget=0, single_max=0, rcache=-1,
         pack=1) -> Plan:
    """The planner's team-kernel programs for one class and shape (store: False/True, or 2 for the
    solid-harmonic store plan; rcache: the planner's choice of cached R tables, -1 default, 0 never,
    1 wherever they fit; pack: small ket z-pairs share column groups)."""
    lib = _load()
    err = ctypes.create_string_buffer(256)
    if lib.shim_build(la, lb, lc, ld, Kb, Kk, int(onec), int(store), T, budget, single_max, rcache, int(pack), err, 256):
        raise PlanError(err.value.decode())
    sc = np.zeros(64, dtype=np.int32)
    n = lib.shim_scalars(sc.ctypes.data, 64)
    assert n == len(SCALARS)
    s = {k: int(v) for k, v in zip(SCALARS, sc[:n])}
    return Plan(s, _array(lib, lib.shim_array, 0, GROUP), _array(lib, lib.shim_array, 1, STEP),
                _array(lib, lib.shim_array, 2, STEP), _array(lib, lib.shim_array, 3, B23),
                _array(lib, lib.shim_array, 4, np.uint16), _array(lib, lib.shim_rprog, 0, np.uint32),
                _array(lib, lib.shim_rprog, 1, np.int32), float(lib.shim_exec_fma()))


def boys_table():
    """The library's Boys table as [grid][m][k] and the grid's 1/h."""
    lib = _load()
    dims = np.zeros(3, dtype=np.int32)
    inv_h = ctypes.c_double(0.0)
    n = lib.shim_boys(None, 0, dims.ctypes.data, ctypes.byref(inv_h))
    tab = np.zeros(n)
    lib.shim_boys(tab.ctypes.data, n, dims.ctypes.data, ctypes.byref(inv_h))
    return tab.reshape(int(dims[0]), int(dims[1]), int(dims[2])), inv_h.value


def boys_interpolate(tab, inv_h, m, T):
    """F_m(T) as the kernel forms it inside the table: nearest grid point
    T0 = i h (round to nearest), then Horner's rule in -d = T0 - T over the
    row's coefficients F_{m+k}(T0)/k!."""
    i = int(math.floor(T * inv_h + 0.5))
    nd = i / inv_h - T
    c = tab[i, m]
    f = c[-1]
    for k in range(len(c) - 2, -1, -1):
        f = f * nd + c[k]
    return f


def solid_table(l):
    """The library's real solid harmonics of one l: [2l+1][ncart(l)]."""
    lib = _load()
    nc = (l + 1) * (l + 2) // 2
    out = np.zeros((2 * l + 1) * nc)
    assert lib.shim_solid(l, out.ctypes.data, len(out)) == len(out)
    return out.reshape(2 * l + 1, nc)


# ----------------------------------------------------------------- records
def _etab_blocks(la, lb):
    """(a, b, offset) of each (a, b) block of a per-axis table, t contiguous, a-major."""
    o = 0
    for a in range(la + 1):
        for b in range(lb + 1):
            yield a, b, o
            o += a + b + 1


def rec_size(la, lb):
    tab = sum(a + b + 1 for a in range(la + 1) for b in range(lb + 1))
    return (REC_HEADER + 3 * tab + 1) & ~1


def pair_record(la, lb, za, zb, ca, cb, A, B, signed):
    """Primitive-pair record: header [zeta_p, 1/zeta_p, P, prefactor, 0, 0], then
    the x, y, z tables (E)_{ab}^t scaled to E_00^0 = 1 (Eqs. E2rr1/E2rr2);
    signed: (-1)^t folded in (Eq. pq). lb = -1: one-centre bra (Eq. E1rr)."""
    one = lb < 0
    lb = max(lb, 0)
    A = np.asarray(A, dtype=np.float64)
    B = A if one else np.asarray(B, dtype=np.float64)
    p = za + (0.0 if one else zb)
    P = A if one else (za * A + zb * B) / p
    pref = ca * (1.0 if one else cb * math.exp(-za * zb * float(np.sum((A - B) ** 2)) / p))
    tabs = []
    for ax in range(3):
        if one:
            E1 = oracle.e1c(la, za)
            E = np.zeros((la + 1, 1, la + 1))
            E[:, 0, :] = E1 / E1[0, 0]
        else:
            E = oracle.e2c(la, lb, za, zb, float(A[ax]), float(B[ax]))
            E = E / E[0, 0, 0]
        t = []
        for a, b, _ in _etab_blocks(la, lb):
            blk = E[a, b, :a + b + 1].copy()
            if signed:
                blk[1::2] *= -1.0
            t.append(blk)
        tabs.append(np.concatenate(t))
    rec = np.zeros(rec_size(la, lb))
    rec[:REC_HEADER] = [p, 1.0 / p, P[0], P[1], P[2], pref, 0.0, 0.0]
    body = np.concatenate(tabs)
    rec[REC_HEADER:REC_HEADER + len(body)] = body
    return rec


def shell_pair_records(basis, i, j, signed):
    """Records of all primitive pairs of shells (i, j) of `basis`; j = None: one-centre."""
    li = int(basis.l[i])
    pi = range(int(basis.prim_off[i]), int(basis.prim_off[i] + basis.nprim[i]))
    if j is None:
        return [pair_record(li, -1, basis.exps[a], 0.0, basis.coefs[a], 1.0, basis.center[i], None, signed)
                for a in pi]
    lj = int(basis.l[j])
    pj = range(int(basis.prim_off[j]), int(basis.prim_off[j] + basis.nprim[j]))
    return [pair_record(li, lj, basis.exps[a], basis.exps[b], basis.coefs[a], basis.coefs[b], basis.center[i],
                        basis.center[j], signed) for a in pi for b in pj]


# ----------------------------------------------------------------- hazards
def check_hazards(pl: Plan):
    """No entry of a ket step reads or writes what another entry of that step
    writes, and every access stays inside the team workspace."""
    W = pl.s["team_doubles"]
    for g in pl.groups:
        for off, n in ((g["k1_off"], g["k1_n"]), (g["k2_off"], g["k2_n"]), (g["k3_off"], g["k3_n"])):
            ent = pl.kprog[off:off + n]
            outs = ent["out"].astype(np.int64)
            assert len(np.unique(outs)) == len(outs), "two entries of one step write the same word"
            n_max = int(ent["n"].max()) if n else 0
            reads = set()
            for k in range(n_max):
                live = ent["n"] > k
                reads |= set((ent["coef"][live].astype(np.int64) + k * ent["stride"][live]).tolist())
                reads |= set((ent["src"][live].astype(np.int64) + k * ent["stride"][live]).tolist())
            assert not (reads & set(outs.tolist())), "a step reads a word another entry of it writes"
            assert outs.max(initial=0) < W and max(reads, default=0) < W


# ----------------------------------------------------------------- execution
def _run_step(ws, ent, acc, count):
    if len(ent) == 0:
        return
    count["fma"] += int(ent["n"].astype(np.int64).sum())
    out = ent["out"].astype(np.int64)
    coef = ent["coef"].astype(np.int64)
    src = ent["src"].astype(np.int64)
    st = ent["stride"].astype(np.int64)
    n = ent["n"].astype(np.int64)
    v = ws[out].copy() if acc else np.zeros(len(ent))
    for k in range(int(n.max())):
        live = n > k
        v[live] += ws[coef[live] + k * st[live]] * ws[src[live] + k * st[live]]
    ws[out] = v


def rlevel_programs():
    """The planner's R-level program words and the start of each total order."""
    lib = _load()
    return _array(lib, lib.shim_rprog, 0, np.uint32), _array(lib, lib.shim_rprog, 1, np.int32)


def _level(rprog, roff, N, src, g):
    """Entries of total order N of one R level from the previous level `src`:
    PQ[axis] * src[first source] + k * src[second source], with k the word's
    coefficient field (the kernel looks k up in a table of small integers as
    doubles) and entry 0 the Boys seed g[0]."""
    cnt = (N + 1) * (N + 2) * (N + 3) // 6
    w = rprog[roff[N]:roff[N] + cnt].astype(np.int64)
    ax = (w >> 24) & 3
    s1 = w & 0xFFF
    s2 = (w >> 12) & 0xFFF
    c = (w >> 26).astype(np.float64)
    val = g[1][ax] * src[s1] + c * src[s2]
    val[0] = g[0]
    return val


def hermite_R(rprog, roff, L, G, PQ):
    """[tuv]^(0) of total order <= L from the seeds G[m] = [000]^(m) by the
    program words alone, in the layout (t, u, v) -> roff(L, t, u) + v."""
    PQ = np.asarray(PQ, dtype=np.float64)
    cur = np.array([G[L]])
    for nn in range(L - 1, -1, -1):
        cur = _level(rprog, roff, L - nn, cur, (G[nn], PQ))
    return cur


def simplex_offset(N, t, u):
    """Start of row (t, u) of a [t][u][v] simplex of total order N."""
    tet = lambda n: 0 if n < 0 else n * (n + 1) * (n + 2) // 6
    tri = lambda n: 0 if n < 0 else n * (n + 1) // 2
    return tet(N + 1) - tet(N - t + 1) + tri(N - t + 1) - tri(N - t - u + 1)


def _compute_R(pl: Plan, ws, count):
    s = pl.s
    L = s["L"]
    # the kernel's count: 8 per Boys order (Horner and the power of -2 rho),
    # one per R entry below the top of each level
    count["fma"] += 8 * (L + 1) + sum((L - nn + 1) * (L - nn + 2) * (L - nn + 3) // 6 - 1 for nn in range(L))
    rb = ws[s["o_recb"]:s["o_recb"] + REC_HEADER]
    rk = ws[s["o_reck"]:s["o_reck"] + REC_HEADER]
    PQ = rb[2:5] - rk[2:5]
    zp, zq = rb[0], rk[0]
    rho = zp * zq / (zp + zq)
    Tb = rho * float(PQ @ PQ)
    pref = TWO_PI_52 / (zp * zq * math.sqrt(zp + zq)) * rb[5] * rk[5]
    F = oracle.boys(L, Tb)
    G = np.array([(-2.0 * rho) ** m * pref * F[m] for m in range(L + 1)])
    ws[s["o_G"]:s["o_G"] + L + 1] = G
    o0, o1 = s["o_R0"], s["o_R1"]
    if L == 0:
        ws[o0] = G[0]
        return
    ws[o1 if L & 1 else o0] = G[L]
    # levels alternate between the R0 and R1 regions of the workspace, as in the kernel
    for nn in range(L - 1, -1, -1):
        N = L - nn
        dst, src = (o1, o0) if nn & 1 else (o0, o1)
        val = _level(pl.rprog, pl.roff, N, ws[src:], (G[nn], PQ))
        ws[dst:dst + len(val)] = val


def _fill_R_cache(pl: Plan, ws, bra_recs, ket_recs_signed, count, pbs=None):
    """cache_R == 2: the R table of every primitive quartet, computed once into the region o_Rc;
    cache_R == 3: those of the bra primitives `pbs` (one at a time), table pk."""
    s = pl.s
    nR = (s["L"] + 1) * (s["L"] + 2) * (s["L"] + 3) // 6
    pbs = range(s["Kb"]) if pbs is None else pbs
    ntab = s["Kb"] * s["Kk"] if s["cache_R"] == 2 else s["Kk"]
    assert s["rstride"] >= nR and s["o_Rc"] + ntab * s["rstride"] <= s["team_doubles"]
    for i, pb in enumerate(pbs):
        for pk in range(s["Kk"]):
            ws[s["o_recb"]:s["o_recb"] + s["recb"]] = bra_recs[pb][:s["recb"]]
            ws[s["o_reck"]:s["o_reck"] + s["reck"]] = ket_recs_signed[pk][:s["reck"]]
            _compute_R(pl, ws, count)
            o = s["o_Rc"] + (i * s["Kk"] + pk) * s["rstride"]
            ws[o:o + nR] = ws[s["o_R0"]:s["o_R0"] + nR]


def _load_cached_R(pl: Plan, ws, i, nR):
    s = pl.s
    o = s["o_Rc"] + i * s["rstride"]
    ws[s["o_R0"]:s["o_R0"] + nR] = ws[o:o + nR]


def emulate(pl: Plan, bra_recs, ket_recs_signed, count=None) -> np.ndarray:
    """Run one quartet through the plan's programs (store epilogue); returns
    the shellset [Nb][Nk] (row-major, bra Cartesian pair major). `count`, a
    dict, receives the FP64 FMAs the programs execute ("fma")."""
    if count is None:
        count = {}
    count.setdefault("fma", 0)
    s = pl.s
    Nb, Nk, hb, c1size = s["Nb"], s["Nk"], s["hb"], s["c1size"]
    assert len(bra_recs) == s["Kb"] and len(ket_recs_signed) == s["Kk"]
    ws = np.zeros(s["team_doubles"])
    out = np.full(Nb * Nk, np.nan)
    ob, ok = s["o_recb"], s["o_reck"]

    def load_bra(r):
        ws[ob:ob + s["recb"]] = r[:s["recb"]]

    def load_ket(r):
        ws[ok:ok + s["reck"]] = r[:s["reck"]]

    nR = (s["L"] + 1) * (s["L"] + 2) * (s["L"] + 3) // 6
    if s["cache_R"] == 1:
        load_bra(bra_recs[0])
        load_ket(ket_recs_signed[0])
        _compute_R(pl, ws, count)
    elif s["cache_R"] == 2:
        _fill_R_cache(pl, ws, bra_recs, ket_recs_signed, count)
    b1 = pl.b1
    b23 = pl.b23
    for g in pl.groups:
        ncols = int(g["ncols"])
        cols = np.arange(ncols)
        cm = pl.colmap[g["col_off"]:g["col_off"] + ncols].astype(np.int64)
        for pb in range(s["Kb"]):
            if s["cache_R"] != 1:
                load_bra(bra_recs[pb])
            for pk in range(s["Kk"]):
                if s["cache_R"] != 1:
                    load_ket(ket_recs_signed[pk])
                    if s["cache_R"] == 2:
                        _load_cached_R(pl, ws, pb * s["Kk"] + pk, nR)
                    else:
                        _compute_R(pl, ws, count)
                if g["k1_n"] > 0:
                    _run_step(ws, pl.kprog[g["k1_off"]:g["k1_off"] + g["k1_n"]], False, count)
                _run_step(ws, pl.kprog[g["k2_off"]:g["k2_off"] + g["k2_n"]], False, count)
                _run_step(ws, pl.kprog[g["k3_off"]:g["k3_off"] + g["k3_n"]], pk > 0, count)
            # b1: C1[col][out] = sum_k E[coef + k st] X[col][src + k st]
            count["fma"] += int(b1["n"].astype(np.int64).sum()) * ncols
            count["fma"] += int((b23["nv"].astype(np.int64) * (b23["nu"].astype(np.int64) + 1)).sum()) * ncols
            for e in b1:
                k = np.arange(int(e["n"])) * int(e["stride"])
                c = ws[int(e["coef"]) + k]
                x = ws[s["o_X"] + cols[:, None] * hb + int(e["src"]) + k[None, :]]
                ws[s["o_C1"] + cols * c1size + int(e["out"])] = x @ c
            # b23: OUT[out][col] (+)= sum_v Ez[v] sum_u Ey[u] C1[col][row(v) + u]
            to_global = pb == s["Kb"] - 1
            for e in b23:
                r1 = int(e["r"]) + 1
                iu = np.arange(int(e["nu"])) * int(e["su"])
                ey = ws[int(e["ey"]) + iu]
                acc = np.zeros(ncols)
                for iv in range(int(e["nv"])):
                    va = int(e["v0"]) + iv * int(e["sv"])
                    row = int(e["src"]) + int(e["u0"]) + va * r1 - va * (va - 1) // 2
                    c1 = ws[s["o_C1"] + cols[:, None] * c1size + row + iu[None, :]]
                    acc += ws[int(e["ez"]) + iv * int(e["sv"])] * (c1 @ ey)
                o = s["o_OUT"] + int(e["out"]) * ncols + cols
                if pb > 0:
                    acc = ws[o] + acc
                if to_global:
                    out[int(e["out"]) * Nk + cm] = acc
                else:
                    ws[o] = acc
    return out.reshape(Nb, Nk)


def emulate_sph(pl: Plan, bra_recs, ket_recs_signed, count=None) -> np.ndarray:
    """Run one quartet through a solid-harmonic plan (store = 2) the way k_quartets_sph does: the ket
    groups' Cartesian columns staged in a global area, the passes d -> d' and c -> c', the bra steps on
    groups of ncols_s spherical columns, the passes b -> b' (into the C1 slots) and a -> a'. Returns the
    shellset [2la+1][2lb+1][2lc+1][2ld+1] flattened to [Nb_sph][Nk_sph]. Every shared-memory access is
    checked against the team workspace."""
    if count is None:
        count = {}
    count.setdefault("fma", 0)
    s = pl.s
    assert s["sph"] == 1
    la, lb, lc, ld = s["la"], s["lb"], s["lc"], s["ld"]
    na, nb, nc, nd = [(l + 1) * (l + 2) // 2 for l in (la, lb, lc, ld)]
    nsa, nsb, nsc, nsd = s["nsa"], s["nsb"], s["nsc"], s["nsd"]
    Ca, Cb, Cc, Cd = solid_table(la), solid_table(lb), solid_table(lc), solid_table(ld)
    hb, hbp, c1s, ncs = s["hb"], s["hbp"], s["c1s"], s["ncols_s"]
    nks = nsc * nsd
    W = s["team_doubles"]
    ws = np.zeros(W)
    xg = np.full((s["Nk"], hbp), np.nan)
    out = np.zeros((nsa * nsb, nks))
    ob, ok = s["o_recb"], s["o_reck"]

    def span(lo, n):
        assert 0 <= lo and lo + n <= W, "workspace access out of range"
        return slice(lo, lo + n)

    nR = (s["L"] + 1) * (s["L"] + 2) * (s["L"] + 3) // 6
    if s["cache_R"] == 1:
        ws[span(ob, s["recb"])] = bra_recs[0][:s["recb"]]
        ws[span(ok, s["reck"])] = ket_recs_signed[0][:s["reck"]]
        _compute_R(pl, ws, count)
    elif s["cache_R"] == 2:
        span(s["o_Rc"], s["Kb"] * s["Kk"] * s["rstride"])
        _fill_R_cache(pl, ws, bra_recs, ket_recs_signed, count)
    for pb in range(s["Kb"]):
        if s["cache_R"] == 3:
            span(s["o_Rc"], s["Kk"] * s["rstride"])
            _fill_R_cache(pl, ws, bra_recs, ket_recs_signed, count, [pb])
        if s["cache_R"] != 1:
            ws[span(ob, s["recb"])] = bra_recs[pb][:s["recb"]]
        for g in pl.groups:
            ncols = int(g["ncols"])
            for pk in range(s["Kk"]):
                if s["cache_R"] != 1:
                    ws[span(ok, s["reck"])] = ket_recs_signed[pk][:s["reck"]]
                    if s["cache_R"] >= 2:
                        _load_cached_R(pl, ws, pb * s["Kk"] + pk if s["cache_R"] == 2 else pk, nR)
                    else:
                        _compute_R(pl, ws, count)
                if g["k1_n"] > 0:
                    _run_step(ws, pl.kprog[g["k1_off"]:g["k1_off"] + g["k1_n"]], False, count)
                _run_step(ws, pl.kprog[g["k2_off"]:g["k2_off"] + g["k2_n"]], False, count)
                _run_step(ws, pl.kprog[g["k3_off"]:g["k3_off"] + g["k3_n"]], pk > 0, count)
            cm = pl.colmap[g["col_off"]:g["col_off"] + ncols].astype(np.int64)
            for col in range(ncols):
                xg[cm[col]] = ws[span(s["o_X"] + col * hb, hbp)]
        assert not np.isnan(xg).any(), "a Cartesian ket column was never staged"
        Y = np.einsum("ed,cdp->cep", Cd, xg.reshape(nc, nd, hbp))          # pass d -> d'
        count["fma"] += hbp * (nc * int((Cd != 0).sum()) + int((Cc != 0).sum()) * nsd)
        for c0 in range(0, nks, ncs):
            ncols = min(ncs, nks - c0)
            cols = np.arange(ncols)
            for col in range(ncols):                                       # pass c -> c'
                cp, dp = divmod(c0 + col, nsd)
                ws[span(s["o_Xs"] + col * hb, hbp)] = Cc[cp] @ Y[:, dp, :]
            if s["top_only"]:
                # one-centre bra: OUT[m] = (2 zeta)^-la sum_a C_ma X[top(a)] (the lower Hermite terms of a
                # solid harmonic's Cartesian expansion cancel)
                L = la
                top = []
                for ax in range(L, -1, -1):
                    for ay in range(L - ax, -1, -1):
                        az = L - ax - ay
                        row = (L + 1) * (L + 2) * (L + 3) // 6 - (L - ay + 1) * (L - ay + 2) * (L - ay + 3) // 6 \
                            + (L - ay + 1) * (L - ay + 2) // 2 - (L - ay - az + 1) * (L - ay - az + 2) // 2
                        top.append(row + ax)
                f = (0.5 / ws[ob]) ** L
                Xt = np.stack([ws[span(s["o_Xs"] + col * hb, hbp)][top] for col in range(ncols)], -1)
                out[:, c0:c0 + ncols] += f * (Ca @ Xt)
                count["fma"] += ncols * int((Ca != 0).sum())
                continue
            count["fma"] += int(pl.b1["n"].astype(np.int64).sum()) * ncols
            count["fma"] += int((pl.b23["nv"].astype(np.int64) * (pl.b23["nu"].astype(np.int64) + 1)).sum()) * ncols
            for e in pl.b1:                                                # b1 into the C1 slots
                k = np.arange(int(e["n"])) * int(e["stride"])
                c = ws[int(e["coef"]) + k]
                assert int(e["out"]) < c1s and s["o_Xs"] + (ncols - 1) * hb + int(e["src"]) + k[-1] < W
                x = ws[s["o_Xs"] + cols[:, None] * hb + int(e["src"]) + k[None, :]]
                ws[s["o_C1s"] + cols * c1s + int(e["out"])] = x @ c
            OUT = np.zeros((s["Nb"], ncols))
            for e in pl.b23:                                               # b23, fresh per bra primitive
                r1 = int(e["r"]) + 1
                iu = np.arange(int(e["nu"])) * int(e["su"])
                ey = ws[int(e["ey"]) + iu]
                acc = np.zeros(ncols)
                for iv in range(int(e["nv"])):
                    va = int(e["v0"]) + iv * int(e["sv"])
                    row = int(e["src"]) + int(e["u0"]) + va * r1 - va * (va - 1) // 2
                    c1 = ws[s["o_C1s"] + cols[:, None] * c1s + row + iu[None, :]]
                    acc += ws[int(e["ez"]) + iv * int(e["sv"])] * (c1 @ ey)
                OUT[int(e["out"])] = acc
            ws[span(s["o_OUTs"], s["Nb"] * ncols)] = OUT.reshape(-1)
            T1 = np.einsum("eb,abk->aek", Cb, OUT.reshape(na, nb, ncols))   # pass b -> b'
            assert na * nsb <= c1s
            for col in range(ncols):
                ws[span(s["o_C1s"] + col * c1s, na * nsb)] = T1[:, :, col].reshape(-1)
            T1 = np.stack([ws[span(s["o_C1s"] + col * c1s, na * nsb)].reshape(na, nsb) for col in range(ncols)], -1)
            out[:, c0:c0 + ncols] += np.einsum("fa,aek->fek", Ca, T1).reshape(nsa * nsb, ncols)   # pass a -> a'
            count["fma"] += ncols * (na * int((Cb != 0).sum()) + int((Ca != 0).sum()) * nsb)
    return out


# ----------------------------------------------------------------- lane efficiency
def lane_efficiency(pl: Plan):
    """Share of FP64 lane slots that do useful work when a team runs the plan's
    ket steps and its b23 step, under the kernel's lane assignment: in a ket
    step lane tl runs entries tl and tl + T side by side (2 chains), then moves
    on by 2T; in b23 lane tl runs (entry, column) items tl, tl + T, ... with
    the column fastest. A warp instruction costs as many slots as the longest
    chain of its 32 lanes needs. Returns (ket, b23) as fractions."""
    T = pl.s["T"]
    width = min(T, 32)

    def warp_share(work_per_lane_round):
        W = work_per_lane_round.reshape(work_per_lane_round.shape[0], -1, width)
        used = W.sum()
        slots = (W.max(axis=2) * width).sum()
        return used, slots

    ku = ks = bu = bs = 0
    w23 = pl.b23["nv"].astype(np.int64) * (pl.b23["nu"].astype(np.int64) + 1)
    for g in pl.groups:
        for off, n in ((g["k1_off"], g["k1_n"]), (g["k2_off"], g["k2_n"]), (g["k3_off"], g["k3_n"])):
            if n == 0:
                continue
            nn = pl.kprog["n"][off:off + n].astype(np.int64)
            rounds = (n + 2 * T - 1) // (2 * T)
            pad = np.zeros(rounds * 2 * T, dtype=np.int64)
            pad[:n] = nn
            u, s_ = warp_share(pad.reshape(rounds, 2, T).sum(axis=1))
            ku += u
            ks += s_
        ncols = int(g["ncols"])
        n = len(pl.b23) * ncols
        rounds = (n + T - 1) // T
        pad = np.zeros(rounds * T, dtype=np.int64)
        pad[:n] = w23[np.arange(n) // ncols]
        u, s_ = warp_share(pad.reshape(rounds, T))
        bu += u
        bs += s_
    return ku / ks, bu / bs
