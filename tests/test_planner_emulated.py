"""Host logic on the CPU: the planner's step programs, run in an emulator of the
team kernel (tests/team_emulator.py), reproduce the oracle's shellsets.

The team kernel executes whatever programs the host planner emits for a class
(R levels, ket steps k1/k2/k3, bra steps b1/b23, column map) with fixed
per-entry semantics. Running those programs here checks, without a GPU, that
for every class shape the planner produces (one group or many, z-pair groups
sharing one k1 output, contracted classes, one-centre bras, store-only plans)
the programs compute [ab|cd] of Eqs. ket-from-hermite and bra-from-hermite and
that no entry of a step depends on another entry of the same step.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import parity
import team_emulator as te
from paper_2405_01834_gb300 import inputs


def _basis_4c(lq, K, seed, n=2):
    """n x n quartets of class lq: random bra and ket pairs in a 1.5-bohr box
    (overlapping shells, so integrals are O(1)), exponents log-uniform [0.2, 4]."""
    b, q = inputs.class_sweep(lq, n_bra=n, n_ket=n, seed=seed, box=1.5, zlo=0.2, zhi=4.0, K=K)
    return b, q


def _emulate_4c(pl, b, q):
    out = []
    for a, bb, c, d in q:
        br = te.shell_pair_records(b, a, bb, signed=False)
        kr = te.shell_pair_records(b, c, d, signed=True)
        out.append(te.emulate(pl, br, kr).reshape(-1))
    return np.concatenate(out)


def _check_4c(lq, K=(1, 1, 1, 1), seed=11, n=2, **shape):
    b, q = _basis_4c(lq, K, seed, n)
    pl = te.plan(*lq, K[0] * K[1], K[2] * K[3], **shape)
    te.check_hazards(pl)
    got = _emulate_4c(pl, b, q)
    ref, off = oracle.eri4(b, q)
    assert np.max(np.abs(ref)) > 1e-3   # the inputs give integrals of a meaningful size
    parity.check(got, ref, off, what="emulated %s K=%s %s" % (lq, K, shape), evaluate=parity.Eri4Evaluator(b, q))
    return pl


def test_rlevel_programs_reproduce_hermite_integrals():
    """The R-level program words (Eq. r), run alone, give the oracle's
    [tuv]^(0) for every total order the engine uses (L <= 25: l = 6 gradients)."""
    rprog, roff = te.rlevel_programs()
    rng = np.random.default_rng(3)
    for L in list(range(0, 26)):
        rho = float(rng.uniform(0.3, 2.0))
        PQ = rng.uniform(-1.0, 1.0, 3)
        T = rho * float(PQ @ PQ)
        F = oracle.boys(L, T)
        G = np.array([(-2.0 * rho) ** m * F[m] for m in range(L + 1)])
        R = te.hermite_R(rprog, roff, L, G, PQ)
        ref = oracle.rtable(L, rho, PQ)
        scale = np.max(np.abs(ref))
        for t in range(L + 1):
            for u in range(L + 1 - t):
                o = te.simplex_offset(L, t, u)
                got = R[o:o + L + 1 - t - u]
                np.testing.assert_allclose(got, ref[t, u, :L + 1 - t - u], rtol=0, atol=1e-12 * scale,
                                           err_msg="L=%d t=%d u=%d" % (L, t, u))


@pytest.mark.parametrize("lq", [q for q in itertools.product(range(3), repeat=4)])
def test_uncontracted_low_l(lq):
    """Every class with all l <= 2, one primitive per shell."""
    _check_4c(lq, seed=100 + sum(x * 3 ** i for i, x in enumerate(lq)))


@pytest.mark.parametrize("lq", [(3, 3, 3, 3), (4, 3, 2, 1), (1, 2, 3, 4), (0, 4, 4, 0), (4, 4, 4, 4),
                                (5, 4, 3, 2), (6, 6, 1, 0), (6, 6, 6, 6)])
def test_uncontracted_high_l(lq):
    """Higher l, including [gg|gg] and [ii|ii] (workspace split into many column groups)."""
    pl = _check_4c(lq, seed=7, n=1 if sum(lq) >= 20 else 2)
    if sum(lq) >= 16:
        assert pl.s["ngroups"] > 1


@pytest.mark.parametrize("lq,K", [((0, 0, 0, 0), (6, 6, 6, 6)), ((1, 0, 1, 0), (3, 6, 3, 6)),
                                  ((1, 1, 1, 1), (3, 2, 2, 1)), ((2, 1, 0, 0), (1, 3, 6, 6)),
                                  ((2, 2, 2, 2), (2, 2, 1, 2)), ((3, 1, 2, 0), (1, 3, 2, 6)),
                                  ((3, 3, 2, 2), (2, 1, 1, 2)), ((0, 0, 0, 0), (32, 32, 1, 2)),
                                  ((1, 1, 0, 0), (32, 4, 2, 2))])
def test_contracted(lq, K):
    """Contracted shells: primitive loops over bra and ket pairs, R per primitive
    quartet; up to the largest contraction degree the engine accepts (32)."""
    pl = _check_4c(lq, K=K, seed=21)
    assert pl.s["cache_R"] in (0, 2)


@pytest.mark.parametrize("lq,K,store", [((1, 1, 1, 1), (1, 1, 1, 1), True), ((2, 2, 2, 2), (1, 1, 1, 1), True),
                                        ((3, 2, 3, 2), (1, 1, 1, 1), True), ((2, 1, 2, 1), (1, 1, 2, 3), True),
                                        ((2, 1, 2, 1), (2, 1, 1, 1), True)])
def test_store_only_plans(lq, K, store):
    """Store plans: no OUT region when the bra has one primitive pair (b23 writes the shellset)."""
    pl = _check_4c(lq, K=K, seed=31, store=store)
    assert pl.s["has_out"] == (0 if K[0] * K[1] == 1 else 1)


@pytest.mark.parametrize("lq,K,single_max,budget", [((2, 2, 2, 2), (1, 1, 1, 1), 4000, 0),
                                                    ((2, 2, 2, 2), (1, 1, 1, 1), 4000, 8 * 1024),
                                                    ((3, 2, 2, 2), (1, 1, 1, 1), 4000, 12 * 1024),
                                                    ((2, 2, 2, 1), (2, 1, 2, 1), 4000, 8 * 1024),
                                                    ((3, 3, 3, 3), (1, 1, 1, 1), 4000, 24 * 1024)])
def test_forced_column_groups(lq, K, single_max, budget):
    """Small workspace caps force one group per ket z-pair (split into chunks);
    uncontracted classes share one k1 output between the groups of a z-pair."""
    pl = _check_4c(lq, K=K, seed=41, single_max=single_max, budget=budget)
    assert pl.s["ngroups"] > 1
    if K == (1, 1, 1, 1) and budget:
        assert np.any(pl.groups["k1_n"] == 0)   # some group reuses its z-pair's A
    if K != (1, 1, 1, 1):
        assert np.all(pl.groups["k1_n"] > 0)    # contracted: every group recomputes A


def _basis_3c(la, lc, ld, Ka, Kc, Kd, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    aux, orb = inputs.BasisBuilder(), inputs.BasisBuilder()
    for _ in range(2):
        inputs.random_shell(rng, aux, la, rng.uniform(0, 1.5, 3), Ka, 0.2, 4.0)
        inputs.random_shell(rng, orb, lc, rng.uniform(0, 1.5, 3), Kc, 0.2, 4.0)
        inputs.random_shell(rng, orb, ld, rng.uniform(0, 1.5, 3), Kd, 0.2, 4.0)
    trip = np.array([[a, 2 * k, 2 * k + 1] for a in range(2) for k in range(2)], dtype=np.int32)
    return aux.build(), orb.build(), trip


@pytest.mark.parametrize("store", [False, True])
@pytest.mark.parametrize("la,lc,ld,K", [(0, 0, 0, (1, 1, 1)), (1, 1, 0, (1, 3, 1)), (2, 1, 1, (1, 1, 1)),
                                        (3, 2, 1, (1, 1, 1)), (4, 0, 0, (1, 6, 6)), (5, 1, 0, (1, 3, 6)),
                                        (6, 2, 2, (1, 1, 1)), (6, 3, 3, (1, 1, 1)), (2, 2, 0, (2, 1, 1))])
def test_three_center(la, lc, ld, K, store):
    """[a|cd] with a one-centre bra (Eq. E1rr; the bra steps skip the zero
    parity terms with stride-2 entries), with and without the OUT region."""
    aux, orb, trip = _basis_3c(la, lc, ld, *K, seed=51 + la)
    pl = te.plan(la, 0, lc, ld, K[0], K[1] * K[2], onec=True, store=store)
    te.check_hazards(pl)
    got = []
    for a, c, d in trip:
        br = te.shell_pair_records(aux, a, None, signed=False)
        kr = te.shell_pair_records(orb, c, d, signed=True)
        got.append(te.emulate(pl, br, kr).reshape(-1))
    got = np.concatenate(got)
    ref, off = oracle.eri3(aux, orb, trip)
    assert np.max(np.abs(ref)) > 1e-3
    parity.check(got, ref, off, what="emulated [%d|%d%d]" % (la, lc, ld), evaluate=parity.Eri3Evaluator(aux, orb, trip))


def test_emulator_detects_a_corrupted_program():
    """The comparison is sensitive: one ket-step entry pointed at the wrong E
    coefficient, or one bra entry with a shortened sum, makes the result differ."""
    lq = (2, 1, 2, 1)
    b, q = _basis_4c(lq, (1, 1, 1, 1), 61)
    ref, off = oracle.eri4(b, q)
    pl = te.plan(*lq)
    g = pl.groups[0]
    k3 = pl.kprog[g["k3_off"]:g["k3_off"] + g["k3_n"]]
    i = int(np.argmax(k3["n"]))
    bad = pl.kprog.copy()
    bad[g["k3_off"] + i]["coef"] += 1
    pl_bad = te.Plan(pl.s, pl.groups, bad, pl.b1, pl.b23, pl.colmap, pl.rprog, pl.roff)
    with pytest.raises(AssertionError):
        parity.check(_emulate_4c(pl_bad, b, q), ref, off, what="corrupted k3", evaluate=parity.Eri4Evaluator(b, q))
    b23 = pl.b23.copy()
    j = int(np.argmax(b23["nu"]))
    b23[j]["nu"] -= 1
    pl_bad = te.Plan(pl.s, pl.groups, pl.kprog, pl.b1, b23, pl.colmap, pl.rprog, pl.roff)
    with pytest.raises(AssertionError):
        parity.check(_emulate_4c(pl_bad, b, q), ref, off, what="corrupted b23", evaluate=parity.Eri4Evaluator(b, q))
    parity.check(_emulate_4c(pl, b, q), ref, off, what="intact", evaluate=parity.Eri4Evaluator(b, q))


def test_boys_table_interpolation():
    """The library's Boys table, evaluated the way the kernel does (nearest grid
    point, 8-term Taylor series by Horner's rule), against the oracle's
    long-double F_m for every order the engine uses (m <= 25) across the
    tabulated range T < 100."""
    tab, inv_h = te.boys_table()
    assert tab.shape[1] >= 26
    rng = np.random.default_rng(5)
    Ts = np.concatenate([[0.0, 1e-12, 0.03125, 1.0 / 32 - 1e-13, 99.96875, 99.99999],
                         rng.uniform(0.0, 100.0, 300), rng.uniform(0.0, 2.0, 100)])
    worst = 0.0
    for T in Ts:
        ref = oracle.boys(25, float(T), precision=1)
        for m in range(26):
            got = te.boys_interpolate(tab, inv_h, m, float(T))
            worst = max(worst, abs(got - ref[m]) / ref[m])
    # Taylor truncation <= (1/32)^8/8! relative; the rest is FP64 rounding of the Horner steps
    assert worst <= 4e-16, worst


@pytest.mark.parametrize("l", range(7))
def test_solid_harmonic_tables(l):
    """The library's solid-harmonic coefficients (built by recurrences in l)
    equal the oracle's explicit closed form."""
    np.testing.assert_allclose(te.solid_table(l), oracle.solid_coefs(l), rtol=0, atol=1e-13)


@pytest.mark.parametrize("lq,K,shape", [((1, 1, 1, 1), (1, 1, 1, 1), {}), ((2, 2, 2, 2), (1, 1, 1, 1), {}),
                                        ((3, 3, 3, 3), (1, 1, 1, 1), {}), ((4, 4, 4, 4), (1, 1, 1, 1), {}),
                                        ((2, 1, 2, 1), (2, 3, 1, 2), {}),
                                        ((2, 2, 2, 1), (2, 1, 2, 1), {"single_max": 4000, "budget": 8 * 1024}),
                                        ((3, 2, 2, 2), (1, 1, 1, 1), {"single_max": 4000, "budget": 12 * 1024})])
def test_planner_fma_count_matches_programs(lq, K, shape):
    """The FP64 FMA count per shellset the planner reports (the numerator of
    the benchmark's executed-FLOP rates) equals the FMAs its programs execute
    when run: Boys and R per primitive quartet (per group when R is not
    cached), the ket steps per primitive quartet and the bra steps per bra
    primitive pair and column."""
    b, q = _basis_4c(lq, K, 71, n=1)
    pl = te.plan(*lq, K[0] * K[1], K[2] * K[3], **shape)
    count = {}
    a, bb, c, d = q[0]
    te.emulate(pl, te.shell_pair_records(b, a, bb, False), te.shell_pair_records(b, c, d, True), count)
    assert count["fma"] == pl.exec_fma, (count["fma"], pl.exec_fma)


def test_random_shapes():
    """Seeded random classes (l <= 3), contraction degrees, shared-memory budgets,
    single-group caps and store flags: the shapes the autotuner may ask for.
    Every plan the planner accepts computes the oracle's shellset."""
    rng = np.random.default_rng(2024)
    done = 0
    while done < 60:
        lq = tuple(int(x) for x in rng.integers(0, 4, 4))
        K = tuple(int(rng.choice([1, 1, 1, 2, 3])) for _ in range(4))
        budget = int(rng.choice([0, 8, 12, 16, 24, 32, 64, 128, 200])) * 1024
        single_max = int(rng.choice([0, 2000, 4000, 16000, 48000]))
        store = bool(rng.integers(0, 2))
        try:
            pl = te.plan(*lq, K[0] * K[1], K[2] * K[3], store=store, budget=budget, single_max=single_max)
        except te.PlanError:
            continue   # a budget too small for the class: the planner refuses, which is its contract
        te.check_hazards(pl)
        b, q = _basis_4c(lq, K, int(rng.integers(0, 10 ** 6)), n=1)
        got = _emulate_4c(pl, b, q)
        ref, off = oracle.eri4(b, q)
        parity.check(got, ref, off, what="random shape %s K=%s b=%d s=%d store=%d" % (lq, K, budget, single_max, store),
                     evaluate=parity.Eri4Evaluator(b, q))
        done += 1


@pytest.mark.parametrize("lq,k_min,b23_min", [((3, 3, 3, 3), 0.95, 0.85), ((4, 4, 4, 4), 0.97, 0.90),
                                              ((5, 5, 5, 5), 0.98, 0.90), ((6, 6, 6, 6), 0.98, 0.90)])
def test_planner_lane_efficiency(lq, k_min, b23_min):
    """Regression guard on the plans' shape: the share of FP64 lane slots doing
    useful work in the ket steps and in b23 (sorted entries, columns fastest),
    for the uncontracted [ll|ll] classes the benchmark times."""
    k, b23 = te.lane_efficiency(te.plan(*lq, store=True))
    assert k >= k_min and b23 >= b23_min, (k, b23)


def test_boys_asymptotic_form_above_the_table():
    """Above the table (T >= 100) the kernel uses F_m(T) = c_m T^-(m+1/2) with
    c_0 = sqrt(pi)/2 and c_(m+1) = c_m (2m+1)/2, dropping the exp(-T) terms;
    against the oracle's long-double F_m the dropped part is below 1e-17
    relative for m <= 25, so only rounding remains."""
    c = [math.sqrt(math.pi) / 2.0]
    for m in range(25):
        c.append(c[-1] * (2 * m + 1) / 2.0)
    worst = 0.0
    for T in (100.0, 100.5, 137.25, 400.0, 1e3, 1e4):
        ref = oracle.boys(25, T, precision=1)
        for m in range(26):
            got = c[m] * T ** (-(m + 0.5))
            worst = max(worst, abs(got - ref[m]) / ref[m])
    assert worst <= 2e-15, worst


def _emulate_sph(pl, b, q):
    out = []
    for a, bb, c, d in q:
        br = te.shell_pair_records(b, a, bb, signed=False)
        kr = te.shell_pair_records(b, c, d, signed=True)
        out.append(te.emulate_sph(pl, br, kr).reshape(-1))
    return np.concatenate(out)


@pytest.mark.parametrize("lq,K,budget", [((2, 1, 2, 1), (1, 1, 1, 1), 0), ((3, 3, 3, 3), (1, 1, 1, 1), 0),
                                         ((2, 2, 3, 1), (2, 1, 1, 3), 0), ((4, 2, 3, 3), (1, 1, 1, 1), 48),
                                         ((6, 6, 1, 0), (1, 1, 1, 1), 0), ((0, 0, 5, 4), (1, 1, 1, 1), 0),
                                         ((4, 4, 4, 4), (1, 1, 1, 1), 0), ((1, 3, 2, 2), (2, 2, 1, 1), 24)])
def test_solid_harmonic_plans(lq, K, budget):
    """Solid-harmonic store plans (Cartesian ket groups staged, ket passes d -> d' and c -> c', bra steps
    on spherical columns, bra passes b -> b' and a -> a') reproduce the oracle's solid-harmonic shellsets,
    including plans squeezed into small shared-memory budgets (many ket and bra-pass groups) and
    contracted bras (summed over bra primitives in the output)."""
    b, q = _basis_4c(lq, K, 71)
    pl = te.plan(*lq, K[0] * K[1], K[2] * K[3], store=2, budget=budget * 1024)
    assert pl.s["sph"] == 1
    te.check_hazards(pl)
    cnt = {}
    got = _emulate_sph(pl, b, q)
    ref, off = oracle.eri4_sph(b, q)
    assert np.max(np.abs(ref)) > 1e-4
    parity.check(got, ref, off, what="emulated sph %s K=%s" % (lq, K), evaluate=parity.Eri4SphEvaluator(b, q))
    te.emulate_sph(pl, te.shell_pair_records(b, *q[0][:2], signed=False),
                   te.shell_pair_records(b, *q[0][2:], signed=True), cnt)
    assert cnt["fma"] == pytest.approx(pl.exec_fma, rel=1e-9)


def test_solid_harmonic_plan_executes_fewer_operations():
    """At [ii|ii] the solid-harmonic plan executes well under half the FP64 multiply-adds of the
    Cartesian plan followed by the index-by-index transform."""
    cart = te.plan(6, 6, 6, 6, store=True).exec_fma
    sph = te.plan(6, 6, 6, 6, store=2).exec_fma
    ncs = 28 * 28
    transform = ncs * (28 * 70 + 70 * 13) + 169 * (28 * 70 + 70 * 13)   # k_cart2sph, zeros skipped
    assert sph < 0.5 * (cart + transform)


@pytest.mark.parametrize("lq,K,store,shape", [((2, 2, 2, 1), (2, 1, 2, 1), True, {"single_max": 4000, "budget": 24 * 1024}),
                                              ((3, 2, 2, 2), (1, 1, 2, 3), True, {"single_max": 4000}),
                                              ((2, 1, 2, 2), (2, 2, 1, 1), False, {"single_max": 3000}),
                                              ((3, 3, 3, 3), (1, 1, 1, 3), 2, {}),
                                              ((2, 2, 3, 1), (2, 1, 1, 3), 2, {"budget": 24 * 1024}),
                                              ((3, 3, 3, 2), (2, 2, 1, 2), 2, {"budget": 48 * 1024})])
def test_cached_R_tables(lq, K, store, shape):
    """Contracted classes of several column groups keep the R table of every primitive quartet in a
    region of their own (computed once, copied into R0 before each group's k1) instead of computing it
    once per group: both plans give the oracle's shellsets, and the cached plan executes fewer FP64
    operations, exactly as many as the planner reports."""
    b, q = _basis_4c(lq, K, 81)
    emul, ref_fn, ev = ((_emulate_sph, oracle.eri4_sph, parity.Eri4SphEvaluator) if store == 2 else
                        (_emulate_4c, oracle.eri4, parity.Eri4Evaluator))
    ref, off = ref_fn(b, q)
    fma = {}
    for rc in (0, 1):
        pl = te.plan(*lq, K[0] * K[1], K[2] * K[3], store=store, rcache=rc, **shape)
        assert pl.s["ngroups"] > 1
        assert pl.s["cache_R"] in ((2, 3) if rc else (0,))
        te.check_hazards(pl)
        parity.check(emul(pl, b, q), ref, off, what="cached R %d %s K=%s" % (rc, lq, K), evaluate=ev(b, q))
        cnt = {}
        recs = (te.shell_pair_records(b, *q[0][:2], signed=False), te.shell_pair_records(b, *q[0][2:], signed=True))
        (te.emulate_sph if store == 2 else te.emulate)(pl, *recs, cnt)
        assert cnt["fma"] == pytest.approx(pl.exec_fma, rel=1e-12)
        fma[rc] = pl.exec_fma
    assert fma[1] < fma[0]


@pytest.mark.parametrize("lq,K,store", [((3, 3, 3, 3), (1, 1, 1, 1), True), ((3, 2, 3, 2), (1, 1, 1, 1), True),
                                        ((3, 3, 2, 2), (1, 2, 1, 1), False), ((3, 3, 3, 2), (1, 1, 1, 1), 2)])
def test_packed_zpair_groups(lq, K, store):
    """Small ket z-pairs packed whole into shared column groups (each group computes the A blocks of all
    its z-pairs) give the oracle's shellsets, like one group per z-pair, with fewer groups and no more FP64
    operations (R per group, where it is not cached, runs fewer times)."""
    b, q = _basis_4c(lq, K, 91)
    emul, ref_fn, ev = ((_emulate_sph, oracle.eri4_sph, parity.Eri4SphEvaluator) if store == 2 else
                        (_emulate_4c, oracle.eri4, parity.Eri4Evaluator))
    ref, off = ref_fn(b, q)
    pls = {pk: te.plan(*lq, K[0] * K[1], K[2] * K[3], store=store, pack=pk, single_max=4000) for pk in (0, 1)}
    for pk, pl in pls.items():
        te.check_hazards(pl)
        parity.check(emul(pl, b, q), ref, off, what="packed %d %s K=%s" % (pk, lq, K), evaluate=ev(b, q))
    assert pls[1].s["ngroups"] < pls[0].s["ngroups"]
    assert pls[1].exec_fma <= pls[0].exec_fma * (1 + 1e-12)


def test_team_shape_rules():
    """The planner's team shapes: teams of up to 32 lanes fill whole warps of a CTA; single-group classes with
    a high total angular momentum and few Cartesian components ([l0|l0]) take at least half as many lanes as
    the largest R level has entries; solid-harmonic plans of several groups that hold one team per SM take
    1024 lanes."""
    for lq in [(2, 0, 2, 0), (3, 0, 3, 0), (1, 1, 1, 1), (2, 1, 2, 0), (0, 0, 3, 3)]:
        for store in (True, 2):
            s = te.plan(*lq, store=store).s
            if s["T"] < 32:
                assert (s["T"] * s["teams_per_cta"]) % 32 == 0, (lq, store, s["T"], s["teams_per_cta"])
    for lq, tmin in [((4, 0, 4, 0), 64), ((5, 0, 5, 0), 128), ((6, 0, 6, 0), 128)]:
        for store in (True, 2):
            s = te.plan(*lq, store=store).s
            assert s["ngroups"] == 1 and s["T"] >= tmin, (lq, store, s["T"])
    for lq in [(4, 4, 4, 4), (5, 5, 5, 5), (6, 6, 6, 6)]:
        assert te.plan(*lq, store=2).s["T"] == 1024
        assert te.plan(*lq, store=True).s["T"] == 512


@pytest.mark.parametrize("lq,K", [((5, 5, 5, 5), (1, 5)), ((6, 6, 6, 6), (1, 5)), ((5, 5, 5, 5), (5, 5))])
def test_cached_R_fallback_budget(lq, K):
    """Contracted solid-harmonic classes whose R tables do not fit next to a full-budget workspace get the
    plan with a smaller budget and the tables cached by default: R once per primitive quartet, fewer FP64
    operations than the uncached plan."""
    dflt = te.plan(*lq, Kb=K[0], Kk=K[1], store=2)
    plain = te.plan(*lq, Kb=K[0], Kk=K[1], store=2, rcache=0)
    assert dflt.s["cache_R"] >= 2 and plain.s["cache_R"] == 0
    assert dflt.exec_fma < plain.exec_fma


@pytest.mark.parametrize("la,lc,ld,K", [(3, 2, 1, (1, 3, 1)), (6, 0, 0, (1, 6, 6)), (4, 3, 3, (1, 1, 1)),
                                        (5, 2, 2, (2, 1, 1)), (2, 4, 4, (1, 1, 1))])
def test_three_center_solid_harmonic_plans(la, lc, ld, K):
    """Solid-harmonic plans of 3-center classes reproduce the oracle's solid-harmonic [a|cd], including several
    column groups and contracted kets. The one-centre bra over solid harmonics needs only the top Hermite
    shell (the lower terms of a solid harmonic's Cartesian expansion cancel): the k3 step forms those rows
    alone and the bra step is one sparse sum per component, fewer operations than the Cartesian plan."""
    aux, orb, trip = _basis_3c(la, lc, ld, *K, seed=61 + la)
    pl = te.plan(la, 0, lc, ld, K[0], K[1] * K[2], onec=True, store=2)
    assert pl.s["sph"] == 1
    te.check_hazards(pl)
    got = []
    for a, c, d in trip:
        br = te.shell_pair_records(aux, a, None, signed=False)
        kr = te.shell_pair_records(orb, c, d, signed=True)
        got.append(te.emulate_sph(pl, br, kr).reshape(-1))
    got = np.concatenate(got)
    ref, off = oracle.eri3_sph(aux, orb, trip)
    assert np.max(np.abs(ref)) > 1e-4
    parity.check(got, ref, off, what="emulated sph [%d|%d%d]" % (la, lc, ld),
                 evaluate=parity.Eri3SphEvaluator(aux, orb, trip))
    # only the top Hermite shell of the bra is formed, and the planner counts what the programs execute
    assert pl.s["top_only"] == 1
    cnt = {}
    te.emulate_sph(pl, te.shell_pair_records(aux, trip[0][0], None, signed=False),
                   te.shell_pair_records(orb, trip[0][1], trip[0][2], signed=True), cnt)
    assert cnt["fma"] == pytest.approx(pl.exec_fma, rel=1e-9)
    assert pl.exec_fma < te.plan(la, 0, lc, ld, K[0], K[1] * K[2], onec=True, store=True).exec_fma
