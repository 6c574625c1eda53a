"""Tolerance rule of the parity comparisons (test infrastructure, like the rest of oracle/).

The bar for every integral the engine computes, against the FP64 oracle on the same inputs:
  * abs: max |engine - oracle| <= 1e-12 * max |oracle|, over the whole batch compared and over
    every shellset whose largest integral is above 1e-10 (the floor of the relative bound; a
    shellset below it, e.g. one that vanishes by symmetry, has a rounding remnant for its largest
    value, which sets no scale);
  * rel: every integral with |oracle| > 1e-10 has |engine - oracle| <= 1e-10 |oracle|.

A value that misses a bound against the FP64 oracle is judged again against the oracle's
long-double build: a miss that the FP64 oracle's own rounding causes is no miss.

Exception (cancellation). An integral many orders of magnitude below the terms the method adds
to form it cannot be resolved to 1e-10 relative by any FP64 evaluation: its rounding error is set
by the size of those terms, not by its own size. A miss against the long-double value is excused
only if the engine's error stays within WITHIN times the FP64 oracle's own rounding error on that
same integral, measured against the long-double build. The oracle's error is taken as an
envelope: the largest of its errors on the given input and on ENVELOPE_RUNS copies of the input
moved by one or two units in the last place (equal input values move together, so shells that
share a centre or an exponent keep sharing it). A single FP64 evaluation is one draw of rounding
noise, and on cancellation-limited integrals that noise is dominated by a few discrete roundings
(measured: one [ff|ff] integral of 1.2e-10 came out -4e-21 off in most draws and +2.5e-20 in a
sixth of them), so one draw can sit far below the typical size; the envelope measures the size.
The same exception applies to the absolute bounds (a shellset or a batch whose largest integral
is itself a cancellation remnant). Nothing else is widened. The count of excused integrals,
shellsets and batches is returned (`n_cancel`, with the worst cases) and must stay at or below
MAX_CANCEL_PER_ELEMENT of the integrals compared (at least MIN_CANCEL_ALLOWED), or at or below
twice the number of misses the FP64 oracle itself makes on the same batch against its long-double
build (plus MIN_CANCEL_ALLOWED): some batches are full of cancellation-limited values
(solid-harmonic combinations of distant, diffuse shells cancel the dominant Cartesian terms by
factors up to 1e7), and there the oracle's own count is the yardstick.
"""
from __future__ import annotations

import copy

import numpy as np

ABS = 1e-12
REL = 1e-10
FLOOR = 1e-10
WITHIN = 10.0
ENVELOPE_RUNS = 6
MAX_CANCEL_PER_ELEMENT = 1e-5
MIN_CANCEL_ALLOWED = 4
_ULP1 = 2.0 ** -52   # spacing of doubles just above 1


def _moves(a, seed):
    """-2..2 per value, a function of the value's bits and the seed (equal values move alike)."""
    bits = np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)
    h = (bits ^ np.uint64((0x9E3779B97F4A7C15 * (seed + 1)) & 0xFFFFFFFFFFFFFFFF)) * np.uint64(0xBF58476D1CE4E5B9)
    h ^= h >> np.uint64(31)
    return (h % np.uint64(5)).astype(np.float64) - 2.0


def _perturbed(basis, seed):
    """Copy of `basis` whose centres, exponents and coefficients are moved by -2..2 ulp."""
    b = copy.copy(basis)
    for name in ("center", "exps", "coefs"):
        a = np.asarray(getattr(basis, name), dtype=np.float64)
        with np.errstate(over="ignore"):
            r = _moves(a, seed)
        setattr(b, name, a * (1.0 + r * _ULP1))
    return b


class Eri4Evaluator:
    """Oracle [ab|cd] of a subset of the quartets, optionally on a perturbed basis."""

    def __init__(self, basis, quartets):
        import oracle
        self.oracle, self.basis = oracle, basis
        self.q = np.asarray(quartets, dtype=np.int32).reshape(-1, 4)

    def __call__(self, sel, precision, seed=None):
        b = self.basis if seed is None else _perturbed(self.basis, seed)
        return self.oracle.eri4(b, self.q[sel], precision=precision)[0]


class Eri4SphEvaluator(Eri4Evaluator):
    """Oracle solid-harmonic [ab|cd] of a subset of the quartets, optionally on a perturbed basis."""

    def __call__(self, sel, precision, seed=None):
        b = self.basis if seed is None else _perturbed(self.basis, seed)
        return self.oracle.eri4_sph(b, self.q[sel], precision=precision)[0]


class Eri3Evaluator:
    """Oracle [a|cd] of a subset of the triplets, optionally on perturbed bases."""

    def __init__(self, aux, orb, triplets):
        import oracle
        self.oracle, self.aux, self.orb = oracle, aux, orb
        self.t = np.asarray(triplets, dtype=np.int32).reshape(-1, 3)

    def __call__(self, sel, precision, seed=None):
        a = self.aux if seed is None else _perturbed(self.aux, seed)
        o = self.orb if seed is None else _perturbed(self.orb, 1000 + seed)
        return self.oracle.eri3(a, o, self.t[sel], precision=precision)[0]


class Eri3SphEvaluator(Eri3Evaluator):
    """Oracle solid-harmonic [a|cd] of a subset of the triplets, optionally on perturbed bases."""

    def __call__(self, sel, precision, seed=None):
        a = self.aux if seed is None else _perturbed(self.aux, seed)
        o = self.orb if seed is None else _perturbed(self.orb, 1000 + seed)
        return self.oracle.eri3_sph(a, o, self.t[sel], precision=precision)[0]


def _envelope(evaluate, sets, ld):
    """The FP64 oracle's rounding error on shellsets `sets`: the largest over the input and ENVELOPE_RUNS
    ulp-level perturbations of it, each against the long-double build of the same input."""
    env = np.abs(evaluate(sets, 0) - ld)
    for r in range(ENVELOPE_RUNS):
        env = np.maximum(env, np.abs(evaluate(sets, 0, r) - evaluate(sets, 1, r)))
    return env


def _oracle_misses(evaluate, ref, off, sets):
    """Integrals (relative bound) and shellsets (absolute bound) where the FP64 oracle itself misses the
    bar against its long-double build."""
    ld = evaluate(sets, 1)
    e = np.abs(ref - ld)
    n = int(np.sum((np.abs(ld) > FLOOR) & (e > REL * np.abs(ld))))
    for s in sets:
        a, b = int(off[s]), int(off[s + 1])
        if b > a:
            m = float(np.max(np.abs(ld[a:b])))
            n += int(m > FLOOR and float(np.max(e[a:b])) > ABS * m)
    return n


def check(gpu, ref, offsets, what="", evaluate=None, max_cancel=None):
    """Compare engine values with the FP64 oracle's (`ref`), shellset by shellset (`offsets`, n+1).
    `evaluate(sel, precision, seed)` recomputes shellsets `sel` with the oracle (precision 1: long
    double; seed: perturbed input); it is only called for shellsets that miss a bound against the
    FP64 oracle. Those are judged again against the long-double value (a miss caused by the FP64
    oracle's own rounding is no miss); what still misses needs the cancellation exception."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    off = np.asarray(offsets, dtype=np.int64)
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    assert off[0] == 0 and off[-1] == ref.size, what + ": offsets do not cover the values"
    assert np.all(np.isfinite(gpu)), what + ": non-finite values"
    n_sets = len(off) - 1
    err = np.abs(gpu - ref)
    sizes = np.diff(off)
    nonempty = sizes > 0
    starts = off[:-1][nonempty]
    set_of = np.repeat(np.arange(n_sets), sizes)
    scale = np.zeros(n_sets)
    worst = np.zeros(n_sets)
    if ref.size:
        scale[nonempty] = np.maximum.reduceat(np.abs(ref), starts)
        worst[nonempty] = np.maximum.reduceat(err, starts)
    batch_scale = float(np.max(np.abs(ref))) if ref.size else 0.0
    batch_worst = float(np.max(err)) if err.size else 0.0
    all_sets = np.arange(n_sets)
    batch_excused = False
    if batch_worst > ABS * batch_scale:
        # the batch-wide bound: judged against the long-double values, then the cancellation exception
        assert evaluate is not None, "%s: max abs error %.3e > %.0e * %.3e over the batch" % (
            what, batch_worst, ABS, batch_scale)
        ld_all = evaluate(all_sets, 1)
        e_all = float(np.max(np.abs(gpu - ld_all)))
        if e_all > ABS * float(np.max(np.abs(ld_all))):
            env_all = _envelope(evaluate, all_sets, ld_all)
            assert e_all <= WITHIN * float(np.max(env_all)), (
                "%s: max abs error %.3e over the batch (largest value %.3e), oracle envelope %.3e" % (
                    what, e_all, batch_scale, float(np.max(env_all))))
            batch_excused = True
    abs_fail = (scale > FLOOR) & (worst > ABS * scale)
    big = np.abs(ref) > FLOOR
    rel = np.zeros_like(err)
    rel[big] = err[big] / np.abs(ref[big])
    rel_fail = rel > REL
    bad_sets = np.unique(np.concatenate([np.where(abs_fail)[0], set_of[rel_fail]]))
    n_cancel_rel = n_cancel_abs = 0
    exceptions = []
    if len(bad_sets):
        assert evaluate is not None, "%s: %d shellsets miss the bound (%d integrals above rel %.0e, worst %.3e)" % (
            what, len(bad_sets), int(rel_fail.sum()), REL, float(rel.max()))
        idx = np.concatenate([np.arange(off[s], off[s + 1]) for s in bad_sets])
        ld = evaluate(bad_sets, 1)
        g = gpu[idx]
        e_ld = np.abs(g - ld)
        rf = (np.abs(ld) > FLOOR) & (e_ld > REL * np.abs(ld))    # misses against the long-double value
        local = np.concatenate([[0], np.cumsum([int(off[s + 1] - off[s]) for s in bad_sets])])
        af = np.zeros(len(bad_sets), dtype=bool)
        for k in range(len(bad_sets)):
            a, b = local[k], local[k + 1]
            m = np.max(np.abs(ld[a:b])) if b > a else 0.0
            af[k] = m > FLOOR and np.max(e_ld[a:b]) > ABS * m
        if np.any(rf) or np.any(af):
            env = _envelope(evaluate, bad_sets, ld)
            for k in np.where(rf)[0]:
                exceptions.append({"kind": "rel", "value": float(ld[k]), "engine_error": float(e_ld[k]),
                                   "oracle_envelope": float(env[k]), "bound": float(REL * abs(ld[k]))})
            for k in np.where(af)[0]:
                a, b = local[k], local[k + 1]
                exceptions.append({"kind": "abs", "value": float(np.max(np.abs(ld[a:b]))),
                                   "engine_error": float(np.max(e_ld[a:b])),
                                   "oracle_envelope": float(np.max(env[a:b])),
                                   "bound": float(ABS * np.max(np.abs(ld[a:b])))})
            bad = [x for x in exceptions if not x["engine_error"] <= WITHIN * x["oracle_envelope"]]
            if bad:
                x = bad[0]
                raise AssertionError("%s: %d %s misses not explained by cancellation (e.g. value %.6e, engine error "
                                     "%.3e, bound %.3e, oracle envelope %.3e)" % (
                                         what, len(bad), x["kind"], x["value"], x["engine_error"], x["bound"],
                                         x["oracle_envelope"]))
            n_cancel_rel = int(rf.sum())
            n_cancel_abs = int(af.sum())
    n_elem = int(ref.size)
    ceiling = max(MIN_CANCEL_ALLOWED, int(MAX_CANCEL_PER_ELEMENT * n_elem)) if max_cancel is None else max_cancel
    n_cancel = n_cancel_rel + n_cancel_abs + int(batch_excused)
    oracle_misses = None
    if n_cancel > ceiling and max_cancel is None and evaluate is not None:
        oracle_misses = _oracle_misses(evaluate, ref, off, all_sets)
        ceiling = max(ceiling, 2 * oracle_misses + MIN_CANCEL_ALLOWED)
    assert n_cancel <= ceiling, "%s: %d cancellation exceptions, ceiling %d (FP64 oracle's own misses: %s)" % (
        what, n_cancel, ceiling, oracle_misses)
    ratio = np.where(scale > FLOOR, worst / np.where(scale > FLOOR, scale, 1.0), 0.0)
    return {"what": what, "elements": n_elem, "shellsets": n_sets,
            "max_abs_over_scale": float(ratio.max()) if n_sets else 0.0,
            "max_rel": float(rel.max()) if rel.size else 0.0,
            "n_cancel": n_cancel, "n_cancel_rel": n_cancel_rel, "n_cancel_abs": n_cancel_abs,
            "cancel_ceiling": ceiling, "oracle_own_misses": oracle_misses,
            "exceptions": sorted(exceptions, key=lambda x: -x["engine_error"] / max(x["bound"], 1e-300))[:8]}
