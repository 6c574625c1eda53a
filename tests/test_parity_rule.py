"""The tolerance rule of the parity tests (oracle/parity.py), on the CPU.

It must pass independent FP64 evaluations of the same integrals and reject
plausible mistakes: a relative error above the bound on an integral that is not
cancellation-limited, an absolute error above the bound in one shellset, a
non-finite value, and misses for which no oracle re-evaluation is possible."""
import numpy as np
import pytest

import oracle
from oracle import parity
from paper_2405_01834_gb300 import inputs


@pytest.fixture(scope="module")
def ff():
    b, q = inputs.class_sweep((3, 3, 3, 3), n_bra=12, n_ket=10, seed=1002)
    ref, off = oracle.eri4(b, q)
    return b, q, ref, off


def test_identical_values_pass(ff):
    b, q, ref, off = ff
    r = parity.check(ref.copy(), ref, off, "self", parity.Eri4Evaluator(b, q))
    assert r["n_cancel"] == 0 and r["max_rel"] == 0.0


def test_independent_fp64_rounding_passes(ff):
    """Another FP64 evaluation of the same exact values (the oracle's rounding noise on a copy of
    the input moved by 1-2 ulp, added to the long-double values) passes, cancellation counted."""
    b, q, ref, off = ff
    ld, _ = oracle.eri4(b, q, precision=1)
    for seed in (31, 32):
        bp = parity._perturbed(b, seed)
        noise = oracle.eri4(bp, q)[0] - oracle.eri4(bp, q, precision=1)[0]
        r = parity.check(ld + noise, ref, off, "draw %d" % seed, parity.Eri4Evaluator(b, q))
        assert r["n_cancel"] <= r["cancel_ceiling"]


def test_relative_error_is_caught(ff):
    b, q, ref, off = ff
    g = ref.copy()
    k = int(np.argmin(np.abs(np.abs(ref) - 1e-3)))   # an integral of about 1e-3
    g[k] *= 1 + 3e-10
    with pytest.raises(AssertionError):
        parity.check(g, ref, off, "planted rel", parity.Eri4Evaluator(b, q))


def test_shellset_absolute_error_is_caught(ff):
    """2e-12 of its shellset's largest integral, in a shellset much smaller than the batch's largest
    (so the batch-wide bound alone would let it pass)."""
    b, q, ref, off = ff
    top = np.max(np.abs(ref))
    sizes = np.array([np.max(np.abs(ref[off[s]:off[s + 1]])) for s in range(len(off) - 1)])
    ok = (sizes > 1e-9) & (sizes < 1e-3 * top)
    assert np.any(ok)
    s = int(np.argmax(np.where(ok, sizes, 0.0)))
    g = ref.copy()
    k = off[s] + int(np.argmax(np.abs(ref[off[s]:off[s + 1]])))
    g[k] += 2e-12 * sizes[s]
    with pytest.raises(AssertionError):
        parity.check(g, ref, off, "planted abs", parity.Eri4Evaluator(b, q))


def test_batch_bound_and_nonfinite_are_caught(ff):
    b, q, ref, off = ff
    g = ref.copy()
    g[0] = np.nan
    with pytest.raises(AssertionError):
        parity.check(g, ref, off, "nan", parity.Eri4Evaluator(b, q))
    g = ref.copy()
    g[5] += 2e-12 * np.max(np.abs(ref))
    with pytest.raises(AssertionError):
        parity.check(g, ref, off, "batch abs", parity.Eri4Evaluator(b, q))


def test_miss_without_oracle_is_an_error(ff):
    b, q, ref, off = ff
    g = ref.copy()
    g[int(np.argmax(np.abs(ref)))] *= 1 + 1e-9
    with pytest.raises(AssertionError):
        parity.check(g, ref, off, "no evaluator")


def test_perturbation_keeps_equal_values_equal():
    b = inputs.small_molecule(n_atoms=2)
    bp = parity._perturbed(b, 3)
    for i in range(b.n_shells):
        for j in range(b.n_shells):
            if np.array_equal(b.center[i], b.center[j]):
                assert np.array_equal(bp.center[i], bp.center[j])
    moved = np.abs(bp.exps / b.exps - 1.0)
    assert np.all(moved <= 2.5 * 2.0 ** -52) and np.any(moved > 0)


def test_ceiling_follows_the_oracles_own_misses():
    """A batch full of cancellation-limited values (solid-harmonic shellsets of distant, diffuse shells:
    the combinations cancel the dominant Cartesian terms by up to 1e7) needs many exceptions for any
    FP64 evaluation; the ceiling then follows the FP64 oracle's own misses on the batch."""
    rng = np.random.Generator(np.random.PCG64(31))
    bb = inputs.BasisBuilder()
    for i in range(10):
        l = [0, 1, 2, 3, 4, 6, 5, 2, 3, 1][i]
        inputs.random_shell(rng, bb, l, rng.uniform(0, 4, 3), 1 + (i % 2 if l < 3 else 0), 0.1, 20.0)
    b = bb.build()
    q = inputs.random_quartets(b, 60, seed=5)
    q = q[b.l[q].sum(axis=1) <= 16]
    ref, off = oracle.eri4_sph(b, q)
    ld, _ = oracle.eri4_sph(b, q, precision=1)
    bp = parity._perturbed(b, 50)
    draw = ld + (oracle.eri4_sph(bp, q)[0] - oracle.eri4_sph(bp, q, precision=1)[0])
    r = parity.check(draw, ref, off, "solid draw", parity.Eri4SphEvaluator(b, q))
    assert r["n_cancel"] > parity.MIN_CANCEL_ALLOWED and r["oracle_own_misses"] > 0
    assert r["n_cancel"] <= 2 * r["oracle_own_misses"] + parity.MIN_CANCEL_ALLOWED
    # the same values with one planted error are still caught
    g = draw.copy()
    k = int(np.argmax(np.abs(ref)))
    g[k] *= 1 + 1e-9
    with pytest.raises(AssertionError):
        parity.check(g, ref, off, "solid planted", parity.Eri4SphEvaluator(b, q))
