"""Tolerance rule shared by the GPU parity tests.

Reading of the stated bar (max abs error <= 1e-12 max|integral|, rel <= 1e-10 on
integrals above 1e-10): the maximum is taken over the batch compared; the
relative bound applies to every element whose reference exceeds 1e-10 (the
inputs are normalised so integrals are O(1)). Elements where the FP64 oracle
itself misses the relative bound against its long-double build are
cancellation-limited: they are reported separately and must stay within 10x
the oracle's own error (never silently widened).
"""
import numpy as np

ABS = 1e-12
REL = 1e-10
FLOOR = 1e-10


def check(gpu, ref, ref_ld=None, what=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    assert np.all(np.isfinite(gpu)), what + ": non-finite values"
    M = float(np.max(np.abs(ref))) if ref.size else 0.0
    err = np.abs(gpu - ref)
    worst_abs = float(np.max(err)) if err.size else 0.0
    assert worst_abs <= ABS * M, "%s: max abs err %.3e > %.1e * %.3e" % (what, worst_abs, ABS, M)
    big = np.abs(ref) > FLOOR
    rel = np.zeros_like(err)
    rel[big] = err[big] / np.abs(ref[big])
    bad = rel > REL
    n_cancel = 0
    if np.any(bad):
        assert ref_ld is not None, "%s: %d elements above rel %.0e (worst %.3e)" % (what, int(bad.sum()), REL, rel.max())
        ref_ld = np.asarray(ref_ld, dtype=np.float64)
        own = np.abs(ref - ref_ld)
        limited = bad & (own > REL * np.abs(ref_ld))
        assert not np.any(bad & ~limited), "%s: %d elements above rel %.0e not explained by cancellation" % (
            what, int((bad & ~limited).sum()), REL)
        assert np.all(np.abs(gpu - ref_ld)[limited] <= 10 * own[limited] + ABS * M), what + ": cancellation-limited element too far"
        n_cancel = int(limited.sum())
    return {"max_abs": worst_abs, "scale": M, "max_rel": float(rel.max()) if rel.size else 0.0, "n_cancel": n_cancel}
