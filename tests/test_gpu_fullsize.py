"""Parity at the benchmark's full size and launch configuration: each class of the
224 x 224 sweep is evaluated exactly as bench.py does (prepared batches over 2 GiB output
chunks, autotuned team shapes), and a seeded sample of quartets is checked against the oracle."""
import numpy as np
import pytest
import torch

import bench
import oracle
import parity
from paper_2405_01834_gb300 import inputs, mdx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    e = mdx.Engine(0)
    yield e
    e.close()


@pytest.mark.parametrize("l", [1, 2, 3, 4, 5, 6])
def test_sweep_class_full_size_sampled(eng, l):
    b, q = inputs.class_sweep((l, l, l, l), n_bra=224, n_ket=224)
    db = mdx.DeviceBasis(b)
    per_q = inputs.ncart(l) ** 4
    cq = max(1, min(len(q), bench.CHUNK_BYTES // (per_q * 8)))
    batches = [eng.batch_eri4(db, q[s:s + cq]) for s in range(0, len(q), cq)]
    out = torch.empty(max(bt.total for bt in batches), dtype=torch.float64, device="cuda")
    batches[0].autotune(out, max_trial=max(304, min(len(q), 4096 // l)))
    for bt in batches:
        bt.close()
    batches = [eng.batch_eri4(db, q[s:s + cq]) for s in range(0, len(q), cq)]
    rng = np.random.Generator(np.random.PCG64(500 + l))
    nsample = {1: 400, 2: 200, 3: 60, 4: 24, 5: 10, 6: 6}[l]
    picks = np.sort(rng.choice(len(q), nsample, replace=False))
    got = np.zeros(nsample * per_q)
    for k, bt in enumerate(batches):
        bt.run(out)
        torch.cuda.synchronize()
        lo, hi = k * cq, min(len(q), (k + 1) * cq)
        for n, p in enumerate(picks):
            if lo <= p < hi:
                got[n * per_q:(n + 1) * per_q] = out[(p - lo) * per_q:(p - lo + 1) * per_q].cpu().numpy()
    eng.sync()
    ref, off = oracle.eri4(b, q[picks])
    ref_ld, _ = oracle.eri4(b, q[picks], precision=1)
    parity.check(got, ref, ref_ld, "full-size sweep l=%d" % l, off)
    for bt in batches:
        bt.close()
