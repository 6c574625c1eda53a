"""Parity at the benchmark's full size and launch configuration: each class of the
224 x 224 sweep is evaluated exactly as bench.py does (prepared batches over the same output
chunks, the same autotuner trial), and a seeded sample of quartets is checked against the oracle:
400 [pp|pp], 200 [dd|dd], 100 [ff|ff], 80 [gg|gg], 60 [hh|hh] and 60 [ii|ii] shellsets."""
import numpy as np
import pytest
import torch

import bench
import oracle
from oracle import parity
from paper_2405_01834_gb300 import inputs, mdx

pytestmark = pytest.mark.gpu

SAMPLES = {1: 400, 2: 200, 3: 100, 4: 80, 5: 60, 6: 60}


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
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cq = bench.chunk_quartets(l, len(q), sms)
    batches = [eng.batch_eri4(db, q[s:s + cq]) for s in range(0, len(q), cq)]
    out = torch.empty(max(bt.total for bt in batches), dtype=torch.float64, device="cuda")
    batches[0].autotune(out, max_trial=bench.autotune_trial(l, len(q)))
    for bt in batches:
        bt.close()
    batches = [eng.batch_eri4(db, q[s:s + cq]) for s in range(0, len(q), cq)]
    rng = np.random.Generator(np.random.PCG64(500 + l))
    nsample = SAMPLES[l]
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
    print(parity.check(got, ref, off, "full-size sweep l=%d" % l, parity.Eri4Evaluator(b, q[picks])))
    for bt in batches:
        bt.close()
