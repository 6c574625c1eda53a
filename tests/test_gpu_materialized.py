"""The materialized-Hermite variant (dense [p|q] matrices and batched DGEMMs, the
paper's Sec. 3 third variant) against the oracle and the default kernels."""
import numpy as np
import pytest
import torch

import oracle
from oracle import parity
from paper_2405_01834_gb300 import inputs, mdx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    e = mdx.Engine(0)
    yield e
    e.close()


@pytest.mark.parametrize("lq", [(0, 0, 0, 0), (1, 0, 0, 0), (1, 1, 1, 1), (2, 1, 2, 0), (0, 2, 3, 1), (3, 3, 2, 2),
                                (4, 1, 3, 2), (6, 6, 6, 6)])
def test_materialized_matches_oracle_and_default(eng, lq):
    nb, nk = (4, 3) if max(lq) < 6 else (2, 2)
    b, q = inputs.class_sweep(lq, n_bra=nb, n_ket=nk, seed=91)
    bt = eng.batch_eri4(mdx.DeviceBasis(b), q)
    out_a = torch.empty(bt.total, dtype=torch.float64, device="cuda")
    out_b = torch.empty(bt.total, dtype=torch.float64, device="cuda")
    bt.run(out_a)
    n = bt.run_materialized(out_b)
    torch.cuda.synchronize()
    eng.sync()
    assert n >= 7
    off = bt.offsets().cpu().numpy()
    ref, roff = oracle.eri4(b, q)
    assert np.array_equal(off, roff)
    vb = out_b.cpu().numpy()
    print(parity.check(vb[: off[-1]], ref, off, "materialized %s" % (lq,), parity.Eri4Evaluator(b, q)))
    va = out_a.cpu().numpy()
    assert np.max(np.abs(va - vb)) <= 1e-12 * np.max(np.abs(ref))
    bt.close()


def test_materialized_rejects_contracted(eng):
    b, q = inputs.class_sweep((1, 0, 0, 0), n_bra=2, n_ket=2, seed=3, K=(2, 1, 1, 1))
    bt = eng.batch_eri4(mdx.DeviceBasis(b), q)
    out = torch.empty(bt.total, dtype=torch.float64, device="cuda")
    with pytest.raises(mdx.MdxError):
        bt.run_materialized(out)
    bt.close()
