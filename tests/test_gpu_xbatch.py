"""Batched exchange of several uneven molecules: per-class launches, one persistent launch
and the hybrid of both (optionally replayed from a CUDA graph) against per-molecule
mdx_exchange and the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_01834_gb300 import inputs, mdx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    e = mdx.Engine(0)
    yield e
    e.close()


def _molecules():
    mols = [inputs.small_molecule(seed=80 + i, n_atoms=1 + i % 3, shells=(0, 1, 2), K=1 + i % 3) for i in range(5)]
    mols.append(inputs.molecule(seed=90, n_atoms=2))        # heavy/light shells up to g, K = 6 s shells
    return mols


def _pairs(b):
    return np.array([(i, j) for i in range(b.n_shells) for j in range(i + 1)], dtype=np.int32)


def _register_launches(eng, xb):
    return sum(eng.plan_info(*xb.launch_info(i)[0]).register_kernel != 0 for i in range(xb.n_class_launches))


@pytest.mark.parametrize("persistent", [0, 1, 2])
def test_batched_exchange_matches_single(eng, persistent):
    mols = _molecules()
    bases = [mdx.DeviceBasis(b) for b in mols]
    Ds = [torch.from_numpy(inputs.density(b.nao, 3 + i)) for i, b in enumerate(mols)]
    xb = eng.xbatch(bases, Ds, tau=0.0)
    n = xb.run(persistent=persistent)
    torch.cuda.synchronize()
    eng.sync()
    n_reg = _register_launches(eng, xb)
    assert 0 < n_reg < xb.n_class_launches
    assert n == {0: 2 + xb.n_class_launches, 1: 3, 2: 3 + n_reg}[persistent]
    tot = 0
    for i, (b, db) in enumerate(zip(mols, bases)):
        p = _pairs(b)
        Q = eng.schwarz(db, p)
        K1 = eng.exchange(db, p, Q, Ds[i], 0.0).cpu().numpy()
        tot += eng.last_quartet_count()
        K = xb.Ks[i].cpu().numpy()
        np.testing.assert_allclose(K, K1, rtol=0, atol=1e-13 * np.max(np.abs(K1)))
    assert xb.n_quartets == tot
    # two molecules straight against the oracle
    for i in (0, 2):
        ref = oracle.exchange(mols[i], Ds[i].numpy())
        np.testing.assert_allclose(xb.Ks[i].cpu().numpy(), ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
    xb.close()


@pytest.mark.parametrize("persistent", [0, 1, 2])
def test_persistent_launch_in_cuda_graph(eng, persistent):
    """Every mode of mdx_xbatch_run (per-class launches, one persistent launch, the hybrid) captured in a
    CUDA graph and replayed gives the directly launched K."""
    mols = _molecules()[:4]
    bases = [mdx.DeviceBasis(b) for b in mols]
    Ds = [torch.from_numpy(inputs.density(b.nao, 30 + i)) for i, b in enumerate(mols)]
    xb = eng.xbatch(bases, Ds, tau=1e-12)
    xb.run(persistent=persistent)
    torch.cuda.synchronize()
    ref = [K.clone() for K in xb.Ks]
    for K in xb.Ks:
        K.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            xb.run(persistent=persistent)
    torch.cuda.synchronize()
    for _ in range(2):
        for K in xb.Ks:
            K.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for K, R in zip(xb.Ks, ref):
            torch.testing.assert_close(K, R, rtol=0, atol=1e-13 * float(R.abs().max()))
    eng.sync()
    xb.close()


def test_class_launches_one_by_one(eng):
    """Every per-class launch run alone, then K + K^T, reproduces the batched K; the
    launch info adds up to the batch totals."""
    mols = _molecules()[:3]
    bases = [mdx.DeviceBasis(b) for b in mols]
    Ds = [torch.from_numpy(inputs.density(b.nao, 60 + i)) for i, b in enumerate(mols)]
    xb = eng.xbatch(bases, Ds, tau=1e-12)
    xb.run(persistent=False)
    torch.cuda.synchronize()
    ref = [K.clone() for K in xb.Ks]
    nq, mf = 0, 0.0
    for K in xb.Ks:
        K.zero_()
    for i in range(xb.n_class_launches):
        lk, n, f = xb.launch_info(i)
        assert all(0 <= l <= 6 for l in lk[:4]) and lk[4] >= 1 and lk[5] >= 1 and n > 0 and f > 0
        nq += n
        mf += f
        xb.run_class(i)
    torch.cuda.synchronize()
    eng.sync()
    assert nq == xb.n_quartets
    assert mf == pytest.approx(xb.model_flops, rel=1e-12)
    for K, R in zip(xb.Ks, ref):
        np.testing.assert_allclose((K + K.T).cpu().numpy(), R.cpu().numpy(), rtol=0,
                                   atol=1e-13 * float(R.abs().max()))
    with pytest.raises(mdx.MdxError):
        xb.launch_info(xb.n_class_launches)
    xb.close()


def test_autotuned_batched_exchange_keeps_K():
    """The batched-exchange autotuner (register kernel or team shape per class launch, timed with the
    digestion epilogue) changes only the summation order: K of the per-class and hybrid launches after
    tuning equals K before it, and the oracle's. Own context: the tuned shapes stay with it."""
    e = mdx.Engine(0)
    mols = _molecules()
    bases = [mdx.DeviceBasis(b) for b in mols]
    Ds = [torch.from_numpy(inputs.density(b.nao, 3 + i)) for i, b in enumerate(mols)]
    xb = e.xbatch(bases, Ds, tau=0.0)
    xb.run(persistent=0)
    torch.cuda.synchronize()
    K0 = [K.clone() for K in xb.Ks]
    xb.autotune(max_trial=64)
    for mode in (0, 2, 1):
        xb.run(persistent=mode)
        torch.cuda.synchronize()
        e.sync()
        for K, Kr in zip(xb.Ks, K0):
            np.testing.assert_allclose(K.cpu().numpy(), Kr.cpu().numpy(), rtol=0,
                                       atol=1e-13 * float(Kr.abs().max()))
    ref = oracle.exchange(mols[1], Ds[1].numpy())
    np.testing.assert_allclose(xb.Ks[1].cpu().numpy(), ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
    xb.close()
    e.close()
