"""GPU parity of the exchange build K_ik = sum_jl D_jl (ij|kl) against the oracle's dense K."""
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


def _pairs(b):
    return np.array([(i, j) for i in range(b.n_shells) for j in range(i + 1)], dtype=np.int32)


def _run(eng, b, D, tau, seed_shuffle=None):
    db = mdx.DeviceBasis(b)
    pairs = _pairs(b)
    if seed_shuffle is not None:
        rng = np.random.Generator(np.random.PCG64(seed_shuffle))
        pairs = pairs[rng.permutation(len(pairs))]
        flip = rng.uniform(size=len(pairs)) < 0.5
        pairs[flip] = pairs[flip][:, ::-1]
    Q = eng.schwarz(db, pairs)
    K = eng.exchange(db, pairs, Q, torch.from_numpy(D), tau)
    torch.cuda.synchronize()
    return K.cpu().numpy(), eng.last_quartet_count(), len(pairs)


def test_exchange_small_molecule_no_screening(eng):
    """Small molecule of 3 atoms (s,p,d, K=3), random symmetric D, every unique quartet."""
    b = inputs.small_molecule(n_atoms=3)
    D = inputs.random_symmetric(b.nao, 5)
    K, nq, npair = _run(eng, b, D, 0.0, seed_shuffle=1)
    assert nq == npair * (npair + 1) // 2
    ref = oracle.exchange(b, D)
    np.testing.assert_allclose(K, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
    np.testing.assert_array_equal(K, K.T)


def test_exchange_high_l_molecule(eng):
    """Heavy/light clusters with f and g shells and K = 6 s shells (the batched-exchange molecules), D = C C^T."""
    b = inputs.molecule(seed=21, n_atoms=3)
    D = inputs.density(b.nao, 4)
    K, nq, npair = _run(eng, b, D, 0.0)
    ref = oracle.exchange(b, D)
    np.testing.assert_allclose(K, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
    assert np.sum(D * K) > 0


def test_exchange_screening(eng):
    """With tau > 0 fewer quartets are kept and K moves by less than the dropped-quartet
    bound: every kept-out quartet has Q_ij Q_kl max|D| < tau, so each of its <= 8 block
    updates changes a K entry by less than (#terms <= 28^2) * tau."""
    b = inputs.molecule(seed=22, n_atoms=3)
    D = inputs.density(b.nao, 6)
    K0, n0, npair = _run(eng, b, D, 0.0)
    tau = 1e-7
    K1, n1, _ = _run(eng, b, D, tau)
    assert n1 < n0
    ref = oracle.exchange(b, D)
    np.testing.assert_allclose(K0, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
    assert np.max(np.abs(K1 - K0)) <= 8 * 28 * 28 * (n0 - n1) * tau


def test_exchange_rejects_duplicate_pairs(eng):
    b = inputs.small_molecule(n_atoms=1)
    db = mdx.DeviceBasis(b)
    pairs = np.array([[1, 0], [0, 1]], dtype=np.int32)
    with pytest.raises(mdx.MdxError, match="EINVAL"):
        eng.exchange(db, pairs, torch.ones(2, dtype=torch.float64), torch.eye(b.nao, dtype=torch.float64))
