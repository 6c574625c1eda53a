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


def test_exchange_energy_from_the_library(eng):
    """mdx_exchange's energy output: E_x = alpha sum D o K, against the oracle's."""
    b = inputs.molecule(seed=23, n_atoms=3)
    D = inputs.density(b.nao, 9)
    db = mdx.DeviceBasis(b)
    pairs = _pairs(b)
    Q = eng.schwarz(db, pairs)
    K, E = eng.exchange(db, pairs, Q, torch.from_numpy(D), 0.0, alpha=-1.0)
    Eref = -oracle.exchange_energy(b, D)
    assert abs(float(E) - Eref) <= 1e-12 * abs(Eref)
    assert abs(float(E) + float(torch.sum(torch.from_numpy(D).cuda() * K))) <= 1e-13 * abs(Eref)


def _rule_kept(b, pairs, Q, D, tau):
    """Plain restatement of the screening rule over every unordered pair of pairs (FP64)."""
    nc = (b.l + 1) * (b.l + 2) // 2
    n = b.n_shells
    dmax = np.zeros((n, n))
    for i in range(n):
        for k in range(n):
            dmax[i, k] = np.max(np.abs(D[b.ao_off[i]:b.ao_off[i] + nc[i], b.ao_off[k]:b.ao_off[k] + nc[k]]))
    kept = set()
    for p in range(len(pairs)):
        i, j = pairs[p]
        for q in range(p + 1):
            k, l = pairs[q]
            d = max(max(dmax[i, k], dmax[i, l]), max(dmax[j, k], dmax[j, l]))
            if Q[p] * Q[q] * d >= tau:
                kept.add(frozenset((p, q)))
    return kept


@pytest.mark.parametrize("tau", [0.0, 1e-9, 1e-6])
def test_screening_kept_set_matches_the_rule(eng, tau):
    """The quartets the GPU screening keeps (mdx_exchange_screen) are exactly those of a plain
    restatement of the rule, in any pair order and orientation; the count per class agrees too."""
    b = inputs.molecule(seed=24, n_atoms=3)
    D = inputs.density(b.nao, 3)
    db = mdx.DeviceBasis(b)
    rng = np.random.Generator(np.random.PCG64(8))
    pairs = _pairs(b)[rng.permutation(b.n_shells * (b.n_shells + 1) // 2)]
    flip = rng.uniform(size=len(pairs)) < 0.5
    pairs[flip] = pairs[flip][:, ::-1]
    Q = eng.schwarz(db, pairs)
    kept, n, mf = eng.exchange_screen(db, pairs, Q, torch.from_numpy(D), tau)
    got = {frozenset((int(x), int(y))) for x, y in kept.cpu().numpy()}
    assert len(got) == n == kept.shape[0]
    ref = _rule_kept(b, pairs, Q.cpu().numpy(), D, tau)
    assert got == ref
    assert mf > 0
    if tau > 0:
        assert n < len(pairs) * (len(pairs) + 1) // 2
    _, n2, _ = eng.exchange_screen(db, pairs, Q, torch.from_numpy(D), tau, list_quartets=False)
    assert n2 == n
