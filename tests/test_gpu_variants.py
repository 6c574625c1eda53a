"""The register kernel (one thread per quartet) and the team kernel on the same
classes, both against the oracle: integrals, 3-center integrals and the
exchange digestion, with the class's shape fixed through mdx_set_class_shape."""
import numpy as np
import pytest
import torch

import oracle
from oracle import parity
from paper_2405_01834_gb300 import inputs, mdx

pytestmark = pytest.mark.gpu

# small classes (register kernels exist) with several contraction depths
CLASSES = [((0, 0, 0, 0), (3, 2, 3, 1)), ((1, 0, 0, 0), (3, 3, 1, 2)), ((1, 1, 1, 0), (1, 2, 3, 1)),
           ((2, 1, 0, 0), (1, 1, 2, 1)), ((0, 1, 0, 2), (2, 1, 1, 1)), ((1, 0, 1, 1), (2, 1, 2, 1)),
           ((3, 0, 0, 0), (1, 1, 3, 3)), ((0, 0, 4, 0), (2, 2, 1, 1)), ((2, 0, 0, 1), (1, 1, 1, 1)),
           ((1, 3, 0, 0), (1, 1, 2, 2)), ((0, 2, 1, 0), (1, 1, 1, 1))]


def _kb(K):
    return K[0] * K[1], K[2] * K[3]


@pytest.mark.parametrize("lq,K", CLASSES)
def test_register_and_team_kernels_match_oracle(lq, K):
    b, q = inputs.class_sweep(lq, n_bra=7, n_ket=5, seed=41, K=K)
    ref, roff = oracle.eri4(b, q)
    ev = parity.Eri4Evaluator(b, q)
    assert mdx.plan_info(*lq, *_kb(K)).register_kernel == 1
    got = {}
    for variant in (1, 2):
        eng = mdx.Engine(0)
        eng.set_class_shape(*lq, *_kb(K), variant=variant)
        assert eng.plan_info(*lq, *_kb(K)).register_kernel == (variant == 2)
        v, off = eng.eri4(mdx.DeviceBasis(b), q)
        torch.cuda.synchronize()
        eng.sync()
        v, off = v.cpu().numpy(), off.cpu().numpy()
        assert np.array_equal(off, roff)
        print(parity.check(v[: off[-1]], ref, off, "%s K=%s variant %d" % (lq, K, variant), ev))
        got[variant] = v[: off[-1]]
        eng.close()
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got[1] - got[2])) <= 1e-13 * scale


@pytest.mark.parametrize("la", [0, 1, 2, 3, 4])
def test_three_center_register_kernel(la):
    """[a|cd] with a contracted orbital pair (s K=6 / p K=3) through the register kernel."""
    aux, orb = inputs.df_cluster(seed=1003, n_atoms=3)
    rng = np.random.Generator(np.random.PCG64(40 + la))
    A = rng.choice(np.where(aux.l == la)[0], 3, replace=False)
    pairs = [(c, d) for c in range(orb.n_shells) for d in range(c + 1) if orb.l[c] + orb.l[d] <= 1]
    P = np.array(pairs)[rng.choice(len(pairs), 6, replace=False)]
    trip = np.array([(a, c, d) for a in A for c, d in P], dtype=np.int32)
    eng = mdx.Engine(0)
    v, off = eng.eri3(mdx.DeviceBasis(aux), mdx.DeviceBasis(orb), trip)
    torch.cuda.synchronize()
    eng.sync()
    ref, roff = oracle.eri3(aux, orb, trip)
    print(parity.check(v.cpu().numpy()[: roff[-1]], ref, roff, "3c reg la=%d" % la, parity.Eri3Evaluator(aux, orb, trip)))
    eng.close()


def test_exchange_digestion_both_kernels():
    """Exchange of a 3-atom s,p,d molecule (K = 3): small classes digested by the
    register kernel (default) and by the team kernel give the oracle's K."""
    b = inputs.small_molecule(n_atoms=3)
    D = inputs.random_symmetric(b.nao, 11)
    ref = oracle.exchange(b, D)
    pairs = np.array([(i, j) for i in range(b.n_shells) for j in range(i + 1)], dtype=np.int32)
    Ks = []
    for force_team in (False, True):
        eng = mdx.Engine(0)
        if force_team:
            for la in range(3):
                for lb in range(3):
                    for lc in range(3):
                        for ld in range(3):
                            if mdx.plan_info(la, lb, lc, ld, 9, 9).register_kernel:
                                eng.set_class_shape(la, lb, lc, ld, 9, 9, variant=1)
        db = mdx.DeviceBasis(b)
        Q = eng.schwarz(db, pairs)
        K = eng.exchange(db, pairs, Q, torch.from_numpy(D), 0.0).cpu().numpy()
        eng.sync()
        np.testing.assert_allclose(K, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
        Ks.append(K)
        eng.close()
    assert np.max(np.abs(Ks[0] - Ks[1])) <= 1e-13 * np.max(np.abs(ref))


def test_shape_setter_rejects():
    eng = mdx.Engine(0)
    with pytest.raises(mdx.MdxError):
        eng.set_class_shape(3, 3, 3, 3, variant=2)      # no register kernel for [ff|ff]
    with pytest.raises(mdx.MdxError):
        eng.set_class_shape(1, 1, 1, 1, team_threads=3)
    with pytest.raises(mdx.MdxError):
        eng.set_class_shape(1, 1, 1, 1, variant=5)
    eng.close()


# classes of total angular momentum 5-6 (and L = 4 ones too large for registers alone):
# R in registers, [p|cd] and the shellset in shared memory
XS_CLASSES = [((3, 0, 1, 0), (1, 3, 2, 3)), ((1, 1, 1, 1), (2, 1, 1, 2)), ((2, 1, 1, 0), (1, 2, 3, 1)),
              ((6, 0, 0, 0), (1, 1, 2, 2)), ((2, 0, 1, 1), (1, 2, 2, 1)), ((5, 0, 0, 0), (1, 1, 2, 2)),
              ((1, 0, 0, 3), (2, 2, 1, 1)), ((3, 0, 0, 1), (1, 1, 2, 2)), ((4, 0, 1, 0), (1, 1, 1, 1)),
              ((3, 0, 1, 1), (1, 2, 2, 1)), ((5, 0, 1, 0), (1, 1, 2, 2)), ((2, 2, 1, 0), (1, 1, 2, 1)),
              ((2, 1, 1, 1), (1, 1, 1, 2))]


@pytest.mark.parametrize("lq,K", XS_CLASSES)
def test_shared_memory_register_variant(lq, K):
    b, q = inputs.class_sweep(lq, n_bra=6, n_ket=5, seed=43, K=K)
    ref, roff = oracle.eri4(b, q)
    ev = parity.Eri4Evaluator(b, q)
    got = {}
    for variant in (1, 2):
        eng = mdx.Engine(0)
        eng.set_class_shape(*lq, *_kb(K), variant=variant)
        v, off = eng.eri4(mdx.DeviceBasis(b), q)
        torch.cuda.synchronize()
        eng.sync()
        v, off = v.cpu().numpy(), off.cpu().numpy()
        assert np.array_equal(off, roff)
        print(parity.check(v[: off[-1]], ref, off, "%s K=%s variant %d" % (lq, K, variant), ev))
        got[variant] = v[: off[-1]]
        eng.close()
    assert np.max(np.abs(got[1] - got[2])) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("la", [5, 6])
def test_three_center_shared_memory_variant(la):
    """[a|ss] and [a|ps] with contracted orbital pairs (K = 36 / 18) in the shared-memory variant."""
    aux, orb = inputs.df_cluster(seed=1003, n_atoms=3)
    rng = np.random.Generator(np.random.PCG64(70 + la))
    A = rng.choice(np.where(aux.l == la)[0], 2, replace=False)
    pairs = [(c, d) for c in range(orb.n_shells) for d in range(c + 1) if orb.l[c] + orb.l[d] <= 1]
    P = np.array(pairs)[rng.choice(len(pairs), 6, replace=False)]
    trip = np.array([(a, c, d) for a in A for c, d in P], dtype=np.int32)
    eng = mdx.Engine(0)
    for lc, ld in ((0, 0), (1, 0), (0, 1)):
        kc = {0: 6, 1: 3}
        try:
            eng.set_class_shape(la, 0, lc, ld, 1, kc[lc] * kc[ld], one_centre=True, variant=2)
        except mdx.MdxError:
            pass    # [i|ps] is above the size limit of the variant: stays on the team kernel
    v, off = eng.eri3(mdx.DeviceBasis(aux), mdx.DeviceBasis(orb), trip)
    torch.cuda.synchronize()
    eng.sync()
    ref, roff = oracle.eri3(aux, orb, trip)
    print(parity.check(v.cpu().numpy()[: roff[-1]], ref, roff, "3c xs la=%d" % la, parity.Eri3Evaluator(aux, orb, trip)))
    eng.close()
