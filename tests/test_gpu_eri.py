"""GPU parity: the CUDA engine (through the C ABI) against the CPU oracle.

Inputs are seeded and synthetic (paper_2405_01834_gb300.inputs); the oracle
is the plain CPU McMurchie-Davidson code in oracle/. Tolerance: oracle/parity.py.
"""
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


def _gpu4(eng, basis, q):
    db = mdx.DeviceBasis(basis)
    v, off = eng.eri4(db, q)
    torch.cuda.synchronize()
    return v.cpu().numpy(), off.cpu().numpy()


def test_small_molecule_all_unique_quartets(eng):
    """Small molecule: 6 atoms with s,p,d shells, K = 3, every unique quartet."""
    b = inputs.small_molecule()
    q = inputs.unique_quartets(b.n_shells)
    assert len(q) == 14706
    v, off = _gpu4(eng, b, q)
    ref, roff = oracle.eri4(b, q)
    assert np.array_equal(off, roff)
    r = parity.check(v[: off[-1]], ref, off, "small molecule", parity.Eri4Evaluator(b, q))
    print(r)


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4, 5, 6])
def test_class_sweep_grid(eng, l):
    """Per-class random quartet grid at a size the oracle finishes in seconds: a 5 x 3 grid of
    random bra/ket pairs of class [ll|ll], K = 1, exponents in [0.05, 50]."""
    nb, nk = (5, 3) if l < 6 else (3, 2)
    b, q = inputs.class_sweep((l, l, l, l), n_bra=nb, n_ket=nk, seed=77)
    v, off = _gpu4(eng, b, q)
    ref, roff = oracle.eri4(b, q)
    assert np.array_equal(off, roff)
    print(parity.check(v[: off[-1]], ref, off, "sweep l=%d" % l, parity.Eri4Evaluator(b, q)))


MIXED = [(0, 1, 2, 3), (3, 2, 1, 0), (6, 0, 0, 0), (0, 0, 0, 6), (2, 6, 1, 4), (5, 0, 4, 1), (1, 3, 6, 2),
         (4, 4, 0, 2), (6, 5, 1, 1), (0, 6, 6, 0)]


@pytest.mark.parametrize("lq", MIXED)
def test_mixed_classes_contracted(eng, lq):
    """Unequal angular momenta in every position, contraction degrees 1-3."""
    K = tuple(1 + (x % 3) for x in lq) if max(lq) < 5 else (1, 2, 1, 2)
    b, q = inputs.class_sweep(lq, n_bra=3, n_ket=2, seed=5, K=K)
    v, off = _gpu4(eng, b, q)
    ref, _ = oracle.eri4(b, q)
    print(parity.check(v[: off[-1]], ref, off, "mixed %s" % (lq,), parity.Eri4Evaluator(b, q)))


def test_random_quartets_many_classes(eng):
    """200 random quartets over a basis of s..i shells with K in 1..3: many
    classes in one call, ragged class sizes, shells repeated across quartets."""
    rng = np.random.Generator(np.random.PCG64(99))
    bb = inputs.BasisBuilder()
    for i in range(14):
        l = i % 7
        K = 1 if l >= 4 else 1 + i % 3
        inputs.random_shell(rng, bb, l, rng.uniform(0, 5, 3), K, 0.1, 20.0)
    b = bb.build()
    q = inputs.random_quartets(b, 200, seed=3)
    # keep the oracle time modest: drop quartets with total L > 14
    L = b.l[q].sum(axis=1)
    q = q[L <= 14]
    v, off = _gpu4(eng, b, q)
    ref, _ = oracle.eri4(b, q)
    print(parity.check(v[: off[-1]], ref, off, "random", parity.Eri4Evaluator(b, q)))


def test_empty_and_single(eng):
    b = inputs.small_molecule(n_atoms=1)
    db = mdx.DeviceBasis(b)
    v, off = eng.eri4(db, np.zeros((0, 4), dtype=np.int32))
    assert off.cpu().numpy().tolist() == [0]
    q = np.array([[2, 2, 2, 2]], dtype=np.int32)
    v, off = eng.eri4(db, q)
    ref, roff = oracle.eri4(b, q)
    print(parity.check(v.cpu().numpy()[: int(off[-1])], ref, roff, "single", parity.Eri4Evaluator(b, q)))


def test_errors_are_reported(eng):
    b = inputs.small_molecule(n_atoms=1)
    db = mdx.DeviceBasis(b)
    with pytest.raises(mdx.MdxError, match="EINVAL"):
        eng.eri4(db, np.array([[0, 0, 0, 99]], dtype=np.int32))
    with pytest.raises(mdx.MdxError, match="ECAPACITY"):
        eng.eri4(db, np.array([[2, 2, 2, 2]], dtype=np.int32), out=torch.empty(10, dtype=torch.float64, device="cuda"))
    bad = inputs.small_molecule(n_atoms=1)
    bad.l = bad.l.copy()
    bad.l[0] = 7
    with pytest.raises(mdx.MdxError, match="EUNSUPPORTED"):
        eng.eri4(mdx.DeviceBasis(bad), np.array([[0, 0, 0, 0]], dtype=np.int32))
    # the context stays usable (two atoms: no shellset that vanishes by symmetry)
    b2 = inputs.small_molecule(n_atoms=2)
    v, off = eng.eri4(mdx.DeviceBasis(b2), np.array([[0, 4, 2, 3]], dtype=np.int32))
    ref, roff = oracle.eri4(b2, [[0, 4, 2, 3]])
    print(parity.check(v.cpu().numpy()[: int(off[-1])], ref, roff, "after errors", parity.Eri4Evaluator(b2, [[0, 4, 2, 3]])))


@pytest.mark.parametrize("la", [0, 1, 2, 3, 4, 5, 6])
def test_three_center(eng, la):
    """[a|cd]: auxiliary shell a (K=1) against contracted orbital pairs (K 6/3/1)."""
    aux_all, orb = inputs.df_cluster(seed=11, n_atoms=3)
    sel = np.where(aux_all.l == la)[0][:2]
    rng = np.random.Generator(np.random.PCG64(la))
    pairs = rng.integers(0, orb.n_shells, (6, 2))
    t = np.array([[a, c, d] for a in sel for c, d in pairs], dtype=np.int32)
    daux, dorb = mdx.DeviceBasis(aux_all), mdx.DeviceBasis(orb)
    v, off = eng.eri3(daux, dorb, t)
    torch.cuda.synchronize()
    ref, roff = oracle.eri3(aux_all, orb, t)
    assert np.array_equal(off.cpu().numpy(), roff)
    print(parity.check(v.cpu().numpy()[: roff[-1]], ref, roff, "3c la=%d" % la, parity.Eri3Evaluator(aux_all, orb, t)))


def test_prepared_batch_runs_repeatably(eng):
    """mdx_batch_eri4 + mdx_batch_run twice gives the mdx_eri4 result bit for bit."""
    b, q = inputs.class_sweep((2, 1, 2, 0), n_bra=7, n_ket=5, seed=8, K=(2, 1, 3, 1))
    db = mdx.DeviceBasis(b)
    v, off = eng.eri4(db, q)
    bt = eng.batch_eri4(db, q)
    assert bt.n == len(q) and bt.total == int(off[-1])
    assert torch.equal(bt.offsets(), off)
    for _ in range(2):
        w = torch.full((bt.total,), float("nan"), dtype=torch.float64, device="cuda")
        nl = bt.run(w)
        torch.cuda.synchronize()
        eng.sync()
        assert nl == 2
        assert torch.equal(w, v[: bt.total])
    bt.close()


def test_schwarz(eng):
    b = inputs.small_molecule(n_atoms=3)
    pairs = np.array([(i, j) for i in range(b.n_shells) for j in range(i + 1)], dtype=np.int32)
    Q = eng.schwarz(mdx.DeviceBasis(b), pairs).cpu().numpy()
    q4 = np.array([(i, j, i, j) for i, j in pairs], dtype=np.int32)
    ref, off = oracle.eri4(b, q4)
    refQ = []
    for n, (i, j) in enumerate(pairs):
        m = inputs.ncart(int(b.l[i])) * inputs.ncart(int(b.l[j]))
        blk = ref[off[n]:off[n + 1]].reshape(m, m)
        refQ.append(np.sqrt(np.max(np.abs(np.diag(blk)))))
    np.testing.assert_allclose(Q, refQ, rtol=1e-12, atol=0)


def test_autotuned_batch_matches(eng):
    """The autotuner keeps results (only the summation order may change)."""
    b, q = inputs.class_sweep((3, 2, 2, 1), n_bra=9, n_ket=7, seed=12, K=(1, 2, 1, 3))
    db = mdx.DeviceBasis(b)
    v, off = eng.eri4(db, q)
    bt = eng.batch_eri4(db, q)
    w = torch.empty(bt.total, dtype=torch.float64, device="cuda")
    bt.autotune(w, max_trial=32)
    w.fill_(float("nan"))
    bt.run(w)
    torch.cuda.synchronize()
    eng.sync()
    ref, _ = oracle.eri4(b, q)
    print(parity.check(w.cpu().numpy(), ref, off.cpu().numpy(), "autotuned", parity.Eri4Evaluator(b, q)))
    bt.close()


SPH = [(0, 0, 0, 0), (1, 1, 1, 1), (2, 2, 2, 2), (3, 3, 3, 3), (4, 4, 4, 4), (5, 5, 5, 5), (6, 6, 6, 6),
       (2, 1, 0, 3), (3, 3, 2, 2), (4, 2, 4, 1), (6, 5, 6, 4), (6, 0, 6, 0), (5, 5, 0, 0), (0, 6, 2, 6)]


@pytest.mark.parametrize("lq", SPH)
def test_solid_harmonic_eri4(eng, lq):
    """mdx_eri4_sph against the oracle's solid-harmonic shellsets (m = -l..l): the classes of the team
    kernel contract the solid-harmonic coefficients into the transforms, the small classes transform
    Cartesian shellsets index by index. Contracted bras and kets where the class is small enough."""
    K = (1, 2, 1, 2) if max(lq) < 4 else ((2, 1, 1, 1) if sum(lq) <= 12 else (1, 1, 1, 1))
    nb, nk = (3, 2) if sum(lq) < 20 else (2, 2)
    # overlapping shells (3-bohr box, exponents 0.2-5): integrals of a meaningful size at every l
    b, q = inputs.class_sweep(lq, n_bra=nb, n_ket=nk, seed=13, K=K, box=3.0, zlo=0.2, zhi=5.0)
    db = mdx.DeviceBasis(b)
    v, off = eng.eri4_sph(db, q)
    torch.cuda.synchronize()
    ref, roff = oracle.eri4_sph(b, q)
    assert np.array_equal(off.cpu().numpy(), roff)
    print(parity.check(v.cpu().numpy()[: roff[-1]], ref, roff, "solid %s" % (lq,), parity.Eri4SphEvaluator(b, q)))


def test_solid_harmonic_batch_repeats_and_matches(eng):
    """A prepared solid-harmonic batch (mixed classes: team-kernel and register-kernel ones) gives the
    mdx_eri4_sph result bit for bit, run after run, and reports solid-harmonic sizes."""
    rng = np.random.Generator(np.random.PCG64(31))
    bb = inputs.BasisBuilder()
    for i in range(10):
        l = [0, 1, 2, 3, 4, 6, 5, 2, 3, 1][i]
        inputs.random_shell(rng, bb, l, rng.uniform(0, 4, 3), 1 + (i % 2 if l < 3 else 0), 0.1, 20.0)
    b = bb.build()
    q = inputs.random_quartets(b, 60, seed=5)
    q = q[b.l[q].sum(axis=1) <= 16]
    db = mdx.DeviceBasis(b)
    v, off = eng.eri4_sph(db, q)
    bt = eng.batch_eri4_sph(db, q)
    assert bt.n == len(q) and bt.total == int(off[-1])
    assert torch.equal(bt.offsets(), off)
    for _ in range(2):
        w = torch.full((bt.total,), float("nan"), dtype=torch.float64, device="cuda")
        bt.run(w)
        torch.cuda.synchronize()
        eng.sync()
        assert torch.equal(w, v[: bt.total])
    ref, roff = oracle.eri4_sph(b, q)
    print(parity.check(v.cpu().numpy()[: roff[-1]], ref, roff, "solid batch", parity.Eri4SphEvaluator(b, q)))
    with pytest.raises(mdx.MdxError, match="EUNSUPPORTED"):
        bt.run_materialized(w)
    bt.close()


@pytest.mark.parametrize("lq,K", [((3, 3, 3, 3), (1, 1, 1, 3)), ((4, 0, 4, 0), (1, 1, 1, 1)), ((2, 2, 3, 1), (2, 1, 1, 3))])
def test_solid_harmonic_batch_autotuned(lq, K):
    """The autotuner on a solid-harmonic batch (team sizes, budgets, cached R tables of contracted classes)
    keeps the oracle's results, and the tuned batch repeats them bit for bit."""
    e = mdx.Engine(0)
    b, q = inputs.class_sweep(lq, n_bra=3, n_ket=3, seed=17, K=K, box=3.0, zlo=0.2, zhi=5.0)
    db = mdx.DeviceBasis(b)
    bt = e.batch_eri4_sph(db, q)
    w = torch.full((bt.total,), float("nan"), dtype=torch.float64, device="cuda")
    bt.autotune(w, max_trial=9)
    w2 = torch.full((bt.total,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        bt.run(w)
        bt.run(w2)
        torch.cuda.synchronize()
        e.sync()
        assert torch.equal(w, w2)
    ref, roff = oracle.eri4_sph(b, q)
    assert np.array_equal(bt.offsets().cpu().numpy(), roff)
    print(parity.check(w.cpu().numpy(), ref, roff, "autotuned solid %s K=%s" % (lq, K), parity.Eri4SphEvaluator(b, q)))
    bt.close()
    e.close()


def test_bound_screens_quartets(eng):
    """mdx_eri4's bound input: quartets with bound < tau are written as zeros without evaluation, the
    others are the unscreened values bit for bit; bound = NULL and tau = 0 keep every quartet."""
    b = inputs.small_molecule(n_atoms=3)
    db = mdx.DeviceBasis(b)
    q = inputs.unique_quartets(b.n_shells)[::7]
    pairs = np.array([(i, j) for i in range(b.n_shells) for j in range(i + 1)], dtype=np.int32)
    Q = eng.schwarz(db, pairs).cpu().numpy()
    pid = {(int(i), int(j)): n for n, (i, j) in enumerate(pairs)}
    key = lambda i, j: pid[(max(i, j), min(i, j))]
    bound = np.array([Q[key(a, bb)] * Q[key(c, d)] for a, bb, c, d in q])
    v0, off0 = eng.eri4(db, q)
    tau = float(np.quantile(bound, 0.4))
    v1, off1 = eng.eri4(db, q, bound=bound, tau=tau)
    v2, off2 = eng.eri4(db, q, bound=bound, tau=0.0)
    torch.cuda.synchronize()
    assert torch.equal(off0, off1) and torch.equal(off0, off2)
    off = off0.cpu().numpy()
    v0, v1, v2 = v0.cpu().numpy(), v1.cpu().numpy(), v2.cpu().numpy()
    assert np.array_equal(v0[: off[-1]], v2[: off[-1]])
    dropped = bound < tau
    assert 0 < dropped.sum() < len(q)
    for n in range(len(q)):
        a, z = off[n], off[n + 1]
        if dropped[n]:
            assert np.all(v1[a:z] == 0.0)
            # the bound holds: the dropped integrals are below it
            assert np.max(np.abs(v0[a:z])) <= bound[n] * (1 + 1e-12)
        else:
            assert np.array_equal(v1[a:z], v0[a:z])
    with pytest.raises(mdx.MdxError, match="EINVAL"):
        eng.eri4(db, q, bound=bound, tau=-1.0)


def test_bound_screens_triplets(eng):
    """mdx_eri3's bound input, as mdx_eri4's."""
    aux, orb = inputs.df_cluster(seed=11, n_atoms=2)
    t = np.array([[a, c, d] for a in range(0, aux.n_shells, 3) for c in range(orb.n_shells) for d in range(c + 1)][:300],
                 dtype=np.int32)
    rng = np.random.Generator(np.random.PCG64(4))
    bound = rng.uniform(0, 1, len(t))
    daux, dorb = mdx.DeviceBasis(aux), mdx.DeviceBasis(orb)
    v0, off = eng.eri3(daux, dorb, t)
    v1, _ = eng.eri3(daux, dorb, t, bound=bound, tau=0.5)
    torch.cuda.synchronize()
    off = off.cpu().numpy()
    v0, v1 = v0.cpu().numpy(), v1.cpu().numpy()
    for n in range(len(t)):
        a, z = off[n], off[n + 1]
        if bound[n] < 0.5:
            assert np.all(v1[a:z] == 0.0)
        else:
            assert np.array_equal(v1[a:z], v0[a:z])


@pytest.mark.parametrize("lq,K,nb,nk", [((6, 6, 6, 6), (1, 1, 1, 1), 24, 19), ((5, 5, 5, 5), (1, 1, 5, 1), 12, 10),
                                        ((4, 0, 4, 0), (1, 1, 1, 1), 64, 64)])
def test_solid_harmonic_rotation_invariance_at_scale(lq, K, nb, nk):
    """A property that holds at any size: rotating the whole geometry leaves the Frobenius norm of every
    solid-harmonic shellset unchanged (the harmonics of each l map onto one another orthogonally). Checked
    on the GPU for every shellset of a batch the size of one benchmark chunk ([ii|ii]: 456 quartets), with
    the autotuned shape."""
    e = mdx.Engine(0)
    b, q = inputs.class_sweep(lq, n_bra=nb, n_ket=nk, seed=33, K=K, box=3.0, zlo=0.2, zhi=5.0)
    rng = np.random.Generator(np.random.PCG64(34))
    R, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    norms = []
    for rot in (False, True):
        bb, _ = inputs.class_sweep(lq, n_bra=nb, n_ket=nk, seed=33, K=K, box=3.0, zlo=0.2, zhi=5.0)
        if rot:
            bb.center = np.ascontiguousarray(bb.center @ R.T)
        bt = e.batch_eri4_sph(mdx.DeviceBasis(bb), q)
        out = torch.empty(bt.total, dtype=torch.float64, device="cuda")
        bt.autotune(out, max_trial=len(q))
        bt.run(out)
        off = bt.offsets()
        torch.cuda.synchronize()
        e.sync()
        per = int(off[1] - off[0])
        norms.append(out.view(-1, per).norm(dim=1).cpu().numpy())
        bt.close()
    big = norms[0] > 1e-8 * norms[0].max()
    np.testing.assert_allclose(norms[1][big], norms[0][big], rtol=1e-11)
    e.close()


def _basis_3c_sph(la, lc, ld, K, seed, n=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    aux, orb = inputs.BasisBuilder(), inputs.BasisBuilder()
    for _ in range(n):
        inputs.random_shell(rng, aux, la, rng.uniform(0, 3.0, 3), K[0], 0.2, 5.0)
        inputs.random_shell(rng, orb, lc, rng.uniform(0, 3.0, 3), K[1], 0.2, 5.0)
        inputs.random_shell(rng, orb, ld, rng.uniform(0, 3.0, 3), K[2], 0.2, 5.0)
    trip = np.array([[a, 2 * k, 2 * k + 1] for a in range(n) for k in range(n)], dtype=np.int32)
    return aux.build(), orb.build(), trip


@pytest.mark.parametrize("la,lc,ld,K", [(5, 0, 0, (1, 6, 6)), (6, 1, 0, (1, 6, 3)), (4, 1, 1, (1, 3, 3)),
                                        (2, 2, 1, (1, 1, 3))])
def test_three_center_batch_autotuned(la, lc, ld, K):
    """A Cartesian [a|cd] batch after the autotuner (register kernel or team shapes of the one-centre classes,
    as the density-fitting benchmark tunes them) against the oracle. Own context: the tuned shapes stay
    with it."""
    aux, orb, trip = _basis_3c_sph(la, lc, ld, K, 61 + la + lc)
    e = mdx.Engine(0)
    bt = e.batch_eri3(mdx.DeviceBasis(aux), mdx.DeviceBasis(orb), trip)
    w = torch.full((bt.total,), float("nan"), dtype=torch.float64, device="cuda")
    bt.autotune(w, max_trial=len(trip))
    bt.run(w)
    torch.cuda.synchronize()
    e.sync()
    ref, roff = oracle.eri3(aux, orb, trip)
    assert np.array_equal(bt.offsets().cpu().numpy(), roff)
    print(parity.check(w.cpu().numpy(), ref, roff, "tuned 3c [%d|%d%d]" % (la, lc, ld),
                       parity.Eri3Evaluator(aux, orb, trip)))
    bt.close()
    e.close()


@pytest.mark.parametrize("la,lc,ld,K", [(1, 0, 0, (1, 3, 1)), (3, 2, 1, (1, 3, 1)), (6, 0, 0, (1, 6, 6)),
                                        (4, 3, 3, (1, 1, 1)), (6, 3, 3, (1, 1, 1)), (2, 4, 4, (1, 1, 3)),
                                        (5, 5, 5, (1, 1, 1)), (6, 6, 6, (1, 1, 1))])
def test_solid_harmonic_eri3(eng, la, lc, ld, K):
    """mdx_eri3_sph (and its prepared batch, autotuned) against the oracle's solid-harmonic [a|cd]:
    register-kernel classes transformed index by index, team-kernel classes with the coefficients
    contracted into the transforms (one-centre bra)."""
    aux, orb, trip = _basis_3c_sph(la, lc, ld, K, 41 + la + lc)
    da, do = mdx.DeviceBasis(aux), mdx.DeviceBasis(orb)
    v, off = eng.eri3_sph(da, do, trip)
    torch.cuda.synchronize()
    ref, roff = oracle.eri3_sph(aux, orb, trip)
    assert np.array_equal(off.cpu().numpy(), roff)
    ev = parity.Eri3SphEvaluator(aux, orb, trip)
    print(parity.check(v.cpu().numpy()[: roff[-1]], ref, roff, "solid [%d|%d%d]" % (la, lc, ld), ev))
    e = mdx.Engine(0)
    bt = e.batch_eri3_sph(da, do, trip)
    w = torch.full((bt.total,), float("nan"), dtype=torch.float64, device="cuda")
    bt.autotune(w, max_trial=len(trip))
    bt.run(w)
    torch.cuda.synchronize()
    e.sync()
    print(parity.check(w.cpu().numpy(), ref, roff, "solid batch [%d|%d%d]" % (la, lc, ld), ev))
    bt.close()
    e.close()
