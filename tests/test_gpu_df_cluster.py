"""Density-fitting cluster at full size: 100 atoms, orbital 4s3p2d1f (K 6/3/1/1), auxiliary s..i.
Schwarz factors of all 500,500 orbital shell pairs on the GPU (checked on a sample against the
oracle), pairs screened at Q >= 1e-12, then a seeded sample of [a|cd] triplets over the kept
pairs and every auxiliary class compared with the oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import parity
from paper_2405_01834_gb300 import inputs, mdx

pytestmark = pytest.mark.gpu


def test_df_cluster_full_size_sampled():
    eng = mdx.Engine(0)
    aux, orb = inputs.df_cluster()
    assert orb.n_atoms == 100 and orb.n_shells == 1000 and aux.n_shells == 2300
    dorb, daux = mdx.DeviceBasis(orb), mdx.DeviceBasis(aux)
    ii, jj = np.tril_indices(orb.n_shells)
    pairs = np.stack([ii, jj], axis=1).astype(np.int32)
    Q = eng.schwarz(dorb, pairs).cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(3003))
    pick = rng.choice(len(pairs), 300, replace=False)
    q4 = np.array([(i, j, i, j) for i, j in pairs[pick]], dtype=np.int32)
    ref, off = oracle.eri4(orb, q4)
    refQ = [np.sqrt(np.max(np.abs(np.diag(ref[off[n]:off[n + 1]].reshape(int(np.sqrt(off[n + 1] - off[n])), -1)))))
            for n in range(len(pick))]
    np.testing.assert_allclose(Q[pick], refQ, rtol=1e-12, atol=0)
    kept = pairs[Q >= 1e-12]
    assert 0 < len(kept) < len(pairs)
    # one sample per auxiliary angular momentum, several pairs each
    trip = []
    for la in range(7):
        a_sh = rng.choice(np.where(aux.l == la)[0], 4, replace=False)
        for a in a_sh:
            for c, d in kept[rng.choice(len(kept), 12, replace=False)]:
                trip.append((a, c, d))
    trip = np.array(trip, dtype=np.int32)
    v, voff = eng.eri3(daux, dorb, trip)
    torch.cuda.synchronize()
    r3, r3off = oracle.eri3(aux, orb, trip)
    print(parity.check(v.cpu().numpy()[: r3off[-1]], r3, r3off, "df cluster", parity.Eri3Evaluator(aux, orb, trip)))
    eng.close()
