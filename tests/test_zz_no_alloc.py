"""mdx_eri4_noalloc (C ABI) against mdx_eri4.

Callers whose device memory is owned by their own pool or budget cannot let a
library call cudaMalloc; mdx_eri4_noalloc serves them from a fixed 32 MiB
__device__ scratch array. This file is collected last on purpose: it must pass
alone in a fresh process (first call sets the device up) and after the other
GPU tests.
"""
import numpy as np
import pytest
import torch

from oracle import parity
from paper_2405_01834_gb300 import inputs, mdx

pytestmark = pytest.mark.gpu


def _cases():
    b1 = inputs.small_molecule(seed=17, n_atoms=3)            # s,p,d shells, K = 3
    q1 = inputs.unique_quartets(b1.n_shells)
    b2, q2 = inputs.class_sweep((4, 2, 3, 1), n_bra=6, n_ket=5, seed=23, K=(1, 2, 1, 3))
    return [(b1, q1), (b2, q2)]


@pytest.mark.parametrize("case", [0, 1])
def test_noalloc_matches_eri4_twice(case):
    b, q = _cases()[case]
    eng = mdx.Engine(0)
    db = mdx.DeviceBasis(b)
    ref, ref_off = eng.eri4(db, q)
    torch.cuda.synchronize()
    total = int(ref_off[-1])
    for _ in range(2):   # two calls in a row: the shared scratch is reused
        out = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
        st, off = mdx.eri4_noalloc(db, q, out)
        torch.cuda.synchronize()
        assert st == 0, mdx.STATUS.get(st, st)
        assert torch.equal(off, ref_off)
        print(parity.check(out.cpu().numpy(), ref[:total].cpu().numpy(), off.cpu().numpy(), "noalloc vs eri4"))
    eng.close()


def test_noalloc_rejects_oversize_request():
    """A request needing more than the 32 MiB scratch is refused cleanly; the next call works."""
    # [ss|ss] with 32 primitives per shell: 200 shell pairs x 1024 primitive-pair
    # records x 2 copies x 96 bytes = 39 MB of records for a 80 KB output
    b, q = inputs.class_sweep((0, 0, 0, 0), n_bra=100, n_ket=100, seed=3, K=(32, 32, 32, 32))
    db = mdx.DeviceBasis(b)
    out = torch.empty(len(q) - 1, dtype=torch.float64, device="cuda")
    st, _ = mdx.eri4_noalloc(db, q, out)
    assert mdx.STATUS[st] == "MDX_ECAPACITY"          # output too small: checked first
    out = torch.empty(len(q), dtype=torch.float64, device="cuda")
    st, _ = mdx.eri4_noalloc(db, q, out)
    assert mdx.STATUS[st] == "MDX_ESCRATCH"
    b2 = inputs.small_molecule(seed=18, n_atoms=2)
    q2 = inputs.unique_quartets(b2.n_shells)[:50]
    db2 = mdx.DeviceBasis(b2)
    eng = mdx.Engine(0)
    ref, ref_off = eng.eri4(db2, q2)
    out = torch.empty(int(ref_off[-1]), dtype=torch.float64, device="cuda")
    st, off = mdx.eri4_noalloc(db2, q2, out)
    torch.cuda.synchronize()
    assert st == 0
    print(parity.check(out.cpu().numpy(), ref[: int(ref_off[-1])].cpu().numpy(), off.cpu().numpy(),
                       "noalloc after refusal"))
    eng.close()
