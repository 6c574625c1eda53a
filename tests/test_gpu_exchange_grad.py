"""GPU exchange-energy gradient (shifted-class derivative integrals contracted with
D (x) D in the kernel) against the oracle's explicit gradient and central finite differences."""
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


def _grad(eng, b, D, tau=0.0, alpha=-1.0):
    db = mdx.DeviceBasis(b)
    pairs = _pairs(b)
    Q = eng.schwarz(db, pairs)
    g, e = eng.exchange_grad(db, pairs, Q, torch.from_numpy(D), tau=tau, alpha=alpha, n_atoms=b.n_atoms)
    torch.cuda.synchronize()
    return g.cpu().numpy(), float(e.cpu())


@pytest.mark.parametrize("shells,K,natoms", [((0, 1, 2), 2, 3), ((1, 3), 1, 2), ((0, 2, 4), 1, 2)])
def test_gradient_matches_oracle(eng, shells, K, natoms):
    b = inputs.small_molecule(seed=51 + len(shells), n_atoms=natoms, shells=shells, K=K)
    D = inputs.density(b.nao, 10, occ_fraction=0.4)
    g, E = _grad(eng, b, D)
    ref = -oracle.exchange_grad(b, D)
    Eref = -oracle.exchange_energy(b, D)
    scale = np.max(np.abs(ref))
    np.testing.assert_allclose(g, ref, rtol=0, atol=1e-11 * max(scale, 1e-3))
    assert abs(E - Eref) <= 1e-11 * abs(Eref)
    np.testing.assert_allclose(g.sum(axis=0), 0.0, atol=1e-12 * max(scale, 1e-3))


def _energy(eng, b, D):
    """E_x = -sum D o K through the forward exchange build (independent of the gradient code)."""
    db = mdx.DeviceBasis(b)
    pairs = _pairs(b)
    Q = eng.schwarz(db, pairs)
    K = eng.exchange(db, pairs, Q, torch.from_numpy(D), 0.0)
    return -float(torch.sum(torch.from_numpy(D).cuda() * K).cpu())


def test_gradient_against_finite_differences(eng):
    """Central differences (h = 1e-4 bohr) of the GPU forward energy, every atom and axis of a
    contracted heavy/light molecule (the batched-exchange and gradient molecules)."""
    b = inputs.molecule(seed=61, n_atoms=3)
    D = inputs.density(b.nao, 11)
    g, E = _grad(eng, b, D)
    assert abs(E - _energy(eng, b, D)) <= 1e-11 * abs(E)
    h = 1e-4
    for A in range(b.n_atoms):
        for x in range(3):
            vals = []
            for d in (h, -h):
                bb = inputs.molecule(seed=61, n_atoms=3)
                bb.center = bb.center.copy()
                bb.center[bb.atom == A, x] += d
                vals.append(_energy(eng, bb, D))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(g[A, x] - fd) <= 2e-7 * max(1.0, abs(fd)), (A, x, g[A, x], fd)


def test_autograd_function(eng):
    """torch.autograd through ExchangeEnergy: d/dcoords = mdx_exchange_grad, d/dD = 2 alpha K."""
    b = inputs.small_molecule(seed=71, n_atoms=3, shells=(0, 1, 2), K=2)
    D = torch.from_numpy(inputs.density(b.nao, 12)).cuda().requires_grad_(True)
    coords = torch.from_numpy(b.atoms).cuda().requires_grad_(True)
    db = mdx.DeviceBasis(b)
    E = mdx.exchange_energy(eng, db, coords, D, alpha=-1.0)
    gc, gD = torch.autograd.grad(E, (coords, D))
    ref_g = -oracle.exchange_grad(b, D.detach().cpu().numpy())
    np.testing.assert_allclose(gc.cpu().numpy(), ref_g, rtol=0, atol=1e-11 * np.max(np.abs(ref_g)))
    K = oracle.exchange(b, D.detach().cpu().numpy())
    np.testing.assert_allclose(gD.cpu().numpy(), -2.0 * K, rtol=0, atol=1e-11 * np.max(np.abs(K)))
    E = float(E.detach())
    assert abs(E + float(np.sum(D.detach().cpu().numpy() * K))) <= 1e-11 * abs(E)


def test_gradient_ten_atom_cluster_fd_eight_atoms(eng):
    """The 400-atom gradient workload at reduced size: a 10-atom heavy/light cluster (quadruple-zeta-like shells,
    Schwarz x density screening at 1e-11); dE_x/dR against central differences of the GPU forward
    energy on 8 seeded atoms (one seeded axis each), and translational invariance."""
    b = inputs.molecule(seed=1005, n_atoms=10)
    D = inputs.density(b.nao, 1005)
    tau = 1e-11
    db = mdx.DeviceBasis(b)
    pairs = _pairs(b)
    Q = eng.schwarz(db, pairs)
    g, E = eng.exchange_grad(db, pairs, Q, torch.from_numpy(D), tau=tau, alpha=-1.0, n_atoms=b.n_atoms)
    g = g.cpu().numpy()
    np.testing.assert_allclose(g.sum(axis=0), 0.0, atol=1e-9 * np.max(np.abs(g)))
    rng = np.random.Generator(np.random.PCG64(1005))
    atoms = rng.choice(b.n_atoms, 8, replace=False)
    axes = rng.integers(0, 3, 8)
    h = 1e-4

    def energy(bb):
        dbb = mdx.DeviceBasis(bb)
        Qb = eng.schwarz(dbb, pairs)
        K = eng.exchange(dbb, pairs, Qb, torch.from_numpy(D), tau)
        return -float(torch.sum(torch.from_numpy(D).cuda() * K).cpu())

    for A, x in zip(atoms, axes):
        vals = []
        for d in (h, -h):
            bb = inputs.molecule(seed=1005, n_atoms=10)
            bb.center = bb.center.copy()
            bb.center[bb.atom == A, x] += d
            vals.append(energy(bb))
        fd = (vals[0] - vals[1]) / (2 * h)
        # screening at tau moves E by far less than the FD resolution here
        assert abs(g[A, x] - fd) <= 1e-6 * max(1.0, abs(fd)), (A, x, g[A, x], fd)


def test_autograd_with_cpu_coordinates(eng):
    """Coordinates on the host in float32: the centres go to the device in float64, and the gradient
    comes back on the host in float32."""
    b = inputs.small_molecule(seed=72, n_atoms=2, shells=(0, 1), K=2)
    D = torch.from_numpy(inputs.density(b.nao, 13)).cuda()
    coords = torch.from_numpy(b.atoms).to(torch.float32).requires_grad_(True)
    db = mdx.DeviceBasis(b)
    E = mdx.exchange_energy(eng, db, coords, D, alpha=-1.0)
    (gc,) = torch.autograd.grad(E, (coords,))
    assert gc.device.type == "cpu" and gc.dtype == torch.float32
    bf = inputs.small_molecule(seed=72, n_atoms=2, shells=(0, 1), K=2)
    bf.center = coords.detach().double().numpy()[bf.atom]
    ref = -oracle.exchange_grad(bf, D.cpu().numpy())
    np.testing.assert_allclose(gc.numpy(), ref, rtol=0, atol=1e-6 * np.max(np.abs(ref)))


def test_autograd_rejects_asymmetric_density(eng):
    b = inputs.small_molecule(seed=73, n_atoms=2, shells=(0, 1), K=1)
    D = torch.from_numpy(inputs.density(b.nao, 14)).cuda()
    D[0, 1] += 1e-3
    with pytest.raises(mdx.MdxError, match="symmetric"):
        mdx.exchange_energy(eng, mdx.DeviceBasis(b), torch.from_numpy(b.atoms).cuda(), D)


def test_gradient_ten_atoms_against_the_oracle(eng):
    """The oracle's exchange-energy gradient on ten atoms (s, p, d shells in a 9-bohr box, every unique
    quartet): all 30 components and the energy at the parity bar. (The quadruple-zeta-like shells of the
    cluster workload would take the CPU oracle hours at ten atoms; their gradient is checked against
    central differences above.)"""
    b = inputs.small_molecule(seed=1010, n_atoms=10, box=9.0, shells=(0, 1, 2), K=1)
    D = inputs.density(b.nao, 1010)
    g, E = _grad(eng, b, D)
    ref = -oracle.exchange_grad(b, D)
    Eref = -oracle.exchange_energy(b, D)
    scale = np.max(np.abs(ref))
    np.testing.assert_allclose(g, ref, rtol=0, atol=1e-11 * scale)
    assert abs(E - Eref) <= 1e-11 * abs(Eref)
