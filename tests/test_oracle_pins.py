"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names the passage of Asadchev & Valeev (arXiv:2405.01834) whose
formula it checks and the independent fact it checks it against: closed
forms, mpmath quadrature / differentiation at 30 digits, textbook special
cases, invariants of the integrals and an independent Obara-Saika recursion.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2405_01834_gb300 import inputs

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 30

rng0 = np.random.Generator(np.random.PCG64(4242))


# ------------------------------------------------------------------ Boys (Eq. boys)
def test_boys_at_zero():
    F = oracle.boys(25, 0.0)
    np.testing.assert_allclose(F, [1.0 / (2 * m + 1) for m in range(26)], rtol=1e-15, atol=0)


@pytest.mark.parametrize("T", [1e-8, 1e-3, 0.3, 1.0, 7.5, 29.0, 31.0, 44.0, 120.0, 900.0])
def test_boys_f0_is_erf(T):
    ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert abs(oracle.boys(0, T)[0] - ref) <= 2e-15 * ref


@pytest.mark.parametrize("T", [0.0, 2e-4, 0.37, 3.3, 12.0, 29.5, 30.5, 54.9, 55.1, 56.0, 80.0, 250.0])
def test_boys_against_incomplete_gamma(T):
    """F_m(T) = gamma(m+1/2, T) / (2 T^(m+1/2)), the closed form of Eq. boys via the
    lower incomplete gamma function (mpmath, 30 digits); F_m(0) = 1/(2m+1)."""
    F = oracle.boys(25, T)
    for m in range(26):
        if T == 0.0:
            ref = 1.0 / (2 * m + 1)
        else:
            ref = float(mpmath.gammainc(m + 0.5, 0, T) / (2 * mpmath.mpf(T) ** (m + 0.5)))
        assert abs(F[m] - ref) <= 5e-15 * abs(ref), (m, F[m], ref)


@pytest.mark.parametrize("T", [0.37, 5.0, 29.5])
def test_boys_against_quadrature(T):
    """F_m(T) = int_0^1 y^2m exp(-T y^2) dy (Eq. boys) by mpmath quadrature, for
    moderate T where the integrand is not sharply peaked."""
    F = oracle.boys(12, T)
    for m in range(13):
        ref = float(mpmath.quad(lambda y: y ** (2 * m) * mpmath.exp(-T * y * y), [0, 0.25, 0.5, 0.75, 1]))
        assert abs(F[m] - ref) <= 5e-15 * abs(ref), (m, F[m], ref)


def test_boys_recursion_consistency():
    """Downward recursion F_m = (2T F_{m+1} + e^-T)/(2m+1) holds for the oracle's values."""
    for T in [0.01, 1.0, 10.0, 29.0, 35.0, 60.0]:
        F = oracle.boys(24, T)
        for m in range(24):
            lhs = F[m]
            rhs = (2 * T * F[m + 1] + math.exp(-T)) / (2 * m + 1)
            assert abs(lhs - rhs) <= 4e-15 * lhs


def test_boys_long_double_agrees():
    for T in np.concatenate([np.linspace(0, 40, 81), [55.0, 70.0, 200.0]]):
        a = oracle.boys(25, T, 0)
        b = oracle.boys(25, T, 1)
        np.testing.assert_allclose(a, b, rtol=3e-15, atol=0)


# ------------------------------------------------------------------ E coefficients
def hermite_gaussian(t, p, xP):
    """Lambda_t = (d/dP)^t exp(-p (x-P)^2) = p^(t/2) H_t(sqrt(p) xP) exp(-p xP^2)."""
    c = np.zeros(t + 1); c[t] = 1.0
    return p ** (t / 2) * np.polynomial.hermite.hermval(math.sqrt(p) * xP, c) * np.exp(-p * xP * xP)


@pytest.mark.parametrize("la,lb", [(0, 0), (1, 0), (0, 1), (2, 1), (1, 3), (4, 4), (6, 6)])
def test_e2c_reproduces_gaussian_product(la, lb):
    """Eq. cart2herm-2 along one axis: x_A^i x_B^j exp(-a x_A^2 - b x_B^2) = sum_t E_ij^t Lambda_t."""
    rng = np.random.Generator(np.random.PCG64(100 + 10 * la + lb))
    for _ in range(3):
        za, zb = np.exp(rng.uniform(np.log(0.2), np.log(5.0), 2))
        A, B = rng.uniform(-1.0, 1.0, 2)
        p = za + zb
        P = (za * A + zb * B) / p
        E = oracle.e2c(la, lb, za, zb, A, B)
        xs = P + rng.uniform(-1.5, 1.5, 7) / math.sqrt(p)
        for i in range(la + 1):
            for j in range(lb + 1):
                lhs = (xs - A) ** i * (xs - B) ** j * np.exp(-za * (xs - A) ** 2 - zb * (xs - B) ** 2)
                rhs = sum(E[i, j, t] * hermite_gaussian(t, p, xs - P) for t in range(i + j + 1))
                scale = max(1.0, np.max(np.abs(lhs)))
                np.testing.assert_allclose(rhs, lhs, rtol=0, atol=1e-12 * scale)
                # zero above i+j (Eq. E2-abp)
                assert np.all(E[i, j, i + j + 1:] == 0)


@pytest.mark.parametrize("la", [0, 1, 2, 3, 6])
def test_e1c_reproduces_cartesian(la):
    """Eq. cart2herm-1 along one axis: x^a exp(-z x^2) = sum_t E_a^t Lambda_t, zero for odd a+t."""
    z = 0.73
    E = oracle.e1c(la, z)
    xs = np.linspace(-2, 2, 9)
    for a in range(la + 1):
        lhs = xs ** a * np.exp(-z * xs * xs)
        rhs = sum(E[a, t] * hermite_gaussian(t, z, xs) for t in range(a + 1))
        np.testing.assert_allclose(rhs, lhs, rtol=0, atol=1e-13)
        for t in range(la + 1):
            if (a + t) % 2 == 1 or t > a:
                assert E[a, t] == 0.0


def test_e2c_top_hermite():
    """Eq. E2-abab: E_ab^(a+b) = E_00^0 / (2 zeta_p)^(a+b)."""
    za, zb, A, B = 0.9, 2.3, 0.1, -0.8
    p = za + zb
    E = oracle.e2c(6, 6, za, zb, A, B)
    for i in range(7):
        for j in range(7):
            assert abs(E[i, j, i + j] - E[0, 0, 0] / (2 * p) ** (i + j)) <= 1e-15 * abs(E[0, 0, 0]) / (2 * p) ** (i + j) * 4


def test_e2c_overlap_integral():
    """E_ij^0 sqrt(pi/p) is the 1-D overlap integral (quadrature of the definition)."""
    from scipy.integrate import quad
    za, zb, A, B = 1.3, 0.4, 0.25, -0.6
    p = za + zb
    E = oracle.e2c(3, 3, za, zb, A, B)
    for i in range(4):
        for j in range(4):
            f = lambda x: (x - A) ** i * (x - B) ** j * math.exp(-za * (x - A) ** 2 - zb * (x - B) ** 2)
            ref = quad(f, -12, 12, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
            assert abs(E[i, j, 0] * math.sqrt(math.pi / p) - ref) <= 1e-13


# ------------------------------------------------------------------ R (Eqs. 0m, r)
@pytest.mark.parametrize("L", [0, 1, 3, 5])
def test_rtable_is_derivative_of_f0(L):
    """[tuv]^(0) / pref = d^t/dX d^u/dY d^v/dZ F_0(rho (X^2+Y^2+Z^2)) at X = P-Q."""
    rho = 0.8
    PQ = np.array([0.31, -0.52, 0.77])
    R = oracle.rtable(L, rho, PQ)

    def F0(X, Y, Z):
        T = rho * (X * X + Y * Y + Z * Z)
        return mpmath.sqrt(mpmath.pi) / 2 * mpmath.erf(mpmath.sqrt(T)) / mpmath.sqrt(T)

    scale = np.max(np.abs(R))
    for t in range(L + 1):
        for u in range(L + 1 - t):
            for v in range(L + 1 - t - u):
                ref = float(mpmath.diff(F0, (mpmath.mpf(PQ[0]), mpmath.mpf(PQ[1]), mpmath.mpf(PQ[2])), (t, u, v)))
                assert abs(R[t, u, v] - ref) <= 1e-12 * scale, (t, u, v, R[t, u, v], ref)


# ------------------------------------------------------------------ whole integrals
def _two_shell_basis(specs):
    bb = inputs.BasisBuilder()
    for l, xyz, z, c in specs:
        bb.add_shell(l, xyz, z, c)
    return bb.build()


def test_ssss_closed_form():
    """(ss|ss) = 2 pi^(5/2)/(p q sqrt(p+q)) exp(-mu_ab AB^2) exp(-mu_cd CD^2) F_0(rho PQ^2)."""
    rng = np.random.Generator(np.random.PCG64(7))
    for _ in range(10):
        cen = rng.uniform(-2, 2, (4, 3))
        z = np.exp(rng.uniform(np.log(0.05), np.log(50), 4))
        b = _two_shell_basis([(0, cen[i], [z[i]], [1.0]) for i in range(4)])
        v, _ = oracle.eri4(b, [[0, 1, 2, 3]])
        p, q = z[0] + z[1], z[2] + z[3]
        P = (z[0] * cen[0] + z[1] * cen[1]) / p
        Q = (z[2] * cen[2] + z[3] * cen[3]) / q
        rho = p * q / (p + q)
        T = rho * np.sum((P - Q) ** 2)
        F0 = 1.0 if T < 1e-300 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
        ref = (2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * math.exp(-z[0] * z[1] / p * np.sum((cen[0] - cen[1]) ** 2))
               * math.exp(-z[2] * z[3] / q * np.sum((cen[2] - cen[3]) ** 2)) * F0)
        assert abs(v[0] - ref) <= 1e-14 * abs(ref)


OS_CASES = [
    ((0, 0, 0, 0), 1), ((1, 0, 0, 0), 1), ((0, 0, 1, 0), 1), ((0, 1, 0, 0), 1), ((0, 0, 0, 1), 1),
    ((1, 1, 1, 1), 1), ((2, 1, 0, 1), 2), ((1, 0, 2, 1), 2), ((2, 2, 2, 2), 1), ((3, 0, 1, 2), 1),
    ((0, 3, 2, 0), 1), ((3, 3, 0, 0), 1), ((4, 0, 0, 2), 1),
]


@pytest.mark.parametrize("lq,K", OS_CASES)
def test_eri4_against_obara_saika(lq, K):
    """Contracted [ab|cd] (Eqs. def-abcd, 3) against the independent OS/HGP recursion."""
    import os_reference as osr
    rng = np.random.Generator(np.random.PCG64(hash(lq) % 2**32 + K))
    specs = []
    for l in lq:
        z = np.exp(rng.uniform(np.log(0.1), np.log(8.0), K))
        c = rng.uniform(0.2, 1.0, K) * inputs.primitive_norm(l, z)
        specs.append((l, rng.uniform(-1.5, 1.5, 3), z, c))
    b = _two_shell_basis(specs)
    v, _ = oracle.eri4(b, [[0, 1, 2, 3]])
    ref = np.array(osr.eri4_shellset(*lq, *[s[1] for s in specs],
                                     *[x for s in specs for x in (list(s[2]), list(s[3]))])).reshape(-1)
    scale = np.max(np.abs(ref))
    np.testing.assert_allclose(v, ref, rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("la,lc,ld", [(0, 0, 0), (1, 0, 0), (0, 1, 1), (2, 1, 0), (3, 2, 1), (4, 1, 1), (6, 0, 0)])
def test_eri3_against_obara_saika(la, lc, ld):
    """[a|cd] (Eq. def-acd, 1-center bra via Eq. E1rr) against OS with phi_b = 1."""
    import os_reference as osr
    rng = np.random.Generator(np.random.PCG64(31 * la + 7 * lc + ld))
    za = [float(np.exp(rng.uniform(np.log(0.1), np.log(5.0))))]
    ca = [1.3]
    aux = _two_shell_basis([(la, rng.uniform(-1, 1, 3), za, ca)])
    specs = []
    for l in (lc, ld):
        z = np.exp(rng.uniform(np.log(0.1), np.log(8.0), 2))
        specs.append((l, rng.uniform(-1.5, 1.5, 3), z, rng.uniform(0.2, 1.0, 2)))
    orb = _two_shell_basis(specs)
    v, _ = oracle.eri3(aux, orb, [[0, 0, 1]])
    ref = np.array(osr.eri3_shellset(la, lc, ld, aux.center[0], specs[0][1], specs[1][1], za, ca,
                                     list(specs[0][2]), list(specs[0][3]),
                                     list(specs[1][2]), list(specs[1][3]))).reshape(-1)
    scale = np.max(np.abs(ref))
    np.testing.assert_allclose(v, ref, rtol=0, atol=1e-12 * scale)


def _random_basis(ls, seed, K=2):
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for l in ls:
        z = np.exp(rng.uniform(np.log(0.1), np.log(8.0), K))
        specs.append((l, rng.uniform(-1.5, 1.5, 3), z, rng.uniform(0.2, 1.0, K) * inputs.primitive_norm(l, z)))
    return _two_shell_basis(specs), specs


def _shellset(b, q):
    v, _ = oracle.eri4(b, [q])
    return v.reshape([inputs.ncart(int(b.l[s])) for s in q])


def test_permutational_symmetry():
    """The 8 index permutations of (ab|cd) are transposes of one another (Eq. def-abcd)."""
    b, _ = _random_basis([2, 1, 3, 0], 11)
    ref = _shellset(b, [0, 1, 2, 3])
    np.testing.assert_allclose(_shellset(b, [1, 0, 2, 3]), ref.transpose(1, 0, 2, 3), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(_shellset(b, [0, 1, 3, 2]), ref.transpose(0, 1, 3, 2), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(_shellset(b, [2, 3, 0, 1]), ref.transpose(2, 3, 0, 1), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(_shellset(b, [3, 2, 1, 0]), ref.transpose(3, 2, 1, 0), rtol=1e-12, atol=1e-15)


def test_translation_invariance():
    b, _ = _random_basis([2, 2, 1, 1], 12)
    ref = _shellset(b, [0, 1, 2, 3])
    b.center = b.center + np.array([3.7, -1.1, 0.45])
    np.testing.assert_allclose(_shellset(b, [0, 1, 2, 3]), ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))


def test_axis_permutation_covariance():
    """Swapping x and y coordinates swaps a_x and a_y in every Cartesian component."""
    ls = [2, 1, 1, 2]
    b, _ = _random_basis(ls, 13)
    ref = _shellset(b, [0, 1, 2, 3])
    b.center = b.center[:, [1, 0, 2]].copy()
    sw = _shellset(b, [0, 1, 2, 3])
    perms = []
    for l in ls:
        comps = [(ax, ay, l - ax - ay) for ax in range(l, -1, -1) for ay in range(l - ax, -1, -1)]
        perms.append([comps.index((c[1], c[0], c[2])) for c in comps])
    ref_sw = ref[np.ix_(*perms)]
    np.testing.assert_allclose(sw, ref_sw, rtol=0, atol=1e-13 * np.max(np.abs(ref)))


def test_far_separation_limit():
    """[ss|ss] -> S_ab S_cd / R for bra and ket distributions far apart."""
    z = [0.7, 1.9, 0.4, 1.1]
    Rsep = 500.0
    cen = [np.zeros(3), np.array([0.3, 0, 0]), np.array([Rsep, 0.2, 0]), np.array([Rsep, -0.1, 0.3])]
    b = _two_shell_basis([(0, cen[i], [z[i]], [1.0]) for i in range(4)])
    v, _ = oracle.eri4(b, [[0, 1, 2, 3]])
    def S(za, zb, A, B):
        p = za + zb
        return (math.pi / p) ** 1.5 * math.exp(-za * zb / p * np.sum((A - B) ** 2))
    P = (z[0] * cen[0] + z[1] * cen[1]) / (z[0] + z[1])
    Q = (z[2] * cen[2] + z[3] * cen[3]) / (z[2] + z[3])
    ref = S(z[0], z[1], cen[0], cen[1]) * S(z[2], z[3], cen[2], cen[3]) / np.linalg.norm(P - Q)
    assert abs(v[0] - ref) <= 1e-13 * ref


def test_long_double_certifies_double():
    """The FP64 oracle agrees with its long-double build on a mixed sample.

    Scale is the largest integral of the sample: some shellsets here vanish by
    symmetry (odd one-centre classes such as [ds|ps] on one atom), where FP64
    leaves ~1e-15 of rounding noise on an exact zero."""
    b = inputs.small_molecule(seed=5, n_atoms=3)
    q = inputs.unique_quartets(b.n_shells)[::7]
    v, off = oracle.eri4(b, q, precision=0)
    w, _ = oracle.eri4(b, q, precision=1)
    M = np.max(np.abs(w))
    assert np.max(np.abs(v - w)) <= 1e-13 * M
    big = np.abs(w) > 1e-10 * M
    assert np.max(np.abs(v - w)[big] / np.abs(w)[big]) <= 1e-10


# ------------------------------------------------------------------ exchange (Sec. 6)
def test_exchange_digestion_matches_einsum():
    """K_ik = sum_jl D_jl (ij|kl): the oracle digestion against an einsum over the
    full AO integral tensor assembled shell by shell, symmetric K, Tr(DK) > 0."""
    b = inputs.small_molecule(seed=9, n_atoms=2, shells=(0, 1), K=2)
    nao = b.nao
    ns = b.n_shells
    full = np.zeros((nao,) * 4)
    quart = np.array([[i, j, k, l] for i in range(ns) for j in range(ns) for k in range(ns) for l in range(ns)],
                     dtype=np.int32)
    v, off = oracle.eri4(b, quart)
    nc = [inputs.ncart(int(x)) for x in b.l]
    ao = b.ao_off
    for n, (i, j, k, l) in enumerate(quart):
        blk = v[off[n]:off[n + 1]].reshape(nc[i], nc[j], nc[k], nc[l])
        full[ao[i]:ao[i] + nc[i], ao[j]:ao[j] + nc[j], ao[k]:ao[k] + nc[k], ao[l]:ao[l] + nc[l]] = blk
    D = inputs.density(nao, 3, occ_fraction=0.4)
    K = oracle.exchange(b, D)
    np.testing.assert_allclose(K, np.einsum("ijkl,jl->ik", full, D), rtol=0, atol=1e-13 * np.max(np.abs(K)))
    np.testing.assert_allclose(K, K.T, rtol=0, atol=1e-13 * np.max(np.abs(K)))
    assert np.sum(D * K) > 0
    # row-restricted form gives the same rows
    Kr = oracle.exchange(b, D, row_shells=[1])
    r0, r1 = ao[1], ao[1] + nc[1]
    np.testing.assert_allclose(Kr[r0:r1], K[r0:r1], rtol=0, atol=1e-15)


# ------------------------------------------------------------------ exchange gradient
def test_exchange_gradient_against_finite_differences():
    """dS/dR of S = sum D_ik D_jl (ij|kl) (all four centres differentiated with
    d/dA x_A^a e^(-z x_A^2) = 2z x_A^(a+1) e - a x_A^(a-1) e) against central finite
    differences (h = 1e-4 bohr) of the oracle's own S; and sum over atoms = 0."""
    b = inputs.small_molecule(seed=41, n_atoms=3, shells=(0, 1, 2), K=2)
    D = inputs.density(b.nao, 8, occ_fraction=0.4)
    g = oracle.exchange_grad(b, D)
    np.testing.assert_allclose(g.sum(axis=0), 0.0, atol=1e-12 * np.max(np.abs(g)))
    h = 1e-4
    for A, x in [(0, 0), (1, 2), (2, 1)]:
        def S(delta):
            bb = inputs.small_molecule(seed=41, n_atoms=3, shells=(0, 1, 2), K=2)
            bb.center = bb.center.copy()
            bb.center[bb.atom == A, x] += delta
            return oracle.exchange_energy(bb, D)
        fd = (S(h) - S(-h)) / (2 * h)
        assert abs(g[A, x] - fd) <= 1e-7 * max(1.0, abs(fd)), (A, x, g[A, x], fd)


def test_exchange_gradient_high_l_invariance():
    """f shells (derivatives reach l = 4) on two atoms: translational invariance and FD."""
    b = inputs.small_molecule(seed=42, n_atoms=2, shells=(1, 3), K=1)
    D = inputs.density(b.nao, 9, occ_fraction=0.4)
    g = oracle.exchange_grad(b, D)
    np.testing.assert_allclose(g.sum(axis=0), 0.0, atol=1e-12 * np.max(np.abs(g)))
    h = 1e-4
    bb = inputs.small_molecule(seed=42, n_atoms=2, shells=(1, 3), K=1)
    c0 = bb.center.copy()
    bb.center = c0.copy(); bb.center[bb.atom == 1, 0] += h
    sp = oracle.exchange_energy(bb, D)
    bb.center = c0.copy(); bb.center[bb.atom == 1, 0] -= h
    sm = oracle.exchange_energy(bb, D)
    fd = (sp - sm) / (2 * h)
    assert abs(g[1, 0] - fd) <= 1e-7 * max(1.0, abs(fd))


# ------------------------------------------------------------------ solid harmonics (Eqs. solid2herm)
def _sphere_moment(a, b, c):
    """int x^a y^b z^c dOmega over the unit sphere (zero unless a, b, c are even)."""
    if a % 2 or b % 2 or c % 2:
        return 0.0
    return 2.0 * math.gamma((a + 1) / 2) * math.gamma((b + 1) / 2) * math.gamma((c + 1) / 2) / math.gamma((a + b + c + 3) / 2)


@pytest.mark.parametrize("l", range(7))
def test_solid_harmonics_orthonormal_on_sphere(l):
    """int S_lm S_lm' dOmega = 4 pi / (2l+1) delta_mm' (the angular norm of z^l), exact monomial moments."""
    C = oracle.solid_coefs(l)
    comps = [(ax, ay, l - ax - ay) for ax in range(l, -1, -1) for ay in range(l - ax, -1, -1)]
    M = np.array([[_sphere_moment(a[0] + b[0], a[1] + b[1], a[2] + b[2]) for b in comps] for a in comps])
    np.testing.assert_allclose(C @ M @ C.T, 4 * math.pi / (2 * l + 1) * np.eye(2 * l + 1), atol=1e-12)


@pytest.mark.parametrize("l", range(7))
def test_solid_harmonics_are_spherical_harmonics(l):
    """S_lm(r) = c_l r^l Y_lm(theta, phi) with real Y built from scipy's complex harmonics; |c_l| equal
    for every m (per-m sign is the convention)."""
    sp = pytest.importorskip("scipy.special")
    rng = np.random.Generator(np.random.PCG64(l))
    pts = rng.normal(size=(40, 3))
    r = np.linalg.norm(pts, axis=1)
    theta = np.arccos(pts[:, 2] / r)
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    C = oracle.solid_coefs(l)
    comps = [(ax, ay, l - ax - ay) for ax in range(l, -1, -1) for ay in range(l - ax, -1, -1)]
    mono = np.array([pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c for a, b, c in comps])
    S = C @ mono
    ratios = []
    for m in range(-l, l + 1):
        if hasattr(sp, "sph_harm_y"):
            Y = sp.sph_harm_y(l, abs(m), theta, phi)
        else:
            Y = sp.sph_harm(abs(m), l, phi, theta)
        if m > 0:
            Yr = math.sqrt(2) * Y.real
        elif m < 0:
            Yr = math.sqrt(2) * Y.imag
        else:
            Yr = Y.real
        ratio = S[m + l] / (r ** l * Yr)
        np.testing.assert_allclose(ratio, ratio[0], rtol=1e-10)
        ratios.append(abs(ratio[0]))
    np.testing.assert_allclose(ratios, ratios[0], rtol=1e-12)
    assert abs(ratios[0] - math.sqrt(4 * math.pi / (2 * l + 1))) < 1e-12


def test_spherical_eri_transform():
    """[ab|cd] over solid harmonics = C_a C_b C_c C_d applied to the Cartesian shellset, checked with
    einsum; s and p shells are the Cartesian values reordered (y, z, x)."""
    b, _ = _random_basis([2, 1, 3, 0], 44)
    v, _ = oracle.eri4(b, [[0, 1, 2, 3]])
    w, _ = oracle.eri4_sph(b, [[0, 1, 2, 3]])
    cart = v.reshape(6, 3, 10, 1)
    Cs = [oracle.solid_coefs(l) for l in (2, 1, 3, 0)]
    ref = np.einsum("ai,bj,ck,dl,ijkl->abcd", *Cs, cart).reshape(-1)
    np.testing.assert_allclose(w, ref, rtol=0, atol=1e-14 * np.max(np.abs(ref)))
    np.testing.assert_allclose(w.reshape(5, 3, 7, 1)[:, [2, 0, 1]], np.einsum("ai,ck,ijkl->ajcl", Cs[0], Cs[2], cart),
                               rtol=0, atol=1e-14 * np.max(np.abs(ref)))


@pytest.mark.parametrize("ls", [(2, 0, 0, 0), (3, 1, 0, 0), (2, 2, 1, 0), (4, 0, 2, 1)])
def test_spherical_eri_rotation_invariance(ls):
    """A rotation of the whole geometry maps the real solid harmonics of each shell onto one another by an
    orthogonal matrix, so the Frobenius norm of a solid-harmonic shellset does not change (a wrong
    coefficient breaks the orthogonality); the Cartesian shellset's norm does change (its components are
    not orthonormal), which shows the test has teeth."""
    _, specs = _random_basis(list(ls), 91)
    rng = np.random.Generator(np.random.PCG64(92))
    Qr, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    rot = [(l, Qr @ np.asarray(xyz), z, c) for (l, xyz, z, c) in specs]
    w0, _ = oracle.eri4_sph(_two_shell_basis(specs), [[0, 1, 2, 3]])
    w1, _ = oracle.eri4_sph(_two_shell_basis(rot), [[0, 1, 2, 3]])
    n0, n1 = np.linalg.norm(w0), np.linalg.norm(w1)
    assert n0 > 1e-6
    assert abs(n1 - n0) <= 1e-12 * n0, (n0, n1)
    v0, _ = oracle.eri4(_two_shell_basis(specs), [[0, 1, 2, 3]])
    v1, _ = oracle.eri4(_two_shell_basis(rot), [[0, 1, 2, 3]])
    assert abs(np.linalg.norm(v1) - np.linalg.norm(v0)) > 1e-6 * np.linalg.norm(v0)


def _basis_3c_pin(la, lc, ld, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    aux, orb = inputs.BasisBuilder(), inputs.BasisBuilder()
    z = np.exp(rng.uniform(np.log(0.2), np.log(4.0), 2))
    aux.add_shell(la, rng.uniform(-1, 1, 3), z, rng.uniform(0.2, 1.0, 2) * inputs.primitive_norm(la, z))
    for l in (lc, ld):
        z = np.exp(rng.uniform(np.log(0.2), np.log(4.0), 2))
        orb.add_shell(l, rng.uniform(-1, 1, 3), z, rng.uniform(0.2, 1.0, 2) * inputs.primitive_norm(l, z))
    return aux.build(), orb.build()


@pytest.mark.parametrize("la,lc,ld", [(3, 1, 2), (6, 0, 0), (2, 4, 3)])
def test_three_center_solid_harmonic_oracle(la, lc, ld):
    """The oracle's [a|cd] over solid harmonics equals the coefficient matrices applied to its Cartesian
    shellset (einsum), in FP64 and in long double, and keeps its norm when the geometry is rotated."""
    aux, orb = _basis_3c_pin(la, lc, ld, 95 + la)
    t = [[0, 0, 1]]
    Cs = [oracle.solid_coefs(l) for l in (la, lc, ld)]
    for prec in (0, 1):
        v, _ = oracle.eri3(aux, orb, t, precision=prec)
        vc = v.reshape(inputs.ncart(la), inputs.ncart(lc), inputs.ncart(ld))
        ref = np.einsum("ai,ck,dl,ikl->acd", *Cs, vc)
        # the combinations cancel: bound the rounding by the sum of the magnitudes they combine
        mag = np.einsum("ai,ck,dl,ikl->acd", *[np.abs(C) for C in Cs], np.abs(vc))
        w, off = oracle.eri3_sph(aux, orb, t, precision=prec)
        assert off[-1] == (2 * la + 1) * (2 * lc + 1) * (2 * ld + 1)
        assert np.all(np.abs(w - ref.reshape(-1)) <= 1e-14 * mag.reshape(-1) + 1e-300), prec
    rng = np.random.Generator(np.random.PCG64(96))
    R, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    aux.center = np.ascontiguousarray(aux.center @ R.T)
    orb.center = np.ascontiguousarray(orb.center @ R.T)
    w1, _ = oracle.eri3_sph(aux, orb, t, precision=1)
    assert abs(np.linalg.norm(w1) - np.linalg.norm(w)) <= 1e-12 * np.linalg.norm(w)


# ------------------------------------------------------------------ textbook values
def test_h2_sto3g_textbook_integrals():
    """H2 / STO-3G at 1.4 bohr: the four distinct two-electron integrals printed
    in a standard textbook worked example (tests/golden/h2_sto3g_two_electron.txt,
    four decimals). Pins contraction, primitive normalisation and the whole
    [ss|ss] path to numbers computed outside this project."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "h2_sto3g_two_electron.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    kv = {r[0]: r[1:] for r in rows}
    a = np.array([float(x) for x in kv["exps"]])
    c = np.array([float(x) for x in kv["coefs"]])
    R = float(kv["R"][0])
    bb = inputs.BasisBuilder()
    for z in (0.0, R):
        at = bb.add_atom([0.0, 0.0, z])
        bb.add_shell(0, [0.0, 0.0, z], a, c * inputs.primitive_norm(0, a), atom=at)
    b = bb.build()
    idx = {"1": 0, "2": 1}
    for key, vals in kv.items():
        if not key.startswith("("):
            continue
        i, j, k, l = (idx[ch] for ch in key if ch in "12")
        v, _ = oracle.eri4(b, np.array([[i, j, k, l]], dtype=np.int32))
        assert abs(v[0] - float(vals[0])) <= 0.5e-4, (key, v[0], vals[0])


def test_eri3_is_eri4_with_a_constant_function():
    """A Gaussian of exponent 0 is the constant 1, so [a|cd] (Eq. def-acd, one-centre
    E of Eq. E1rr) equals [a b|cd] with b an s function of exponent 0 and coefficient
    1 placed anywhere (two-centre E of Eqs. E2rr1/E2rr2)."""
    rng = np.random.Generator(np.random.PCG64(5))
    aux, orb = inputs.BasisBuilder(), inputs.BasisBuilder()
    for la in range(5):
        inputs.random_shell(rng, aux, la, rng.uniform(0, 2, 3), 2, 0.3, 3.0)
    for l in (0, 1, 2):
        inputs.random_shell(rng, orb, l, rng.uniform(0, 2, 3), 2, 0.3, 3.0)
    A, O = aux.build(), orb.build()
    t = np.array([[a, c, d] for a in range(A.n_shells) for c in range(O.n_shells) for d in range(O.n_shells)],
                 dtype=np.int32)
    v3, _ = oracle.eri3(A, O, t)
    bb = inputs.BasisBuilder()
    for B_, shells in ((A, range(A.n_shells)), (None, [None]), (O, range(O.n_shells))):
        for s in shells:
            if B_ is None:
                bb.add_shell(0, [0.3, -0.2, 0.1], np.array([0.0]), np.array([1.0]))
                continue
            p0, n = int(B_.prim_off[s]), int(B_.nprim[s])
            bb.add_shell(int(B_.l[s]), B_.center[s], B_.exps[p0:p0 + n], B_.coefs[p0:p0 + n])
    unit = A.n_shells
    q = np.array([[a, unit, unit + 1 + c, unit + 1 + d] for a, c, d in t], dtype=np.int32)
    v4, _ = oracle.eri4(bb.build(), q)
    np.testing.assert_allclose(v3, v4, rtol=0, atol=1e-13 * np.max(np.abs(v3)))
