"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
library special functions, quadrature, invariants of symmetric inputs, brute
force, finite differences, or values printed in the paper.  A plausible slip in
the oracle (dropped term, wrong sign, wrong index, transposed operand, wrong
normalisation) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(1234)


# --------------------------------------------------------------- special functions
@pytest.mark.parametrize("alpha", [1.5, 3.5, 9.5, 21.5])
def test_gegenbauer_endpoints_and_library(alpha):
    for n in range(0, 21):
        c1 = math.exp(math.lgamma(n + 2 * alpha) - math.lgamma(n + 1) - math.lgamma(2 * alpha))
        assert oracle.gegenbauer(n, alpha, 1.0) == pytest.approx(c1, rel=1e-12)
        assert oracle.gegenbauer(n, alpha, -1.0) == pytest.approx((-1) ** n * c1, rel=1e-12)
        for xi in (-0.83, -0.2, 0.0, 0.37, 0.91):
            ref = special.eval_gegenbauer(n, alpha, xi)
            assert oracle.gegenbauer(n, alpha, xi) == pytest.approx(ref, rel=1e-10, abs=1e-12 * c1)


@pytest.mark.parametrize("alpha", [1.5, 5.5])
def test_gegenbauer_orthogonality(alpha):
    def w(x):
        return (1 - x * x) ** (alpha - 0.5)
    for n in range(0, 6):
        for k in range(0, 6):
            val, _ = integrate.quad(lambda x: w(x) * oracle.gegenbauer(n, alpha, x) * oracle.gegenbauer(k, alpha, x),
                                    -1, 1, epsabs=1e-13, limit=200)
            if n == k:
                norm = math.pi * 2 ** (1 - 2 * alpha) * math.exp(math.lgamma(n + 2 * alpha) - math.lgamma(n + 1) -
                                                                 2 * math.lgamma(alpha)) / (n + alpha)
                assert val == pytest.approx(norm, rel=1e-9)
            else:
                assert abs(val) < 1e-9


def test_plm_matches_library_with_condon_shortley_phase():
    for l in range(0, 13):
        for m in range(0, l + 1):
            for x in (-1.0, -0.7, -0.1, 0.0, 0.33, 0.95, 1.0):
                assert oracle.plm(l, m, x) == pytest.approx(special.lpmv(m, l, x), rel=1e-11, abs=1e-11)


def test_spherical_harmonic_addition_theorem():
    # sum_m Y_lm(1) Y*_lm(2) = (2l+1)/(4 pi) P_l(cos gamma), written in the real form.
    for _ in range(5):
        t1, t2 = RNG.uniform(0, np.pi, 2)
        p1, p2 = RNG.uniform(0, 2 * np.pi, 2)
        cg = math.cos(t1) * math.cos(t2) + math.sin(t1) * math.sin(t2) * math.cos(p1 - p2)
        for l in range(0, 11):
            s = 0.0
            for m in range(0, l + 1):
                term = oracle.nlm2(l, m) * oracle.plm(l, m, math.cos(t1)) * oracle.plm(l, m, math.cos(t2))
                s += term if m == 0 else 2 * term * math.cos(m * (p1 - p2))
            assert s == pytest.approx((2 * l + 1) / (4 * math.pi) * special.eval_legendre(l, cg), abs=1e-12)


def test_harmonic_normalisation_by_quadrature():
    for l, m in [(0, 0), (3, 0), (4, 2), (7, 7)]:
        val, _ = integrate.quad(lambda t: oracle.nlm2(l, m) * oracle.plm(l, m, math.cos(t)) ** 2 * math.sin(t),
                                0, math.pi, epsabs=1e-13)
        # int |Y_lm|^2 dOmega = 1 (phi integral of cos^2 or |e^{im phi}|^2 gives 2 pi)
        assert 2 * math.pi * val == pytest.approx(1.0, rel=1e-10)


def test_legendre_derivative_identities_by_finite_difference():
    h = 1e-6
    for l in range(0, 10):
        for m in range(0, l + 1):
            for th in (0.2, 1.1, 2.5):
                fd = (oracle.plm(l, m, math.cos(th + h)) - oracle.plm(l, m, math.cos(th - h))) / (2 * h)
                assert oracle.dplm_dtheta(l, m, math.cos(th)) == pytest.approx(fd, rel=1e-6, abs=1e-6)
                if m > 0:
                    ref = m * oracle.plm(l, m, math.cos(th)) / math.sin(th)
                    assert oracle.mplm_over_sin(l, m, math.cos(th)) == pytest.approx(ref, rel=1e-11, abs=1e-11)


# --------------------------------------------------------------- radial basis
@pytest.mark.parametrize("b", [1.0, 0.31])
def test_inl_closed_form_matches_quadrature(b):
    assert oracle.inl(0, 0, b) == pytest.approx(-1 / (12 * math.pi * b), rel=1e-14)
    for n in range(0, 9):
        for l in range(0, 7):
            f = lambda r: r * r * oracle.rho_nl(n, l, b, r) * oracle.phi_nl(n, l, b, r)
            # substitute r = b t/(1-t) to map [0, inf) to [0, 1)
            g = lambda t: f(b * t / (1 - t)) * b / (1 - t) ** 2 if t < 1 else 0.0
            val, _ = integrate.quad(g, 0, 1, epsabs=0, epsrel=1e-13, limit=400)
            assert val == pytest.approx(oracle.inl(n, l, b), rel=1e-10)


def test_radial_biorthogonality():
    b = 0.7
    for l in (0, 2, 5):
        for n in range(0, 5):
            for k in range(0, 5):
                if n == k:
                    continue
                g = lambda t: (lambda r: r * r * oracle.rho_nl(n, l, b, r) * oracle.phi_nl(k, l, b, r))(
                    b * t / (1 - t)) * b / (1 - t) ** 2 if t < 1 else 0.0
                val, _ = integrate.quad(g, 0, 1, epsabs=1e-13, limit=400)
                assert abs(val) < 1e-9 * abs(oracle.inl(n, l, b))


def test_poisson_equation_radial_by_finite_difference():
    # (1/r^2) d/dr (r^2 dPhi/dr) - l(l+1) Phi / r^2 = 4 pi rho  for each (n, l)
    b = 0.8
    for n in range(0, 6):
        for l in range(0, 5):
            for r in (0.13, 0.9, 3.7):
                h = 1e-3 * r
                f = lambda x: x * x * oracle.dphi_nl_dr(n, l, b, x)
                d = (-f(r + 2 * h) + 8 * f(r + h) - 8 * f(r - h) + f(r - 2 * h)) / (12 * h)   # 4th order
                lap = d / (r * r) - l * (l + 1) * oracle.phi_nl(n, l, b, r) / (r * r)
                assert lap == pytest.approx(4 * math.pi * oracle.rho_nl(n, l, b, r), rel=1e-8, abs=1e-10)


def test_radial_derivative_by_finite_difference():
    b = 0.45
    for n in range(0, 8):
        for l in range(0, 6):
            for r in (0.05, 0.6, 4.0):
                h = 1e-6 * r
                fd = (oracle.phi_nl(n, l, b, r + h) - oracle.phi_nl(n, l, b, r - h)) / (2 * h)
                assert oracle.dphi_nl_dr(n, l, b, r) == pytest.approx(fd, rel=1e-6, abs=1e-9)
                if l >= 1:
                    assert oracle.phi_nl_over_r(n, l, b, r) == pytest.approx(oracle.phi_nl(n, l, b, r) / r, rel=1e-12)


# --------------------------------------------------------------- coefficients
def _hernquist_quadrature_shell(b, nodes=120):
    """Weighted 'particles' on the x axis that integrate a Hernquist sphere's
    mass exactly: M(<r) = s^2/(1+s)^2 with s = t/(1-t), dM = 2t dt (t = sqrt u).
    Only l = 0 coefficients of such a set carry meaning."""
    x, w = np.polynomial.legendre.leggauss(nodes)
    t = 0.5 * (x + 1)
    wt = 0.5 * w * 2 * t
    r = b * t / (1 - t)
    pos = np.zeros((nodes, 4))
    pos[:, 0] = r
    pos[:, 3] = wt
    return pos


@pytest.mark.parametrize("b", [1.0, 0.3])
def test_hernquist_sphere_has_only_a000(b):
    nmax = 12
    pos = _hernquist_quadrature_shell(b)
    A = oracle.coeffs(pos, nmax, 0, b)
    S = A[: oracle.n_coef(nmax, 0)]
    assert S[0] == pytest.approx(1.0, rel=1e-12)
    assert np.max(np.abs(S[1:])) < 1e-11
    # potential and force of that expansion: -1/(r+b) and -x/(r (r+b)^2)
    pts = np.array([[0.2, 0.1, -0.3, 0], [2.0, -1.0, 0.5, 0], [0.0, 0.0, 0.7, 0]])
    f = oracle.field(pts, A, nmax, 0, b)
    r = np.linalg.norm(pts[:, :3], axis=1)
    assert np.allclose(f[:, 3], -1 / (r + b), rtol=1e-11)
    assert np.allclose(f[:, :3], -pts[:, :3] / (r * (r + b) ** 2)[:, None], rtol=1e-10, atol=1e-12)


def test_hernquist_sample_monte_carlo():
    b = 0.4
    pos = workloads.hernquist_positions(40000, b, seed=9)
    A = oracle.coeffs(pos, 4, 4, b)
    nc = oracle.n_coef(4, 4)
    # S_000 = 3 <1/(1+s)> with <1/(1+s)> = 1/3: statistical error ~ 1/sqrt(N)
    assert A[0] == pytest.approx(1.0, abs=5 * 0.25 / math.sqrt(40000))
    others = np.abs(np.delete(A, [0]))
    assert others.max() < 0.1


def test_single_particle_at_origin():
    nmax, lmax, b, mass = 8, 5, 0.6, 0.37
    pos = np.array([[0.0, 0.0, 0.0, mass]])
    A = oracle.coeffs(pos, nmax, lmax, b)
    nc = oracle.n_coef(nmax, lmax)
    for n in range(nmax + 1):
        # Phi_n0(0) = -(1/b) C_n^{3/2}(-1) = -(1/b) (-1)^n (n+1)(n+2)/2 ; S = Phi N_00^2 m / I_n0
        ref = mass * (-(1 / b) * (-1) ** n * (n + 1) * (n + 2) / 2) / (4 * math.pi) / oracle.inl(n, 0, b)
        assert A[oracle.idx(n, 0, 0, lmax)] == pytest.approx(ref, rel=1e-13)
        for l in range(1, lmax + 1):
            for m in range(l + 1):
                assert A[oracle.idx(n, l, m, lmax)] == 0.0
                assert A[nc + oracle.idx(n, l, m, lmax)] == 0.0


def test_mirror_symmetric_sample_kills_odd_terms():
    nmax, lmax, b = 6, 6, 0.5
    base, _ = workloads.plummer(300, seed=4)
    pos = workloads.mirror8(base)
    A = oracle.coeffs(pos, nmax, lmax, b)
    nc = oracle.n_coef(nmax, lmax)
    scale = np.max(np.abs(A))
    assert np.max(np.abs(A[nc:])) < 1e-13 * scale        # y-reflection: every T vanishes
    for n in range(nmax + 1):
        for l in range(lmax + 1):
            for m in range(l + 1):
                v = A[oracle.idx(n, l, m, lmax)]
                if m % 2 == 1 or l % 2 == 1:                 # x- and z-reflections
                    assert abs(v) < 1e-13 * scale
    # and the even terms are not all trivially zero
    assert abs(A[oracle.idx(1, 2, 2, lmax)]) > 1e-6 * scale


def test_k_fold_rotation_keeps_only_multiples_of_k():
    nmax, lmax, b, K = 4, 7, 0.5, 3
    base, _ = workloads.plummer(200, seed=5)
    pos = workloads.rotate_copies(base, K)
    A = oracle.coeffs(pos, nmax, lmax, b)
    nc = oracle.n_coef(nmax, lmax)
    scale = np.max(np.abs(A))
    for n in range(nmax + 1):
        for l in range(lmax + 1):
            for m in range(l + 1):
                if m % K:
                    i = oracle.idx(n, l, m, lmax)
                    assert abs(A[i]) < 1e-13 * scale and abs(A[nc + i]) < 1e-13 * scale
    assert abs(A[oracle.idx(0, 3, 3, lmax)]) > 1e-8 * scale


def test_mask_excludes_particles():
    pos, _ = workloads.plummer(400, seed=6)
    mask = (np.arange(400) % 3 != 0).astype(np.uint8)
    A1 = oracle.coeffs(pos, 5, 4, 0.4, mask=mask)
    A2 = oracle.coeffs(pos[mask.astype(bool)], 5, 4, 0.4)
    assert np.allclose(A1, A2, rtol=1e-13, atol=1e-15)


def test_power_spectrum_spherical_and_origin():
    # a particle at the origin is spherically symmetric: E_l = 0 for l > 0 (Sec. 4.2)
    A = oracle.coeffs(np.array([[0, 0, 0, 1.0]]), 6, 4, 0.5)
    El = oracle.power_l(A, 6, 4, 0.5)
    assert El[0] > 0 and np.all(El[1:] == 0)
    # absolute value from Eq. 3b with the bi-orthonormal basis
    # psi_n00 = Phi_n0 Y_00 / sqrt|I_n0|: a_n00 = -m psi*_n00(0)
    ref = sum(oracle.phi_nl(n, 0, 0.5, 0.0) ** 2 / (4 * math.pi * abs(oracle.inl(n, 0, 0.5))) for n in range(7))
    assert El[0] == pytest.approx(ref, rel=1e-13)
    # a random isotropic sample: E_l>0 / E_0 = O(1/N)
    pos, _ = workloads.plummer(4000, seed=8)
    El = oracle.power_l(oracle.coeffs(pos, 6, 4, 0.3), 6, 4, 0.3)
    assert np.all(El[1:] / El[0] < 20.0 / 4000)


# --------------------------------------------------------------- field
def test_force_is_minus_gradient_of_potential():
    nmax, lmax, b = 7, 6, 0.35
    pos, _ = workloads.plummer(600, seed=10)
    A = oracle.coeffs(pos, nmax, lmax, b)
    pts = np.array([[0.3, -0.2, 0.5, 0], [1e-3, 2e-3, 0.9, 0], [0.0, 0.0, -0.4, 0], [2.5, 1.0, -3.0, 0],
                    [0.0, 0.0, 0.2, 0]])
    f = oracle.field(pts, A, nmax, lmax, b)
    h = 1e-4
    for k in range(len(pts)):
        g = np.zeros(3)
        for d in range(3):
            def pot(dx):
                p = pts[k:k + 1].copy()
                p[0, d] += dx
                return oracle.field(p, A, nmax, lmax, b)[0, 3]
            g[d] = -(-pot(2 * h) + 8 * pot(h) - 8 * pot(-h) + pot(-2 * h)) / (12 * h)   # 4th order
        assert np.allclose(f[k, :3], g, rtol=1e-9, atol=1e-9 * np.abs(g).max())


def test_lmax0_force_is_radial():
    pos, _ = workloads.plummer(500, seed=11)
    A = oracle.coeffs(pos, 10, 0, 0.3)
    pts = RNG.normal(size=(20, 4))
    f = oracle.field(pts, A, 10, 0, 0.3)
    cross = np.cross(f[:, :3], pts[:, :3])
    assert np.max(np.linalg.norm(cross, axis=1) / np.linalg.norm(f[:, :3], axis=1)) < 1e-12


def test_gravitational_constant_scales_field():
    pos, _ = workloads.plummer(200, seed=12)
    A = oracle.coeffs(pos, 4, 3, 0.3)
    f1 = oracle.field(pos[:10], A, 4, 3, 0.3, G=1.0)
    f2 = oracle.field(pos[:10], A, 4, 3, 0.3, G=2.5)
    assert np.allclose(f2, 2.5 * f1, rtol=1e-14)


def _offset_plummer_quadrature(x0, a, b, nr=64, nth=32, nph=40):
    """Weighted points that integrate a Plummer sphere (mass 1, scale a) centred
    at x0 exactly enough for the tests: Gauss-Legendre in t with r = b t/(1-t),
    Gauss-Legendre in cos(theta), uniform in phi."""
    t, wt = np.polynomial.legendre.leggauss(nr)
    t = 0.5 * (t + 1)
    wt = 0.5 * wt
    r = b * t / (1 - t)
    dr = b / (1 - t) ** 2 * wt
    c, wc = np.polynomial.legendre.leggauss(nth)
    ph = 2 * np.pi * np.arange(nph) / nph
    R, C, PH = np.meshgrid(r, c, ph, indexing="ij")
    W = (dr[:, None, None] * wc[None, :, None] * (2 * np.pi / nph)) * R ** 2
    S = np.sqrt(1 - C ** 2)
    X = np.stack([R * S * np.cos(PH), R * S * np.sin(PH), R * C], -1).reshape(-1, 3)
    rho = 3 / (4 * np.pi * a ** 3) * (1 + ((X - x0) ** 2).sum(1) / a ** 2) ** -2.5
    pos = np.zeros((len(X), 4))
    pos[:, :3] = X
    pos[:, 3] = rho * W.reshape(-1)
    return pos


def test_expansion_of_offset_plummer_converges_to_exact_field():
    """The truncation error of Eq. 1a-3b for a smooth, off-centre (so every
    l, m appears) density: potential and acceleration converge to the exact
    Plummer field -1/sqrt(|x-x0|^2+a^2) as (nmax, lmax) grows."""
    x0, a, b = np.array([0.1, 0.05, -0.08]), 0.3, 0.3
    pos = _offset_plummer_quadrature(x0, a, b)
    assert pos[:, 3].sum() == pytest.approx(1.0, rel=1e-12)
    u = RNG.normal(size=(30, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    tgt = np.zeros((30, 4))
    tgt[:, :3] = u * RNG.uniform(0.1, 3.0, 30)[:, None]
    d = tgt[:, :3] - x0
    dd = (d ** 2).sum(1) + a * a
    acc_exact = -d / dd[:, None] ** 1.5
    errs = []
    for nmax, lmax in [(4, 2), (10, 6), (20, 10)]:
        A = oracle.coeffs(pos, nmax, lmax, b)
        f = oracle.field(tgt, A, nmax, lmax, b)
        e = np.linalg.norm(f[:, :3] - acc_exact, axis=1) / np.linalg.norm(acc_exact, axis=1)
        errs.append(np.max(e))
        assert np.max(np.abs(f[:, 3] + 1 / np.sqrt(dd)) * np.sqrt(dd)) < 10 * np.max(e) + 1e-12
    assert errs[0] > 10 * errs[1] > 100 * errs[2]
    assert errs[2] < 1e-5


def test_scf_residual_against_direct_summation_small_n():
    """Sec. 4.1 compares model accelerations with direct N-body summation.  For
    a discrete sample (N <= 512, compact) the expansion of point masses
    converges only algebraically in nmax, so the check is a bounded residual
    that shrinks from (4,2) to (20,10) at points outside the sample."""
    pos = workloads.hernquist_positions(2000, 0.3, seed=13)
    pos = pos[np.linalg.norm(pos[:, :3], axis=1) < 0.5][:400]
    pos[:, 3] = 1.0 / len(pos)
    u = RNG.normal(size=(24, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    tgt = np.zeros((24, 4))
    tgt[:, :3] = u * RNG.uniform(0.7, 2.5, 24)[:, None]
    ref = oracle.direct(pos, tgt)
    errs = []
    for nmax, lmax in [(4, 2), (20, 10)]:
        f = oracle.field(tgt, oracle.coeffs(pos, nmax, lmax, 0.3), nmax, lmax, 0.3)
        errs.append(np.median(np.linalg.norm(f[:, :3] - ref[:, :3], axis=1) / np.linalg.norm(ref[:, :3], axis=1)))
    assert errs[1] < 0.7 * errs[0]
    assert errs[1] < 0.02


# --------------------------------------------------------------- host (App. A)
def _host_phys(components, G):
    return oracle.host_struct(components, G=G)


def test_host_forces_are_minus_gradient():
    G = 1.0
    comps = [(oracle.HOST_HERNQUIST, 2.0, 0.7, 0), (oracle.HOST_NFW, 5.0, 3.0, 0), (oracle.HOST_MN, 3.0, 2.0, 0.3)]
    for c in comps:
        h = _host_phys([c], G)
        for x in ([1.0, 0.5, -0.2], [4.0, -3.0, 2.0], [0.1, 0.0, 0.05]):
            a, _ = oracle.host_accel(h, np.array(x))
            g = np.zeros(3)
            eps = 1e-6
            for d in range(3):
                xp = np.array(x, float)
                xm = xp.copy()
                xp[d] += eps
                xm[d] -= eps
                g[d] = -(oracle.host_accel(h, xp)[1] - oracle.host_accel(h, xm)[1]) / (2 * eps)
            assert np.allclose(a, g, rtol=1e-7, atol=1e-10)


def test_host_potentials_match_paper_table1():
    """E and L_z' of Orbits 0-9 (Table 1) from their initial conditions
    (Table A3) in MilkyWayPotential2022 (Table A2)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "mw2022_orbits.txt"))
    h = _host_phys(workloads.mw2022_physical(), workloads.G_PC_KMS2_MSUN * 1e-3)
    for row in rows:
        x, v = row[1:4], row[4:7]
        Lz = x[0] * v[1] - x[1] * v[0]
        _, psi = oracle.host_accel(h, x)
        E = 0.5 * float(v @ v) + psi
        assert abs(Lz / 1e3 - row[7]) <= 0.0051, (row[0], Lz)
        assert abs(E / 1e5 - row[8]) <= 0.0051, (row[0], E)


def test_unit_conversion_matches_nbody_input_deck():
    # App. B: the deck's 202.0992878224309 pc/Myr is the 197.61111164 km/s of Table A3.
    assert 197.61111164 * workloads.KMS_TO_PC_MYR == pytest.approx(202.0992878224309, rel=1e-9)


def test_tidal_difference_is_linear_for_small_offsets():
    h = _host_phys(workloads.host_in_units(workloads.galaxy_host_physical(), workloads.Units(1e5, 3.7)), 1.0)
    R = np.array([2100.0, 300.0, 150.0])
    x = np.array([0.3, -0.2, 0.1])
    t1 = oracle.tidal(h, R, x)
    t2 = oracle.tidal(h, R, 2 * x)
    t3 = oracle.tidal(h, R, -x)
    # a_tid(x) = T x + O(x^2): odd part doubles, even part is second order
    assert np.allclose(t2, 2 * t1, rtol=1e-3)
    assert np.allclose(t3, -t1, rtol=1e-3)
    # and it equals the plain double difference up to that difference's rounding
    aRx, _ = oracle.host_accel(h, R + x)
    aR, _ = oracle.host_accel(h, R)
    assert np.allclose(t1, aRx - aR, rtol=1e-8, atol=1e-15)


# --------------------------------------------------------------- integrator
def _static_setup():
    pos, vel = workloads.plummer(64, seed=14)
    nmax, lmax, b = 6, 4, 0.3
    big, _ = workloads.plummer(2000, seed=15)
    A = oracle.coeffs(big, nmax, lmax, b)
    acc = oracle.forces(pos, A, nmax, lmax, b)
    return pos, vel, acc, A, nmax, lmax, b


def _energy(pos, vel, A, nmax, lmax, b):
    f = oracle.field(pos, A, nmax, lmax, b)
    return 0.5 * (vel[:, :3] ** 2).sum(1) + f[:, 3]


def test_leapfrog_static_potential_energy_is_second_order():
    pos, vel, acc, A, nmax, lmax, b = _static_setup()
    E0 = _energy(pos, vel, A, nmax, lmax, b)
    errs = []
    for dt, n in [(0.02, 50), (0.01, 100)]:
        p, v, a, _, _ = oracle.step(pos, vel, acc, nmax, lmax, b, dt, n, A_frozen=A)
        errs.append(np.max(np.abs(_energy(p, v, A, nmax, lmax, b) - E0)))
    assert errs[1] < errs[0] / 3.0
    assert errs[1] < 1e-3


def test_leapfrog_time_reversible():
    pos, vel, acc, A, nmax, lmax, b = _static_setup()
    p, v, a, _, _ = oracle.step(pos, vel, acc, nmax, lmax, b, 0.01, 40, A_frozen=A)
    v[:, :3] *= -1
    p2, v2, _, _, _ = oracle.step(p, v, a, nmax, lmax, b, 0.01, 40, A_frozen=A)
    assert np.allclose(p2[:, :3], pos[:, :3], atol=1e-11)
    assert np.allclose(-v2[:, :3], vel[:, :3], atol=1e-11)


def test_com_orbit_conserves_lz_in_axisymmetric_host():
    units = workloads.Units(1e5, 3.7)
    h = _host_phys(workloads.host_in_units(workloads.galaxy_host_physical(), units), 1.0)
    com = np.array([2000.0, 0.0, 300.0, 0.0, 60.0, 5.0])
    pos = np.zeros((0, 4))
    E0 = 0.5 * com[3:] @ com[3:] + oracle.host_accel(h, com[:3])[1]
    Lz0 = com[0] * com[4] - com[1] * com[3]
    dE = []
    for dt, n in [(0.5, 400), (0.25, 800)]:
        _, _, _, c1, _ = oracle.step(pos, pos, pos, 0, 0, 0.3, dt, n, com=com, host=h)
        assert c1[0] * c1[4] - c1[1] * c1[3] == pytest.approx(Lz0, rel=1e-12)
        dE.append(abs(0.5 * c1[3:] @ c1[3:] + oracle.host_accel(h, c1[:3])[1] - E0))
    assert dE[1] < dE[0] / 3.0          # second order in dt
    assert dE[1] < 1e-4 * abs(E0)


def test_plummer_sample_is_in_henon_units():
    pos, vel = workloads.plummer(4000, seed=16)
    K = 0.5 * (pos[:, 3] * (vel[:, :3] ** 2).sum(1)).sum()
    U = 0.5 * (pos[:, 3] * oracle.direct(pos, pos)[:, 3]).sum()
    assert K + U == pytest.approx(-0.25, abs=0.02)
    assert 2 * K / abs(U) == pytest.approx(1.0, abs=0.05)
