"""Pins of the oracle's Zhao (1996) radial family (Eq. 4) away from alpha = 1.

Eq. 4 prints the lowest-order potential U_00 ~ (1 + (r/b)^(1/alpha))^-alpha;
the rest of the family (the Gegenbauer index (2l+1) alpha + 1/2, the density
constant K_nl, the normalisation I_nl) is written out in the oracle's header.
Each test checks it against something other than itself:

* alpha = 1/2 is the Clutton-Brock (1973) basis, whose lowest pair is the
  Plummer sphere (textbook potential -1/sqrt(r^2 + b^2));
* the Poisson equation, by finite differences of the potential, fixes K_nl;
* Gauss-Jacobi quadrature of the lowest-order density (mass from its
  enclosed-mass profile, not from K_nl or I_nl) must give S_000 = 1 and no
  other coefficient: this fixes I_nl through the coefficient pass;
* quadrature of r^2 rho_nl Phi_n'l gives the closed-form I_nl and zero off
  the diagonal;
* finite differences fix dPhi_nl/dr and the field's gradient;
* a particle at the origin gives Phi_n0(0) = -(1/b) C_n^(alpha+1/2)(-1).
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle
import workloads

ALPHAS = [0.5, 0.75, 1.5, 2.0]


def _radial_quad(f, b, alpha):
    """int_0^inf f(r) dr with r = b (p/(1-p))^alpha, p in (0, 1)."""
    def g(p):
        if p <= 0.0 or p >= 1.0:
            return 0.0
        r = b * (p / (1 - p)) ** alpha
        return f(r) * r * alpha / (p * (1 - p))
    val, _ = integrate.quad(g, 0, 1, epsabs=0, epsrel=1e-11, limit=500)
    return val


def test_alpha_half_is_the_clutton_brock_basis():
    b = 0.7
    for r in (0.0, 0.05, 0.7, 3.0, 40.0):
        # lowest pair: the Plummer potential and density (mass 1, scale b)
        assert oracle.phi_nl(0, 0, b, r, alpha=0.5) == pytest.approx(-1 / math.sqrt(r * r + b * b), rel=1e-14)
        assert oracle.rho_nl(0, 0, b, r, alpha=0.5) == pytest.approx(
            3 / (4 * math.pi * b ** 3) * (1 + (r / b) ** 2) ** -2.5, rel=1e-13)
        # Clutton-Brock: -(1/b) s^l (1+s^2)^-(l+1/2) C_n^(l+1)((s^2-1)/(s^2+1))
        s = r / b
        for n in range(5):
            for l in range(4):
                ref = -(1 / b) * s ** l * (1 + s * s) ** -(l + 0.5) * special.eval_gegenbauer(n, l + 1.0, (s * s - 1) / (s * s + 1))
                assert oracle.phi_nl(n, l, b, r, alpha=0.5) == pytest.approx(ref, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("alpha", ALPHAS + [1.0])
def test_u00_is_the_printed_form(alpha):
    b = 0.4
    for r in (0.01, 0.4, 2.0, 25.0):
        ref = -(1 / b) * (1 + (r / b) ** (1 / alpha)) ** -alpha
        assert oracle.phi_nl(0, 0, b, r, alpha=alpha) == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("alpha", [0.5, 0.7, 1.5, 2.0])
def test_poisson_equation_by_finite_difference(alpha):
    # (1/r^2) d/dr (r^2 dPhi/dr) - l(l+1) Phi / r^2 = 4 pi rho
    b = 0.8
    for n in range(0, 5):
        for l in range(0, 4):
            for r in (0.13, 0.9, 3.7):
                h = 1e-3 * r
                f = lambda x: x * x * oracle.dphi_nl_dr(n, l, b, x, alpha=alpha)
                d = (-f(r + 2 * h) + 8 * f(r + h) - 8 * f(r - h) + f(r - 2 * h)) / (12 * h)
                lap = d / (r * r) - l * (l + 1) * oracle.phi_nl(n, l, b, r, alpha=alpha) / (r * r)
                rho = oracle.rho_nl(n, l, b, r, alpha=alpha)
                assert lap == pytest.approx(4 * math.pi * rho, rel=1e-7, abs=1e-9 * abs(oracle.rho_nl(0, l, b, r, alpha=alpha)))


@pytest.mark.parametrize("alpha", [0.5, 0.75, 1.5, 2.0])
def test_radial_derivative_by_finite_difference(alpha):
    b = 0.45
    for n in range(0, 7):
        for l in range(0, 5):
            for r in (0.02, 0.6, 4.0):
                h = 1e-6 * r
                fd = (oracle.phi_nl(n, l, b, r + h, alpha=alpha) - oracle.phi_nl(n, l, b, r - h, alpha=alpha)) / (2 * h)
                scale = abs(oracle.dphi_nl_dr(0, l, b, r, alpha=alpha)) + 1e-12
                assert oracle.dphi_nl_dr(n, l, b, r, alpha=alpha) == pytest.approx(fd, rel=1e-6, abs=1e-8 * scale)
                if l >= 1:
                    assert oracle.phi_nl_over_r(n, l, b, r, alpha=alpha) == pytest.approx(
                        oracle.phi_nl(n, l, b, r, alpha=alpha) / r, rel=1e-12)


@pytest.mark.parametrize("alpha", ALPHAS)
def test_inl_closed_form_and_biorthogonality_by_quadrature(alpha):
    b = 0.6
    for l in range(0, 4):
        for n in range(0, 6):
            inl = oracle.inl(n, l, b, alpha=alpha)
            for k in range(0, 6):
                val = _radial_quad(lambda r: r * r * oracle.rho_nl(n, l, b, r, alpha=alpha) *
                                   oracle.phi_nl(k, l, b, r, alpha=alpha), b, alpha)
                if k == n:
                    assert val == pytest.approx(inl, rel=1e-9)
                else:
                    assert abs(val) < 1e-9 * abs(inl)


def _zhao_sphere(b, alpha, nodes=80):
    """Weighted points on the x axis whose sums of Phi_n0 are the integrals of
    Phi_n0 over the lowest-order density of the family (mass 1): its enclosed
    mass is p^(alpha+1) with p = t/(1+t), t = (r/b)^(1/alpha), and
    Phi_n0 = -(1/b) (1-p)^alpha C_n(2p - 1), so with x = 2p - 1 the integral
    of Phi_n0 dM = (alpha+1) p^alpha dp is 2^(-2 alpha - 1) (alpha+1) times
    that of a polynomial against the Jacobi weight (1-x)^alpha (1+x)^alpha:
    Gauss-Jacobi, each node's mass divided by its (1-p)^alpha."""
    x, w = special.roots_jacobi(nodes, alpha, alpha)
    p = 0.5 * (x + 1)
    pos = np.zeros((nodes, 4))
    pos[:, 0] = b * (p / (1 - p)) ** alpha
    pos[:, 3] = (alpha + 1) * 2.0 ** (-2 * alpha - 1) * w / (1 - p) ** alpha
    return pos


@pytest.mark.parametrize("alpha", ALPHAS)
def test_lowest_order_sphere_has_only_a000(alpha):
    b, nmax = 0.35, 10
    pos = _zhao_sphere(b, alpha)
    A = oracle.coeffs(pos, nmax, 0, b, alpha=alpha)
    S = A[: oracle.n_coef(nmax, 0)]
    assert S[0] == pytest.approx(1.0, rel=1e-11)
    assert np.max(np.abs(S[1:])) < 1e-10
    # the expansion's field is that sphere's: U_00 and -M(<r)/r^2 r_hat
    pts = np.array([[0.2, 0.1, -0.3, 0], [2.0, -1.0, 0.5, 0], [0.0, 0.0, 0.7, 0], [0.01, 0.0, 0.0, 0]])
    f = oracle.field(pts, A, nmax, 0, b, alpha=alpha)
    r = np.linalg.norm(pts[:, :3], axis=1)
    t = (r / b) ** (1 / alpha)
    assert np.allclose(f[:, 3], -(1 / b) * (1 + t) ** -alpha, rtol=1e-10)
    M = (t / (1 + t)) ** (alpha + 1)
    assert np.allclose(f[:, :3], -pts[:, :3] * (M / r ** 3)[:, None], rtol=1e-9, atol=1e-12)


def test_plummer_sphere_in_the_clutton_brock_basis():
    """alpha = 1/2, b = the Plummer scale: the textbook Plummer field."""
    b = 0.59
    A = oracle.coeffs(_zhao_sphere(b, 0.5), 8, 0, b, alpha=0.5)
    pts = RNG_PTS
    f = oracle.field(pts, A, 8, 0, b, alpha=0.5)
    r2 = np.sum(pts[:, :3] ** 2, axis=1)
    assert np.allclose(f[:, 3], -1 / np.sqrt(r2 + b * b), rtol=1e-11)
    assert np.allclose(f[:, :3], -pts[:, :3] / ((r2 + b * b) ** 1.5)[:, None], rtol=1e-10)


RNG_PTS = np.random.default_rng(77).normal(size=(12, 4))


@pytest.mark.parametrize("alpha", [0.5, 1.5, 2.0])
def test_single_particle_at_origin(alpha):
    nmax, lmax, b, mass = 7, 4, 0.6, 0.37
    A = oracle.coeffs(np.array([[0.0, 0.0, 0.0, mass]]), nmax, lmax, b, alpha=alpha)
    lam = alpha + 0.5
    for n in range(nmax + 1):
        c = (-1) ** n * math.exp(math.lgamma(n + 2 * lam) - math.lgamma(n + 1) - math.lgamma(2 * lam))
        ref = mass * (-(1 / b) * c) / (4 * math.pi) / oracle.inl(n, 0, b, alpha=alpha)
        assert A[oracle.idx(n, 0, 0, lmax)] == pytest.approx(ref, rel=1e-12)
    nz = [i for i in range(A.size) if i % oracle.n_coef(nmax, lmax) not in
          [oracle.idx(n, 0, 0, lmax) for n in range(nmax + 1)]]
    assert np.all(A[nz] == 0.0)


@pytest.mark.parametrize("alpha", [0.6, 1.7])
def test_force_is_minus_gradient_of_potential(alpha):
    nmax, lmax, b = 6, 5, 0.35
    pos, _ = workloads.plummer(500, seed=13)
    A = oracle.coeffs(pos, nmax, lmax, b, alpha=alpha)
    pts = np.array([[0.3, -0.2, 0.5, 0], [1e-3, 2e-3, 0.9, 0], [0.0, 0.0, -0.4, 0], [2.5, 1.0, -3.0, 0]])
    f = oracle.field(pts, A, nmax, lmax, b, alpha=alpha)
    h = 1e-4
    for k in range(len(pts)):
        g = np.zeros(3)
        for d in range(3):
            def pot(dx):
                p = pts[k:k + 1].copy()
                p[0, d] += dx
                return oracle.field(p, A, nmax, lmax, b, alpha=alpha)[0, 3]
            g[d] = -(-pot(2 * h) + 8 * pot(h) - 8 * pot(-h) + pot(-2 * h)) / (12 * h)
        assert np.allclose(f[k, :3], g, rtol=1e-8, atol=1e-8 * np.abs(g).max())


@pytest.mark.parametrize("alpha", [0.5, 2.0])
def test_field_at_the_origin_is_finite(alpha):
    """At r = 0 the l = 0 radial term has no direction (for alpha > 1 it is
    unbounded next to the centre) and is left out; the l = 1 terms give the
    gradient there, which the field approaches off the origin for alpha <= 1."""
    nmax, lmax, b = 5, 3, 0.5
    pos, _ = workloads.plummer(300, seed=14)
    A = oracle.coeffs(pos, nmax, lmax, b, alpha=alpha)
    f0 = oracle.field(np.zeros((1, 4)), A, nmax, lmax, b, alpha=alpha)[0]
    assert np.all(np.isfinite(f0))
    A1 = A.copy()
    nc = oracle.n_coef(nmax, lmax)
    for n in range(nmax + 1):          # keep l = 1 only
        for l in range(lmax + 1):
            if l != 1:
                for m in range(l + 1):
                    A1[oracle.idx(n, l, m, lmax)] = A1[nc + oracle.idx(n, l, m, lmax)] = 0.0
    f1 = oracle.field(np.zeros((1, 4)), A1, nmax, lmax, b, alpha=alpha)[0]
    assert np.allclose(f0[:3], f1[:3], rtol=1e-13, atol=1e-15)
    if alpha <= 1:
        e = oracle.field(np.array([[1e-7, -2e-7, 1.5e-7, 0]]), A, nmax, lmax, b, alpha=alpha)[0]
        assert np.allclose(e[:3] - f0[:3], 0, atol=1e-3 * np.abs(f0[:3]).max())


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5])
def test_half_mass_scale(alpha):
    r50 = 0.83
    b = oracle.zhao_half_mass_scale(r50, alpha)
    t = (r50 / b) ** (1 / alpha)
    assert (t / (1 + t)) ** (alpha + 1) == pytest.approx(0.5, rel=1e-14)
    if alpha == 1.0:
        assert b == pytest.approx(r50 / (1 + math.sqrt(2)), rel=1e-15)
    if alpha == 0.5:   # Plummer: r_h = a / sqrt(2^(2/3) - 1) ~ 1.305 a
        assert r50 / b == pytest.approx(1.0 / math.sqrt(2 ** (2 / 3) - 1), rel=1e-15)
        assert r50 / b == pytest.approx(1.3048, abs=1e-4)


def test_alpha_one_is_unchanged():
    """The keyword defaults give the Hernquist-Ostriker values (I_00 = -1/(12 pi b))."""
    b = 0.3
    assert oracle.inl(0, 0, b) == oracle.inl(0, 0, b, alpha=1.0)
    assert oracle.inl(0, 0, b) == pytest.approx(-1 / (12 * math.pi * b), rel=1e-14)
    assert oracle.knl(3, 2) == pytest.approx(2 * (0.5 * 3 * (3 + 8 + 3) + 3 * 5), rel=1e-15)
    pos, _ = workloads.plummer(50, seed=15)
    assert np.array_equal(oracle.coeffs(pos, 4, 3, b), oracle.coeffs(pos, 4, 3, b, alpha=1.0))


def _random_rotation(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    q *= np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5])
def test_rotation_invariance(alpha):
    """A rotation of the sample leaves each degree's power E_l unchanged and
    rotates the field: psi(R x; R sample) = psi(x; sample), a(R x) = R a(x).
    This ties the relative normalisation of every order m (the (2 - delta_m0)
    factor, N_lm, the sine terms) to geometry rather than to a formula."""
    nmax, lmax, b = 6, 5, 0.35
    pos, _ = workloads.plummer(600, seed=90)
    pos[:, :3] += np.array([0.07, -0.04, 0.05])      # not centred: every m is present
    Rm = _random_rotation(91)
    rot = pos.copy()
    rot[:, :3] = pos[:, :3] @ Rm.T
    A = oracle.coeffs(pos, nmax, lmax, b, alpha=alpha)
    Ar = oracle.coeffs(rot, nmax, lmax, b, alpha=alpha)
    E, Er = oracle.power_l(A, nmax, lmax, b, alpha), oracle.power_l(Ar, nmax, lmax, b, alpha)
    assert np.allclose(E, Er, rtol=1e-11, atol=0)
    pts = np.random.default_rng(92).normal(size=(8, 4)) * 0.5
    f = oracle.field(pts, A, nmax, lmax, b, alpha=alpha)
    pr = pts.copy()
    pr[:, :3] = pts[:, :3] @ Rm.T
    fr = oracle.field(pr, Ar, nmax, lmax, b, alpha=alpha)
    assert np.allclose(fr[:, 3], f[:, 3], rtol=1e-11)
    assert np.allclose(fr[:, :3], f[:, :3] @ Rm.T, rtol=1e-10, atol=1e-12 * np.abs(f[:, :3]).max())


@pytest.mark.parametrize("alpha", [0.5, 1.0, 2.0])
def test_joint_scaling_of_positions_and_b(alpha):
    """Positions and b scaled together by lam: U_nl -> U_nl / lam and
    I_nl -> I_nl / lam, so the coefficients are unchanged, the potential
    scales as 1/lam and the acceleration as 1/lam^2 (every power of b in the
    normalisation and the field is tied down)."""
    nmax, lmax, b, lam = 6, 4, 0.3, 3.7
    pos, _ = workloads.plummer(400, seed=93)
    pos[:, :3] += np.array([0.03, 0.02, -0.05])
    big = pos.copy()
    big[:, :3] *= lam
    A = oracle.coeffs(pos, nmax, lmax, b, alpha=alpha)
    Ab = oracle.coeffs(big, nmax, lmax, lam * b, alpha=alpha)
    assert np.allclose(Ab, A, rtol=1e-11, atol=1e-13 * np.abs(A).max())
    pts = np.random.default_rng(94).normal(size=(6, 4)) * 0.4
    f = oracle.field(pts, A, nmax, lmax, b, alpha=alpha)
    ptsb = pts.copy()
    ptsb[:, :3] *= lam
    fb = oracle.field(ptsb, Ab, nmax, lmax, lam * b, alpha=alpha)
    assert np.allclose(fb[:, 3], f[:, 3] / lam, rtol=1e-11)
    assert np.allclose(fb[:, :3], f[:, :3] / lam ** 2, rtol=1e-10, atol=1e-12 * np.abs(f[:, :3]).max())
