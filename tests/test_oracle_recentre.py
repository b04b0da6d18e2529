"""Pins of the oracle's re-centring (Sec. 2.1): the SCF centre at the maximum
of a_000, the expansion's density, the core radius and the core velocity.

* a sample symmetric under the eight reflections about a point c has its
  centre exactly at c, and its core velocity is the bulk velocity added to
  velocities reflected with the positions;
* the centre is a stationary point and a local maximum of a_000, which is
  computed here directly from the coefficient pass (S_000 of the particles
  shifted by -x_c), not from the iteration's profile;
* the expansion's density is the Zhao lowest-order density for the projected
  lowest-order sphere (Plummer at alpha = 1/2, Hernquist at alpha = 1) and
  equals the Laplacian of the potential over 4 pi (Eq. 1b against Eq. 1a) for
  a general expansion, by finite differences;
* the core radius of a Plummer sample in its own basis (alpha = 1/2, b = a)
  is that of the Plummer density, r_core^2 = int rho^3 r^4 dr / int rho^3 r^2 dr
  = 0.3 a^2, within sampling noise;
* re-centring leaves host-frame positions and velocities unchanged.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
import workloads


def _a000(pos, xc, b, alpha, mask=None):
    p = pos.copy()
    p[:, :3] -= xc
    return oracle.coeffs(p, 0, 0, b, mask=mask, alpha=alpha)[0]


def _symmetric(n, seed, c, V0):
    pos, vel = workloads.plummer(n, seed=seed)
    P, V = [], []
    for sx in (1, -1):
        for sy in (1, -1):
            for sz in (1, -1):
                sgn = np.array([sx, sy, sz])
                q, u = pos.copy(), vel.copy()
                q[:, :3] *= sgn
                u[:, :3] *= sgn
                q[:, 3] /= 8
                P.append(q)
                V.append(u)
    P, V = np.concatenate(P), np.concatenate(V)
    P[:, :3] += c
    V[:, :3] += V0
    return P, V


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5])
def test_symmetric_sample_centre_and_core_velocity(alpha):
    c, V0 = np.array([0.11, -0.05, 0.023]), np.array([0.3, -0.2, 0.1])
    pos, vel = _symmetric(3000, 21, c, V0)
    xc, it = oracle.expansion_centre(pos, 0.3, alpha)
    assert np.allclose(xc, c, rtol=0, atol=1e-12)
    p2, v2, com, xc2, V, rc, _ = oracle.recentre(pos, vel, np.zeros(6), 6, 4, 0.3, alpha)
    assert np.allclose(V, V0, rtol=0, atol=1e-12)
    assert 0.0 < rc < 1.0


@pytest.mark.parametrize("alpha", [0.5, 1.0])
def test_centre_is_the_maximum_of_a000(alpha):
    pos, _ = workloads.plummer(5000, seed=22)
    pos[:, :3] += np.array([0.05, 0.02, -0.04])
    b = 0.3
    mask = np.arange(pos.shape[0]) % 7 != 3
    xc, it = oracle.expansion_centre(pos, b, alpha, mask=mask)
    assert it < 100
    a0 = _a000(pos, xc, b, alpha, mask)
    rng = np.random.default_rng(3)
    for _ in range(12):
        d = rng.normal(size=3)
        d *= 1e-3 * b / np.linalg.norm(d)
        assert _a000(pos, xc + d, b, alpha, mask) < a0
    if alpha != 1.0:   # smooth profile: the gradient vanishes (central differences)
        h = 1e-5 * b
        g = [(_a000(pos, xc + h * e, b, alpha, mask) - _a000(pos, xc - h * e, b, alpha, mask)) / (2 * h)
             for e in np.eye(3)]
        assert np.max(np.abs(g)) < 1e-7 * a0 / b


def _zhao_sphere(b, alpha, nodes=80):
    x, w = special.roots_jacobi(nodes, alpha, alpha)
    p = 0.5 * (x + 1)
    pos = np.zeros((nodes, 4))
    pos[:, 0] = b * (p / (1 - p)) ** alpha
    pos[:, 3] = (alpha + 1) * 2.0 ** (-2 * alpha - 1) * w / (1 - p) ** alpha
    return pos


def test_density_of_the_lowest_order_spheres():
    pts = np.random.default_rng(4).normal(size=(10, 4))
    r = np.linalg.norm(pts[:, :3], axis=1)
    b = 0.45
    A = oracle.coeffs(_zhao_sphere(b, 0.5), 6, 0, b, alpha=0.5)          # Plummer
    assert np.allclose(oracle.density(pts, A, 6, 0, b, 0.5), 3 / (4 * math.pi * b ** 3) * (1 + (r / b) ** 2) ** -2.5,
                       rtol=1e-10)
    A = oracle.coeffs(_zhao_sphere(b, 1.0), 6, 0, b, alpha=1.0)          # Hernquist
    assert np.allclose(oracle.density(pts, A, 6, 0, b, 1.0), b / (2 * math.pi * r * (r + b) ** 3), rtol=1e-10)


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.7])
def test_density_is_laplacian_of_potential(alpha):
    nmax, lmax, b = 5, 4, 0.4
    pos, _ = workloads.plummer(400, seed=23)
    A = oracle.coeffs(pos, nmax, lmax, b, alpha=alpha)
    pts = np.array([[0.3, -0.2, 0.5, 0], [0.7, 0.1, -0.2, 0], [-0.1, 0.45, 0.3, 0]])
    rho = oracle.density(pts, A, nmax, lmax, b, alpha)
    h = 2e-3
    for k in range(len(pts)):
        lap = 0.0
        for d in range(3):
            def pot(dx):
                p = pts[k:k + 1].copy()
                p[0, d] += dx
                return oracle.field(p, A, nmax, lmax, b, alpha=alpha)[0, 3]
            lap += (-pot(2 * h) + 16 * pot(h) - 30 * pot(0) + 16 * pot(-h) - pot(-2 * h)) / (12 * h * h)
        assert lap == pytest.approx(4 * math.pi * rho[k], rel=1e-6)


def test_plummer_core_radius():
    n, a = 200000, 3 * math.pi / 16     # Henon-unit Plummer scale
    pos, vel = workloads.plummer(n, seed=24)
    A = oracle.coeffs(pos, 6, 0, a, alpha=0.5)
    rc, V = oracle.core_frame(pos, vel, A, 6, 0, a, 0.5)
    print(f"Plummer r_core / a = {rc / a:.4f} (density of the Plummer sphere: sqrt(0.3) = {math.sqrt(0.3):.4f})")
    assert rc / a == pytest.approx(math.sqrt(0.3), rel=0.02)
    assert np.linalg.norm(V) < 0.05       # an isotropic sample at rest


def test_recentre_keeps_host_frame_state():
    pos, vel = workloads.plummer(3000, seed=25)
    pos[:, :3] += 0.07
    vel[:, :3] += 0.02
    com = np.array([10.0, -3.0, 1.0, 0.1, 0.2, -0.3])
    p2, v2, c2, xc, V, rc, it = oracle.recentre(pos, vel, com, 8, 4, 0.3, 1.0)
    assert np.allclose(p2[:, :3] + c2[:3], pos[:, :3] + com[:3], rtol=0, atol=1e-13)
    assert np.allclose(v2[:, :3] + c2[3:], vel[:, :3] + com[3:], rtol=0, atol=1e-14)
    assert np.linalg.norm(xc - 0.07) < 0.1 and np.linalg.norm(V - 0.02) < 0.2   # sampling noise of the core


# --------------------------------------------------------------- b at the maximum of a_000
@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5])
def test_a000_scale_of_the_lowest_order_sphere_is_its_own(alpha):
    """The projection of a density onto the unit-energy lowest pair is largest
    when the pair's density is the density itself (Cauchy-Schwarz in the
    energy inner product): the search returns the sphere's own scale."""
    b_true = 0.37
    pos = _zhao_sphere(b_true, alpha, nodes=120)
    for b0 in (0.2, 0.37, 0.9):
        b = oracle.a000_scale(pos, b0, alpha)
        assert b == pytest.approx(b_true, rel=1e-12)


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5])
def test_a000_scale_slope_is_the_derivative_of_ln_a000(alpha):
    """The stationarity condition the maximiser solves is d ln a_000 / d ln b,
    by 4th-order central differences of the closed form a_000(b)."""
    pos, _ = workloads.plummer(3000, seed=30)
    mask = np.arange(3000) % 5 != 4
    for b in (0.15, 0.3, 0.8):
        x, h = math.log(b), 1e-3
        f = lambda y: math.log(oracle.a000_biorth(pos, math.exp(y), alpha, mask=mask))
        fd = (-f(x + 2 * h) + 8 * f(x + h) - 8 * f(x - h) + f(x - 2 * h)) / (12 * h)
        assert oracle.a000_scale_slope(pos, x, alpha, mask=mask) == pytest.approx(fd, abs=1e-10)


def test_a000_scale_of_samples():
    a = 3 * math.pi / 16
    pos, _ = workloads.plummer(200000, seed=26)
    assert oracle.a000_scale(pos, 0.3, 0.5) / a == pytest.approx(1.0, abs=0.01)      # Plummer in its own basis
    hp = workloads.hernquist_positions(200000, 0.4, seed=27)
    assert oracle.a000_scale(hp, 0.3, 1.0) / 0.4 == pytest.approx(1.0, abs=0.01)     # Hernquist in its own


def test_a000_scale_is_a_maximum_of_a000():
    pos, _ = workloads.plummer(5000, seed=28)
    mask = np.arange(5000) % 4 != 1
    for alpha in (0.5, 1.0):
        b = oracle.a000_scale(pos, 0.3, alpha, mask=mask)
        a0 = oracle.a000_biorth(pos, b, alpha, mask=mask)
        # a_000 from the coefficient pass (S_000 sqrt|I_00| / N_00) agrees with the closed form
        S = oracle.coeffs(pos, 0, 0, b, mask=mask, alpha=alpha)[0]
        assert S * math.sqrt(abs(oracle.inl(0, 0, b, alpha))) * math.sqrt(4 * math.pi) == pytest.approx(a0, rel=1e-12)
        for f in (1 - 1e-3, 1 + 1e-3, 1 - 1e-6, 1 + 1e-6):
            assert oracle.a000_biorth(pos, b * f, alpha, mask=mask) < a0
        assert abs(oracle.a000_scale_slope(pos, math.log(b), alpha, mask=mask)) < 1e-14
    assert oracle.a000_scale(pos, 0.3, 1.0, mask=np.zeros(5000, bool)) == 0.3     # empty set keeps b


def test_recentre_degenerate_sets():
    pos, vel = workloads.plummer(200, seed=29)
    # nothing in the set: the frame stays, no core
    p2, v2, c2, xc, V, rc, it = oracle.recentre(pos, vel, np.zeros(6), 4, 2, 0.3, 1.0, mask=np.zeros(200, bool))
    assert it == 0 and np.all(xc == 0) and np.all(V == 0) and rc == 0.0
    assert np.array_equal(p2, pos) and np.array_equal(v2, vel)
    # one particle: the centre moves onto it; at r = 0 it has no core
    one, v1 = pos[:1].copy(), vel[:1].copy()
    p2, v2, c2, xc, V, rc, it = oracle.recentre(one, v1, np.zeros(6), 4, 2, 0.3, 1.0)
    assert np.allclose(xc, one[0, :3], rtol=0, atol=1e-15) and rc == 0.0 and np.all(V == 0)


# --------------------------------------------------------------- alpha and b at the maximum of a_000
def test_lowest_pair_normalisation_derivative():
    """d ln|I_00|/d alpha (digamma form) against central differences of the
    oracle's own closed-form I_00(alpha)."""
    for al in (0.3, 0.7, 1.0, 1.9, 3.0):
        h = 1e-5
        fd = (math.log(abs(oracle.inl(0, 0, 1.0, al + h))) - math.log(abs(oracle.inl(0, 0, 1.0, al - h)))) / (2 * h)
        assert oracle.dln_i00_dalpha(al) == pytest.approx(fd, rel=1e-8)


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5])
def test_a000_alpha_slope_is_the_derivative_of_ln_a000(alpha):
    pos, _ = workloads.plummer(3000, seed=31)
    mask = np.arange(3000) % 7 != 2
    for b in (0.2, 0.45):
        h = 1e-4
        f = lambda al: math.log(oracle.a000_biorth(pos, b, al, mask=mask))
        fd = (-f(alpha + 2 * h) + 8 * f(alpha + h) - 8 * f(alpha - h) + f(alpha - 2 * h)) / (12 * h)
        assert oracle.a000_alpha_slope(pos, alpha, b, mask=mask) == pytest.approx(fd, abs=1e-9)


@pytest.mark.parametrize("alpha0", [0.5, 0.7, 1.0, 1.5])
def test_alpha_and_b_of_the_lowest_order_sphere_are_its_own(alpha0):
    """Cauchy-Schwarz in the energy inner product over the whole family: the
    unit-energy lowest pair of (alpha, b) projects a density most strongly
    when its density is that density, so the joint maximum of a_000 over
    (alpha, b) returns the projected sphere's own exponent and scale."""
    pos = _zhao_sphere(0.37, alpha0, nodes=160)
    al, b = oracle.a000_alpha_scale(pos, 1.0, 0.3)
    assert al == pytest.approx(alpha0, rel=1e-8)
    assert b[0] == pytest.approx(0.37, rel=1e-10)


def test_alpha_and_b_of_samples_and_of_a_batch():
    a = 3 * math.pi / 16
    pos, _ = workloads.plummer(10000, seed=26)                # the alpha = 1/2 lowest-order sphere
    al, b = oracle.a000_alpha_scale(pos, 1.0, 0.3)
    assert al == pytest.approx(0.5, rel=0.02) and b[0] == pytest.approx(a, rel=0.02)
    hp = workloads.hernquist_positions(10000, 0.4, seed=28)   # the alpha = 1 one
    al, b = oracle.a000_alpha_scale(hp, 0.7, 0.3)
    assert al == pytest.approx(1.0, rel=0.03) and b[0] == pytest.approx(0.4, rel=0.03)
    # a joint maximum: a_000 falls when alpha moves with b re-maximised
    def H(x):
        return math.log(oracle.a000_biorth(hp, oracle.a000_scale(hp, 0.4, x), x))
    for f in (1 - 1e-3, 1 + 1e-3):
        assert H(al * f) < H(al)
    # a batch shares alpha; each progenitor keeps its own b; an empty one keeps b0
    p1, _ = workloads.plummer(5000, seed=1)
    p2, _ = workloads.plummer(6000, seed=2)
    p2[:, :3] *= 0.6
    P = np.concatenate([p1, p2])
    mask = np.ones(11000, bool)
    al, b = oracle.a000_alpha_scale(np.concatenate([P, P[:10]]), 1.0, [0.3, 0.2, 0.25],
                                    offsets=[0, 5000, 11000, 11010],
                                    mask=np.concatenate([mask, np.zeros(10, bool)]))
    assert al == pytest.approx(0.5, rel=0.03)
    assert b[0] == pytest.approx(a, rel=0.03) and b[1] == pytest.approx(0.6 * a, rel=0.03) and b[2] == 0.25
