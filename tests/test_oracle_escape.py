"""Pins of the oracle's escape physics (oracle.boundedness, oracle.tidal_scales).

* Boundedness (Sec. 2.2 footnote): the escape speed of a two-body pair, a
  distant test star against the point-mass escape speed of a Plummer sample,
  and the near-total boundedness of an equilibrium Plummer sample; the
  kinetic factor (1 as printed, 1/2 as the standard energy) moves the
  threshold by sqrt(2).
* The energy-based Lagrange radius r_x (Sec. 2.2) against a brute-force scan
  of its definition (the smallest radius that encloses at least the fraction
  x of the bound particles), on small inputs, at x = 1 (the bound radius r_b)
  and with nothing bound.
* Tidal scales: for a point-mass host the tidal tensor has eigenvalues
  GM/R^3 (2, -1, -1), so r_t is the Jacobi radius R (M_c / 3M)^(1/3) and
  dt_int = sqrt(eta) sqrt(R^3 / GM) (Sec. 2.2, Sec. 3.1 footnote); the trace
  of the tidal tensor is -4 pi G rho_host (Poisson's equation) for each host
  component.
* The complete refresh: on a Hernquist sphere of scale a the retuned basis
  scale is a (r_50 = (1 + sqrt 2) a), and b changes only at refreshes.
* The evolve schedule (Sec. 2.2): with every star bound and inside r_x it is
  the plain leapfrog bit for bit; an unbound star beyond r_x leaves the
  cluster's evolution bit for bit unchanged (and changes it when left in the
  coefficient sum); on a circular orbit about a point mass, where dt_int is
  constant and known in closed form, the run splits into ceil(n / k) pieces.
"""
import math

import numpy as np
import pytest

import oracle
import workloads


def _pair(v0, v1):
    pos = np.array([[-0.5, 0.0, 0.0, 0.5], [0.5, 0.0, 0.0, 0.5]])
    vel = np.array([[0.0, v0, 0.0, 0.0], [0.0, 0.0, -v1, 0.0]])
    return pos, vel


def test_pair_escape_speed():
    # each star sees the other's potential G m / d = 0.5: bound iff kin v^2 < 0.5
    pos, vel = _pair(0.999, 1.001)
    E, bound, _, _, Mb = oracle.boundedness(pos, vel)
    assert bound.tolist() == [True, False]
    assert abs(E[0] - (0.5 * 0.999**2 - 0.5)) < 1e-15 and Mb == 0.5
    # the printed form (kin = 1) lowers the escape speed to sqrt(1/2)
    pos, vel = _pair(0.7, 0.71)
    assert oracle.boundedness(pos, vel, kin=1.0)[1].tolist() == [True, False]
    assert oracle.boundedness(pos, vel, kin=0.5)[1].tolist() == [True, True]


def test_distant_star_point_mass_escape_speed():
    pos, vel = workloads.plummer(2048, seed=11)
    D = 60.0
    v_esc = math.sqrt(2.0 * pos[:, 3].sum() / D)     # the cluster is a point mass at D >> r_V
    for f, want in [(0.0, True), (0.9, True), (1.1, False)]:
        p = np.vstack([pos, [[0.0, D, 0.0, 1e-9]]])
        v = np.vstack([vel, [[f * v_esc, 0.0, 0.0, 0.0]]])
        assert bool(oracle.boundedness(p, v)[1][-1]) is want, f


def test_equilibrium_plummer_is_bound():
    pos, vel = workloads.plummer(4096, seed=12)
    _, bound, _, _, Mb = oracle.boundedness(pos, vel)
    assert bound.mean() > 0.995 and Mb > 0.995


def _brute_rx2(r2, bound, frac):
    nb = int(bound.sum())
    if nb == 0:
        return 0.0
    for c in np.sort(r2):                     # candidate radii, smallest first
        if np.count_nonzero(bound & (r2 <= c)) >= frac * nb:
            return float(c)
    raise AssertionError("no candidate")


@pytest.mark.parametrize("frac", [0.01, 0.5, 0.9, 0.999, 1.0])
def test_lagrange_radius_brute_force(frac):
    rng = np.random.default_rng(13)
    n = 61
    pos = np.zeros((n, 4))
    pos[:, :3] = rng.normal(size=(n, 3)) * rng.uniform(0.2, 3.0, size=(n, 1))
    pos[:, 3] = rng.uniform(0.5, 1.5, size=n) / n
    vel = np.zeros((n, 4))
    vel[:, :3] = rng.normal(scale=0.35, size=(n, 3))
    E, bound, rx2, mask, _ = oracle.boundedness(pos, vel, frac=frac)
    assert 5 < bound.sum() < n                 # some of each
    r2 = pos[:, 0] ** 2 + pos[:, 1] ** 2 + pos[:, 2] ** 2
    want = _brute_rx2(r2, bound, frac)
    assert rx2 == want
    assert np.array_equal(mask, r2 <= want)
    if frac == 1.0:                            # the bound radius r_b encloses every bound star
        assert rx2 == r2[bound].max()


def test_nothing_bound():
    pos, vel = workloads.plummer(128, seed=14)
    vel[:, :3] *= 50.0
    E, bound, rx2, mask, Mb = oracle.boundedness(pos, vel)
    assert not bound.any() and rx2 == 0.0 and not mask.any() and Mb == 0.0


def test_tidal_scales_point_mass():
    GM, Mc, eta = 3.0e5, 2.0, 1.0 / 400.0
    R = np.array([[80.0, 30.0, -20.0], [0.0, 0.0, 150.0]])
    host = oracle.host_struct([(oracle.HOST_HERNQUIST, GM, 1e-9, 0.0)])
    out = oracle.tidal_scales(host, R, np.array([Mc, Mc]), eta)
    for i, Ri in enumerate(np.linalg.norm(R, axis=1)):
        w = GM / Ri**3
        assert np.allclose(out[i, 9:12], [2 * w, -w, -w], rtol=1e-7, atol=1e-7 * w)
        assert abs(out[i, 12] - math.sqrt(6.0) * w) < 1e-7 * w
        assert abs(out[i, 14] - Ri * (Mc / (3.0 * GM)) ** (1.0 / 3.0)) < 1e-7 * out[i, 14]
        assert abs(out[i, 15] - math.sqrt(eta) * math.sqrt(Ri**3 / GM)) < 1e-7 * out[i, 15]
        T = out[i, :9].reshape(3, 3)
        n_hat = R[i] / Ri
        assert np.allclose(T, w * (3 * np.outer(n_hat, n_hat) - np.eye(3)), atol=1e-7 * w)


def _rho(kind, M, a, b, P):
    x, y, z = P
    r = math.sqrt(x * x + y * y + z * z)
    if kind == oracle.HOST_HERNQUIST:
        return M * a / (2 * math.pi * r * (r + a) ** 3)
    if kind == oracle.HOST_NFW:
        return M / (4 * math.pi * r * (r + a) ** 2)
    Rc2, zb = x * x + y * y, math.sqrt(z * z + b * b)
    return (b * b * M / (4 * math.pi)) * (a * Rc2 + (a + 3 * zb) * (a + zb) ** 2) / (
        (Rc2 + (a + zb) ** 2) ** 2.5 * zb**3)


@pytest.mark.parametrize("kind,M,a,b", [(oracle.HOST_HERNQUIST, 2.0e3, 1.5, 0.0),
                                        (oracle.HOST_NFW, 5.0e4, 20.0, 0.0),
                                        (oracle.HOST_MN, 1.0e4, 3.0, 0.3)])
def test_tidal_trace_is_minus_four_pi_G_rho(kind, M, a, b):
    host = oracle.host_struct([(kind, M, a, b)])
    pts = np.array([[2.0, 1.0, 0.5], [10.0, -4.0, 0.2], [0.3, 0.2, -1.0]])
    out = oracle.tidal_scales(host, pts, np.ones(3))
    for i, P in enumerate(pts):
        tr = out[i, 0] + out[i, 4] + out[i, 8]
        scale = np.max(np.abs(out[i, 9:12]))
        assert abs(tr + 4 * math.pi * _rho(kind, M, a, b, P)) < 1e-10 * scale, (i, tr)
        assert abs(out[i, 9:12].sum() - tr) < 1e-10 * scale
        assert out[i, 9] >= out[i, 10] >= out[i, 11]


# ---------------------------------------------------------------- the evolve schedule
def test_evolve_without_escapers_is_the_plain_leapfrog():
    # every particle bound and inside r_100: the coefficient set is everything,
    # so refreshing at every integration timestep changes nothing
    pos, vel = workloads.plummer(256, seed=15)
    b = workloads.basis_scale(workloads.half_mass_radius(pos))
    nmax, lmax, dt = 4, 2, 0.01
    assert oracle.boundedness(pos, vel, frac=1.0)[3].all()
    acc = oracle.forces(pos, oracle.coeffs(pos, nmax, lmax, b), nmax, lmax, b)
    p1, v1, a1, _, _ = oracle.step(pos, vel, acc, nmax, lmax, b, dt, 7)
    p2, v2, a2, _, bound, mask, stats, n_int, _ = oracle.evolve(pos, vel, acc, nmax, lmax, b, dt, 7, frac=1.0,
                                                                max_steps=3)
    assert n_int == 3 and mask.all() and stats[3] == 256
    assert np.array_equal(p1, p2) and np.array_equal(v1, v2) and np.array_equal(a1, a2)


def test_escaper_beyond_r_x_does_not_feed_back():
    # an unbound star far outside r_x is left out of Eq. 3b, so the cluster
    # evolves exactly as without it; with the star in the coefficients it would not
    pos, vel = workloads.plummer(384, seed=16)
    b = workloads.basis_scale(workloads.half_mass_radius(pos))
    nmax, lmax, dt, n = 4, 2, 0.01, 384
    D = 40.0
    v_esc = math.sqrt(2.0 / D)
    p_e = np.vstack([pos, [[0.0, 0.0, D, 1.0 / n]]])
    v_e = np.vstack([vel, [[0.0, 0.0, 3.0 * v_esc, 0.0]]])
    E = oracle.boundedness(pos, vel)[0]
    assert np.min(np.abs(E)) > 1e-2 * (1.0 / n) * 40   # no marginal star the escaper's potential could flip
    acc = oracle.forces(pos, oracle.coeffs(pos, nmax, lmax, b), nmax, lmax, b)
    acc_e = oracle.forces(p_e, oracle.coeffs(p_e, nmax, lmax, b, mask=np.r_[np.ones(n), 0]), nmax, lmax, b)
    r1 = oracle.evolve(pos, vel, acc, nmax, lmax, b, dt, 6, max_steps=2)
    r2 = oracle.evolve(p_e, v_e, acc_e, nmax, lmax, b, dt, 6, max_steps=2)
    assert not r2[4][-1] and not r2[5][-1]
    assert np.array_equal(r1[0], r2[0][:n]) and np.array_equal(r1[1], r2[1][:n])
    assert r1[6][0] == r2[6][0] and r1[6][2] == r2[6][2]
    p3 = oracle.step(p_e, v_e, acc_e, nmax, lmax, b, dt, 6)[0]        # escaper left in the sum
    assert np.max(np.abs(p3[:n] - r1[0])) > 1e-12


def test_integration_timestep_count_on_a_circular_orbit():
    # point-mass host: dt_int = sqrt(eta) sqrt(R^3 / GM) is constant on a circular
    # orbit; with dt_int / dt = 7.4 the run is split into ceil(30 / 7) pieces
    GM, eta, dt = 1.0e4, 1.0 / 400.0, 0.01
    R = (7.4 * dt / math.sqrt(eta)) ** (2.0 / 3.0) * GM ** (1.0 / 3.0)
    host = oracle.host_struct([(oracle.HOST_HERNQUIST, GM, 1e-9 * R, 0.0)])
    com = np.array([R, 0.0, 0.0, 0.0, math.sqrt(GM / R), 0.0])
    pos, vel = workloads.plummer(128, seed=17)
    b = workloads.basis_scale(workloads.half_mass_radius(pos))
    acc = oracle.forces(pos, oracle.coeffs(pos, 2, 1, b), 2, 1, b, com=com, host=host)
    out = oracle.evolve(pos, vel, acc, 2, 1, b, dt, 30, com=com, host=host, eta=eta)
    assert out[7] == 5
    ts = oracle.tidal_scales(host, out[3][:3], np.array([1.0]), eta)[0]
    assert 7.0 < ts[15] / dt < 8.0


def test_complete_refresh_retunes_b_to_the_hernquist_scale():
    # a Hernquist sphere of scale a has r_50 = (1 + sqrt 2) a, so the retuned
    # b is the sample's scale (to sampling noise); with no retuning b stays
    a = 0.7
    pos = workloads.hernquist_positions(20000, a, seed=18, rmax_over_b=200.0)
    vel = np.zeros_like(pos)                       # every star bound
    acc = np.zeros_like(pos)
    out = oracle.evolve(pos, vel, acc, 2, 1, 0.3, 1e-4, 1, max_steps=1, retune_every=5)
    assert abs(out[8] - a) < 0.03 * a, out[8]
    assert oracle.evolve(pos, vel, acc, 2, 1, 0.3, 1e-4, 1, max_steps=1)[8] == 0.3
    # a step of 1e-4 barely moves the stars, so retuning at integration
    # timesteps 0 and 2 of 3 gives the same scale as retuning once
    out3 = oracle.evolve(pos, vel, acc, 2, 1, 0.3, 1e-4, 3, max_steps=1, retune_every=2)
    assert out3[7] == 3 and abs(out3[8] - out[8]) < 1e-6 * a
