"""Pins of the oracle's reverse mode (oracle/reverse.py) against definitions
that do not go through it:

* the tidal tensors of App. A against fourth-order differences of the
  oracle's host acceleration, and their symmetry (they are Hessians);
* one level's pull-back (own-position term, the term through the
  coefficients, tidal and centre terms, host parameters) against brute-force
  central differences of the scalar sum_i d_i . a_i(x, R) + w Vbar . g(R)
  with respect to every coordinate of every particle, R and the host
  parameters (a dropped term, a wrong sign or a transposed tensor fails it);
* the whole sweep against central differences of a loss through the
  oracle's forward leapfrog (x_0, v_0, centre state and host parameters).
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle import reverse

NMAX, LMAX = 4, 2


def small_case(n=24, seed=5):
    """A small Plummer cluster in the King-workload units, on the 8 kpc circle."""
    pos, vel = workloads.plummer(n, seed=seed)
    wl = workloads.king_circular(n=512, seed=2, nsteps=1)
    b = workloads.basis_scale(workloads.half_mass_radius(pos))
    return pos, vel, wl.com.copy(), list(wl.host), b


def fd4(f, x0, h):
    return (-f(x0 + 2 * h) + 8 * f(x0 + h) - 8 * f(x0 - h) + f(x0 - 2 * h)) / (12 * h)


@pytest.mark.parametrize("kind", ["hernquist", "nfw", "mn", "all"])
def test_tidal_tensor_matches_force_differences(kind):
    comps = workloads.host_in_units(workloads.galaxy_host_physical(), workloads.Units(1e5, 1.0))
    pick = {"nfw": [comps[0]], "mn": [comps[1]], "hernquist": [comps[2]], "all": comps}[kind]
    host = oracle.host_struct(pick)
    pts = np.array([[3000.0, 500.0, 200.0], [0.0, 0.0, 100.0], [800.0, -300.0, 0.0], [0.0, 0.0, 0.5],
                    [-120.0, 40.0, -900.0]])
    T = oracle.tidal_tensor(host, pts)
    for k, x in enumerate(pts):
        e = 2e-4 * max(np.linalg.norm(x), 1.0)
        J = np.zeros((3, 3))
        for j in range(3):
            dx = np.zeros(3)
            dx[j] = 1.0
            J[:, j] = fd4(lambda s: oracle.host_accel(host, x + s * dx)[0], 0.0, e)
        scale = np.max(np.abs(T[k]))
        assert np.max(np.abs(J - T[k])) < 1e-9 * scale, (kind, k)
        assert np.max(np.abs(T[k] - T[k].T)) <= 1e-14 * scale


def _psi(x, R, Vbar, d, w, b, comps):
    """sum_i d_i . a_i(x, R) + w Vbar . g(R), straight from the oracle's forward pieces."""
    host = oracle.host_struct(comps)
    A = oracle.coeffs(x, NMAX, LMAX, b)
    a = oracle.forces(x, A, NMAX, LMAX, b, com=R, host=host)[:, :3]
    g = oracle.host_accel(host, R[:3])[0]
    return np.sum(d * a) + w * g @ Vbar


def test_level_pullback_matches_brute_force_differences():
    pos, _, com, comps, b = small_case()
    rng = np.random.default_rng(11)
    d = rng.normal(size=(pos.shape[0], 3))
    Vbar = rng.normal(size=3)
    w = 0.01
    dx, dR, dth = reverse.level(pos, com, Vbar, d, w, NMAX, LMAX, b, 1.0, comps)
    # every particle coordinate
    ref = np.zeros_like(dx)
    for k in range(pos.shape[0]):
        for j in range(3):
            def f(s, k=k, j=j):
                x = pos.copy()
                x[k, j] += s
                return _psi(x, com, Vbar, d, w, b, comps)
            ref[k, j] = fd4(f, 0.0, 1e-3 * b)
    assert np.max(np.abs(dx - ref)) < 1e-7 * np.max(np.abs(ref))
    # the centre position
    refR = np.zeros(3)
    for j in range(3):
        def f(s, j=j):
            R = com.copy()
            R[j] += s
            return _psi(pos, R, Vbar, d, w, b, comps)
        refR[j] = fd4(f, 0.0, 0.3)   # well below the disk scale height (~75 length units)
    assert np.max(np.abs(dR - refR)) < 1e-6 * np.max(np.abs(refR))
    # host parameters: GM_c (G = 1) and the scale length a_c
    for c in range(len(comps)):
        for q, rel in ((1, 1e-4), (2, 1e-3)):
            def f(s, c=c, q=q):
                cc = [list(x) for x in comps]
                cc[c][q] *= (1 + s)
                return _psi(pos, com, Vbar, d, w, b, [tuple(x) for x in cc])
            ref_q = fd4(f, 0.0, rel) / comps[c][q]
            got = dth[c, 0 if q == 1 else 1]
            assert abs(got - ref_q) < 1e-6 * abs(ref_q) + 1e-14, (c, q, got, ref_q)


def _loss(pos0, vel0, com0, comps, b, dt, nsteps, gx, gv, gc):
    _, _, p, v, c = reverse.forward(pos0, vel0, com0, NMAX, LMAX, b, dt, nsteps, 1.0, comps)
    return np.sum(gx * p[:, :3]) + np.sum(gv * v[:, :3]) + gc @ c


def test_sweep_matches_differences_of_the_forward_loss():
    pos, vel, com, comps, b = small_case(n=20, seed=6)
    dt, nsteps = 0.01, 3
    rng = np.random.default_rng(12)
    gx = rng.normal(size=(pos.shape[0], 3))
    gv = rng.normal(size=(pos.shape[0], 3))
    gc = rng.normal(size=6) * np.array([1e-3, 1e-3, 1e-3, 1.0, 1.0, 1.0])
    X, C, *_ = reverse.forward(pos, vel, com, NMAX, LMAX, b, dt, nsteps, 1.0, comps)
    xb, vb, cb, th = reverse.sweep(X, C, gx, gv, gc, NMAX, LMAX, b, dt, 1.0, comps)
    # directional derivative along random (dx0, dv0)
    ux = rng.normal(size=(pos.shape[0], 3))
    uv = rng.normal(size=(pos.shape[0], 3))

    def f(s):
        p = pos.copy()
        v = vel.copy()
        p[:, :3] += s * ux
        v[:, :3] += s * uv
        return _loss(p, v, com, comps, b, dt, nsteps, gx, gv, gc)
    ref = fd4(f, 0.0, 1e-3 * b)
    got = np.sum(xb * ux) + np.sum(vb * uv)
    assert abs(got - ref) < 1e-7 * abs(ref)
    # centre state
    for j in range(6):
        def f(s, j=j):
            c = com.copy()
            c[j] += s
            return _loss(pos, vel, c, comps, b, dt, nsteps, gx, gv, gc)
        step = 0.3 if j < 3 else 1e-3 * np.linalg.norm(com[3:])
        ref = fd4(f, 0.0, step)
        assert abs(cb[j] - ref) < 1e-6 * max(abs(ref), 1e-3 * np.max(np.abs(cb))), (j, cb[j], ref)
    # host parameters
    for c in range(len(comps)):
        for q, rel in ((1, 1e-4), (2, 1e-3)):
            def f(s, c=c, q=q):
                cc = [list(x) for x in comps]
                cc[c][q] *= (1 + s)
                return _loss(pos, vel, com, [tuple(x) for x in cc], b, dt, nsteps, gx, gv, gc)
            ref = fd4(f, 0.0, rel) / comps[c][q]
            got = th[c, 0 if q == 1 else 1]
            assert abs(got - ref) < 1e-6 * abs(ref) + 1e-14, (c, q, got, ref)
