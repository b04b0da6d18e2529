"""Pins of the oracle's energy diagnostic (oracle.energy / or_energy):

* the tidal term: the gradient of phi_tid(x) = psi_host(R + x) - psi_host(R)
  + x . a_host(R) is minus the frame's tidal acceleration a_host(R + x) -
  a_host(R) (Sec. 2.1), by fourth-order differences (a dropped x . a_host(R)
  or a wrong sign fails it);
* the self energy W = 1/2 sum m psi_SCF against the direct-summation
  potential energy of the same particles (within the expansion's truncation);
* a Plummer sample in Henon units has E = K + W = -1/4 up to sampling noise;
* the live self-consistent run conserves K + W to second order in dt: the
  expansion's potential is psi(x_i) = sum_j m_j K(x_i, x_j) with a symmetric
  kernel, so the N-body system it defines is Hamiltonian with energy K + W,
  and the leapfrog's energy error falls 4x when dt halves.
"""
import numpy as np

import oracle
import workloads


def fd4(f, x0, h):
    return (-f(x0 + 2 * h) + 8 * f(x0 + h) - 8 * f(x0 - h) + f(x0 - 2 * h)) / (12 * h)


def test_tidal_potential_gradient_is_minus_tidal_acceleration():
    wl = workloads.king_circular(n=256, seed=2, nsteps=1)
    host = oracle.host_struct(wl.host)
    R = wl.com.copy()
    rng = np.random.default_rng(7)
    nmax, lmax, b = 2, 1, 1.0
    A = np.zeros(2 * oracle.n_coef(nmax, lmax))     # no self field: energy = K + U
    for x in rng.normal(scale=5.0, size=(4, 3)):
        def U(s, j):
            p = np.zeros((1, 4))
            p[0, :3] = x
            p[0, j] += s
            p[0, 3] = 1.0
            return oracle.energy(p, np.zeros((1, 4)), A, nmax, lmax, b, com=R, host=host)[2]
        grad = np.array([fd4(lambda s, j=j: U(s, j), 0.0, 1e-2) for j in range(3)])
        tid = oracle.tidal(host, R[:3], x)
        assert np.max(np.abs(grad + tid)) < 1e-7 * np.max(np.abs(tid)), (grad, tid)


def test_self_energy_close_to_direct_summation():
    pos, vel = workloads.plummer(4096, seed=1)
    b = workloads.basis_scale(workloads.half_mass_radius(pos))
    W_direct = 0.5 * np.sum(pos[:, 3] * oracle.direct(pos, pos)[:, 3])
    for nmax, lmax in [(10, 6), (20, 10)]:
        A = oracle.coeffs(pos, nmax, lmax, b)
        W = oracle.energy(pos, vel, A, nmax, lmax, b)[1]
        assert abs(W - W_direct) < 0.01 * abs(W_direct), (nmax, lmax, W, W_direct)


def test_plummer_sample_energy_is_minus_a_quarter():
    pos, vel = workloads.plummer(4096, seed=1)
    b = workloads.basis_scale(workloads.half_mass_radius(pos))
    A = oracle.coeffs(pos, 10, 6, b)
    K, W, U, E = oracle.energy(pos, vel, A, 10, 6, b)
    assert U == 0.0 and abs(E - (K + W)) < 1e-15
    assert abs(E + 0.25) < 0.03
    assert abs(2 * K / abs(W) - 1.0) < 0.1


def test_live_scf_energy_error_is_second_order_in_dt():
    pos, vel = workloads.plummer(512, seed=4)
    b = workloads.basis_scale(workloads.half_mass_radius(pos))
    nmax, lmax = 6, 4
    worst = []
    for dt in (0.02, 0.01, 0.005):
        p, v = pos.copy(), vel.copy()
        A = oracle.coeffs(p, nmax, lmax, b)
        a = oracle.forces(p, A, nmax, lmax, b)
        E0 = oracle.energy(p, v, A, nmax, lmax, b)[3]
        errs = []
        for _ in range(5):      # checkpoints every 0.1 time units
            p, v, a, _, A = oracle.step(p, v, a, nmax, lmax, b, dt, int(round(0.1 / dt)))
            errs.append(abs(oracle.energy(p, v, A, nmax, lmax, b)[3] - E0))
        worst.append(max(errs))
    assert worst[0] / worst[1] > 3.0 and worst[1] / worst[2] > 3.0, worst
    assert worst[2] < 1e-5 * abs(E0)
