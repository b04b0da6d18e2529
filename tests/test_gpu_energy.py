"""scf_energy (kinetic, self, tidal energy per progenitor) on the GPU.

* Against the oracle's or_energy on the same state: kinetic and self energy
  to 1e-10 relative in double precision, the tidal energy to 1e-8 of its size
  (it is a second-order remainder psi(R+x) - psi(R) + x.a(R), evaluated in
  double on the GPU and in long double by the oracle); mixed precision to
  1e-6.
* Energy drift after the first 10 steps, the comparison used once chaos
  separates the trajectories: the isolated Plummer workload (N = 4096,
  (10,6), dt = 0.01, 100 steps) run by the GPU in FP64 and by the oracle, with
  the energy every 10 steps; the two energy histories agree to 1e-8 of |E0|
  and both drift by less than 1e-4 |E0|; the mixed-precision run's history
  agrees with the FP64 one to 1e-5 |E0|.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scf():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2602_13385_gb300 as pkg
    return pkg


def dev(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), device="cuda", dtype=dtype)


def test_energy_matches_oracle_fp64_with_host(scf):
    wl = workloads.king_circular(n=20000, seed=81, nsteps=1)
    host = oracle.host_struct(wl.host)
    A = oracle.coeffs(wl.pos, wl.nmax, wl.lmax, wl.b)
    ref = oracle.energy(wl.pos, wl.vel, A, wl.nmax, wl.lmax, wl.b, com=wl.com, host=host)
    cfg = scf.Config(nmax=wl.nmax, lmax=wl.lmax, b=wl.b, dt=wl.dt, host=list(wl.host))
    sim = scf.SCF(cfg, n=wl.n)
    p, v, c = dev(wl.pos), dev(wl.vel), dev(wl.com[None])
    acc = sim.forces(p, dev(A[None]), com=c)
    E = sim.energy(p, v, acc, com=c).cpu().numpy()[0]
    E2 = sim.energy(p, v, acc, com=c).cpu().numpy()[0]
    print("energy GPU", E, "oracle", ref)
    assert np.array_equal(E, E2)                         # fixed summation order
    assert abs(E[0] - ref[0]) < 1e-10 * abs(ref[0])
    assert abs(E[1] - ref[1]) < 1e-10 * abs(ref[1])
    assert abs(E[2] - ref[2]) < 1e-8 * abs(ref[2])
    assert abs(E[3] - ref[3]) < 1e-10 * (abs(ref[0]) + abs(ref[1]) + abs(ref[2]))
    assert sim.status() == (0, 0)


def test_energy_matches_oracle_mixed(scf):
    wl = workloads.plummer_eccentric(n=50000, seed=82, nsteps=1)
    p32 = wl.pos.astype(np.float32).astype(np.float64)
    v32 = wl.vel.astype(np.float32).astype(np.float64)
    host = oracle.host_struct(wl.host)
    A = oracle.coeffs(p32, wl.nmax, wl.lmax, wl.b)
    ref = oracle.energy(p32, v32, A, wl.nmax, wl.lmax, wl.b, com=wl.com, host=host)
    cfg = scf.Config(nmax=wl.nmax, lmax=wl.lmax, b=wl.b, dt=wl.dt, host=list(wl.host), precision="mixed")
    sim = scf.SCF(cfg, n=wl.n)
    p, v, c = dev(wl.pos, torch.float32), dev(wl.vel, torch.float32), dev(wl.com[None])
    acc = sim.forces(p, dev(A[None]), com=c)
    E = sim.energy(p, v, acc, com=c).cpu().numpy()[0]
    print("mixed energy GPU", E, "oracle", ref)
    for i in range(3):
        assert abs(E[i] - ref[i]) < 1e-6 * abs(ref[i]), (i, E[i], ref[i])


def test_energy_per_progenitor(scf):
    sizes = [3000, 0, 17, 9000]
    pos_l, vel_l = [], []
    for i, n in enumerate(sizes):
        p, v = workloads.plummer(max(n, 1), seed=90 + i)
        pos_l.append(p[:n])
        vel_l.append(v[:n])
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    bs = [0.3 + 0.02 * i for i in range(len(sizes))]
    cfg = scf.Config(nmax=8, lmax=4, b=0.3)
    sim = scf.SCF(cfg, offsets=offsets, b_per_prog=bs)
    p, v = dev(np.concatenate(pos_l)), dev(np.concatenate(vel_l))
    A = sim.coeffs(p)
    acc = sim.forces(p, A)
    E = sim.energy(p, v, acc).cpu().numpy()
    for i, n in enumerate(sizes):
        if n == 0:
            assert np.all(E[i] == 0)
            continue
        ref = oracle.energy(pos_l[i], vel_l[i], A[i].cpu().numpy(), 8, 4, bs[i])
        assert np.max(np.abs(E[i] - ref)) < 1e-10 * np.max(np.abs(ref)), (i, E[i], ref)


def _gpu_history(scf, wl, precision, every=10):
    dtype = torch.float64 if precision == "fp64" else torch.float32
    cfg = scf.Config(nmax=wl.nmax, lmax=wl.lmax, b=wl.b, dt=wl.dt, precision=precision)
    sim = scf.SCF(cfg, n=wl.n)
    p, v = dev(wl.pos, dtype), dev(wl.vel, dtype)
    acc = sim.forces(p, sim.coeffs(p))
    hist = [sim.energy(p, v, acc).cpu().numpy()[0, 3]]
    for _ in range(wl.nsteps // every):
        sim.step(p, v, acc, nsteps=every)
        hist.append(sim.energy(p, v, acc).cpu().numpy()[0, 3])
    assert sim.status() == (0, 0)
    return np.array(hist)


def test_energy_drift_fp64_against_oracle_and_mixed(scf):
    wl = workloads.plummer_isolated()           # N = 4096, (10,6), dt = 0.01, 100 steps
    every = 10
    p, v = wl.pos.copy(), wl.vel.copy()
    A = oracle.coeffs(p, wl.nmax, wl.lmax, wl.b)
    a = oracle.forces(p, A, wl.nmax, wl.lmax, wl.b)
    ref = [oracle.energy(p, v, A, wl.nmax, wl.lmax, wl.b)[3]]
    for _ in range(wl.nsteps // every):
        p, v, a, _, A = oracle.step(p, v, a, wl.nmax, wl.lmax, wl.b, wl.dt, every)
        ref.append(oracle.energy(p, v, A, wl.nmax, wl.lmax, wl.b)[3])
    ref = np.array(ref)
    g64 = _gpu_history(scf, wl, "fp64", every)
    g32 = _gpu_history(scf, wl, "mixed", every)
    E0 = abs(ref[0])
    print("energy drift |E-E0|/|E0|: oracle", np.max(np.abs(ref - ref[0])) / E0,
          "GPU fp64", np.max(np.abs(g64 - g64[0])) / E0, "mixed", np.max(np.abs(g32 - g32[0])) / E0)
    print("fp64 vs oracle", np.max(np.abs(g64 - ref)) / E0, "mixed vs fp64", np.max(np.abs(g32 - g64)) / E0)
    assert np.max(np.abs(g64 - ref)) < 1e-8 * E0
    assert np.max(np.abs(ref - ref[0])) < 1e-4 * E0
    assert np.max(np.abs(g64 - g64[0])) < 1e-4 * E0
    assert np.max(np.abs(g32 - g64)) < 1e-5 * E0
