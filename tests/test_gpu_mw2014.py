"""MWPotential2014 on the GPU (App. A): the exponentially cut-off power-law
bulge next to the Miyamoto-Nagai disk and NFW halo, in every kernel that
evaluates the host -- the field kernel's tidal term (double, and single
precision in its cancellation-free form), the centre orbit of kernel 2, the
tidal tensor of scf_tidal and the tidal energy of scf_energy -- against the
FP64 oracle, on the paper's validation progenitor and orbits (Sec. 3, Table A3).
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


def rel_acc(a, b):
    na = np.linalg.norm(b[:, :3], axis=1)
    return np.linalg.norm(a[:, :3] - b[:, :3], axis=1) / np.maximum(na, 1e-6 * np.median(na))


@pytest.mark.parametrize("orbit", ["circular_5kpc", "circular_20kpc", "eccentric"])
def test_fp64_forces_and_tidal_term(scf, orbit):
    wl = workloads.mw2014_validation(orbit, n=5000, seed=81)
    host = oracle.host_struct(wl.host)
    A = oracle.coeffs(wl.pos, wl.nmax, wl.lmax, wl.b)
    ref = oracle.forces(wl.pos, A, wl.nmax, wl.lmax, wl.b, com=wl.com, host=host)
    sim = scf.SCF(scf.Config(nmax=wl.nmax, lmax=wl.lmax, b=wl.b, host=list(wl.host)), n=wl.n)
    acc = sim.forces(dev(wl.pos), dev(A[None]), com=dev(wl.com[None])).cpu().numpy()
    e = rel_acc(acc, ref)
    assert e.max() < 1e-10
    # the tidal term alone (zero coefficients), with particles spread to 2 kpc
    far = wl.pos.copy()
    far[:, :3] *= np.geomspace(1.0, 2e3 / wl.units.rv_pc / 20.0, wl.n)[:, None]
    tid = sim.forces(dev(far), dev(np.zeros_like(A)[None]), com=dev(wl.com[None])).cpu().numpy()[:, :3]
    tref = oracle.tidal_many(host, wl.com, far)
    et = np.linalg.norm(tid - tref, axis=1) / np.linalg.norm(tref, axis=1)
    print(f"{orbit}: FP64 acceleration max {e.max():.1e}, tidal term median {np.median(et):.1e} max {et.max():.1e}")
    assert np.median(et) < 1e-12 and et.max() < 1e-9
    assert sim.status() == (0, 0)


@pytest.mark.parametrize("orbit", ["circular_5kpc", "circular_20kpc", "eccentric"])
def test_mixed_tidal_term_without_cancellation(scf, orbit):
    """The single-precision tidal difference of the bulge (divided differences,
    Gauss-Legendre increments of the incomplete gamma function) keeps a few
    float ulps of the term itself, near the centre and far out."""
    wl = workloads.mw2014_validation(orbit, n=5000, seed=82)
    host = oracle.host_struct(wl.host)
    pos = wl.pos.copy()
    pos[:, :3] *= np.geomspace(1e-3, 2e3 / wl.units.rv_pc / 20.0, wl.n)[:, None]
    p32 = pos.astype(np.float32).astype(np.float64)
    com32 = wl.com.copy()
    com32[:3] = wl.com[:3].astype(np.float32)
    nc = oracle.n_coef(wl.nmax, wl.lmax)
    sim = scf.SCF(scf.Config(nmax=wl.nmax, lmax=wl.lmax, b=wl.b, precision="mixed", host=list(wl.host)), n=wl.n)
    tid = sim.forces(dev(p32, torch.float32), dev(np.zeros((1, 2 * nc))), com=dev(com32[None])).cpu().double().numpy()
    tref = oracle.tidal_many(host, com32, p32)
    et = np.linalg.norm(tid[:, :3] - tref, axis=1) / np.linalg.norm(tref, axis=1)
    print(f"{orbit}: mixed tidal term median {np.median(et):.1e}, p99 {np.quantile(et, 0.99):.1e}, max {et.max():.1e}")
    assert np.median(et) < 1e-6 and et.max() < 1e-4
    assert sim.status() == (0, 0)


def test_tidal_scales_and_the_sec31_radii(scf):
    wl = workloads.mw2014_validation("circular_5kpc", n=1000, seed=83)
    host = oracle.host_struct(wl.host)
    u = wl.units                                               # every centre in this cluster's units
    coms = np.array([np.r_[np.array(R) * 1e3 / u.rv_pc, [u.velocity_kms(x) for x in V]]
                     for R, V in workloads.MW2014_ORBITS.values()])
    Mc = np.ones(3)                                            # M_c = 1e5 Msun in these units
    sim = scf.SCF(scf.Config(nmax=2, lmax=1, b=wl.b, host=list(wl.host)), offsets=[0, 10, 20, 30])
    out = sim.tidal(dev(coms), dev(Mc)).cpu().numpy()
    ref = oracle.tidal_scales(host, coms[:, :3], Mc)
    for i in range(3):
        s = np.max(np.abs(ref[i, 9:12]))
        assert np.max(np.abs(out[i, :9] - ref[i, :9])) < 1e-12 * s
        for j in (12, 13, 14, 15):
            assert abs(out[i, j] - ref[i, j]) < 1e-12 * abs(ref[i, j])
    rt_pc = out[:2, 14] * wl.units.rv_pc
    print(f"GPU r_t: 5 kpc {rt_pc[0]:.3f} pc (printed 33.3), 20 kpc {rt_pc[1]:.3f} pc (printed 101.9)")
    assert round(rt_pc[1], 1) == 101.9 and abs(rt_pc[0] / 33.3 - 1) < 0.01


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_leapfrog_on_the_eccentric_validation_orbit(scf, precision):
    """Ten steps (cluster + centre orbit in the MW2014 field) against the
    oracle from the same state; mixed precision at its stated bounds."""
    wl = workloads.mw2014_validation("eccentric", n=4000, seed=84)
    dt = torch.float64 if precision == "fp64" else torch.float32
    pos = wl.pos if precision == "fp64" else wl.pos.astype(np.float32).astype(np.float64)
    vel = wl.vel if precision == "fp64" else wl.vel.astype(np.float32).astype(np.float64)
    host = oracle.host_struct(wl.host)
    A = oracle.coeffs(pos, wl.nmax, wl.lmax, wl.b)
    a0 = oracle.forces(pos, A, wl.nmax, wl.lmax, wl.b, com=wl.com, host=host)
    p1, v1, a1, c1, _ = oracle.step(pos, vel, a0, wl.nmax, wl.lmax, wl.b, wl.dt, 10, com=wl.com, host=host)
    sim = scf.SCF(scf.Config(nmax=wl.nmax, lmax=wl.lmax, b=wl.b, dt=wl.dt, precision=precision,
                             host=list(wl.host)), n=wl.n)
    p, v, a, c = dev(pos, dt), dev(vel, dt), dev(a0, dt), dev(wl.com[None])
    sim.step(p, v, a, com=c, nsteps=10)
    ex = np.max(np.abs(p.cpu().double().numpy()[:, :3] - p1[:, :3]))
    ec = np.max(np.abs(c.cpu().numpy()[0] - c1) / np.abs(c1).max())
    ea = rel_acc(a.cpu().double().numpy(), a1)
    print(f"{precision}: positions {ex:.1e}, centre {ec:.1e}, accelerations median {np.median(ea):.1e}")
    assert ec < 1e-12
    if precision == "fp64":
        assert ex < 1e-10 and ea.max() < 1e-9
    else:
        assert ex < 1e-5 and np.median(ea) < 1e-5
    assert sim.status() == (0, 0)


def test_tidal_energy_with_the_bulge(scf):
    wl = workloads.mw2014_validation("circular_20kpc", n=3000, seed=85)
    host = oracle.host_struct(wl.host)
    A = oracle.coeffs(wl.pos, wl.nmax, wl.lmax, wl.b)
    acc = oracle.forces(wl.pos, A, wl.nmax, wl.lmax, wl.b, com=wl.com, host=host)
    ref = oracle.energy(wl.pos, wl.vel, A, wl.nmax, wl.lmax, wl.b, com=wl.com, host=host)
    sim = scf.SCF(scf.Config(nmax=wl.nmax, lmax=wl.lmax, b=wl.b, host=list(wl.host)), n=wl.n)
    E = sim.energy(dev(wl.pos), dev(wl.vel), dev(acc), com=dev(wl.com[None])).cpu().numpy()[0]
    assert E[2] == pytest.approx(ref[2], rel=1e-8)
    assert E[3] == pytest.approx(ref[3], rel=1e-10)


def test_adjoint_refuses_the_bulge(scf):
    from paper_2602_13385_gb300 import _lib
    wl = workloads.mw2014_validation("circular_5kpc", n=64, seed=86)
    sim = scf.SCF(scf.Config(nmax=2, lmax=1, b=wl.b, host=list(wl.host)), n=wl.n)
    z = torch.zeros(wl.n, 4, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.ScfError, match="UNSUPPORTED"):
        _lib.scf_adjoint_level(sim._h, dev(wl.pos), dev(wl.com[None]), 0.01, True, z, z.clone(),
                               torch.zeros(1, 6, dtype=torch.float64, device="cuda"),
                               torch.zeros(1, 2 * len(wl.host), dtype=torch.float64, device="cuda"))
