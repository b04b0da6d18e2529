"""The float-float kernels of double-precision handles (field kernel:
SCF_OPT_K3_VARIANT = 1; coefficient kernel: SCF_OPT_K1_VARIANT = 2) against
the FP64 oracle and the native kernels.

* Coefficients (several shapes, a mask, particles at the origin and on the
  axis): within the 1e-10 bar of the FP64 path and 1e-12 of the native kernel.

* Forces (with the host's tidal term, particles at the origin, on the z axis
  and far outside) from the oracle's coefficients: within the 1e-10 bar of
  the FP64 path, and within 1e-12 of the native double kernel.
* Ten leapfrog steps with a host, both kernels in float-float: the same
  states as the oracle's (1e-10).
* The adjoint (which always runs the native kernel) gives the same result
  whichever variant the handle's forward kernel uses.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def scf():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2602_13385_gb300 as pkg
    return pkg


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), device="cuda", dtype=torch.float64)


def acc_err(a, b):
    na = np.linalg.norm(b[:, :3], axis=1)
    floor = max(1e-6 * np.median(na), 1e-300)
    return np.linalg.norm(a[:, :3] - b[:, :3], axis=1) / np.maximum(na, floor)


def handle(scf, wl_or_cfg, n, variant):
    sim = scf.SCF(wl_or_cfg, n=n)
    sim.set_tiles(k3_block=128, k3_variant=variant)
    assert sim.tiles()["k3_variant"] == variant
    return sim


@pytest.mark.parametrize("nmax,lmax", [(20, 8), (10, 6), (6, 12)])
def test_ff_forces_match_oracle_and_native(scf, nmax, lmax):
    wl = workloads.king_circular(n=4000, seed=81, nsteps=1)
    pos = wl.pos.copy()
    pos[0, :3] = 0.0
    pos[1, :3] = [0.0, 0.0, 0.3]
    pos[2, :3] = [0.0, 0.0, -0.2]
    pos[3, :3] = [40.0, -30.0, 10.0]
    A = oracle.coeffs(wl.pos, nmax, lmax, wl.b)
    host = oracle.host_struct(wl.host)
    ref = oracle.forces(pos, A, nmax, lmax, wl.b, com=wl.com, host=host)
    cfg = scf.Config(nmax=nmax, lmax=lmax, b=wl.b, host=list(wl.host))
    out = {}
    for variant in (0, 1):
        sim = handle(scf, cfg, len(pos), variant)
        out[variant] = sim.forces(dev(pos), dev(A[None]), com=dev(wl.com[None])).cpu().numpy()
        assert sim.status() == (0, 0)
    e_or, e_nat = acc_err(out[1], ref), acc_err(out[1], out[0])
    print(f"({nmax},{lmax}) float-float kernel 3: vs oracle max {e_or.max():.2e} median {np.median(e_or):.2e}; "
          f"vs native max {e_nat.max():.2e}")
    assert e_or.max() < TOL and e_nat.max() < 1e-12
    assert np.max(np.abs(out[1][:, 3] - ref[:, 3]) / np.abs(ref[:, 3])) < TOL


@pytest.mark.parametrize("nmax,lmax", [(20, 8), (10, 6), (6, 12), (3, 1)])
def test_ff_coefficients_match_oracle_and_native(scf, nmax, lmax):
    pos, _ = workloads.plummer(2500, seed=84)
    pos[0, :3] = 0.0
    pos[1, :3] = [0.0, 0.0, 0.4]
    pos[2, :3] = [30.0, 20.0, -10.0]
    mask = (np.arange(len(pos)) % 7 != 3).astype(np.uint8)
    b = 0.3
    ref = oracle.coeffs(pos, nmax, lmax, b, mask=mask)
    cfg = scf.Config(nmax=nmax, lmax=lmax, b=b)
    out = {}
    for variant in (0, 2):
        sim = scf.SCF(cfg, n=len(pos))
        sim.set_tiles(k1_tile=128)
        sim.set_tiles(k1_variant=variant)
        assert sim.tiles()["k1_variant"] == variant
        out[variant] = sim.coeffs(dev(pos), mask=torch.tensor(mask, device="cuda")).cpu().numpy()[0]
        assert sim.status() == (0, 0)
    scale = np.abs(ref).max()
    e_or, e_nat = np.abs(out[2] - ref).max() / scale, np.abs(out[2] - out[0]).max() / scale
    print(f"({nmax},{lmax}) float-float kernel 1: vs oracle {e_or:.2e}, vs native {e_nat:.2e}")
    assert e_or < TOL and e_nat < 1e-12


def test_ff_leapfrog_matches_oracle(scf):
    wl = workloads.king_circular(n=3000, seed=82, nsteps=10)
    host = oracle.host_struct(wl.host)
    A = oracle.coeffs(wl.pos, wl.nmax, wl.lmax, wl.b)
    a0 = oracle.forces(wl.pos, A, wl.nmax, wl.lmax, wl.b, com=wl.com, host=host)
    rp, rv, ra, rc, _ = oracle.step(wl.pos, wl.vel, a0, wl.nmax, wl.lmax, wl.b, wl.dt, wl.nsteps, com=wl.com,
                                    host=host)
    cfg = scf.Config(nmax=wl.nmax, lmax=wl.lmax, b=wl.b, dt=wl.dt, host=list(wl.host))
    sim = handle(scf, cfg, wl.n, 1)
    sim.set_tiles(k1_variant=2)
    assert sim.tiles()["k1_variant"] == 2
    p, v, c = dev(wl.pos), dev(wl.vel), dev(wl.com[None])
    a = dev(a0)
    sim.step(p, v, a, com=c, nsteps=wl.nsteps)
    P, V = p.cpu().numpy(), v.cpu().numpy()
    ex = np.abs(P[:, :3] - rp[:, :3]).max() / np.abs(rp[:, :3]).max()
    ev = np.abs(V[:, :3] - rv[:, :3]).max() / np.abs(rv[:, :3]).max()
    print(f"float-float 10 steps: position {ex:.2e}, velocity {ev:.2e}")
    assert ex < TOL and ev < TOL
    assert sim.status() == (0, 0)


def test_adjoint_unaffected_by_the_variant(scf):
    wl = workloads.king_circular(n=2000, seed=83, nsteps=1)
    cfg = scf.Config(nmax=10, lmax=6, b=wl.b, dt=wl.dt, host=list(wl.host))
    res = []
    for variant in (0, 1):
        sim = handle(scf, cfg, wl.n, variant)
        rng = np.random.default_rng(5)
        xb = dev(np.c_[rng.normal(size=(wl.n, 3)), np.zeros(wl.n)])
        vb = dev(np.c_[rng.normal(size=(wl.n, 3)), np.zeros(wl.n)])
        cb = torch.zeros((1, 6), dtype=torch.float64, device="cuda")
        th = torch.zeros((1, 2 * len(wl.host)), dtype=torch.float64, device="cuda")
        from paper_2602_13385_gb300 import _lib
        _lib.scf_adjoint_level(sim._h, dev(wl.pos), dev(wl.com[None]), 0.005, 1, xb, vb, cb, th)
        res.append((xb.cpu().numpy(), vb.cpu().numpy(), cb.cpu().numpy(), th.cpu().numpy()))
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_ff_coefficients_after_other_kernels(scf):
    """Kernel 1 in float-float stages its recurrence tables in shared memory;
    it must not depend on what earlier kernels left there (a missing barrier
    once let warps read tables another warp had not yet written).  Other
    kernels that fill shared memory run in between, and every result is
    checked against the oracle."""
    pos, vel = workloads.plummer(2500, seed=85)
    b = 0.3
    ref = oracle.coeffs(pos, 20, 8, b)
    scale = np.abs(ref).max()
    cfg = scf.Config(nmax=20, lmax=8, b=b)
    sim = scf.SCF(cfg, n=len(pos))
    sim.set_tiles(k1_tile=128)
    sim.set_tiles(k1_variant=2)
    other = scf.SCF(scf.Config(nmax=20, lmax=8, b=b), n=len(pos))
    p, v = dev(pos), dev(vel)
    for _ in range(3):
        other.bound(p, v)                                  # shared-memory j tiles and histograms
        other.coeffs(p)                                    # the native kernel's staged rows
        A = sim.coeffs(p).cpu().numpy()[0]
        assert np.abs(A - ref).max() / scale < TOL
    assert sim.status() == (0, 0)
