"""Mixed precision (float basis, field and state; double coefficient sums and
centre orbit) against the FP64 oracle.

Target: median relative acceleration error <= 1e-5 versus FP64.  The other
bounds below are this build's measured error levels with a safety margin,
stated per quantity:
* coefficients, in the bi-orthonormal normalisation of Eq. 3a (a_nlm =
  S_nlm sqrt|I_nl| / ((2 - delta_m0) N_lm), where every l contributes on
  the same scale): max |da| / max |a| <= 1e-6.  The plain real-form
  max |dS| / max |S| is printed too; it is dominated by the l = lmax terms,
  whose real-form values are large numbers that contribute little potential;
* acceleration: median <= 1e-5, max <= 2e-3 (the max sits on particles whose
  acceleration nearly cancels, e.g. next to the centre);
* tidal term on its own: median relative error <= 1e-5.
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


def f32(x):
    return torch.tensor(np.ascontiguousarray(x), device="cuda", dtype=torch.float32)


def f64(x):
    return torch.tensor(np.ascontiguousarray(x), device="cuda", dtype=torch.float64)


def biorth(nmax, lmax):
    """Weights turning real-form S, T into bi-orthonormal amplitudes a_nlm."""
    w = np.zeros(2 * oracle.n_coef(nmax, lmax))
    nc = oracle.n_coef(nmax, lmax)
    for n in range(nmax + 1):
        for l in range(lmax + 1):
            for m in range(l + 1):
                i = oracle.idx(n, l, m, lmax)
                w[i] = w[nc + i] = np.sqrt(abs(oracle.inl(n, l, 1.0))) / ((1 if m == 0 else 2) *
                                                                          np.sqrt(oracle.nlm2(l, m)))
    return w


def coef_errs(A, ref, nmax, lmax):
    w = biorth(nmax, lmax)
    plain = np.max(np.abs(A - ref)) / np.max(np.abs(ref))
    return np.max(np.abs(A - ref) * w) / np.max(np.abs(ref) * w), plain


def rel_acc(a, b):
    na = np.linalg.norm(b[:, :3], axis=1)
    return np.linalg.norm(a[:, :3] - b[:, :3], axis=1) / np.maximum(na, max(1e-6 * np.median(na), 1e-300))


def make(scf, wl, precision="mixed", offsets=None, b_per_prog=None, host=True):
    cfg = scf.Config(nmax=wl.nmax, lmax=wl.lmax, b=wl.b, dt=wl.dt, precision=precision,
                     host=list(wl.host) if host else [])
    return scf.SCF(cfg, n=None if offsets is not None else wl.n, offsets=offsets, b_per_prog=b_per_prog)


@pytest.mark.parametrize("nmax,lmax,n", [(10, 5, 4096), (10, 6, 4096), (20, 8, 20000), (20, 10, 20000)])
def test_mixed_coefficients(scf, nmax, lmax, n):
    pos, _ = workloads.plummer(n, seed=200 + lmax)
    b = workloads.basis_scale(workloads.half_mass_radius(pos))
    cfg = scf.Config(nmax=nmax, lmax=lmax, b=b, precision="mixed")
    sim = scf.SCF(cfg, n=n)
    A = sim.coeffs(f32(pos)).cpu().numpy()[0]
    # the oracle sums the same float-rounded positions
    ref = oracle.coeffs(pos.astype(np.float32).astype(np.float64), nmax, lmax, b)
    err, plain = coef_errs(A, ref, nmax, lmax)
    print(f"mixed coefficient error ({nmax},{lmax}) N={n}: bi-orthonormal {err:.2e}, real form {plain:.2e}")
    assert err < 1e-6
    assert sim.status() == (0, 0)


def test_mixed_forces_and_tidal_term(scf):
    wl = workloads.plummer_eccentric(n=20000, seed=31, nsteps=1)
    p32 = wl.pos.astype(np.float32).astype(np.float64)
    A = oracle.coeffs(p32, wl.nmax, wl.lmax, wl.b)
    host = oracle.host_struct(wl.host)
    ref = oracle.forces(p32, A, wl.nmax, wl.lmax, wl.b, com=wl.com, host=host)
    sim = make(scf, wl)
    acc = sim.forces(f32(wl.pos), f64(A[None]), com=f64(wl.com[None])).cpu().double().numpy()
    e = rel_acc(acc, ref)
    print(f"mixed acceleration error: median {np.median(e):.2e}, p99 {np.quantile(e, 0.99):.2e}, max {e.max():.2e}")
    assert np.median(e) < 1e-5
    assert e.max() < 2e-3
    # the tidal part alone: with every coefficient zero the kernel returns it
    zero = f64(np.zeros_like(A)[None])
    tid = sim.forces(f32(wl.pos), zero, com=f64(wl.com[None])).cpu().double().numpy()[:, :3]
    tid_ref = np.array([oracle.tidal(host, wl.com[:3], x) for x in p32[:2000, :3]])
    et = np.linalg.norm(tid[:2000] - tid_ref, axis=1) / np.linalg.norm(tid_ref, axis=1)
    print(f"mixed tidal term error: median {np.median(et):.2e}, max {et.max():.2e}")
    assert np.median(et) < 1e-5
    assert et.max() < 1e-4
    assert sim.status() == (0, 0)


@pytest.mark.parametrize("nmax,lmax", [(10, 5), (10, 6), (20, 10)])
@pytest.mark.parametrize("block", [64, 128, 256, 320])
def test_mixed_field_kernel_shapes(scf, nmax, lmax, block):
    """The field kernel's shapes fixed at compile time ((10,5), (20,10)) and a
    runtime one ((10,6)), in every block size, against the oracle on the same
    float-rounded positions, with the host's tidal term and a ragged last block."""
    wl = workloads.plummer_eccentric(n=7001, seed=40 + lmax, nsteps=1)
    p32 = wl.pos.astype(np.float32).astype(np.float64)
    A = oracle.coeffs(p32, nmax, lmax, wl.b)
    ref = oracle.forces(p32, A, nmax, lmax, wl.b, com=wl.com, host=oracle.host_struct(wl.host))
    cfg = scf.Config(nmax=nmax, lmax=lmax, b=wl.b, dt=wl.dt, precision="mixed", host=list(wl.host))
    sim = scf.SCF(cfg, n=wl.n)
    sim.set_tiles(k3_block=block)
    acc = sim.forces(f32(wl.pos), f64(A[None]), com=f64(wl.com[None])).cpu().double().numpy()
    e = rel_acc(acc, ref)
    print(f"({nmax},{lmax}) block {block}: acceleration median {np.median(e):.2e}, max {e.max():.2e}")
    assert np.median(e) < 1e-5 and e.max() < 2e-3
    assert sim.status() == (0, 0)


def test_mixed_step_against_fp64_step(scf):
    wl = workloads.plummer_eccentric(n=8192, seed=32, nsteps=1)
    p32 = wl.pos.astype(np.float32).astype(np.float64)
    v32 = wl.vel.astype(np.float32).astype(np.float64)
    host = oracle.host_struct(wl.host)
    A0 = oracle.coeffs(p32, wl.nmax, wl.lmax, wl.b)
    a0 = oracle.forces(p32, A0, wl.nmax, wl.lmax, wl.b, com=wl.com, host=host)
    rp, rv, ra, rc, rA = oracle.step(p32, v32, a0, wl.nmax, wl.lmax, wl.b, wl.dt, 1, com=wl.com, host=host)
    sim = make(scf, wl)
    p, v, a, c = f32(wl.pos), f32(wl.vel), f32(a0), f64(wl.com[None])
    sim.step(p, v, a, com=c, nsteps=1)
    e = rel_acc(a.cpu().double().numpy(), ra)
    A = sim.last_coeffs().cpu().numpy()[0]
    eA, _ = coef_errs(A, rA, wl.nmax, wl.lmax)
    ex = np.max(np.abs(p.cpu().double().numpy()[:, :3] - rp[:, :3]))
    ec = np.max(np.abs(c.cpu().numpy()[0] - rc))
    print(f"mixed step: accel median {np.median(e):.2e}, coeff {eA:.2e}, pos max abs {ex:.2e}, com {ec:.2e}")
    assert np.median(e) < 1e-5
    assert eA < 1e-6
    assert ex < 1e-5
    assert ec < 1e-9 * np.max(np.abs(rc))      # the centre orbit stays in double precision
    assert sim.status() == (0, 0)


def test_mixed_batched_progenitors(scf):
    sizes = [3000, 17, 0, 9000]
    pos_l, b_l = [], []
    for i, n in enumerate(sizes):
        p, _ = workloads.plummer(max(n, 1), seed=40 + i)
        pos_l.append(p[:n])
        b_l.append(0.28 + 0.03 * i)
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    pos = np.concatenate(pos_l)
    cfg = scf.Config(nmax=12, lmax=6, b=0.3, precision="mixed")
    sim = scf.SCF(cfg, offsets=offsets, b_per_prog=b_l)
    A = sim.coeffs(f32(pos)).cpu().numpy()
    for i, n in enumerate(sizes):
        if n == 0:
            assert np.all(A[i] == 0)
            continue
        ref = oracle.coeffs(pos_l[i].astype(np.float32).astype(np.float64), 12, 6, b_l[i])
        assert coef_errs(A[i], ref, 12, 6)[0] < 1e-6


def test_full_size_eccentric_mixed_workload(scf):
    """The N = 1e6, (20, 10) mixed workload in the launch configuration of the
    benchmark: full coefficient vector against the oracle, accelerations at
    500 sampled particles against the oracle's."""
    wl = workloads.plummer_eccentric()
    p32 = wl.pos.astype(np.float32).astype(np.float64)
    sim = make(scf, wl)
    p = f32(wl.pos)
    A = sim.coeffs(p).cpu().numpy()[0]
    ref_A = oracle.coeffs(p32, wl.nmax, wl.lmax, wl.b)
    eA, eA_plain = coef_errs(A, ref_A, wl.nmax, wl.lmax)
    acc = sim.forces(p, f64(ref_A[None]), com=f64(wl.com[None])).cpu().double().numpy()
    idx = np.random.default_rng(1).choice(wl.n, 500, replace=False)
    ref = oracle.forces(p32[idx], ref_A, wl.nmax, wl.lmax, wl.b, com=wl.com, host=oracle.host_struct(wl.host))
    e = rel_acc(acc[idx], ref)
    print(f"full-size mixed: coeff bi-orthonormal {eA:.2e} (real form {eA_plain:.2e}), "
          f"accel median {np.median(e):.2e} max {e.max():.2e}")
    assert eA < 1e-6
    assert np.median(e) < 1e-5
    assert sim.status() == (0, 0)


@pytest.mark.parametrize("nmax,lmax,n,masked", [(0, 0, 17, False), (10, 6, 1, False), (10, 6, 63, False),
                                                (10, 6, 65, True), (10, 5, 2003, True), (20, 8, 5003, False),
                                                (20, 10, 30000, True),
                                                (40, 12, 4099, False), (3, 1, 1000, False)])
def test_register_tiled_kernel_matches_oracle_and_simple_kernel(scf, nmax, lmax, n, masked):
    """The register-tiled coefficient kernel (the mixed-precision default) on
    ragged sizes (a partial last tile, a single particle, orders that leave
    partly filled 7 x 8 output tiles, nmax = 40 with six radial chunks)
    against the oracle and against the one-thread-per-output kernel."""
    pos, _ = workloads.plummer(max(n, 2), seed=300 + n)
    pos = pos[:n]
    b = workloads.basis_scale(workloads.half_mass_radius(pos)) if n > 4 else 0.3
    mask = (np.arange(n) % 3 != 1).astype(np.uint8) if masked else None
    cfg = scf.Config(nmax=nmax, lmax=lmax, b=b, precision="mixed")
    sim = scf.SCF(cfg, n=n)
    assert sim.tiles()["k1_tile"] == 0          # register-tiled kernel by default
    p = f32(pos)
    m = None if mask is None else torch.tensor(mask, device="cuda")
    A_tiled = sim.coeffs(p, mask=m).cpu().numpy()[0]
    sim.set_tiles(k1_tile=128)
    A_simple = sim.coeffs(p, mask=m).cpu().numpy()[0]
    ref = oracle.coeffs(pos.astype(np.float32).astype(np.float64), nmax, lmax, b, mask=mask)
    e_or, _ = coef_errs(A_tiled, ref, nmax, lmax)
    e_si, _ = coef_errs(A_tiled, A_simple, nmax, lmax)
    nc = oracle.n_coef(nmax, lmax)
    t_m0 = [nc + oracle.idx(k, l, 0, lmax) for k in range(nmax + 1) for l in range(lmax + 1)]
    print(f"tiled kernel ({nmax},{lmax}) N={n}: vs oracle {e_or:.2e}, vs simple kernel {e_si:.2e}")
    assert e_or < 1e-6 and e_si < 1e-6
    assert np.all(A_tiled[t_m0] == 0)          # T_nl0 is identically zero
    assert sim.status() == (0, 0)
