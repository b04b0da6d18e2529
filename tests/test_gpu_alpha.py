"""The CUDA path with the radial family of Eq. 4 away from alpha = 1 (the
general coefficient and field kernels) against the oracle.

Bars, as for alpha = 1: double precision within 1e-10 (coefficients:
max |dA| / max |A|; accelerations: per particle, |a| floored at 1e-6 of the
median), mixed precision median acceleration error <= 1e-5 and bi-orthonormal
coefficient error <= 1e-6.
"""
import math

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


def coef_err(A, B):
    return float(np.max(np.abs(np.asarray(A) - np.asarray(B))) / np.max(np.abs(B)))


def acc_err(a, b):
    na = np.linalg.norm(b[:, :3], axis=1)
    floor = max(1e-6 * np.median(na), 1e-300)
    return np.linalg.norm(a[:, :3] - b[:, :3], axis=1) / np.maximum(na, floor)


def biorth_err(A, ref, nmax, lmax, alpha):
    """Coefficient error in the bi-orthonormal normalisation of Eq. 3a."""
    nc = oracle.n_coef(nmax, lmax)
    w = np.zeros(2 * nc)
    for n in range(nmax + 1):
        for l in range(lmax + 1):
            for m in range(l + 1):
                i = oracle.idx(n, l, m, lmax)
                w[i] = w[nc + i] = math.sqrt(abs(oracle.inl(n, l, 1.0, alpha=alpha))) / (
                    (1 if m == 0 else 2) * math.sqrt(oracle.nlm2(l, m)))
    return float(np.max(np.abs(A - ref) * w) / np.max(np.abs(ref) * w))


def dev(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), device="cuda", dtype=dtype)


def make(scf, nmax, lmax, b, alpha, n=None, offsets=None, host=(), dt=0.01, b_per_prog=None, precision="fp64"):
    cfg = scf.Config(nmax=nmax, lmax=lmax, b=b, dt=dt, host=list(host), precision=precision, alpha=alpha)
    return scf.SCF(cfg, n=n, offsets=offsets, b_per_prog=b_per_prog)


@pytest.mark.parametrize("alpha,nmax,lmax,n", [(0.5, 20, 8, 20000), (1.5, 12, 6, 5003), (2.0, 10, 4, 257),
                                               (0.75, 40, 12, 3001), (0.3, 6, 2, 1), (3.0, 8, 10, 1000)])
def test_fp64_coefficients_and_field_match_oracle(scf, alpha, nmax, lmax, n):
    wl = workloads.plummer_eccentric(n=max(n, 2), seed=600 + n, nsteps=1)
    pos = wl.pos[:n]
    b = workloads.basis_scale(workloads.half_mass_radius(wl.pos), alpha)
    host = oracle.host_struct(wl.host)
    sim = make(scf, nmax, lmax, b, alpha, n=n, host=wl.host)
    assert sim.tiles()["k1_tile"] == 128 and sim.tiles()["k3_block"] == 128
    A = sim.coeffs(dev(pos)).cpu().numpy()[0]
    A_ref = oracle.coeffs(pos, nmax, lmax, b, alpha=alpha)
    eA = coef_err(A, A_ref)
    acc = sim.forces(dev(pos), dev(A_ref[None]), com=dev(wl.com[None])).cpu().numpy()
    ref = oracle.forces(pos, A_ref, nmax, lmax, b, com=wl.com, host=host, alpha=alpha)
    e = acc_err(acc, ref)
    ep = np.max(np.abs(acc[:, 3] - ref[:, 3]) / np.abs(ref[:, 3]))
    print(f"alpha {alpha} ({nmax},{lmax}) N={n}: coefficients {eA:.1e}, accelerations max {e.max():.1e}, "
          f"potential {ep:.1e}")
    assert eA < TOL and e.max() < TOL and ep < TOL
    assert sim.status() == (0, 0)


@pytest.mark.parametrize("alpha", [0.5, 2.0])
def test_fp64_origin_and_axis(scf, alpha):
    """Particles at the origin (the l = 0 radial term left out, alpha > 1
    included) and on the +-z axis."""
    pos, _ = workloads.plummer(300, seed=61)
    pos[0, :3] = 0.0
    pos[1, :2] = 0.0
    pos[2, :2] = 0.0
    pos[2, 2] = -abs(pos[2, 2])
    nmax, lmax, b = 10, 6, 0.35
    sim = make(scf, nmax, lmax, b, alpha, n=300)
    A = sim.coeffs(dev(pos)).cpu().numpy()[0]
    A_ref = oracle.coeffs(pos, nmax, lmax, b, alpha=alpha)
    acc = sim.forces(dev(pos), dev(A_ref[None])).cpu().numpy()
    ref = oracle.forces(pos, A_ref, nmax, lmax, b, alpha=alpha)
    assert np.all(np.isfinite(acc))
    assert coef_err(A, A_ref) < TOL
    scale = np.median(np.linalg.norm(ref[:, :3], axis=1))
    assert np.max(np.abs(acc[:3, :3] - ref[:3, :3])) < TOL * scale
    assert acc_err(acc, ref).max() < TOL
    assert sim.status() == (0, 0)


def test_fp64_steps_match_oracle(scf):
    """Ten kick-drift-kick steps with the host's tidal field (alpha = 1/2)."""
    wl = workloads.plummer_eccentric_cb(n=4000, seed=62, nsteps=10)
    host = oracle.host_struct(wl.host)
    nmax, lmax = 12, 6
    A0 = oracle.coeffs(wl.pos, nmax, lmax, wl.b, alpha=wl.alpha)
    a0 = oracle.forces(wl.pos, A0, nmax, lmax, wl.b, com=wl.com, host=host, alpha=wl.alpha)
    rp, rv, ra, rc, rA = oracle.step(wl.pos, wl.vel, a0, nmax, lmax, wl.b, wl.dt, 10, com=wl.com, host=host,
                                     alpha=wl.alpha)
    sim = make(scf, nmax, lmax, wl.b, wl.alpha, n=wl.n, host=wl.host, dt=wl.dt)
    p, v, a, c = dev(wl.pos), dev(wl.vel), dev(a0), dev(wl.com[None])
    sim.step(p, v, a, com=c, nsteps=10)
    ex = np.max(np.abs(p.cpu().numpy()[:, :3] - rp[:, :3])) / np.max(np.abs(rp[:, :3]))
    ev = np.max(np.abs(v.cpu().numpy()[:, :3] - rv[:, :3])) / np.max(np.abs(rv[:, :3]))
    ea = acc_err(a.cpu().numpy(), ra).max()
    eA = coef_err(sim.last_coeffs().cpu().numpy()[0], rA)
    print(f"10 steps alpha 1/2: x {ex:.1e}, v {ev:.1e}, a {ea:.1e}, A {eA:.1e}")
    assert ex < TOL and ev < TOL and ea < TOL and eA < TOL
    assert np.max(np.abs(c.cpu().numpy()[0] - rc)) < 1e-12 * np.max(np.abs(rc))


def test_fp64_batched_progenitors(scf):
    sizes = [3000, 17, 0, 2001]
    alpha = 0.5
    pos_l, b_l = [], []
    for i, n in enumerate(sizes):
        p, _ = workloads.plummer(max(n, 1), seed=70 + i)
        pos_l.append(p[:n])
        b_l.append(0.5 + 0.05 * i)
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    sim = make(scf, 10, 6, 0.5, alpha, offsets=offsets, b_per_prog=b_l)
    A = sim.coeffs(dev(np.concatenate(pos_l))).cpu().numpy()
    for i, n in enumerate(sizes):
        if n == 0:
            assert np.all(A[i] == 0)
            continue
        assert coef_err(A[i], oracle.coeffs(pos_l[i], 10, 6, b_l[i], alpha=alpha)) < TOL


@pytest.mark.parametrize("alpha,nmax,lmax,n", [(0.5, 20, 10, 20000), (0.5, 10, 5, 3001), (1.5, 12, 6, 5003),
                                                  (0.75, 40, 12, 3001)])
def test_mixed_matches_oracle(scf, alpha, nmax, lmax, n):
    wl = workloads.plummer_eccentric(n=n, seed=640 + n, nsteps=1)
    p32 = wl.pos.astype(np.float32).astype(np.float64)
    b = workloads.basis_scale(workloads.half_mass_radius(wl.pos), alpha)
    host = oracle.host_struct(wl.host)
    sim = make(scf, nmax, lmax, b, alpha, n=n, host=wl.host, precision="mixed")
    assert sim.tiles()["k1_tile"] == 0            # the register-tiled kernel by default
    A = sim.coeffs(dev(wl.pos, torch.float32)).cpu().numpy()[0]
    A_ref = oracle.coeffs(p32, nmax, lmax, b, alpha=alpha)
    eA = biorth_err(A, A_ref, nmax, lmax, alpha)
    sim.set_tiles(k1_tile=128)                     # and the one-thread-per-output kernel
    A_simple = sim.coeffs(dev(wl.pos, torch.float32)).cpu().numpy()[0]
    assert biorth_err(A_simple, A_ref, nmax, lmax, alpha) < 1e-6
    sim.set_tiles(k1_tile=0)
    acc = sim.forces(dev(wl.pos, torch.float32), dev(A_ref[None]), com=dev(wl.com[None])).cpu().double().numpy()
    ref = oracle.forces(p32, A_ref, nmax, lmax, b, com=wl.com, host=host, alpha=alpha)
    e = acc_err(acc, ref)
    print(f"mixed alpha {alpha} ({nmax},{lmax}) N={n}: coefficients {eA:.1e}, accelerations median "
          f"{np.median(e):.1e} max {e.max():.1e}")
    assert eA < 1e-6
    assert np.median(e) < 1e-5 and e.max() < 2e-3
    assert sim.status() == (0, 0)


def test_complete_refresh_retunes_b_for_alpha(scf):
    """Escape-physics run with a complete refresh at every integration
    timestep: the retuned b is the Plummer scale of the bound stars'
    half-mass radius (alpha = 1/2), as the oracle's."""
    pos, vel = workloads.plummer(2000, seed=63)
    nmax, lmax, alpha = 8, 4, 0.5
    b0 = 0.3
    a0 = oracle.forces(pos, oracle.coeffs(pos, nmax, lmax, b0, alpha=alpha), nmax, lmax, b0, alpha=alpha)
    ref = oracle.evolve(pos, vel, a0, nmax, lmax, b0, 0.01, 12, max_steps=4, retune_every=1, alpha=alpha)
    sim = make(scf, nmax, lmax, b0, alpha, n=2000)
    p, v, a = dev(pos), dev(vel), dev(a0)
    sim.evolve(p, v, a, None, nsteps=12, max_steps=4, retune_every=1)
    b_gpu = float(sim.scales().cpu().numpy()[0])
    print(f"retuned b (alpha 1/2): GPU {b_gpu:.15g}, oracle {ref[8]:.15g}")
    assert abs(b_gpu - ref[8]) <= 1e-13 * ref[8]
    assert np.max(np.abs(p.cpu().numpy()[:, :3] - ref[0][:, :3])) < 1e-10 * np.max(np.abs(ref[0][:, :3]))


def test_alpha_options_and_limits(scf):
    from paper_2602_13385_gb300 import _lib
    sim = make(scf, 10, 6, 0.3, 0.5, n=1000)
    for kw in ({"k1_tile": 64}, {"k1_tile": 0}, {"k3_block": 256}, {"k3_variant": 1}, {"k1_variant": 2}):
        # (k1_tile 0, the register-tiled kernel, is single precision only)
        with pytest.raises(_lib.ScfError):
            sim.set_tiles(**kw)
    assert sim.tiles()["k1_tile"] == 128 and sim.tiles()["k3_block"] == 128
    res = sim.autotune(dev(workloads.plummer(1000, seed=64)[0]), cache=False)
    assert res["k1_tile"] == 128 and res["k3_block"] == 128
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(_lib.ScfError, match="INVALID_ARG"):
            make(scf, 10, 6, 0.3, bad, n=10)
    for far in (0.05, 5.0):
        with pytest.raises(_lib.ScfError, match="UNSUPPORTED"):
            make(scf, 10, 6, 0.3, far, n=10)
    # single-precision recurrence scales beyond float range at (40, 12) for alpha = 3
    with pytest.raises(_lib.ScfError, match="UNSUPPORTED"):
        make(scf, 40, 12, 0.3, 3.0, n=10, precision="mixed")
    make(scf, 40, 12, 0.3, 3.0, n=10).close()     # double precision takes it
    # the adjoint kernels are written for alpha = 1
    n = 64
    small = make(scf, 4, 2, 0.3, 0.5, n=n)
    pos = dev(workloads.plummer(n, seed=65)[0])
    xbar, vbar = torch.zeros_like(pos), torch.zeros_like(pos)
    with pytest.raises(_lib.ScfError, match="UNSUPPORTED"):
        _lib.scf_adjoint_level(small._h, pos, None, 1.0, False, xbar, vbar, None, None)


# --------------------------------------------------------------- alpha retuned at complete refreshes
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_retune_alpha_matches_oracle_and_moves_the_handle(scf, precision):
    """alpha and b at the joint maximum of a_000 (Secs. 2, 2.2), from an
    alpha = 1 handle: the GPU's bracket + Illinois root and the oracle's
    bracket + bisection find the same exponent and scale to rounding; the
    handle then runs the general kernels at that exponent and its field is the
    oracle's at (alpha, b)."""
    pos, _ = workloads.plummer(8000, seed=66)
    dt = torch.float64 if precision == "fp64" else torch.float32
    p_ref = pos if precision == "fp64" else pos.astype(np.float32).astype(np.float64)
    mask = (np.arange(8000) % 5 != 3).astype(np.uint8)
    al_ref, b_ref = oracle.a000_alpha_scale(p_ref, 1.0, 0.3, mask=mask.astype(bool))
    nmax, lmax = 8, 4
    sim = make(scf, nmax, lmax, 0.3, 1.0, n=8000, precision=precision)
    p = dev(pos, dt)
    al = sim.retune_alpha(p, torch.tensor(mask, device="cuda"))
    b = float(sim.scales().cpu().numpy()[0])
    print(f"{precision}: alpha GPU {al:.15g} oracle {al_ref:.15g}; b GPU {b:.15g} oracle {b_ref[0]:.15g}")
    assert abs(al - al_ref) < 1e-10 * al_ref and abs(b - b_ref[0]) < 1e-10 * b_ref[0]
    assert abs(al - 0.5) < 0.03            # a Plummer sample: the alpha = 1/2 family
    assert sim.config.alpha == al
    # the handle now expands in the family of exponent al
    A = sim.coeffs(p).cpu().numpy()[0]
    A_ref = oracle.coeffs(p_ref, nmax, lmax, b, alpha=al)
    acc = sim.forces(p, dev(A_ref[None])).cpu().double().numpy()
    ref = oracle.forces(p_ref, A_ref, nmax, lmax, b, alpha=al)
    if precision == "fp64":
        assert coef_err(A, A_ref) < TOL and acc_err(acc, ref).max() < TOL
    else:
        assert biorth_err(A, A_ref, nmax, lmax, al) < 1e-6 and np.median(acc_err(acc, ref)) < 1e-5
    assert sim.status() == (0, 0)


def test_retune_alpha_batch_and_limits(scf):
    from paper_2602_13385_gb300 import _lib
    sizes = [3000, 0, 2500]
    pos_l = []
    for i, n in enumerate(sizes):
        q = workloads.hernquist_positions(max(n, 1), 0.25 + 0.1 * i, seed=70 + i)
        pos_l.append(q[:n])
    P = np.concatenate(pos_l)
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    b0 = [0.3, 0.3, 0.2]
    al_ref, b_ref = oracle.a000_alpha_scale(P, 0.7, b0, offsets=offsets)
    sim = scf.SCF(scf.Config(nmax=4, lmax=2, b=0.3, alpha=0.7), offsets=offsets, b_per_prog=b0)
    al = sim.retune_alpha(dev(P))
    b = sim.scales().cpu().numpy()
    print(f"batch alpha GPU {al:.15g} oracle {al_ref:.15g}; b {b} oracle {b_ref}")
    assert abs(al - al_ref) < 1e-10 * al_ref
    assert b[1] == b0[1] and np.allclose(b[[0, 2]], b_ref[[0, 2]], rtol=1e-10, atol=0)
    for lo, hi in ((0.5, 0.5), (-1.0, 2.0), (0.8, 0.4)):
        with pytest.raises(_lib.ScfError, match="INVALID_ARG"):
            sim.retune_alpha(dev(P), alpha_lo=lo, alpha_hi=hi)
    with pytest.raises(_lib.ScfError, match="UNSUPPORTED"):
        sim.retune_alpha(dev(P), alpha_lo=0.05, alpha_hi=2.0)


def test_evolve_with_alpha_refresh_matches_oracle(scf):
    pos, vel = workloads.plummer(2000, seed=67)
    nmax, lmax, b0 = 6, 4, 0.3
    a0 = oracle.forces(pos, oracle.coeffs(pos, nmax, lmax, b0), nmax, lmax, b0)
    ref = oracle.evolve(pos, vel, a0, nmax, lmax, b0, 0.01, 8, max_steps=4, retune_every=1,
                        retune_rule="alpha_a000", return_alpha=True)
    sim = make(scf, nmax, lmax, b0, 1.0, n=2000)
    p, v, a = dev(pos), dev(vel), dev(a0)
    sim.evolve(p, v, a, None, nsteps=8, max_steps=4, retune_every=1, retune_rule="alpha_a000")
    b_gpu = float(sim.scales().cpu().numpy()[0])
    print(f"evolve alpha refresh: alpha GPU {sim.config.alpha:.15g} oracle {ref[9]:.15g}, b {b_gpu:.15g} "
          f"oracle {ref[8]:.15g}")
    assert abs(sim.config.alpha - ref[9]) < 1e-10 * ref[9]
    assert abs(b_gpu - ref[8]) < 1e-10 * ref[8]
    assert np.max(np.abs(p.cpu().numpy()[:, :3] - ref[0][:, :3])) < 1e-9 * np.max(np.abs(ref[0][:, :3]))
