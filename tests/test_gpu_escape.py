"""Escape physics on the GPU (scf_bound, scf_tidal, scf_set_mask, scf_evolve)
against the oracle (oracle.boundedness, oracle.tidal_scales, oracle.evolve).

* Energies: double precision to 1e-12 of the energy scale |kin v^2| + |psi|,
  mixed precision to 5e-6.  Bound flags bit-exact wherever the oracle's
  energy is further from 0 than the tolerance; the radius r_x and the mask
  bit-exact when the flags agree, and in every case r_x is checked to be the
  k-th smallest bound radius of the GPU's own flags.
* Uneven batches (an empty progenitor, a single star, a progenitor with
  nothing bound) progenitor by progenitor; the full-size workloads on a
  sample of particles the oracle sums one by one.
* Tidal scales at the workload centres; the coefficient set inside scf_step;
  the evolve schedule against the oracle's over several integration timesteps.
* The stream comparison used once chaos has separated the trajectories:
  the stream-forming workload (N = 1e5, one radial period of the 5-20 kpc
  orbit, 8000 steps with the escape physics) run in double and in mixed
  precision; the Sec. 3.3 statistics of the unbound stars (density, track,
  width, velocity dispersion, misalignment) agree within 1% on bins of at
  least 500 stars, on the bins of the double-precision run.
"""
import math
import time

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


def _cluster(n, seed, n_fast=0, n_far=0):
    pos, vel = workloads.plummer(n, seed=seed)
    rng = np.random.default_rng(seed + 1000)
    if n_fast:
        k = rng.choice(n, n_fast, replace=False)
        vel[k, :3] *= 3.0
    if n_far:
        k = rng.choice(n, n_far, replace=False)
        pos[k, :3] *= 20.0
    return pos, vel


def _check_rx(pos, bound, frac, rx, mask):
    """r_x is the k-th smallest bound radius for these flags (k = ceil(frac n_b))."""
    r2 = pos[:, 0] * pos[:, 0] + pos[:, 1] * pos[:, 1] + pos[:, 2] * pos[:, 2]
    nb = int(bound.sum())
    if nb == 0:
        assert rx == 0.0
        return
    k = max(1, int(np.ceil(frac * nb)))
    rx2 = rx * rx
    # rx = sqrt(r2_k) exactly: the selected r2 is the bound key whose square root is rx
    sel = r2[bound][np.sqrt(r2[bound]) == rx]
    assert sel.size >= 1
    c = sel[0]
    assert np.count_nonzero(bound & (r2 <= c)) >= k > np.count_nonzero(bound & (r2 < c))
    assert np.array_equal(mask, r2 <= c), "mask is r <= r_x"
    assert abs(rx2 - c) <= 1e-15 * c


def _compare(pos, vel, res, frac, tol, kin=0.5):
    b, m, st, E = res
    b, m, st, E = b.cpu().numpy().astype(bool), m.cpu().numpy().astype(bool), st.cpu().numpy(), E.cpu().numpy()
    E_o, b_o, rx2_o, m_o, Mb_o = oracle.boundedness(pos, vel, kin=kin, frac=frac)
    v2 = vel[:, 0] ** 2 + vel[:, 1] ** 2 + vel[:, 2] ** 2
    scale = kin * v2 + np.abs(E_o - kin * v2)
    err = np.abs(E - E_o) / np.maximum(scale, 1e-300)
    print(f"energy error vs oracle: max {err.max():.3g}, median {np.median(err):.3g}")
    assert err.max() < tol, err.max()
    decided = np.abs(E_o) > 4 * tol * scale
    assert np.array_equal(b[decided], b_o[decided])
    _check_rx(pos, b, frac, st[0, 2] if st.ndim == 2 else st[2], m)
    if np.array_equal(b, b_o):
        assert st[0, 0] == b_o.sum() and st[0, 2] == math.sqrt(rx2_o) and np.array_equal(m, m_o)
        assert abs(st[0, 1] - Mb_o) <= 1e-12 * max(Mb_o, 1e-300) and st[0, 3] == m_o.sum()
    return b, m, st


@pytest.mark.parametrize("frac", [0.5, 0.999, 1.0])
def test_bound_fp64_matches_oracle(scf, frac):
    pos, vel = _cluster(3000, seed=21, n_fast=60, n_far=12)
    sim = scf.SCF(scf.Config(nmax=4, lmax=2, b=0.3), n=3000)
    res = sim.bound(dev(pos), dev(vel), frac=frac, energies=True)
    b, m, st = _compare(pos, vel, res, frac, 1e-12)
    assert 0 < b.sum() < 3000
    res2 = sim.bound(dev(pos), dev(vel), frac=frac, energies=True)
    assert torch.equal(res[3], res2[3]) and torch.equal(res[2], res2[2])      # fixed summation order


def test_bound_kinetic_factor_as_printed(scf):
    pos, vel = _cluster(2000, seed=22, n_fast=30)
    sim = scf.SCF(scf.Config(nmax=4, lmax=2, b=0.3), n=2000)
    res = sim.bound(dev(pos), dev(vel), kin=1.0, frac=0.999, energies=True)
    _compare(pos, vel, res, 0.999, 1e-12, kin=1.0)


def test_bound_mixed_matches_oracle(scf):
    pos, vel = _cluster(4000, seed=23, n_fast=80, n_far=10)
    p32 = pos.astype(np.float32).astype(np.float64)
    v32 = vel.astype(np.float32).astype(np.float64)
    sim = scf.SCF(scf.Config(nmax=4, lmax=2, b=0.3, precision="mixed"), n=4000)
    res = sim.bound(dev(pos, torch.float32), dev(vel, torch.float32), frac=0.999, energies=True)
    _compare(p32, v32, res, 0.999, 5e-6)


def test_bound_uneven_batch(scf):
    sizes = [1500, 0, 1, 800, 1200]
    parts = []
    for i, n in enumerate(sizes):
        p, v = _cluster(max(n, 2), seed=30 + i, n_fast=n // 40)
        p, v = p[:n], v[:n]
        if i == 3:
            v[:, :3] *= 50.0                      # nothing bound
        parts.append((p, v))
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    sim = scf.SCF(scf.Config(nmax=4, lmax=2, b=0.3), offsets=offsets)
    P = np.concatenate([p for p, _ in parts])
    V = np.concatenate([v for _, v in parts])
    b, m, st, E = sim.bound(dev(P), dev(V), frac=0.999, energies=True)
    b, m, st, E = b.cpu().numpy().astype(bool), m.cpu().numpy().astype(bool), st.cpu().numpy(), E.cpu().numpy()
    for i, (p, v) in enumerate(parts):
        s = slice(offsets[i], offsets[i + 1])
        if sizes[i] == 0:
            assert np.all(st[i] == 0)
            continue
        E_o, b_o, rx2_o, m_o, Mb_o = oracle.boundedness(p, v, frac=0.999)
        assert np.array_equal(b[s], b_o), i
        assert np.max(np.abs(E[s] - E_o)) <= 1e-12 * np.max(np.abs(E_o)), i
        assert st[i, 0] == b_o.sum() and st[i, 2] == math.sqrt(rx2_o) and np.array_equal(m[s], m_o), i
        assert abs(st[i, 1] - Mb_o) <= 1e-12 * max(Mb_o, 1e-300) and st[i, 3] == m_o.sum(), i
    assert st[2, 0] == 0 and st[3, 0] == 0 and st[3, 2] == 0.0


@pytest.mark.parametrize("which", ["king_fp64", "plummer_mixed"])
def test_bound_full_size_sampled(scf, which):
    if which == "king_fp64":
        wl, prec, tol = workloads.king_circular(nsteps=1), "fp64", 1e-12
    else:
        wl, prec, tol = workloads.plummer_eccentric(nsteps=1), "mixed", 5e-6
    dtype = torch.float64 if prec == "fp64" else torch.float32
    sim = scf.SCF(scf.Config(nmax=wl.nmax, lmax=wl.lmax, b=wl.b, precision=prec), n=wl.n)
    p, v = dev(wl.pos, dtype), dev(wl.vel, dtype)
    sim.bound(p, v)                                   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b, m, st, E = sim.bound(p, v, energies=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    print(f"{which}: N = {wl.n}, scf_bound {dt * 1e3:.1f} ms, {wl.n**2 / dt:.3g} pairs/s, "
          f"n_bound {st[0, 0].item():.0f}, r_x {st[0, 2].item():.4g}")
    pos = p.double().cpu().numpy()
    vel = v.double().cpu().numpy()
    idx = np.random.default_rng(24).choice(wl.n, 96, replace=False)
    pot = oracle.direct(pos, pos[idx])[:, 3]
    kin = 0.5 * np.sum(vel[idx, :3] ** 2, axis=1)
    E_o = kin + pot
    err = np.abs(E.cpu().numpy()[idx] - E_o) / (kin + np.abs(pot))
    assert err.max() < tol, err.max()
    bb = b.cpu().numpy().astype(bool)
    decided = np.abs(E_o) > 4 * tol * (kin + np.abs(pot))
    assert np.array_equal(bb[idx][decided], E_o[decided] < 0)
    _check_rx(pos, bb, 0.999, st[0, 2].item(), m.cpu().numpy().astype(bool))


def test_tidal_scales_match_oracle(scf):
    cases = [workloads.king_circular(n=1000, nsteps=1), workloads.plummer_eccentric(n=1000, nsteps=1)]
    for wl in cases:
        host = oracle.host_struct(wl.host)
        rng = np.random.default_rng(25)
        coms = np.vstack([wl.com[None]] + [np.r_[wl.com[:3] * rng.uniform(0.3, 1.5) + rng.normal(size=3) * 50,
                                                  wl.com[3:]][None] for _ in range(4)])
        Mc = np.array([1.0, 0.8, 0.5, 0.2, 1e-3])
        cfg = scf.Config(nmax=2, lmax=1, b=wl.b, host=list(wl.host))
        sim = scf.SCF(cfg, offsets=[0, 200, 400, 600, 800, 1000])
        out = sim.tidal(dev(coms), dev(Mc), eta=1.0 / 400.0).cpu().numpy()
        ref = oracle.tidal_scales(host, coms[:, :3], Mc, 1.0 / 400.0)
        for i in range(5):
            s = np.max(np.abs(ref[i, 9:12]))
            assert np.max(np.abs(out[i, :9] - ref[i, :9])) < 1e-12 * s, i
            assert abs(out[i, 9] - ref[i, 9]) < 1e-12 * s and abs(out[i, 13] - ref[i, 13]) < 1e-12 * s, i
            assert np.max(np.abs(out[i, 10:12] - ref[i, 10:12])) < 1e-7 * s, i
            for j in (12, 14, 15):
                assert abs(out[i, j] - ref[i, j]) < 1e-12 * abs(ref[i, j]), (i, j, out[i, j], ref[i, j])
        no_m = sim.tidal(dev(coms), None).cpu().numpy()
        assert np.all(no_m[:, 14] == 0.0)
    iso = scf.SCF(scf.Config(nmax=2, lmax=1, b=0.3), n=10).tidal().cpu().numpy()
    assert np.all(iso[0, :14] == 0.0) and np.isinf(iso[0, 14]) and np.isinf(iso[0, 15])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_step_uses_the_coefficient_set(scf, prec):
    dtype = torch.float64 if prec == "fp64" else torch.float32
    pos, vel = _cluster(5000, seed=26, n_fast=100, n_far=40)
    sim = scf.SCF(scf.Config(nmax=6, lmax=4, b=0.3, precision=prec), n=5000)
    if prec == "mixed":
        sim.set_tiles(k1_tile=128)   # the same coefficient kernel in the step and in coeffs
    p, v = dev(pos, dtype), dev(vel, dtype)
    b, m, st, _ = sim.bound(p, v, frac=0.9)
    assert 0 < m.sum().item() < 5000
    acc = sim.forces(p, sim.coeffs(p, mask=m))
    sim.set_mask(m)
    sim.step(p, v, acc, nsteps=1)
    A_step = sim.last_coeffs()
    assert torch.equal(A_step, sim.coeffs(p, mask=m))
    assert not torch.equal(A_step, sim.coeffs(p))
    sim.set_mask(None)
    sim.step(p, v, acc, nsteps=1)
    assert torch.equal(sim.last_coeffs(), sim.coeffs(p))
    assert sim.status() == (0, 0)


def _evolve_case(scf, prec, host_kind):
    dtype = torch.float64 if prec == "fp64" else torch.float32
    pos, vel = _cluster(2000, seed=27, n_fast=60, n_far=10)
    b = workloads.basis_scale(workloads.half_mass_radius(pos))
    nmax, lmax, dt, eta = 6, 4, 0.01, 1.0 / 400.0
    if host_kind == "point":
        GM = 1.0e4
        R = (7.4 * dt / math.sqrt(eta)) ** (2.0 / 3.0) * GM ** (1.0 / 3.0)
        comps = [(oracle.HOST_HERNQUIST, GM, 1e-9 * R, 0.0)]
        com = np.array([R, 0.0, 0.0, 0.0, math.sqrt(GM / R), 0.0])
        nsteps, max_steps, n_int = 30, 1000, 5
    else:
        wl = workloads.king_circular(n=10, nsteps=1)
        comps, com = list(wl.host), wl.com.copy()
        nsteps, max_steps, n_int = 25, 10, 3
    return dtype, pos, vel, b, nmax, lmax, dt, eta, comps, com, nsteps, max_steps, n_int


@pytest.mark.parametrize("host_kind", ["point", "galaxy"])
def test_evolve_matches_oracle_fp64(scf, host_kind):
    dtype, pos, vel, b, nmax, lmax, dt, eta, comps, com, nsteps, max_steps, n_int = _evolve_case(scf, "fp64",
                                                                                               host_kind)
    host = oracle.host_struct(comps)
    acc0 = oracle.forces(pos, oracle.coeffs(pos, nmax, lmax, b), nmax, lmax, b, com=com, host=host)
    ref = oracle.evolve(pos, vel, acc0, nmax, lmax, b, dt, nsteps, com=com, host=host, eta=eta, max_steps=max_steps)
    assert ref[7] == n_int
    sim = scf.SCF(scf.Config(nmax=nmax, lmax=lmax, b=b, dt=dt, host=comps), n=pos.shape[0])
    p, v, a, c = dev(pos), dev(vel), dev(acc0), dev(com[None])
    bnd, m, st, n = sim.evolve(p, v, a, c, nsteps=nsteps, eta=eta, max_steps=max_steps)
    assert n == n_int
    assert np.array_equal(bnd.cpu().numpy().astype(bool), ref[4])
    assert np.array_equal(m.cpu().numpy().astype(bool), ref[5])
    assert st[0, 0].item() == ref[6][0] and st[0, 2].item() == ref[6][2]
    scale = np.max(np.abs(ref[0][:, :3]))
    assert np.max(np.abs(p.cpu().numpy() - ref[0])) < 1e-10 * scale
    assert np.max(np.abs(v.cpu().numpy() - ref[1])) < 1e-10 * np.max(np.abs(ref[1][:, :3]))
    assert np.max(np.abs(c.cpu().numpy()[0] - ref[3])) < 1e-12 * np.max(np.abs(ref[3]))
    assert sim.status() == (0, 0)


def test_evolve_mixed_against_fp64(scf):
    out = {}
    for prec in ("fp64", "mixed"):
        dtype, pos, vel, b, nmax, lmax, dt, eta, comps, com, nsteps, max_steps, n_int = _evolve_case(scf, prec,
                                                                                                   "galaxy")
        sim = scf.SCF(scf.Config(nmax=nmax, lmax=lmax, b=b, dt=dt, host=comps, precision=prec), n=pos.shape[0])
        p, v, c = dev(pos, dtype), dev(vel, dtype), dev(com[None])
        a = sim.forces(p, sim.coeffs(p), com=c)
        bnd, m, st, n = sim.evolve(p, v, a, c, nsteps=nsteps, eta=eta, max_steps=max_steps)
        out[prec] = (p.double().cpu().numpy(), bnd.cpu().numpy().astype(bool), n)
    assert out["fp64"][2] == out["mixed"][2]
    d = np.abs(out["fp64"][0][:, :3] - out["mixed"][0][:, :3]).max()
    assert d < 1e-4 * np.abs(out["fp64"][0][:, :3]).max(), d
    assert np.mean(out["fp64"][1] != out["mixed"][1]) < 1e-3


@pytest.fixture(scope="module")
def stream_runs(scf):
    wl = workloads.plummer_stream(n=100_000, nsteps=8000)
    out = {}
    for prec in ("fp64", "mixed"):
        dtype = torch.float64 if prec == "fp64" else torch.float32
        sim = scf.SCF(scf.Config(nmax=wl.nmax, lmax=wl.lmax, b=wl.b, dt=wl.dt, host=list(wl.host), precision=prec),
                      n=wl.n)
        p, v, c = dev(wl.pos, dtype), dev(wl.vel, dtype), dev(wl.com[None])
        a = sim.forces(p, sim.coeffs(p), com=c)
        t0 = time.perf_counter()
        _, _, _, n_int = sim.evolve(p, v, a, c, nsteps=wl.nsteps)
        b, m, st, _ = sim.bound(p, v)
        torch.cuda.synchronize()
        cc = c.cpu().numpy()[0]
        out[prec] = dict(X=p.double().cpu().numpy()[:, :3] + cc[:3], V=v.double().cpu().numpy()[:, :3] + cc[3:],
                         com=cc, unbound=b.cpu().numpy() == 0, n_int=n_int, secs=time.perf_counter() - t0)
        assert sim.status() == (0, 0)
    return wl, out


def test_stream_statistics_mixed_against_fp64(stream_runs):
    from paper_2602_13385_gb300 import streams
    wl, out = stream_runs
    f, m = out["fp64"], out["mixed"]
    print("stream run: fp64 %.1f s, mixed %.1f s, %d integration timesteps, %d unbound"
          % (f["secs"], m["secs"], f["n_int"], f["unbound"].sum()))
    assert f["n_int"] == m["n_int"]
    assert np.array_equal(f["com"], m["com"])               # the centre orbit is double precision in both
    assert f["unbound"].sum() > 3000                         # a stream formed
    assert np.mean(f["unbound"] != m["unbound"]) < 1e-3
    results = {}
    for min_count in (500, 100):
        a = streams.stream_stats(f["X"], f["V"], f["com"][:3], f["com"][3:], f["unbound"], min_count=min_count)
        edges = np.concatenate([a["lo"], a["hi"][-1:]])
        b = streams.stream_stats(m["X"], m["V"], m["com"][:3], m["com"][3:], m["unbound"], edges=edges)
        d, ok = streams.compare(a, b, tol=0.01)
        results[min_count] = (len(edges) - 1, d, ok)
        print(f"bins of >= {min_count} stars: {len(edges) - 1} bins, max differences {d}")
    n_bins, d, ok = results[500]
    assert n_bins >= 8 and ok, d
    assert results[100][0] >= 15


def test_evolve_with_complete_refresh_matches_oracle(scf):
    """Complete refreshes (retune_every = 2): b retuned to r_50 / (1 + sqrt 2)
    at integration timesteps 0, 2, 4 as the oracle's schedule does."""
    dtype, pos, vel, b, nmax, lmax, dt, eta, comps, com, nsteps, max_steps, n_int = _evolve_case(scf, "fp64",
                                                                                               "galaxy")
    host = oracle.host_struct(comps)
    acc0 = oracle.forces(pos, oracle.coeffs(pos, nmax, lmax, b), nmax, lmax, b, com=com, host=host)
    ref = oracle.evolve(pos, vel, acc0, nmax, lmax, b, dt, nsteps, com=com, host=host, eta=eta, max_steps=max_steps,
                        retune_every=2)
    assert ref[7] == n_int and ref[8] != b
    sim = scf.SCF(scf.Config(nmax=nmax, lmax=lmax, b=b, dt=dt, host=comps), n=pos.shape[0])
    p, v, a, c = dev(pos), dev(vel), dev(acc0), dev(com[None])
    bnd, m, st, n = sim.evolve(p, v, a, c, nsteps=nsteps, eta=eta, max_steps=max_steps, retune_every=2)
    assert n == n_int
    b_gpu = sim.scales().cpu().numpy()[0]
    print(f"retuned b: GPU {b_gpu:.15g}, oracle {ref[8]:.15g} (initial {b:.6g})")
    assert abs(b_gpu - ref[8]) <= 1e-14 * ref[8]
    assert np.array_equal(bnd.cpu().numpy().astype(bool), ref[4])
    scale = np.max(np.abs(ref[0][:, :3]))
    assert np.max(np.abs(p.cpu().numpy() - ref[0])) < 1e-10 * scale
    assert np.max(np.abs(v.cpu().numpy() - ref[1])) < 1e-10 * np.max(np.abs(ref[1][:, :3]))
    assert sim.status() == (0, 0)
