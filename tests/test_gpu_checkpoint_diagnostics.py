"""Checkpoint / resume and the per-progenitor diagnostics on the GPU.

* A run checkpointed after 3 steps and resumed into a new handle continues
  bit for bit as the uninterrupted run (every reduction has a fixed order),
  in double and in mixed precision, with a host and a coefficient set.
* ``diagnostics.snapshot`` against the oracle: energies, bound count and
  mass, the bound radius, the energy-based Lagrange radii and the count
  outside r_b (bit-exact given the same flags), the tidal radius and
  integration timestep at the centre.
"""
import math

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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_resume_is_bit_for_bit(scf, tmp_path, prec):
    from paper_2602_13385_gb300 import checkpoint
    dtype = torch.float64 if prec == "fp64" else torch.float32
    wl = workloads.king_circular(n=6000, seed=71, nsteps=6)
    cfg = scf.Config(nmax=10, lmax=6, b=wl.b, dt=wl.dt, host=list(wl.host), precision=prec)
    sim = scf.SCF(cfg, n=wl.n)
    p, v, c = dev(wl.pos, dtype), dev(wl.vel, dtype), dev(wl.com[None])
    b, m, st, _ = sim.bound(p, v, frac=0.99)
    sim.set_mask(m)
    a = sim.forces(p, sim.coeffs(p, mask=m), com=c)
    sim.step(p, v, a, com=c, nsteps=3)
    path = str(tmp_path / "run.pt")
    checkpoint.save(path, sim, {"pos": p, "vel": v, "acc": a, "com": c, "mask": m}, step=3)
    sim.step(p, v, a, com=c, nsteps=3)
    torch.cuda.synchronize()
    sim2, state, step = checkpoint.resume(path)
    assert step == 3 and sim2.tiles() == sim.tiles()
    sim2.step(state["pos"], state["vel"], state["acc"], com=state["com"], nsteps=3)
    torch.cuda.synchronize()
    for name, ref in (("pos", p), ("vel", v), ("acc", a), ("com", c)):
        assert torch.equal(state[name], ref), name
    assert sim.status() == (0, 0) and sim2.status() == (0, 0)


def test_diagnostics_snapshot(scf, tmp_path):
    from paper_2602_13385_gb300 import diagnostics
    wl = workloads.king_circular(n=4000, seed=72, nsteps=1)
    vel = wl.vel.copy()
    vel[::40, :3] *= 3.0
    wl.pos[::97, :3] *= 30.0           # some stars far out and unbound: outside r_b
    vel[::97, :3] *= 5.0
    cfg = scf.Config(nmax=8, lmax=4, b=wl.b, dt=wl.dt, host=list(wl.host))
    sim = scf.SCF(cfg, n=wl.n)
    p, v, c = dev(wl.pos), dev(vel), dev(wl.com[None])
    a = sim.forces(p, sim.coeffs(p), com=c)
    rec = diagnostics.snapshot(sim, p, v, a, c, t=1.5)[0]
    E = sim.energy(p, v, a, com=c).cpu().numpy()[0]
    assert (rec["K"], rec["W"], rec["U"], rec["E"]) == tuple(float(e) for e in E)
    _, b_o, rx2_1, _, Mb = oracle.boundedness(wl.pos, vel, frac=1.0)
    assert rec["n_bound"] == b_o.sum() and abs(rec["M_bound"] - Mb) <= 1e-12 * Mb
    assert rec["r_b"] == math.sqrt(rx2_1)
    r2 = wl.pos[:, 0] ** 2 + wl.pos[:, 1] ** 2 + wl.pos[:, 2] ** 2
    assert rec["n_outside_r_b"] == np.count_nonzero(r2 > rx2_1) and 0 < rec["n_outside_r_b"]
    for x in diagnostics.LAGRANGE_FRACTIONS:
        assert rec["lagrange_radii"][f"{x:g}"] == math.sqrt(oracle.boundedness(wl.pos, vel, frac=x)[2]), x
    ts = oracle.tidal_scales(oracle.host_struct(wl.host), wl.com[:3], np.array([rec["M_bound"]]))[0]
    assert abs(rec["r_t"] - ts[14]) <= 1e-12 * ts[14] and abs(rec["dt_int"] - ts[15]) <= 1e-12 * ts[15]
    path = str(tmp_path / "diag.jsonl")
    with diagnostics.JsonlLog(path) as log:
        log.write([rec])
        log.write(diagnostics.snapshot(sim, p, v, a, c, t=2.0))
    back = diagnostics.read_jsonl(path)
    assert len(back) == 2 and back[0] == rec and back[1]["t"] == 2.0
