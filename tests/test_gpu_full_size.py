"""The benchmark's workloads at full size, in the launch configuration the
benchmark uses (the library's autotuner choosing the kernel shapes on the
same particles), against the FP64 oracle.

* Plummer N = 1e6, (nmax, lmax) = (20, 10), FP64, the 5-20 kpc eccentric
  orbit (the headline workload): the full coefficient vector and one
  leapfrog step from the same state (every position, velocity and
  acceleration, and the centre) at the FP64 bound of 1e-10.
* The batch of ten progenitors of uneven N (1.91e6 stars, (20, 10), mixed
  precision): every progenitor's coefficient vector in the bi-orthonormal
  normalisation and accelerations at sampled particles of every progenitor,
  at the mixed-precision bounds (coefficients 1e-6, median acceleration
  error 1e-5).
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


def dev(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), device="cuda", dtype=dtype)


def rel_acc(a, b):
    na = np.linalg.norm(b[:, :3], axis=1)
    return np.linalg.norm(a[:, :3] - b[:, :3], axis=1) / np.maximum(na, max(1e-6 * np.median(na), 1e-300))


def biorth(nmax, lmax):
    """Weights turning real-form S, T into bi-orthonormal amplitudes a_nlm."""
    nc = oracle.n_coef(nmax, lmax)
    w = np.zeros(2 * nc)
    for n in range(nmax + 1):
        for l in range(lmax + 1):
            for m in range(l + 1):
                i = oracle.idx(n, l, m, lmax)
                w[i] = w[nc + i] = np.sqrt(abs(oracle.inl(n, l, 1.0))) / ((1 if m == 0 else 2) *
                                                                          np.sqrt(oracle.nlm2(l, m)))
    return w


def test_headline_fp64_workload_coefficients_and_one_step(scf):
    wl = workloads.plummer_eccentric()
    host = oracle.host_struct(wl.host)
    cfg = scf.Config(nmax=wl.nmax, lmax=wl.lmax, b=wl.b, dt=wl.dt, host=list(wl.host))
    sim = scf.SCF(cfg, n=wl.n)
    p, v, c = dev(wl.pos), dev(wl.vel), dev(wl.com[None])
    sim.autotune(p, com=c, reps=2, cache=False)
    A = sim.coeffs(p).cpu().numpy()[0]
    A_ref = oracle.coeffs(wl.pos, wl.nmax, wl.lmax, wl.b)
    eA = np.max(np.abs(A - A_ref)) / np.max(np.abs(A_ref))
    # one step from the same state: the acceleration at the start is the GPU's
    # (within 1e-13 of the oracle's), given to both
    a = sim.forces(p, sim.coeffs(p), com=c)
    a0 = a.cpu().numpy()
    p1, v1, a1, c1, _ = oracle.step(wl.pos, wl.vel, a0, wl.nmax, wl.lmax, wl.b, wl.dt, 1, com=wl.com, host=host)
    sim.step(p, v, a, com=c, nsteps=1)
    P, V, Acc, C = (t.cpu().numpy() for t in (p, v, a, c))
    ex = np.max(np.abs(P[:, :3] - p1[:, :3])) / np.max(np.abs(p1[:, :3]))
    ev = np.max(np.abs(V[:, :3] - v1[:, :3])) / np.max(np.abs(v1[:, :3]))
    ea = rel_acc(Acc, a1)
    ec = np.max(np.abs(C[0] - c1)) / np.max(np.abs(c1))
    print(f"headline FP64 at full size ({sim.tiles()}): coefficients {eA:.1e}, positions {ex:.1e}, "
          f"velocities {ev:.1e}, accelerations max {ea.max():.1e} median {np.median(ea):.1e}, centre {ec:.1e}")
    assert eA < TOL and ex < TOL and ev < TOL and ea.max() < TOL and ec < TOL
    assert sim.status() == (0, 0)


def test_batch_of_ten_mixed_workload(scf):
    wl = workloads.progenitor_batch()
    host = oracle.host_struct(wl.host)
    off = np.asarray(wl.offsets)
    cfg = scf.Config(nmax=wl.nmax, lmax=wl.lmax, b=wl.b, dt=wl.dt, precision="mixed", host=list(wl.host))
    sim = scf.SCF(cfg, offsets=list(off), b_per_prog=wl.b_per_prog)
    p32 = wl.pos.astype(np.float32).astype(np.float64)
    p = dev(wl.pos, torch.float32)
    c = dev(wl.com_per_prog)
    sim.autotune(p, com=c, reps=2, cache=False)
    A = sim.coeffs(p).cpu().numpy()
    w = biorth(wl.nmax, wl.lmax)
    rng = np.random.default_rng(5)
    A_refs, idx_all = [], []
    for i in range(len(off) - 1):
        s = slice(off[i], off[i + 1])
        ref = oracle.coeffs(p32[s], wl.nmax, wl.lmax, wl.b_per_prog[i])
        e = np.max(np.abs(A[i] - ref) * w) / np.max(np.abs(ref) * w)
        assert e < 1e-6, (i, e)
        A_refs.append(ref)
        idx_all.append(off[i] + rng.choice(off[i + 1] - off[i], 100, replace=False))
    acc = sim.forces(p, dev(np.stack(A_refs)), com=c).cpu().double().numpy()
    errs = []
    for i, idx in enumerate(idx_all):
        ref = oracle.forces(p32[idx], A_refs[i], wl.nmax, wl.lmax, wl.b_per_prog[i], com=wl.com_per_prog[i],
                            host=host)
        errs.append(rel_acc(acc[idx], ref))
    e = np.concatenate(errs)
    print(f"batch of ten at full size ({sim.tiles()}): accelerations median {np.median(e):.1e}, "
          f"p99 {np.quantile(e, 0.99):.1e}, max {e.max():.1e}")
    assert np.median(e) < 1e-5 and e.max() < 2e-3
    assert sim.status() == (0, 0)
