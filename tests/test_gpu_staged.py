"""scf_step_host: one leapfrog step of a state held in host memory.  With
page-locked (mapped) host arrays the step's kernels work on them in place;
with pageable ones the state is staged through device arrays, kernel 3 split
into chunks at block boundaries.  Either way the same kernels run on the same
block maps as scf_step, so the stepped state must be bitwise the one scf_step
gives on device buffers, for any chunk count, precision and progenitor
layout.  Also the FMA-chain peak utility."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2602_13385_gb300 as p
    return p


def _state(n_list, seed, dtype):
    pos_l, vel_l = [], []
    for i, n in enumerate(n_list):
        p, v = workloads.plummer(n, seed=seed + i)
        p[:, 3] /= len(n_list)
        pos_l.append(p)
        vel_l.append(v)
    return np.concatenate(pos_l), np.concatenate(vel_l)


def _run_both(pkg, precision, n_list, chunks, host=True, nmax=10, lmax=6, pinned=True):
    dtype = torch.float64 if precision == "fp64" else torch.float32
    pos, vel = _state(n_list, 11, dtype)
    comps = []
    if host:
        comps = [(workloads.HOST_HERNQUIST, 50.0, 2.0, 0.0), (workloads.HOST_NFW, 300.0, 20.0, 0.0)]
    cfg = pkg.Config(nmax=nmax, lmax=lmax, b=0.3, dt=0.01, precision=precision, host=comps)
    offsets = np.concatenate([[0], np.cumsum(n_list)]).tolist()
    com0 = np.array([[30.0 + i, 0.0, 5.0, 0.0, 0.4, 0.05] for i in range(len(n_list))])
    out = []
    for staged in (False, True):
        sim = pkg.SCF(cfg, offsets=offsets)
        p = torch.tensor(pos, device="cuda", dtype=dtype)
        v = torch.tensor(vel, device="cuda", dtype=dtype)
        c = torch.tensor(com0, device="cuda") if host else None
        a = sim.forces(p, sim.coeffs(p), com=c)
        if staged:
            pin = (lambda t: t.cpu().pin_memory()) if pinned else (lambda t: t.cpu().clone())
            hp, hv, ha = (pin(t) for t in (p, v, a))
            hc = pin(c) if host else None
            p.zero_()      # the call must take the state from the host buffers
            v.zero_()
            a.zero_()
            if host:
                c.zero_()
            for _ in range(2):
                sim.step_host(p, v, a, hp, hv, ha, com=c, host_com=hc, chunks=chunks)
            torch.cuda.synchronize()
            res = [t.numpy().copy() for t in (hp, hv, ha)] + ([hc.numpy().copy()] if host else [])
        else:
            sim.step(p, v, a, com=c, nsteps=2)
            torch.cuda.synchronize()
            res = [t.cpu().numpy() for t in (p, v, a)] + ([c.cpu().numpy()] if host else [])
        rc, st = sim.status()
        assert rc == 0 and st == 0
        sim.close()
        out.append(res)
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("chunks,pinned", [(1, True), (8, True), (1, False), (3, False), (8, False)])
def test_staged_step_is_bitwise_the_device_step(pkg, precision, chunks, pinned):
    ref, got = _run_both(pkg, precision, [20011], chunks, pinned=pinned)
    for r, g in zip(ref, got):
        assert np.array_equal(r, g)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("pinned", [True, False])
def test_staged_step_batch_of_uneven_progenitors(pkg, precision, pinned):
    ref, got = _run_both(pkg, precision, [3001, 17, 12000, 640], 5, pinned=pinned)
    for r, g in zip(ref, got):
        assert np.array_equal(r, g)


def test_staged_step_more_chunks_than_blocks_and_no_host(pkg):
    ref, got = _run_both(pkg, "fp64", [100], 32, host=False, pinned=False)
    for r, g in zip(ref, got):
        assert np.array_equal(r, g)


def test_staged_step_rejects_bad_chunk_counts(pkg):
    from paper_2602_13385_gb300 import _lib
    sim = pkg.SCF(pkg.Config(nmax=4, lmax=2, b=0.3), n=64)
    p = sim.new_particles()
    hp = p.cpu().pin_memory()
    for bad in (0, _lib.SCF_STAGE_MAX_CHUNKS + 1):
        with pytest.raises(_lib.ScfError) as e:
            sim.step_host(p, p.clone(), p.clone(), hp, hp.clone(), hp.clone(), chunks=bad)
        assert e.value.code == -1
    sim.close()


def test_fma_peak_is_plausible(pkg):
    from paper_2602_13385_gb300 import _lib
    f32, ms32 = _lib.scf_fma_peak(_lib.SCF_MIXED, 2000, torch.cuda.current_stream().cuda_stream)
    f64, ms64 = _lib.scf_fma_peak(_lib.SCF_FP64, 50, torch.cuda.current_stream().cuda_stream)
    props = torch.cuda.get_device_properties(0)
    # below the units x SMs x 2.1 GHz ceiling, above a tenth of it
    assert 0.1 * props.multi_processor_count * 128 * 2 * 2.1e9 < f32 < props.multi_processor_count * 128 * 2 * 2.1e9
    assert 0.1 * props.multi_processor_count * 2 * 2 * 2.1e9 < f64 < 1.05 * props.multi_processor_count * 2 * 2 * 2.1e9
    assert ms32 > 0 and ms64 > 0
