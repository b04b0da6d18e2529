"""The centre's next kick-drift-kick computed ahead (SCF_OPT_CENTRE_AHEAD):
scf_step computes it on a second stream beside kernel 3, and kernel 2 of the
next step takes it only when the state it is about to step is bitwise the
one that was stepped ahead.  Since the same arithmetic produces it from the
same inputs, every stepped state must be bitwise the one of the plain path
(kernel 2 stepping the centre itself), with and without graphs, for one
progenitor and a batch, in both precisions, and when the caller changes the
centre between calls (the key no longer matches, kernel 2 steps it)."""
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


def _state(n_list, seed):
    pos_l, vel_l = [], []
    for i, n in enumerate(n_list):
        p, v = workloads.plummer(n, seed=seed + i)
        p[:, 3] /= len(n_list)
        pos_l.append(p)
        vel_l.append(v)
    return np.concatenate(pos_l), np.concatenate(vel_l)


def _run(pkg, precision, n_list, ahead, graphs, calls, shift_at=None):
    from paper_2602_13385_gb300 import _lib
    dtype = torch.float64 if precision == "fp64" else torch.float32
    pos, vel = _state(n_list, 21)
    host = [(workloads.HOST_HERNQUIST, 50.0, 2.0, 0.0), (workloads.HOST_MN, 400.0, 30.0, 3.0),
            (workloads.HOST_NFW, 300.0, 20.0, 0.0)]
    cfg = pkg.Config(nmax=8, lmax=4, b=0.3, dt=0.02, precision=precision, host=host)
    offsets = np.concatenate([[0], np.cumsum(n_list)]).tolist()
    sim = pkg.SCF(cfg, offsets=offsets)
    _lib.scf_set_option(sim._h, _lib.SCF_OPT_CENTRE_AHEAD, 1 if ahead else 0)
    _lib.scf_set_option(sim._h, _lib.SCF_OPT_GRAPHS, 1 if graphs else 0)
    assert _lib.scf_get_option(sim._h, _lib.SCF_OPT_CENTRE_AHEAD) == (1 if ahead else 0)
    p = torch.tensor(pos, device="cuda", dtype=dtype)
    v = torch.tensor(vel, device="cuda", dtype=dtype)
    com0 = np.array([[40.0 + 3 * i, 2.0, 6.0, 0.1, 0.45, 0.03] for i in range(len(n_list))])
    c = torch.tensor(com0, device="cuda")
    a = sim.forces(p, sim.coeffs(p), com=c)
    trace = []
    for k, nsteps in enumerate(calls):
        if k == shift_at:
            c[:, 0] += 1e-3      # the caller moves the centres: nothing computed ahead applies
        sim.step(p, v, a, com=c, nsteps=nsteps)
        trace.append(c.cpu().numpy().copy())
    torch.cuda.synchronize()
    assert sim.status() == (0, 0)
    out = [t.cpu().numpy() for t in (p, v, a)] + trace
    sim.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("graphs", [True, False])
def test_ahead_is_bitwise_the_plain_centre_step(pkg, precision, graphs):
    calls = [1, 3, 1, 5]
    ref = _run(pkg, precision, [4001], False, graphs, calls)
    got = _run(pkg, precision, [4001], True, graphs, calls)
    for r, g in zip(ref, got):
        assert np.array_equal(r, g)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ahead_batch_and_moved_centres(pkg, precision):
    calls = [2, 2, 4, 1]
    ref = _run(pkg, precision, [1500, 37, 2600], False, True, calls, shift_at=2)
    got = _run(pkg, precision, [1500, 37, 2600], True, True, calls, shift_at=2)
    for r, g in zip(ref, got):
        assert np.array_equal(r, g)
    # and the moved centres did change the orbit (the shift was not a no-op)
    base = _run(pkg, precision, [1500, 37, 2600], True, True, calls)
    assert not np.array_equal(base[-1], got[-1])


def test_option_values(pkg):
    from paper_2602_13385_gb300 import _lib
    sim = pkg.SCF(pkg.Config(nmax=2, lmax=1, b=0.3), n=64)
    assert _lib.scf_get_option(sim._h, _lib.SCF_OPT_CENTRE_AHEAD) == 1
    with pytest.raises(_lib.ScfError) as e:
        _lib.scf_set_option(sim._h, _lib.SCF_OPT_CENTRE_AHEAD, 2)
    assert e.value.code == -1
    sim.close()
