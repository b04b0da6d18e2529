"""scf_coeffs_noalloc — the coefficient entry point that allocates nothing.

It serves callers that cannot call cudaMalloc (code inside a memory arena it
must not grow, paths where allocation is not allowed or would synchronise the
device, plugins handed device pointers but no allocator).  Its scratch is a
static device array inside the library.  These tests call it through the C ABI
and compare it with scf_coeffs (on the same coefficient kernel) on two calls
in a row with different inputs
(the scratch keeps the previous call's contents, so the second call checks
that nothing leaks), at the tolerances the other parity tests use: 1e-10 in
double precision, 1e-6 in mixed precision (the two entry points split the
particles into different numbers of blocks, which changes float rounding).
They also compare it with the FP64 oracle directly (its normalisation is its
own code), over particle counts that leave the block map's edge cases (none,
one, less than a tile, a ragged last block), and check that a non-finite
particle is left out and reported by scf_noalloc_status.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10
TOL_BY_PRECISION = {"fp64": 1e-10, "mixed": 1e-6}


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2602_13385_gb300 as p
    from paper_2602_13385_gb300 import _lib
    _lib.load()
    return p


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _noalloc(pkg, cfg, pos, mask=None):
    from paper_2602_13385_gb300 import _lib
    nc = pkg.n_coef(cfg.nmax, cfg.lmax)
    out = torch.full((2 * nc,), float("nan"), dtype=torch.float64, device="cuda")
    _lib.scf_coeffs_noalloc(cfg.to_c(), pos.shape[0], pos, mask, out, torch.cuda.current_stream().cuda_stream)
    return out


def _existing(pkg, cfg, pos, mask=None):
    sim = pkg.SCF(cfg, n=pos.shape[0])
    # scf_coeffs_noalloc runs the one-thread-per-output coefficient kernel;
    # compare with scf_coeffs on that kernel (mixed precision defaults to the
    # register-tiled one, whose float rounding differs)
    sim.set_tiles(k1_tile=128)
    A = sim.coeffs(pos, mask=mask)[0]
    torch.cuda.synchronize()
    sim.close()
    return A


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_scf_coeffs_on_two_calls(pkg, precision):
    dtype = torch.float64 if precision == "fp64" else torch.float32
    cfg1 = pkg.Config(nmax=20, lmax=8, b=0.3, precision=precision)
    pos1, _ = workloads.plummer(30000, seed=71)
    p1 = torch.tensor(pos1, device="cuda", dtype=dtype)
    # second call: different size, degree and a mask, so stale scratch would show
    cfg2 = pkg.Config(nmax=10, lmax=6, b=0.45, precision=precision)
    pos2, _ = workloads.plummer(5003, seed=72)
    p2 = torch.tensor(pos2, device="cuda", dtype=dtype)
    m2 = torch.tensor((np.arange(5003) % 4 != 1).astype(np.uint8), device="cuda")

    A1 = _noalloc(pkg, cfg1, p1)
    A2 = _noalloc(pkg, cfg2, p2, m2)
    torch.cuda.synchronize()
    R1 = _existing(pkg, cfg1, p1)
    R2 = _existing(pkg, cfg2, p2, m2)
    tol = TOL_BY_PRECISION[precision]
    assert _rel(A1.cpu().numpy(), R1.cpu().numpy()) < tol
    assert _rel(A2.cpu().numpy(), R2.cpu().numpy()) < tol


def test_noalloc_allocates_no_device_memory(pkg):
    cfg = pkg.Config(nmax=12, lmax=6, b=0.3)
    pos, _ = workloads.plummer(20000, seed=73)
    p = torch.tensor(pos, device="cuda")
    out = _noalloc(pkg, cfg, p)          # first call on the device: set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    torch_bytes0 = torch.cuda.memory_allocated()
    from paper_2602_13385_gb300 import _lib
    for _ in range(3):
        _lib.scf_coeffs_noalloc(cfg.to_c(), p.shape[0], p, None, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == torch_bytes0
    assert _rel(out.cpu().numpy(), _existing(pkg, cfg, p).cpu().numpy()) < TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(pkg):
    from paper_2602_13385_gb300 import _lib
    cfg = pkg.Config(nmax=40, lmax=12, b=0.3)      # 2 * NC = 7462 > SCF_NOALLOC_MAX_COEFS
    p = torch.zeros((10, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(2 * pkg.n_coef(40, 12), dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.ScfError) as e:
        _lib.scf_coeffs_noalloc(cfg.to_c(), 10, p, None, out, torch.cuda.current_stream().cuda_stream)
    assert e.value.code == -8


def _biorth_err(A, ref, nmax, lmax):
    """max |dA| / max |A| with every coefficient in the bi-orthonormal
    normalisation of Eq. 3a (the scale on which mixed-precision errors are
    stated)."""
    nc = oracle.n_coef(nmax, lmax)
    w = np.zeros(2 * nc)
    for n in range(nmax + 1):
        for l in range(lmax + 1):
            for m in range(l + 1):
                i = oracle.idx(n, l, m, lmax)
                w[i] = w[nc + i] = np.sqrt(abs(oracle.inl(n, l, 1.0))) / ((1 if m == 0 else 2) *
                                                                          np.sqrt(oracle.nlm2(l, m)))
    return float(np.max(np.abs(A - ref) * w) / np.max(np.abs(ref) * w))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nmax,lmax,b", [(20, 10, 0.3), (10, 6, 0.45), (6, 12, 0.25)])
def test_noalloc_matches_oracle(pkg, precision, nmax, lmax, b):
    dtype = torch.float64 if precision == "fp64" else torch.float32
    pos, _ = workloads.plummer(40000, seed=74)
    pos = pos.astype(np.float32).astype(np.float64)      # both precisions see the same values
    cfg = pkg.Config(nmax=nmax, lmax=lmax, b=b, precision=precision)
    A = _noalloc(pkg, cfg, torch.tensor(pos, device="cuda", dtype=dtype)).cpu().numpy()
    ref = oracle.coeffs(pos, nmax, lmax, b)
    if precision == "fp64":
        assert _rel(A, ref) < 1e-10
    else:
        assert _biorth_err(A, ref, nmax, lmax) < 1e-6
    from paper_2602_13385_gb300 import _lib
    assert _lib.scf_noalloc_status(torch.cuda.current_stream().cuda_stream) == (0, 0)


@pytest.mark.parametrize("n", [0, 1, 127, 129, 40000])
def test_noalloc_block_map_edges(pkg, n):
    cfg = pkg.Config(nmax=8, lmax=4, b=0.3)
    pos, _ = workloads.plummer(max(n, 1), seed=75)
    pos = pos[:n]
    A = _noalloc(pkg, cfg, torch.tensor(pos, device="cuda", dtype=torch.float64).reshape(n, 4)).cpu().numpy()
    if n == 0:
        assert np.all(A == 0.0)
        return
    assert _rel(A, oracle.coeffs(pos, 8, 4, 0.3)) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_nonfinite_particle_is_skipped_and_reported(pkg, precision):
    from paper_2602_13385_gb300 import _lib
    dtype = torch.float64 if precision == "fp64" else torch.float32
    pos, _ = workloads.plummer(5000, seed=76)
    pos = pos.astype(np.float32).astype(np.float64)
    bad = pos.copy()
    bad[17, 1] = np.nan
    bad[4001, 3] = np.inf
    keep = np.ones(5000, bool)
    keep[[17, 4001]] = False
    cfg = pkg.Config(nmax=10, lmax=6, b=0.3, precision=precision)
    stream = torch.cuda.current_stream().cuda_stream
    A = _noalloc(pkg, cfg, torch.tensor(bad, device="cuda", dtype=dtype)).cpu().numpy()
    rc, st = _lib.scf_noalloc_status(stream)
    assert rc == -7 and st & _lib.SCF_STATUS_NONFINITE_POS
    ref = oracle.coeffs(pos[keep], 10, 6, 0.3)
    err = _rel(A, ref) if precision == "fp64" else _biorth_err(A, ref, 10, 6)
    assert err < (1e-10 if precision == "fp64" else 1e-6)
    # the next clean call clears the word
    _noalloc(pkg, cfg, torch.tensor(pos, device="cuda", dtype=dtype))
    assert _lib.scf_noalloc_status(stream) == (0, 0)
