"""The C ABI builds, loads and exports what include/scf.h declares; argument
validation returns the documented codes before any device work (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_13385_gb300 import _lib
    return _lib.load()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(scf_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "scf_init" in names and "scf_step" in names and len(names) >= 9
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_2602_13385_gb300 import _lib
    assert sorted(_lib.EXPORTS) == sorted(n for n in declared_functions() if n in _lib.EXPORTS)
    for name in declared_functions():
        assert name in _lib.EXPORTS, f"binding lacks {name}"


def test_library_targets_sm103a():
    from paper_2602_13385_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_strerror_is_static_text(lib):
    for code in range(0, -10, -1):
        s = lib.scf_strerror(code)
        assert isinstance(s, bytes) and len(s) > 0
    assert lib.scf_strerror(-99) == b"unknown error code"


def _cfg(**kw):
    from paper_2602_13385_gb300 import _lib
    c = _lib.scf_config()
    c.nmax, c.lmax, c.alpha, c.b, c.G, c.dt, c.precision, c.n_host = 4, 3, 1.0, 0.3, 1.0, 0.01, 0, 0
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _init(lib, cfg, offsets=(0, 10), b=None):
    off = (ctypes.c_int64 * len(offsets))(*offsets)
    h = ctypes.c_void_p()
    bp = None if b is None else (ctypes.c_double * len(b))(*b)
    return lib.scf_init(ctypes.byref(cfg), len(offsets) - 1, off, bp, None, ctypes.byref(h))


def test_init_rejects_bad_arguments_before_device_work(lib):
    assert lib.scf_init(None, 1, None, None, None, None) == -2
    assert _init(lib, _cfg(alpha=0.0)) == -1          # the radial family needs alpha > 0
    assert _init(lib, _cfg(alpha=float("nan"))) == -1
    assert _init(lib, _cfg(alpha=0.05)) == -4         # outside SCF_ALPHA_MIN..SCF_ALPHA_MAX
    assert _init(lib, _cfg(alpha=5.0)) == -4
    assert _init(lib, _cfg(lmax=13)) == -4
    assert _init(lib, _cfg(nmax=41)) == -4
    assert _init(lib, _cfg(nmax=-1)) == -1
    assert _init(lib, _cfg(precision=7)) == -1
    assert _init(lib, _cfg(), offsets=(1, 10)) == -1   # offsets[0] must be 0
    assert _init(lib, _cfg(), offsets=(0, 10, 5)) == -1
    assert _init(lib, _cfg(), b=[-1.0]) == -1
    c = _cfg(n_host=1)
    c.host[0].kind, c.host[0].M, c.host[0].a = 9, 1.0, 1.0
    assert _init(lib, c) == -1
    c.host[0].kind, c.host[0].a = 2, 0.0
    assert _init(lib, c) == -1


def test_null_handle_is_rejected(lib):
    assert lib.scf_coeffs(None, None, None, None) == -2
    assert lib.scf_forces(None, None, None, None, None) == -2
    assert lib.scf_step(None, None, None, None, None, 1) == -2
    assert lib.scf_status(None, None) == -2
    assert lib.scf_adjoint_level(None, None, None, 0.005, 1, None, None, None, None) == -2
    assert lib.scf_energy(None, None, None, None, None, None) == -2
    assert lib.scf_bound(None, None, None, 0.5, 0.999, None, None, None, None) == -2
    assert lib.scf_tidal(None, None, None, 0.0025, None) == -2
    assert lib.scf_set_mask(None, None) == -2
    assert lib.scf_get_scales(None, None) == -2
    assert lib.scf_evolve(None, None, None, None, None, 1, None, None, None, None, None) == -2
    assert lib.scf_recentre(None, None, None, None, None, None, 100, 1e-12, None) == -2
    assert lib.scf_retune_a000(None, None, None) == -2
    assert lib.scf_free(None) == 0


def test_noalloc_binding_checks_extents_before_any_device_work():
    """The C entry point cannot see tensor extents; the binding rejects
    mismatches before it marshals a pointer (CPU tensors suffice here)."""
    torch = pytest.importorskip("torch")
    from paper_2602_13385_gb300 import _lib
    cfg = _cfg(nmax=4, lmax=2)                     # FP64, NC = 5 x 6, 2*NC = 60
    pos = torch.zeros((10, 4), dtype=torch.float64)
    A = torch.zeros(60, dtype=torch.float64)
    with pytest.raises(ValueError, match="shape"):
        _lib.scf_coeffs_noalloc(cfg, 11, pos, None, A)            # n larger than pos
    with pytest.raises(ValueError, match="shape"):
        _lib.scf_coeffs_noalloc(cfg, 10, pos[:, :3].contiguous(), None, A)
    with pytest.raises(TypeError, match="float64"):
        _lib.scf_coeffs_noalloc(cfg, 10, pos.float(), None, A)    # float pos for an FP64 config
    with pytest.raises(TypeError, match="float32"):
        _lib.scf_coeffs_noalloc(_cfg(nmax=4, lmax=2, precision=1), 10, pos, None, A)
    with pytest.raises(ValueError, match="2\\*NC"):
        _lib.scf_coeffs_noalloc(cfg, 10, pos, None, A[:59])        # short output
    with pytest.raises(TypeError, match="float64"):
        _lib.scf_coeffs_noalloc(cfg, 10, pos, None, A.float())
    with pytest.raises(ValueError, match="entries"):
        _lib.scf_coeffs_noalloc(cfg, 10, pos, torch.ones(9, dtype=torch.uint8), A)
    with pytest.raises(TypeError, match="uint8"):
        _lib.scf_coeffs_noalloc(cfg, 10, pos, torch.ones(10, dtype=torch.bool), A)
    with pytest.raises(ValueError, match=">= 0"):
        _lib.scf_coeffs_noalloc(cfg, -1, pos, None, A)
    with pytest.raises(ValueError, match="CUDA"):
        _lib.scf_coeffs_noalloc(cfg, 10, pos, None, A)             # right extents, but host tensors
