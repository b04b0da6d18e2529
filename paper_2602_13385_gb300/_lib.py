"""ctypes binding of the C ABI in include/scf.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: it turns tensors into device pointers, checks that
they are CUDA tensors of the expected dtype, and raises :class:`ScfError` on
a non-zero return code.  The library is built in-tree (``build.py``); when it
cannot be loaded the import fails loudly — there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

SCF_FP64 = 0
SCF_MIXED = 1
SCF_HOST_HERNQUIST = 1
SCF_HOST_NFW = 2
SCF_HOST_MN = 3
SCF_HOST_POWCUT = 4
SCF_MAX_LMAX = 12
SCF_MAX_NMAX = 40
SCF_MAX_HOST_COMPONENTS = 8
SCF_STATUS_NONFINITE_POS = 1
SCF_STATUS_NONFINITE_ACC = 2
SCF_STAGE_MAX_CHUNKS = 32

ERRORS = {
    -1: "SCF_ERR_INVALID_ARG",
    -2: "SCF_ERR_NULL_POINTER",
    -3: "SCF_ERR_MISALIGNED",
    -4: "SCF_ERR_UNSUPPORTED",
    -5: "SCF_ERR_CUDA",
    -6: "SCF_ERR_OUT_OF_MEMORY",
    -7: "SCF_ERR_DEVICE_STATUS",
    -8: "SCF_ERR_TOO_LARGE",
    -9: "SCF_ERR_ADJOINT_FP64",
}

# every symbol include/scf.h declares
EXPORTS = ["scf_init", "scf_coeffs", "scf_forces", "scf_step", "scf_step_host", "scf_last_coeffs", "scf_status",
           "scf_launches_per_call", "scf_profile", "scf_profile_read", "scf_coeffs_noalloc", "scf_noalloc_status", "scf_set_option",
           "scf_get_option", "scf_autotune", "scf_adjoint_level", "scf_energy", "scf_bound", "scf_tidal",
           "scf_set_mask", "scf_evolve", "scf_get_scales", "scf_recentre", "scf_retune_a000", "scf_retune_alpha", "scf_get_alpha", "scf_fma_peak", "scf_free", "scf_strerror"]
SCF_OPT_GRAPHS = 1
SCF_OPT_K1_TILE = 2
SCF_OPT_K3_BLOCK = 3
SCF_OPT_K1_VARIANT = 4
SCF_OPT_K3_VARIANT = 5
SCF_OPT_CENTRE_AHEAD = 6


class ScfError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({strerror(code)})")


class scf_host_component(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("M", ctypes.c_double), ("a", ctypes.c_double), ("b", ctypes.c_double)]


class scf_escape_params(ctypes.Structure):
    _fields_ = [("kin", ctypes.c_double), ("frac", ctypes.c_double), ("eta", ctypes.c_double),
                ("max_steps", ctypes.c_int), ("retune_every", ctypes.c_int), ("recentre", ctypes.c_int),
                ("retune_rule", ctypes.c_int), ("alpha_lo", ctypes.c_double), ("alpha_hi", ctypes.c_double)]


class scf_config(ctypes.Structure):
    _fields_ = [("nmax", ctypes.c_int), ("lmax", ctypes.c_int), ("alpha", ctypes.c_double), ("b", ctypes.c_double),
                ("G", ctypes.c_double), ("dt", ctypes.c_double), ("precision", ctypes.c_int),
                ("n_host", ctypes.c_int), ("host", scf_host_component * SCF_MAX_HOST_COMPONENTS)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build: bool = True) -> ctypes.CDLL:
    """Loads libscf.so (building it first when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libscf.so missing at {_build.LIB}; run paper_2602_13385_gb300.build")
    lib = ctypes.CDLL(_build.LIB)
    vp, i, i64p, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
    lib.scf_init.argtypes = [ctypes.POINTER(scf_config), i, i64p, dp, vp, ctypes.POINTER(vp)]
    lib.scf_coeffs.argtypes = [vp, vp, vp, vp]
    lib.scf_forces.argtypes = [vp, vp, vp, vp, vp]
    lib.scf_step.argtypes = [vp, vp, vp, vp, vp, i]
    lib.scf_step_host.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, i]
    lib.scf_last_coeffs.argtypes = [vp, vp]
    lib.scf_status.argtypes = [vp, ctypes.POINTER(i)]
    lib.scf_launches_per_call.argtypes = [vp, i]
    lib.scf_profile.argtypes = [vp, i]
    lib.scf_profile_read.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_int64)]
    lib.scf_coeffs_noalloc.argtypes = [ctypes.POINTER(scf_config), ctypes.c_int64, vp, vp, vp, vp]
    lib.scf_noalloc_status.argtypes = [vp, ctypes.POINTER(i)]
    lib.scf_set_option.argtypes = [vp, i, i]
    lib.scf_get_option.argtypes = [vp, i, ctypes.POINTER(i)]
    lib.scf_autotune.argtypes = [vp, vp, vp, vp, i, dp]
    lib.scf_adjoint_level.argtypes = [vp, vp, vp, ctypes.c_double, i, vp, vp, vp, vp]
    lib.scf_energy.argtypes = [vp, vp, vp, vp, vp, vp]
    d = ctypes.c_double
    lib.scf_bound.argtypes = [vp, vp, vp, d, d, vp, vp, vp, vp]
    lib.scf_tidal.argtypes = [vp, vp, vp, d, vp]
    lib.scf_set_mask.argtypes = [vp, vp]
    lib.scf_get_scales.argtypes = [vp, vp]
    lib.scf_recentre.argtypes = [vp, vp, vp, vp, vp, vp, i, d, dp]
    lib.scf_retune_a000.argtypes = [vp, vp, vp]
    lib.scf_retune_alpha.argtypes = [vp, vp, vp, d, d, dp]
    lib.scf_get_alpha.argtypes = [vp, dp]
    lib.scf_evolve.argtypes = [vp, vp, vp, vp, vp, i, ctypes.POINTER(scf_escape_params), vp, vp, vp,
                               ctypes.POINTER(i)]
    lib.scf_fma_peak.argtypes = [i, i, vp, dp, dp]
    lib.scf_free.argtypes = [vp]
    lib.scf_strerror.argtypes = [i]
    lib.scf_strerror.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "scf_strerror":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(x, dtype=None):
    """Device pointer of a CUDA tensor (or an int / None passed through)."""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"expected a torch tensor, got {type(x)}")
    if not x.is_cuda:
        raise ValueError("the SCF library takes CUDA tensors only (no CPU path)")
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and x.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {x.dtype}")
    return ctypes.c_void_p(x.data_ptr())


def _host_ptr(x, dtype=None):
    """Address of a contiguous CPU tensor (page-locked for overlapped copies)."""
    if x is None:
        return None
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"expected a torch tensor, got {type(x)}")
    if x.is_cuda:
        raise ValueError("expected a host (CPU) tensor")
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and x.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {x.dtype}")
    return ctypes.c_void_p(x.data_ptr())


def _check(rc: int, where: str):
    if rc != 0:
        raise ScfError(rc, where)


def strerror(code: int) -> str:
    return load(build=False).scf_strerror(int(code)).decode() if _lib is not None else str(code)


def scf_init(cfg: scf_config, offsets, b_per_prog=None, stream: int = 0):
    lib = load()
    n_prog = len(offsets) - 1
    off = (ctypes.c_int64 * len(offsets))(*[int(o) for o in offsets])
    bp = None if b_per_prog is None else (ctypes.c_double * n_prog)(*[float(b) for b in b_per_prog])
    h = ctypes.c_void_p()
    _check(lib.scf_init(ctypes.byref(cfg), n_prog, off, bp, ctypes.c_void_p(stream), ctypes.byref(h)), "scf_init")
    return h


def scf_coeffs(h, pos, mask, A_out):
    import torch
    _check(load().scf_coeffs(h, _ptr(pos), _ptr(mask, torch.uint8), _ptr(A_out, torch.float64)), "scf_coeffs")


def scf_forces(h, pos, A, com, acc):
    import torch
    _check(load().scf_forces(h, _ptr(pos), _ptr(A, torch.float64), _ptr(com, torch.float64), _ptr(acc)),
           "scf_forces")


def scf_step(h, pos, vel, acc, com, nsteps: int):
    import torch
    _check(load().scf_step(h, _ptr(pos), _ptr(vel), _ptr(acc), _ptr(com, torch.float64), int(nsteps)), "scf_step")


def scf_step_host(h, pos, vel, acc, com, host_pos, host_vel, host_acc, host_com, chunks: int = 8):
    """One step of a state held in host tensors (read and overwritten), staged
    through the device tensors with copies overlapped with the kernels."""
    import torch
    for d, hst, nm in ((pos, host_pos, "pos"), (vel, host_vel, "vel"), (acc, host_acc, "acc"), (com, host_com, "com")):
        if (d is None) != (hst is None):
            raise ValueError(f"{nm}: give both the device and the host tensor, or neither")
        if d is not None and (hst.dtype != d.dtype or hst.numel() < d.numel()):
            raise ValueError(f"host {nm} must match the device tensor's dtype and size")
    _check(load().scf_step_host(h, _ptr(pos), _ptr(vel), _ptr(acc), _ptr(com, torch.float64), _host_ptr(host_pos),
                                _host_ptr(host_vel), _host_ptr(host_acc), _host_ptr(host_com, torch.float64),
                                int(chunks)), "scf_step_host")


def scf_last_coeffs(h, A_out):
    import torch
    _check(load().scf_last_coeffs(h, _ptr(A_out, torch.float64)), "scf_last_coeffs")


def scf_status(h):
    """Returns (return code, status bits); does not raise on device status."""
    st = ctypes.c_int(0)
    rc = load().scf_status(h, ctypes.byref(st))
    if rc not in (0, -7):
        raise ScfError(rc, "scf_status")
    return rc, st.value


def scf_launches_per_call(h, which: int) -> int:
    return int(load().scf_launches_per_call(h, int(which)))


def scf_profile(h, enable: bool):
    _check(load().scf_profile(h, 1 if enable else 0), "scf_profile")


def scf_profile_read(h):
    """Returns ([ms_k1, ms_k2, ms_k3], [launches_k1, launches_k2, launches_k3])."""
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_int64 * 3)()
    _check(load().scf_profile_read(h, ms, n), "scf_profile_read")
    return list(ms), list(n)


def scf_coeffs_noalloc(cfg: scf_config, n: int, pos, mask, A_out, stream: int = 0):
    """Coefficients of one cluster through the entry point that allocates
    nothing (its scratch is a static device array inside the library).  The
    C side cannot see the tensors' extents, so they are checked here: pos
    (n, 4) of the precision's dtype, mask n bytes, A_out 2 NC doubles, all on
    the current device."""
    import torch
    n = int(n)
    nc = (cfg.nmax + 1) * (cfg.lmax + 1) * (cfg.lmax + 2) // 2
    want = {SCF_FP64: torch.float64, SCF_MIXED: torch.float32}.get(cfg.precision)
    for t, nm in ((pos, "pos"), (mask, "mask"), (A_out, "A_out")):
        if t is not None and not isinstance(t, torch.Tensor):
            raise TypeError(f"{nm} must be a torch tensor")
    if n < 0:
        raise ValueError("n must be >= 0")
    if pos is None or A_out is None:
        raise ValueError("pos and A_out are required")
    if tuple(pos.shape) != (n, 4):
        raise ValueError(f"pos must have shape ({n}, 4), got {tuple(pos.shape)}")
    if want is not None and pos.dtype != want:
        raise TypeError(f"pos must be {want} for this precision, got {pos.dtype}")
    if mask is not None:
        if mask.dtype != torch.uint8:
            raise TypeError(f"mask must be uint8, got {mask.dtype}")
        if mask.numel() < n:
            raise ValueError(f"mask has {mask.numel()} entries for {n} particles")
    if A_out.dtype != torch.float64:
        raise TypeError(f"A_out must be float64, got {A_out.dtype}")
    if A_out.numel() < 2 * nc:
        raise ValueError(f"A_out holds {A_out.numel()} doubles, needs 2*NC = {2 * nc}")
    if A_out.is_cuda:
        cur = torch.cuda.current_device()
        for t, nm in ((pos, "pos"), (mask, "mask"), (A_out, "A_out")):
            if t is not None and t.is_cuda and t.device.index != cur:
                raise ValueError(f"{nm} is on cuda:{t.device.index}, the current device is cuda:{cur}")
    _check(load().scf_coeffs_noalloc(ctypes.byref(cfg), n, _ptr(pos), _ptr(mask, torch.uint8),
                                     _ptr(A_out, torch.float64), ctypes.c_void_p(stream)), "scf_coeffs_noalloc")


def scf_noalloc_status(stream: int = 0):
    """(return code, status bits) of the last scf_coeffs_noalloc call on the
    current device; synchronises the stream; does not raise on device status."""
    st = ctypes.c_int(0)
    rc = load().scf_noalloc_status(ctypes.c_void_p(stream), ctypes.byref(st))
    if rc not in (0, -7):
        raise ScfError(rc, "scf_noalloc_status")
    return rc, st.value


def scf_set_option(h, option: int, value: int):
    _check(load().scf_set_option(h, int(option), int(value)), "scf_set_option")


def scf_get_option(h, option: int) -> int:
    v = ctypes.c_int(0)
    _check(load().scf_get_option(h, int(option), ctypes.byref(v)), "scf_get_option")
    return v.value


def scf_autotune(h, pos, com, acc, reps: int = 5):
    """Times the allowed kernel shapes and keeps the fastest; returns the eight
    average times (ms): kernel-1 tiles 64/128/256, kernel-3 blocks 64/128/256,
    the register-tiled kernel 1, kernel-3 blocks of 320 (0 where a shape does
    not apply)."""
    import torch
    ms = (ctypes.c_double * 8)()
    _check(load().scf_autotune(h, _ptr(pos), _ptr(com, torch.float64), _ptr(acc), int(reps), ms), "scf_autotune")
    return list(ms)


def scf_adjoint_level(h, pos, com, weight: float, drift: bool, xbar, vbar, combar, thetabar):
    """One level of the reverse sweep (see include/scf.h)."""
    import torch
    f64 = torch.float64
    _check(load().scf_adjoint_level(h, _ptr(pos, f64), _ptr(com, f64), float(weight), 1 if drift else 0,
                                    _ptr(xbar, f64), _ptr(vbar, f64), _ptr(combar, f64), _ptr(thetabar, f64)),
           "scf_adjoint_level")


def scf_energy(h, pos, vel, acc, com, E_out):
    """Kinetic, self, tidal and total energy per progenitor (see include/scf.h)."""
    import torch
    _check(load().scf_energy(h, _ptr(pos), _ptr(vel), _ptr(acc), _ptr(com, torch.float64),
                             _ptr(E_out, torch.float64)), "scf_energy")


def scf_bound(h, pos, vel, kin: float, frac: float, E_out, bound_out, mask_out, stats_out):
    import torch
    _check(load().scf_bound(h, _ptr(pos), _ptr(vel), float(kin), float(frac), _ptr(E_out, torch.float64),
                            _ptr(bound_out, torch.uint8), _ptr(mask_out, torch.uint8),
                            _ptr(stats_out, torch.float64)), "scf_bound")


def scf_tidal(h, com, M_c, eta: float, out):
    import torch
    _check(load().scf_tidal(h, _ptr(com, torch.float64), _ptr(M_c, torch.float64), float(eta),
                            _ptr(out, torch.float64)), "scf_tidal")


def scf_set_mask(h, mask):
    import torch
    _check(load().scf_set_mask(h, _ptr(mask, torch.uint8)), "scf_set_mask")


def scf_evolve(h, pos, vel, acc, com, nsteps: int, kin: float, frac: float, eta: float, max_steps: int,
               bound, mask, stats, retune_every: int = 0, recentre: bool = False, retune_rule: int = 0,
               alpha_lo: float = 0.25, alpha_hi: float = 2.0) -> int:
    """Returns the number of integration timesteps."""
    import torch
    ep = scf_escape_params(float(kin), float(frac), float(eta), int(max_steps), int(retune_every),
                           1 if recentre else 0, int(retune_rule), float(alpha_lo), float(alpha_hi))
    n = ctypes.c_int(0)
    _check(load().scf_evolve(h, _ptr(pos), _ptr(vel), _ptr(acc), _ptr(com, torch.float64), int(nsteps),
                             ctypes.byref(ep), _ptr(bound, torch.uint8), _ptr(mask, torch.uint8),
                             _ptr(stats, torch.float64), ctypes.byref(n)), "scf_evolve")
    return n.value


def scf_recentre(h, n_prog: int, pos, vel, acc, com, mask, max_iter: int, tol: float):
    """Returns a host array (n_prog, 8) = (x_c, V_core, r_core, iterations)."""
    import numpy as np
    import torch
    out = np.zeros((int(n_prog), 8))
    _check(load().scf_recentre(h, _ptr(pos), _ptr(vel), _ptr(acc), _ptr(com, torch.float64),
                               _ptr(mask, torch.uint8), int(max_iter), float(tol),
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "scf_recentre")
    return out


def scf_retune_a000(h, pos, mask):
    import torch
    _check(load().scf_retune_a000(h, _ptr(pos), _ptr(mask, torch.uint8)), "scf_retune_a000")


def scf_retune_alpha(h, pos, mask, alpha_lo: float = 0.25, alpha_hi: float = 2.0) -> float:
    """Moves the handle to the exponent and scales at the joint maximum of
    a_000; returns the exponent."""
    import torch
    out = ctypes.c_double(0.0)
    _check(load().scf_retune_alpha(h, _ptr(pos), _ptr(mask, torch.uint8), float(alpha_lo), float(alpha_hi),
                                   ctypes.byref(out)), "scf_retune_alpha")
    return out.value


def scf_get_alpha(h) -> float:
    out = ctypes.c_double(0.0)
    _check(load().scf_get_alpha(h, ctypes.byref(out)), "scf_get_alpha")
    return out.value


def scf_get_scales(h, b_out):
    import torch
    _check(load().scf_get_scales(h, _ptr(b_out, torch.float64)), "scf_get_scales")


def scf_fma_peak(precision: int, iters: int, stream: int = 0):
    """(FLOP/s, ms) of independent FMA chains on the FP64 (SCF_FP64) or FP32
    (SCF_MIXED) pipe, best of three launches."""
    f = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    _check(load().scf_fma_peak(int(precision), int(iters), ctypes.c_void_p(stream), ctypes.byref(f),
                               ctypes.byref(ms)), "scf_fma_peak")
    return f.value, ms.value


def scf_free(h):
    _check(load().scf_free(h), "scf_free")
