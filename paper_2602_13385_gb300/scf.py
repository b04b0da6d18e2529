"""User-facing API of the SCF gravity step on one GPU.

PyTorch supplies device memory and the stream; every step of the method runs
in the CUDA kernels of ``libscf.so`` through the C ABI (``_lib``).

Layouts (see include/scf.h): positions ``(N, 4)`` = (x, y, z, m), velocities
``(N, 4)``, accelerations ``(N, 4)`` = (ax, ay, az, psi_SCF), float64 for
``precision="fp64"`` and float32 for ``precision="mixed"``; coefficients
``(n_prog, 2*NC)`` float64 = [S | T]; centre ``(n_prog, 6)`` float64 = (R, V).
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

import torch

from . import _lib

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune_cache.json")

HOST_HERNQUIST = _lib.SCF_HOST_HERNQUIST
HOST_NFW = _lib.SCF_HOST_NFW
HOST_MN = _lib.SCF_HOST_MN
HOST_POWCUT = _lib.SCF_HOST_POWCUT


def n_lm(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


def n_coef(nmax: int, lmax: int) -> int:
    """Entries of one half (S or T) of a coefficient vector."""
    return (nmax + 1) * n_lm(lmax)


@dataclass
class Config:
    nmax: int
    lmax: int
    b: float
    G: float = 1.0
    dt: float = 0.01
    precision: str = "fp64"           # "fp64" or "mixed"
    host: list = field(default_factory=list)   # [(kind, M, a, b)], kinds HOST_*
    alpha: float = 1.0

    def to_c(self) -> _lib.scf_config:
        c = _lib.scf_config()
        c.nmax, c.lmax, c.alpha, c.b, c.G, c.dt = self.nmax, self.lmax, self.alpha, self.b, self.G, self.dt
        c.precision = {"fp64": _lib.SCF_FP64, "mixed": _lib.SCF_MIXED}[self.precision]
        if len(self.host) > _lib.SCF_MAX_HOST_COMPONENTS:
            raise ValueError("too many host components")
        c.n_host = len(self.host)
        for i, (kind, M, a, b) in enumerate(self.host):
            c.host[i].kind, c.host[i].M, c.host[i].a, c.host[i].b = int(kind), float(M), float(a), float(b)
        return c

    @property
    def dtype(self) -> torch.dtype:
        return torch.float64 if self.precision == "fp64" else torch.float32


class SCF:
    """A handle on the GPU: one or more progenitors sharing a configuration.

    ``offsets``: progenitor boundaries (length n_prog+1, offsets[0] = 0), or
    ``n`` for a single cluster.  ``b_per_prog`` overrides ``config.b``."""

    def __init__(self, config: Config, n: int | None = None, offsets=None, b_per_prog=None,
                 device: torch.device | int | None = None, stream: torch.cuda.Stream | None = None):
        if offsets is None:
            if n is None:
                raise ValueError("give n or offsets")
            offsets = [0, int(n)]
        self.config = config
        self.offsets = [int(o) for o in offsets]
        self.b_per_prog = None if b_per_prog is None else [float(x) for x in b_per_prog]
        self.n_prog = len(self.offsets) - 1
        self.n = self.offsets[-1]
        self.nc = n_coef(config.nmax, config.lmax)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        with torch.cuda.device(self.device):
            self.stream = stream or torch.cuda.current_stream(self.device)
            self._h = _lib.scf_init(config.to_c(), self.offsets, b_per_prog, self.stream.cuda_stream)

    # -- allocation helpers (PyTorch owns the memory)
    def new_coeffs(self) -> torch.Tensor:
        return torch.zeros((self.n_prog, 2 * self.nc), dtype=torch.float64, device=self.device)

    def new_particles(self) -> torch.Tensor:
        return torch.zeros((self.n, 4), dtype=self.config.dtype, device=self.device)

    def _check_particles(self, t: torch.Tensor, name: str):
        if t.shape != (self.n, 4):
            raise ValueError(f"{name} must have shape ({self.n}, 4), got {tuple(t.shape)}")
        if t.dtype != self.config.dtype:
            raise TypeError(f"{name} must be {self.config.dtype}, got {t.dtype}")

    # -- the entry points
    def coeffs(self, pos: torch.Tensor, mask: torch.Tensor | None = None, out: torch.Tensor | None = None):
        self._check_particles(pos, "pos")
        out = self.new_coeffs() if out is None else out
        _lib.scf_coeffs(self._h, pos, mask, out)
        return out

    def forces(self, pos: torch.Tensor, A: torch.Tensor, com: torch.Tensor | None = None,
               out: torch.Tensor | None = None):
        self._check_particles(pos, "pos")
        out = self.new_particles() if out is None else out
        _lib.scf_forces(self._h, pos, A, com, out)
        return out

    def step(self, pos, vel, acc, com=None, nsteps: int = 1):
        for t, nm in ((pos, "pos"), (vel, "vel"), (acc, "acc")):
            self._check_particles(t, nm)
        _lib.scf_step(self._h, pos, vel, acc, com, nsteps)

    def step_host(self, pos, vel, acc, host_pos, host_vel, host_acc, com=None, host_com=None, chunks: int = 8):
        """One step of a state held in host tensors ``host_*`` (page-locked for
        overlap; read, then overwritten with the new state), through the
        device tensors ``pos, vel, acc, com`` (scf_step_host)."""
        for t, nm in ((pos, "pos"), (vel, "vel"), (acc, "acc")):
            self._check_particles(t, nm)
        _lib.scf_step_host(self._h, pos, vel, acc, com, host_pos, host_vel, host_acc, host_com, chunks)

    def energy(self, pos, vel, acc, com=None, out: torch.Tensor | None = None):
        """(n_prog, 4) float64 = (kinetic, self, tidal, total) energy per
        progenitor in its frame; ``acc`` must hold the accelerations and
        potential at ``pos`` (as ``step`` and ``forces`` leave them)."""
        for t, nm in ((pos, "pos"), (vel, "vel"), (acc, "acc")):
            self._check_particles(t, nm)
        out = torch.empty((self.n_prog, 4), dtype=torch.float64, device=self.device) if out is None else out
        _lib.scf_energy(self._h, pos, vel, acc, com, out)
        return out

    # -- escape physics (Sec. 2.2)
    def bound(self, pos, vel, kin: float = 0.5, frac: float = 0.999, energies: bool = False):
        """Boundedness by direct summation and the coefficient set r <= r_x.
        Returns ``(bound, mask, stats, E)``: uint8 ``(N,)`` flags, uint8 ``(N,)``
        mask, float64 ``(n_prog, 4)`` = (n_bound, bound mass, r_x, set size),
        and float64 ``(N,)`` energies when ``energies`` (else None)."""
        for t, nm in ((pos, "pos"), (vel, "vel")):
            self._check_particles(t, nm)
        b = torch.empty(self.n, dtype=torch.uint8, device=self.device)
        m = torch.empty(self.n, dtype=torch.uint8, device=self.device)
        st = torch.empty((self.n_prog, 4), dtype=torch.float64, device=self.device)
        E = torch.empty(self.n, dtype=torch.float64, device=self.device) if energies else None
        _lib.scf_bound(self._h, pos, vel, kin, frac, E, b, m, st)
        return b, m, st, E

    def tidal(self, com=None, M_c=None, eta: float = 1.0 / 400.0):
        """(n_prog, 16) float64: tidal tensor (9), eigenvalues (3), Frobenius
        norm, l1e, r_t and dt_int at the centres (see scf_tidal)."""
        out = torch.empty((self.n_prog, 16), dtype=torch.float64, device=self.device)
        _lib.scf_tidal(self._h, com, M_c, eta, out)
        return out

    def set_mask(self, mask=None):
        """Coefficient set of ``step`` (uint8 ``(N,)`` tensor kept alive by the
        caller), or None for every particle."""
        self._mask_ref = mask
        _lib.scf_set_mask(self._h, mask)

    def evolve(self, pos, vel, acc, com=None, nsteps: int = 1, kin: float = 0.5, frac: float = 0.999,
               eta: float = 1.0 / 400.0, max_steps: int = 1000, retune_every: int = 0, recentre: bool = False,
               retune_rule: str = "half_mass", alpha_range=(0.25, 2.0)):
        """``nsteps`` leapfrog steps with boundedness, the r <= r_x coefficient
        set, the tidal integration timestep and, every ``retune_every``
        integration timesteps, a complete refresh of b (``retune_rule``
        "half_mass" or "a000", :meth:`retune_a000`) or of alpha and b
        ("alpha_a000", :meth:`retune_alpha` over ``alpha_range``), preceded
        with ``recentre`` by :meth:`recentre` (scf_evolve).  Returns
        ``(bound, mask, stats, n_int)`` as of the last integration timestep;
        ``self.config.alpha`` follows the handle's exponent."""
        for t, nm in ((pos, "pos"), (vel, "vel"), (acc, "acc")):
            self._check_particles(t, nm)
        if getattr(self, "_evolve_bufs", None) is None:
            self._evolve_bufs = (torch.empty(self.n, dtype=torch.uint8, device=self.device),
                                 torch.empty(self.n, dtype=torch.uint8, device=self.device),
                                 torch.empty((self.n_prog, 4), dtype=torch.float64, device=self.device))
        b, m, st = self._evolve_bufs
        self._mask_ref = m
        n_int = _lib.scf_evolve(self._h, pos, vel, acc, com, nsteps, kin, frac, eta, max_steps, b, m, st,
                                retune_every, recentre, {"half_mass": 0, "a000": 1, "alpha_a000": 2}[retune_rule],
                                alpha_range[0], alpha_range[1])
        self.config.alpha = _lib.scf_get_alpha(self._h)
        return b, m, st, n_int

    def retune_alpha(self, pos, mask=None, alpha_lo: float = 0.25, alpha_hi: float = 2.0) -> float:
        """Moves the handle to the exponent alpha of the radial family and the
        scales b at the joint maximum of a_000 (scf_retune_alpha); returns
        alpha (also in ``self.config.alpha``)."""
        self._check_particles(pos, "pos")
        al = _lib.scf_retune_alpha(self._h, pos, mask, alpha_lo, alpha_hi)
        self.config.alpha = al
        return al

    def retune_a000(self, pos, mask=None):
        """Sets each progenitor's b to the maximum of a_000 of the coefficient
        set (scf_retune_a000); :meth:`scales` reads it."""
        self._check_particles(pos, "pos")
        _lib.scf_retune_a000(self._h, pos, mask)

    def recentre(self, pos, vel, acc, com=None, mask=None, max_iter: int = 100, tol: float = 1e-12):
        """Moves each progenitor's frame to its SCF centre (the maximum of a_000)
        and core velocity (Sec. 2.1; scf_recentre): particles shifted in place,
        ``com`` += (x_c, V_core); ``acc`` is used as scratch.  Returns a numpy
        array (n_prog, 8) = (x_c, V_core, r_core, iterations)."""
        for t, nm in ((pos, "pos"), (vel, "vel"), (acc, "acc")):
            self._check_particles(t, nm)
        return _lib.scf_recentre(self._h, self.n_prog, pos, vel, acc, com, mask, max_iter, tol)

    def scales(self):
        """(n_prog,) float64: the basis scale b of every progenitor."""
        out = torch.empty(self.n_prog, dtype=torch.float64, device=self.device)
        _lib.scf_get_scales(self._h, out)
        return out

    def last_coeffs(self, out: torch.Tensor | None = None):
        out = self.new_coeffs() if out is None else out
        _lib.scf_last_coeffs(self._h, out)
        return out

    def status(self):
        return _lib.scf_status(self._h)

    def launches_per_call(self, which: str) -> int:
        return _lib.scf_launches_per_call(self._h, {"coeffs": 0, "forces": 1, "step": 2}[which])

    def tiles(self) -> dict:
        """Current kernel shapes: coefficient-kernel tile (0 = the register-tiled
        kernel of mixed precision) and field-kernel block."""
        return {"k1_tile": _lib.scf_get_option(self._h, _lib.SCF_OPT_K1_TILE),
                "k3_block": _lib.scf_get_option(self._h, _lib.SCF_OPT_K3_BLOCK),
                "k1_variant": _lib.scf_get_option(self._h, _lib.SCF_OPT_K1_VARIANT),
                "k3_variant": _lib.scf_get_option(self._h, _lib.SCF_OPT_K3_VARIANT)}

    def set_tiles(self, k1_tile: int | None = None, k3_block: int | None = None, k3_variant: int | None = None,
                  k1_variant: int | None = None):
        """``k1_tile``: 64, 128 or 256 particles per tile of the one-thread-per-
        output coefficient kernel, or 0 for the register-tiled kernel (mixed
        precision only); ``k3_block``: 64, 128 or 256 threads per field block (320
        in mixed precision);
        ``k1_variant`` 2 / ``k3_variant`` 1: the float-float coefficient /
        field kernel of double-precision handles (128-wide only), 0 for the
        native ones."""
        if k3_variant is not None:
            _lib.scf_set_option(self._h, _lib.SCF_OPT_K3_VARIANT, int(k3_variant))
        if k1_variant is not None:
            _lib.scf_set_option(self._h, _lib.SCF_OPT_K1_VARIANT, int(k1_variant))
            if int(k1_variant) != 0:
                k1_tile = None
        if k1_tile is not None:
            if int(k1_tile) == 0:
                _lib.scf_set_option(self._h, _lib.SCF_OPT_K1_VARIANT, 1)
            else:
                _lib.scf_set_option(self._h, _lib.SCF_OPT_K1_TILE, int(k1_tile))
        if k3_block is not None:
            _lib.scf_set_option(self._h, _lib.SCF_OPT_K3_BLOCK, int(k3_block))

    def _tune_key(self) -> str:
        n = max(self.n, 1)
        n2 = float(f"{n:.2g}")          # shapes are chosen per problem-size bucket
        return "|".join(str(x) for x in (torch.cuda.get_device_name(self.device), self.config.precision,
                                         self.config.nmax, self.config.lmax, n2, self.n_prog, self.config.alpha))

    def autotune(self, pos, com=None, acc=None, reps: int = 5, cache: bool = True) -> dict:
        """Chooses the kernel shapes by timing every allowed size on ``pos``
        (scf_autotune); with ``cache`` the choice is stored per GPU, precision,
        (nmax, lmax), problem-size bucket and progenitor count, and reused."""
        key = self._tune_key()
        table = {}
        if cache and os.path.exists(_CACHE):
            try:
                with open(_CACHE) as f:
                    table = json.load(f)
            except (OSError, ValueError):
                table = {}
        if cache and key in table:
            self.set_tiles(**{k: table[key][k] for k in ("k1_tile", "k3_block")})
            return dict(table[key], cached=True)
        acc = self.new_particles() if acc is None else acc
        ms = _lib.scf_autotune(self._h, pos, com, acc, reps)
        result = dict(self.tiles(), ms=ms)
        if cache:
            table[key] = result
            tmp = _CACHE + f".{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1)
            os.replace(tmp, _CACHE)
        return dict(result, cached=False)

    def use_graphs(self, enable: bool = True):
        """scf_step replays a captured CUDA graph per step (default) or launches
        the kernels directly."""
        _lib.scf_set_option(self._h, _lib.SCF_OPT_GRAPHS, 1 if enable else 0)

    def profile(self, enable: bool = True):
        _lib.scf_profile(self._h, enable)

    def profile_read(self):
        """([ms of kernel 1, 2, 3], [launch counts]) since the last read."""
        return _lib.scf_profile_read(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.scf_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
