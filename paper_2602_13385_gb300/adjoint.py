"""Differentiable SCF runs: gradients of a loss on the final state with
respect to the initial phase space of the particles and of the cluster
centre, and the host-galaxy parameters.

:class:`SCFRun` is a ``torch.autograd.Function``.  Its forward integrates
with ``scf_step`` (kick-drift-kick, Sec. 2.1) and keeps a checkpoint
(positions, velocities, accelerations, centre) every ``checkpoint_every``
steps.  Its backward goes through the checkpoints from last to first: it
recomputes the segment's states with ``scf_step``, then runs the
hand-written adjoint ``scf_adjoint_level`` (double-precision CUDA kernels,
include/scf.h) from the segment's last level down to its first, and
finally level 0.  Memory: one copy of the particle state per checkpoint
plus the positions of one segment.

Host parameters are a ``(n_host, 2)`` tensor of (M_c, a_c) per component, in
the units of the configuration (the masses are multiplied by G inside the
library); the component kinds and the Miyamoto-Nagai scale heights come from
``config.host``.  :func:`nfw_scale_mass` maps a virial mass and scale
radius to the scale mass of App. A with torch operations, so gradients with
respect to M_vir and r_s follow by the chain rule.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import torch

from . import _lib
from .scf import SCF, Config

# pc (km/s)^2 / Msun and the critical density of App. A's virial definition
G_PC_KMS2_MSUN = 4.30091727e-3


@dataclass
class RunSpec:
    config: Config                  # precision must be "fp64"
    nsteps: int
    checkpoint_every: int = 50
    offsets: list | None = None     # progenitor boundaries, default one cluster
    b_per_prog: list | None = None


def config_with_host(config: Config, host_params: torch.Tensor) -> Config:
    """``config`` with the (M_c, a_c) of every host component replaced."""
    hp = host_params.detach().to("cpu", torch.float64).tolist()
    if len(hp) != len(config.host):
        raise ValueError(f"host_params has {len(hp)} rows, the configuration {len(config.host)} components")
    host = [(kind, float(M), float(a), b) for (kind, _, _, b), (M, a) in zip(config.host, hp)]
    return replace(config, host=host)


def host_params_of(config: Config, device=None) -> torch.Tensor:
    return torch.tensor([[M, a] for (_, M, a, _) in config.host], dtype=torch.float64, device=device)


class SCFRun(torch.autograd.Function):
    """(pos0, vel0, com0, host_params) -> (pos_T, vel_T, com_T) after
    ``spec.nsteps`` leapfrog steps; differentiable in every input except the
    masses (column 3 of ``pos0``, whose gradient is returned as 0)."""

    @staticmethod
    def forward(ctx, pos0, vel0, com0, host_params, spec: RunSpec):
        cfg = config_with_host(spec.config, host_params)
        if cfg.precision != "fp64":
            raise ValueError("the adjoint runs in double precision: use precision='fp64'")
        n = pos0.shape[0]
        offsets = spec.offsets or [0, n]
        sim = SCF(cfg, offsets=offsets, b_per_prog=spec.b_per_prog, device=pos0.device)
        has_host = len(cfg.host) > 0
        pos = pos0.detach().clone().contiguous()
        vel = vel0.detach().clone().contiguous()
        com = com0.detach().reshape(-1, 6).clone().contiguous()
        A = sim.coeffs(pos)
        acc = sim.forces(pos, A, com if has_host else None)
        ckpts = []
        t = 0
        while t < spec.nsteps:
            ckpts.append((t, pos.clone(), vel.clone(), acc.clone(), com.clone()))
            k = min(spec.checkpoint_every, spec.nsteps - t)
            sim.step(pos, vel, acc, com if has_host else None, k)
            t += k
        ctx.sim, ctx.ckpts, ctx.spec, ctx.cfg = sim, ckpts, spec, cfg
        ctx.com_shape = com0.shape
        ctx.hp_device = host_params.device
        return pos, vel, com.reshape(com0.shape)

    @staticmethod
    def backward(ctx, gpos, gvel, gcom):
        sim, ckpts, spec, cfg = ctx.sim, ctx.ckpts, ctx.spec, ctx.cfg
        dev = sim.device
        n_prog, n_host = sim.n_prog, len(cfg.host)
        has_host = n_host > 0

        def start(g, shape):
            return (torch.zeros(shape, dtype=torch.float64, device=dev) if g is None
                    else g.detach().to(torch.float64).reshape(shape).clone().contiguous())
        xbar = start(gpos, (sim.n, 4))
        vbar = start(gvel, (sim.n, 4))
        xbar[:, 3] = 0
        vbar[:, 3] = 0
        combar = start(gcom, (n_prog, 6))
        thetabar = torch.zeros((n_prog, max(2 * n_host, 1)), dtype=torch.float64, device=dev)
        T, dt = spec.nsteps, cfg.dt
        h = 0.5 * dt

        def level(x, c, w, drift):
            _lib.scf_adjoint_level(sim._h, x, c if has_host else None, w, drift, xbar, vbar,
                                   combar if has_host else None, thetabar if has_host else None)

        for (t0, p, v, a, c) in reversed(ckpts):
            t1 = min(t0 + spec.checkpoint_every, T)
            pos, vel, acc, com = p.clone(), v.clone(), a.clone(), c.clone()
            X, C = [p], [c]
            for _ in range(t1 - t0):
                sim.step(pos, vel, acc, com if has_host else None, 1)
                X.append(pos.clone())
                C.append(com.clone())
            for t in range(t1, t0, -1):
                level(X[t - t0], C[t - t0], h if t == T else dt, True)
        if T > 0:
            level(ckpts[0][1], ckpts[0][4], h, False)
        gpos0 = xbar
        gvel0 = vbar
        if has_host:
            ghost = torch.stack([cfg.G * thetabar[:, 0::2].sum(0), thetabar[:, 1::2].sum(0)], dim=1)
        else:
            ghost = torch.zeros((0, 2), dtype=torch.float64, device=dev)
        return gpos0, gvel0, combar.reshape(ctx.com_shape), ghost.to(ctx.hp_device), None


def run(pos0, vel0, com0, host_params, spec: RunSpec):
    """Differentiable forward run; see :class:`SCFRun`."""
    return SCFRun.apply(pos0, vel0, com0, host_params, spec)


# --------------------------------------------------------------------------
# physical parametrisation and the stream-track loss
# --------------------------------------------------------------------------
def nfw_scale_mass(Mvir_msun, rs_pc, H0_kms_mpc: float = 70.0, overdensity: float = 200.0):
    """Scale mass M_NFW of App. A (Msun) from the virial mass and scale radius,
    differentiable: rho_crit = 3 H0^2/(8 pi G), M_vir = (4 pi/3) 200 rho_crit
    R_vir^3, c = R_vir/r_s, M_NFW = M_vir / (ln(1+c) - c/(1+c))."""
    H = H0_kms_mpc * 1e-6                                 # km/s per pc
    rho_crit = 3.0 * H * H / (8.0 * math.pi * G_PC_KMS2_MSUN)
    Rvir = (3.0 * Mvir_msun / (4.0 * math.pi * overdensity * rho_crit)) ** (1.0 / 3.0)
    c = Rvir / rs_pc
    return Mvir_msun / (torch.log1p(c) - c / (1.0 + c))


def escaper_set(pot0: torch.Tensor, vel0: torch.Tensor, frac: float = 0.01) -> torch.Tensor:
    """Indices of the fraction ``frac`` of particles with the highest
    cluster-frame specific energy |v|^2/2 + psi_SCF at t = 0 (a fixed,
    stop-gradient set)."""
    E = 0.5 * (vel0[:, :3] ** 2).sum(1) + pot0
    k = max(1, int(round(frac * E.shape[0])))
    return torch.topk(E, k).indices.sort().values


def nearest_track_point(points: torch.Tensor, track: torch.Tensor) -> torch.Tensor:
    """Index of the nearest track point of every point (stop-gradient)."""
    with torch.no_grad():
        return torch.cdist(points.to(torch.float64), track.to(torch.float64)).argmin(dim=1)


def stream_track_loss(pos_T, com_T, idx, track, assign):
    """Mean squared distance of the selected particles (host frame: R_T +
    x_k) to their assigned points of the reference track."""
    P = com_T.reshape(-1, 6)[0, :3] + pos_T[idx, :3]
    return ((P - track[assign]) ** 2).sum(1).mean()
