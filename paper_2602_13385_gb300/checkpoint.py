"""Checkpoint and resume of a run.

The state of a run is the caller's tensors — positions, velocities,
accelerations (the leapfrog needs a(x) at the current positions), the
centres (R, V) — plus the step count and the configuration; a handle holds
no physical state of its own (its buffers are scratch, its block maps and
kernel shapes follow from the configuration).  Because every reduction runs
in a fixed order, a run resumed from a checkpoint into a new handle with the
same configuration and kernel shapes continues bit for bit as the
uninterrupted run would.
"""
from __future__ import annotations

import dataclasses
import os

import torch

from .scf import SCF, Config

FORMAT = 1


def save(path: str, sim, state: dict, step: int = 0, extra: dict | None = None) -> None:
    """Writes ``state`` (name -> tensor: at least ``pos``, ``vel``, ``acc``;
    ``com`` with a host; ``mask`` if the run uses a coefficient set) with the
    step count and what a handle needs to continue it: the configuration, the
    progenitor layout and the kernel shapes of ``sim`` (an ``SCF``).  Written
    to a temporary file and renamed, so a crash never leaves half a
    checkpoint."""
    blob = {
        "format": FORMAT,
        "config": dataclasses.asdict(sim.config),
        "step": int(step),
        "offsets": list(sim.offsets),
        "b_per_prog": [float(x) for x in sim.scales().cpu()],  # as retuned by complete refreshes
        "tiles": sim.tiles(),
        "state": {k: v.detach().cpu() for k, v in state.items() if v is not None},
        "extra": extra or {},
    }
    tmp = f"{path}.{os.getpid()}.tmp"
    torch.save(blob, tmp)
    os.replace(tmp, path)


def load(path: str, device=None) -> dict:
    """Reads a checkpoint: returns a dict with ``config`` (a Config),
    ``step``, ``offsets``, ``b_per_prog``, ``tiles``, ``extra`` and ``state``
    (tensors on ``device``, default the current CUDA device)."""
    blob = torch.load(path, map_location="cpu", weights_only=False)
    if blob.get("format") != FORMAT:
        raise ValueError(f"{path}: unknown checkpoint format {blob.get('format')}")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    cfg = dict(blob["config"])
    cfg["host"] = [tuple(h) for h in cfg.get("host", [])]
    out = dict(blob)
    out["config"] = Config(**cfg)
    out["state"] = {k: v.to(dev).contiguous() for k, v in blob["state"].items()}
    return out


def resume(path: str, device=None):
    """Loads a checkpoint and opens a handle for it with the same kernel
    shapes.  Returns ``(sim, state, step)``."""
    ck = load(path, device)
    offsets = ck["offsets"]
    sim = SCF(ck["config"], offsets=offsets, b_per_prog=ck["b_per_prog"], device=device)
    if ck["tiles"]:
        t = ck["tiles"]
        sim.set_tiles(k3_block=t["k3_block"], k3_variant=t.get("k3_variant"), k1_variant=t.get("k1_variant"))
        if t.get("k1_variant", 0) != 2:
            sim.set_tiles(k1_tile=t["k1_tile"])
    mask = ck["state"].get("mask")
    if mask is not None:
        sim.set_mask(mask)
    return sim, ck["state"], ck["step"]
