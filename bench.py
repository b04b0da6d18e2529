#!/usr/bin/env python
"""Benchmark of the SCF gravity step: particle-force evaluations per second.

A step is one pass of the whole hot path (scf_step with nsteps = 1): half kick
+ drift, coefficient sums (kernel 1), fixed-order reduction + centre-orbit
step (kernel 2), field + tidal term + half kick (kernel 3).  One step
evaluates one force per particle, so value = particles x steps / device time.

Default workload: King W0 = 6 cluster, N = 1e5 (1e5 Msun, r_h = 3 pc) on a
circular orbit at R = 8 kpc in the NFW + Miyamoto-Nagai + Hernquist host,
nmax = 20, lmax = 8, double precision.  Inputs are seeded and synthetic.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--workload NAME] [--impl ours|reference]

With torchrun (N > 1) every rank runs an independent replica of the workload
(the step has no cross-GPU exchange in this build); value = all ranks'
evaluations / max rank time.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SCF particle-force evals/s on 1 GB300 at stated err vs FP64 oracle; % FP roofline"
UNIT = "particle-force evals/s"
L2_FLUSH_BYTES = 256 << 20           # > 129 MB L2
FP64_FMA_PER_SM_CLK = 2              # measured: 1.20 TFLOP/s FP64 FMA chains at 1995 MHz on 152 SMs
FP32_FMA_PER_SM_CLK = 128
N_SM = 152

WORKLOADS = {
    # name: (workload builder, precision)
    "king_circular_fp64": ("king_circular", "fp64"),
    "king_circular_mixed": ("king_circular", "mixed"),
    "plummer_eccentric_mixed": ("plummer_eccentric", "mixed"),
    "plummer_eccentric_fp64": ("plummer_eccentric", "fp64"),
    "batch10_mixed": ("progenitor_batch", "mixed"),
    "plummer_isolated_fp64": ("plummer_isolated", "fp64"),
    # the paper's stream progenitors (King W0 = 5, 1e5 Msun, r_h = 10 pc, N = 2e5
    # each) on its ten Table A3 orbits in MilkyWayPotential2022, (10, 5)
    "paper_orbits_mixed": ("paper_orbits", "mixed"),
    "paper_orbits_fp64": ("paper_orbits", "fp64"),
    # double-precision particles with the float-float field kernel (SCF_OPT_K3_VARIANT = 1)
    "king_circular_fp64ff": ("king_circular", "fp64"),
    "plummer_eccentric_fp64ff": ("plummer_eccentric", "fp64"),
    # the Plummer cluster in the alpha = 1/2 (Clutton-Brock) member of the radial family
    "plummer_eccentric_cb_mixed": ("plummer_eccentric_cb", "mixed"),
    "plummer_eccentric_cb_fp64": ("plummer_eccentric_cb", "fp64"),
}
FF_WORKLOADS = {"king_circular_fp64ff", "plummer_eccentric_fp64ff"}
BUILDER_ARGS = {"paper_orbits": {"n_per": 200_000}}
# per workload (not builder): the double-precision Clutton-Brock line runs N = 1e5
WORKLOAD_ARGS = {"plummer_eccentric_cb_fp64": {"n": 100_000}}
DEFAULT_WORKLOAD = "king_circular_fp64"


def per_particle_flops(nmax, lmax):
    """Algorithmic flops per particle of the coefficient pass and of the force
    pass (FMA = 2 flops): Nc = (nmax+1) N_lm complex coefficients."""
    nn, nl = nmax + 1, lmax + 1
    nlm = nl * (nl + 1) // 2
    nc = nn * nlm
    k1 = 4 * nc + 6 * nn * nl + 6 * nlm
    k3 = 8 * nc + 12 * nn * nl + 30 * nlm + 100
    return k1, k3


def per_particle_bytes(elem):
    """Algorithmic HBM bytes per particle per step (4-component records)."""
    rec = 4 * elem
    return 5 * rec, 4 * rec      # kernel 1: r pos,vel,acc w pos,vel; kernel 3: r pos,vel w acc,vel


# sources that decide the code and launch shapes of the three step kernels
# the sources of the step kernels' code (kernels 1-3, their device helpers and
# tables); the launch shapes are fixed by --tiles in the capture command
STEP_SOURCES = ["scf_coeffs.cu", "scf_device.cuh", "scf_forces.cu", "scf_tables.cu"]


def src_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2602_13385_gb300", "csrc")
    for fn in STEP_SOURCES:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# --------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3] not in ("[N/A]", ""))}


# --------------------------------------------------------------------- helpers
def build_workload(name, n_override=None):
    import workloads
    builder, precision = WORKLOADS[name]
    fn = getattr(workloads, builder)
    kw = dict(BUILDER_ARGS.get(builder, {}))
    kw.update(WORKLOAD_ARGS.get(name, {}))
    if n_override is not None:
        if "n_per" in kw:
            kw["n_per"] = max(1, n_override // 10)
        else:
            kw["n"] = n_override
    return fn(**kw), precision


def traffic_for(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary of the same kernel
    source, or None when there is none (or it is stale)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        e = d.get(workload, {}).get(kernel)
        if e and e.get("src_hash") == src_hash():
            return e["dram_bytes_per_launch"]
    except (ValueError, OSError):
        pass
    return None


def cpu_baseline(wl, precision, steps=2):
    """The FP64 oracle timed on the host cores on the same workload (full N,
    `steps` leapfrog steps), plus the GPU-vs-oracle error on that first step."""
    import numpy as np
    import oracle
    host = oracle.host_struct(wl.host) if wl.host else None
    com = wl.com if wl.host else np.zeros(6)
    t0 = time.perf_counter()
    A0 = oracle.coeffs(wl.pos, wl.nmax, wl.lmax, wl.b, alpha=wl.alpha)
    acc0 = oracle.forces(wl.pos, A0, wl.nmax, wl.lmax, wl.b, com=com, host=host, alpha=wl.alpha)
    t_init = time.perf_counter() - t0
    t0 = time.perf_counter()
    p1, v1, a1, c1, A1 = oracle.step(wl.pos, wl.vel, acc0, wl.nmax, wl.lmax, wl.b, wl.dt, 1, com=com, host=host,
                                     alpha=wl.alpha)
    t1 = time.perf_counter() - t0
    t_rest = 0.0
    if steps > 1:
        t0 = time.perf_counter()
        oracle.step(p1, v1, a1, wl.nmax, wl.lmax, wl.b, wl.dt, steps - 1, com=c1, host=host, alpha=wl.alpha)
        t_rest = time.perf_counter() - t0
    secs = t1 + t_rest
    return {
        "value": wl.n * steps / secs, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
        "sample": f"{steps} full leapfrog steps of the same workload (N={wl.n}) by the FP64 C oracle "
                  f"(OpenMP, {oracle.num_threads()} threads); initial force evaluation {t_init:.2f} s not counted",
        "seconds": secs,
    }, (wl.pos, wl.vel, acc0, com, p1, v1, a1, A1)


def oracle_error(sim, wl, ref, dtype, torch):
    """Error of one GPU step against the oracle's step from the same state."""
    import numpy as np
    pos, vel, acc0, com, p1, v1, a1, A1 = ref
    dev = sim.device
    p = torch.tensor(pos, device=dev, dtype=dtype)
    v = torch.tensor(vel, device=dev, dtype=dtype)
    a = torch.tensor(acc0, device=dev, dtype=dtype)
    c = torch.tensor(com[None], device=dev, dtype=torch.float64)
    sim.step(p, v, a, com=c if wl.host else None, nsteps=1)
    A = sim.last_coeffs().cpu().numpy()[0]
    ag = a.cpu().double().numpy()
    na = np.linalg.norm(a1[:, :3], axis=1)
    rel = np.linalg.norm(ag[:, :3] - a1[:, :3], axis=1) / np.maximum(na, 1e-6 * np.median(na))
    return {
        "coeff_max_rel": float(np.max(np.abs(A - A1)) / np.max(np.abs(A1))),
        "accel_rel_median": float(np.median(rel)), "accel_rel_max": float(np.max(rel)),
        "pos_max_abs": float(np.max(np.abs(p.cpu().double().numpy()[:, :3] - p1[:, :3]))),
        "what": "one leapfrog step from the same state, GPU vs the FP64 oracle",
    }


# --------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    wl, precision = build_workload(args.workload)
    host = oracle.host_struct(wl.host) if wl.host else None
    import numpy as np
    com = wl.com if wl.host else np.zeros(6)
    # bounded sample: the whole warm-up + timed run near <= 2 minutes of host
    # time (at most 3 s a step)
    per_step = min(3.0, 120.0 / max(1, args.steps + args.warmup))
    t0 = time.perf_counter()
    A0 = oracle.coeffs(wl.pos, wl.nmax, wl.lmax, wl.b, alpha=wl.alpha)
    acc = oracle.forces(wl.pos, A0, wl.nmax, wl.lmax, wl.b, com=com, host=host, alpha=wl.alpha)
    t_full = time.perf_counter() - t0
    n = wl.n
    if t_full > per_step:
        n = max(1000, int(wl.n * per_step / t_full))
    pos, vel, acc = wl.pos[:n].copy(), wl.vel[:n].copy(), acc[:n].copy()
    pos[:, 3] *= wl.n / n
    c = com.copy()
    for _ in range(args.warmup):
        pos, vel, acc, c, _ = oracle.step(pos, vel, acc, wl.nmax, wl.lmax, wl.b, wl.dt, 1, com=c, host=host,
                                          alpha=wl.alpha)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pos, vel, acc, c, _ = oracle.step(pos, vel, acc, wl.nmax, wl.lmax, wl.b, wl.dt, 1, com=c, host=host,
                                          alpha=wl.alpha)
    secs = time.perf_counter() - t0
    value = n * args.steps / secs
    sample = (f"{n} of the workload's {wl.n} particles (mass rescaled), {args.steps} leapfrog steps by the FP64 "
              f"C oracle on {oracle.num_threads()} host threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
        "config": workload_config(wl, "fp64", args.workload),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(wl, precision, name):
    return {"workload": wl.name, "bench_name": name, "N": int(wl.n), "nmax": wl.nmax, "lmax": wl.lmax,
            "alpha": wl.alpha,
            "precision": precision, "n_progenitors": 1 if wl.offsets is None else len(wl.offsets) - 1,
            "host": ("MilkyWayPotential2022 (Table A2)" if wl.name.startswith("paper_orbits") else
                     "NFW(Mvir=1e12,rs=20kpc)+MN(6.8e10,3,0.28kpc)+Hernquist(5e9,0.5kpc)") if wl.host else "none",
            "dt_henon": wl.dt, "l2": "flushed (256 MiB write) before every timed step"}


# --------------------------------------------------------------------- our arm
# Pair terms of the boundedness sum on the FP32 pipe.  Single precision:
# dx, dy, dz (3 adds), r^2 (1 multiply + 2 FMAs) and m / r accumulated
# (1 FMA) = 7 operations; 1/sqrt runs on the special-function unit.  Double
# precision runs the same terms in float-float arithmetic: 86 single-precision
# operations per pair (exact differences, squares with their rounding errors,
# a Newton step for 1/r, a float-float accumulation).
PAIR_OPS = {"mixed": 7, "fp64": 86}


def escape_timing(sim, p, v, offsets, precision, clocks, torch, reps=3):
    """Time one scf_bound call (boundedness by direct summation, r_x and the
    mask) with CUDA events on the handle's stream, after one untimed call."""
    n = sim.n
    bnd = torch.empty(n, dtype=torch.uint8, device=p.device)
    msk = torch.empty_like(bnd)
    st = torch.empty((sim.n_prog, 4), dtype=torch.float64, device=p.device)
    from paper_2602_13385_gb300 import _lib
    stream = sim.stream
    with torch.cuda.stream(stream):
        _lib.scf_bound(sim._h, p, v, 0.5, 0.999, None, bnd, msk, st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            _lib.scf_bound(sim._h, p, v, 0.5, 0.999, None, bnd, msk, st)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    pairs = float(sum((offsets[i + 1] - offsets[i]) ** 2 for i in range(len(offsets) - 1)))
    clock = clocks.get("sm_max_mhz") or 2070.0
    lanes = FP32_FMA_PER_SM_CLK
    ops = PAIR_OPS[precision]
    ceiling = N_SM * lanes / ops * clock * 1e6
    return {"kernel": "scf_bound (k_bound_pairs + k_bound_finish + k_select)", "ms": ms,
            "pairs_per_s": pairs / (ms * 1e-3),
            "roofline": {"bound": "alu", "achieved": pairs / (ms * 1e-3), "peak": ceiling, "unit": "pairs/s",
                         "frac": pairs / (ms * 1e-3) / ceiling,
                         "peak_basis": f"FP32 pipe: {N_SM} SMs x {lanes} lanes/clk / {ops} ops per pair "
                                       f"x {clock:.0f} MHz"},
            "n_bound": float(st[:, 0].sum().item())}


def max_over_ranks(ms: float, device=None) -> float:
    """The slowest rank's time, on every rank (the local time without a
    process group, or with one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, steps: int, world: int, ms_max: float) -> float:
    """Units all ranks processed (independent replicas, weak scaling) per second
    of the slowest rank."""
    return units_per_rank * steps * world / (ms_max * 1e-3)


def refresh_timing(sim, p, v, torch, reps=3):
    """Time the complete-refresh operations on the bench state (copies of the
    particles, after one untimed call each): scf_recentre (the SCF centre,
    density, core frame; 100 iterations at most) and scf_retune_a000 (b at the
    maximum of a_000).  The latter changes the handle's scales, so this runs
    last."""
    from paper_2602_13385_gb300 import _lib
    stream = sim.stream
    pc, vc = p.clone(), v.clone()
    ac = torch.empty_like(p)
    out = {}
    with torch.cuda.stream(stream):
        res = _lib.scf_recentre(sim._h, sim.n_prog, pc, vc, ac, None, None, 100, 1e-12)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            _lib.scf_recentre(sim._h, sim.n_prog, pc, vc, ac, None, None, 100, 1e-12)
        e1.record(stream)
        torch.cuda.synchronize()
        out["recentre_ms"] = e0.elapsed_time(e1) / reps
        out["recentre_iterations"] = float(res[:, 7].max())
        _lib.scf_retune_a000(sim._h, p, None)
        e0.record(stream)
        for _ in range(reps):
            _lib.scf_retune_a000(sim._h, p, None)
        e1.record(stream)
    torch.cuda.synchronize()
    out["retune_a000_ms"] = e0.elapsed_time(e1) / reps
    out["what"] = ("complete-refresh operations (Sec. 2, 2.1), per call on the bench state: re-centring "
                   "(including its host read-back) and the a_000 scale search")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default kernel shapes")
    ap.add_argument("--tiles", default=None,
                    help="K1,K3: fixed kernel shapes instead of the autotuner (K1 = 0 for the register-tiled "
                         "coefficient kernel, else 64/128/256 particles per tile; K3 = 64/128/256 threads)")
    ap.add_argument("--n", type=int, default=None,
                    help="particle count of a smaller case of the same workload (for profiling captures)")
    ap.add_argument("--no-escape", action="store_true",
                    help="skip the timing of the boundedness kernels (scf_bound) reported under 'escape'")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_2602_13385_gb300 import SCF, Config
    wl, precision = build_workload(args.workload, args.n)
    dtype = torch.float64 if precision == "fp64" else torch.float32
    cfg = Config(nmax=wl.nmax, lmax=wl.lmax, b=wl.b, dt=wl.dt, precision=precision, host=list(wl.host),
                 alpha=wl.alpha)
    offsets = [0, wl.n] if wl.offsets is None else list(wl.offsets)
    sim = SCF(cfg, offsets=offsets, b_per_prog=wl.b_per_prog)
    dev = sim.device
    coms = wl.com[None] if wl.com_per_prog is None else wl.com_per_prog
    p = torch.tensor(wl.pos, device=dev, dtype=dtype)
    v = torch.tensor(wl.vel, device=dev, dtype=dtype)
    c = torch.tensor(coms, device=dev, dtype=torch.float64)
    use_com = c if wl.host else None
    if args.workload in FF_WORKLOADS:
        sim.set_tiles(k3_block=128, k3_variant=1, k1_variant=2)
    a = sim.forces(p, sim.coeffs(p), com=use_com)
    tuning = None
    if args.tiles:
        k1t, k3b = (int(x) for x in args.tiles.split(","))
        sim.set_tiles(k1_tile=k1t, k3_block=k3b)
    elif not args.no_autotune:
        # untimed set-up: the library's autotuner picks the kernel shapes
        tuning = sim.autotune(p, com=use_com, acc=torch.empty_like(a), reps=3, cache=False)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = sim.stream

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            flush.fill_(float(i))
            sim.step(p, v, a, com=use_com, nsteps=1)
        torch.cuda.synchronize()
        sim.profile(True)
        sim.profile_read()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        sampler = ClockSampler(local)
        sampler.start()
        barrier()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            sim.step(p, v, a, com=use_com, nsteps=1)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        clocks = sampler.stop()
        ms_total = sum(e0.elapsed_time(e1) for e0, e1 in ev)
        kms, kcount = sim.profile_read()
        sim.profile(False)
    rc, st = sim.status()
    if rc != 0:
        raise RuntimeError(f"device status {st} after the timed steps")

    ms_max = max_over_ranks(ms_total, dev)
    value = whole_job_rate(wl.n, args.steps, world, ms_max)

    # end to end through the public API with host buffers (pinned)
    h_in = [t.cpu().pin_memory() for t in (p, v, a, c)]
    h_out = [torch.empty_like(t) for t in h_in]
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        t0.record(stream)
        for _ in range(e2e_steps):
            for d, hsrc in zip((p, v, a, c), h_in):
                d.copy_(hsrc, non_blocking=True)
            sim.step(p, v, a, com=use_com, nsteps=1)
            for hdst, d in zip(h_out, (p, v, a, c)):
                hdst.copy_(d, non_blocking=True)
        t1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = t0.elapsed_time(t1)
    bytes_io = sum(t.numel() * t.element_size() for t in h_in)
    e2e = {"value": wl.n * e2e_steps / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": bytes_io,
           "d2h_bytes_per_step": bytes_io, "steps": e2e_steps,
           "what": "scf_step through the C ABI with the state copied from pinned host buffers and back every step"}

    # roofline of the dominant kernel (ALU-bound: FP64 pipe in fp64 mode, FP32 in mixed)
    k1f, k3f = per_particle_flops(wl.nmax, wl.lmax)
    elem = 8 if precision == "fp64" else 4
    k1b, k3b = per_particle_bytes(elem)
    dom = 2 if kms[2] >= kms[0] else 0
    avg_ms = kms[dom] / max(1, kcount[dom])
    flops = wl.n * (k3f if dom == 2 else k1f)
    achieved = flops / (avg_ms * 1e-3) / 1e12
    clock = clocks.get("sm_max_mhz") or 2070.0
    fma = FP64_FMA_PER_SM_CLK if precision == "fp64" else FP32_FMA_PER_SM_CLK
    peak = N_SM * fma * 2 * clock * 1e6 / 1e12
    kname = "k3_forces" if dom == 2 else "k1_partials"
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic_for(kname, args.workload),
                "kernel": kname, "kernel_avg_ms": avg_ms,
                "peak_basis": f"{'FP64' if precision == 'fp64' else 'FP32'} pipe: {N_SM} SMs x {fma} FMA/clk x 2 "
                              f"x {clock:.0f} MHz (max SM clock)",
                "frac_at_sampled_clock": (achieved / (N_SM * fma * 2 * clocks["sm_mhz"] * 1e-6)
                                          if clocks.get("sm_mhz") else None),
                "algorithmic_flops_per_launch": flops,
                "algorithmic_bytes_per_launch": wl.n * (k3b if dom == 2 else k1b),
                "kernels_ms_per_step": {"k1_partials": kms[0] / max(1, kcount[0]),
                                        "k2_reduce": kms[1] / max(1, kcount[1]),
                                        "k3_forces": kms[2] / max(1, kcount[2])}}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f64 (kernels 1 and 3 in float-float)" if args.workload in FF_WORKLOADS else "f64")
                 if precision == "fp64" else "f32+f64",
        "data": "synthetic (seeded sample, see config.workload)",
        "config": workload_config(wl, precision, args.workload),
        "roofline": roofline, "e2e": e2e, "gpu_launches": int(sum(kcount)), "clocks": clocks,
        "kernel_shapes": dict(sim.tiles(), autotuned=tuning is not None,
                              candidates_ms=None if tuning is None else tuning["ms"]),
        "src_hash": src_hash(),
    }
    if not args.no_escape:
        line["escape"] = escape_timing(sim, p, v, offsets, precision, clocks, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base, ref = cpu_baseline(wl, precision) if wl.offsets is None else (None, None)
        if base is not None:
            line["cpu_baseline"] = base
            line["error_vs_oracle"] = oracle_error(sim, wl, ref, dtype, torch)
    if not args.no_escape:
        line["refresh"] = refresh_timing(sim, p, v, torch)
    sim.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
