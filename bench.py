#!/usr/bin/env python
"""Benchmark of the SCF gravity step: particle-force evaluations per second.

A step is one pass of the whole hot path (scf_step with nsteps = 1): half kick
+ drift, coefficient sums (kernel 1), fixed-order reduction + centre-orbit
step (kernel 2), field + tidal term + half kick (kernel 3).  One step
evaluates one force per particle, so value = particles x steps / device time.

Default (the headline line): a Plummer cluster of N = 1e6 (2e5 Msun, r_h =
4 pc) on the 5-20 kpc eccentric orbit in the NFW + Miyamoto-Nagai +
Hernquist host, nmax = 20, lmax = 10, double precision: the largest
single-cluster workload, in the paper's precision.  The same run adds, as the
keys "mixed" and "batch", the same cluster in mixed precision (FP32 basis and
field, FP64 sums and centre) and the batch of ten King progenitors of uneven
N (1.91e6 in all) on their own orbits in mixed precision, each with its own
timing, roofline, end-to-end rate, clocks, CPU baseline and error against the
FP64 oracle.  Inputs are seeded and synthetic; samples are rounded to float32
values so that both precisions start from the same state.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--workload NAME] [--impl ours|reference]

With --workload only that line is run.  With torchrun (N > 1) every rank runs
an independent replica of the workload (the step has no cross-GPU exchange in
this build); value = all ranks' evaluations / max rank time.  Prints one JSON
line on rank 0.
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
# Nominal non-tensor FMA units per SM and clock on GB300 (sm_103): 128 FP32
# lanes; FP64 at 1/64 of that rate.  The roofline peak is these unit counts x
# 152 SMs x 2 flops x the maximum SM clock; the FMA-chain kernel scf_fma_peak
# measures the achievable rate beside it ("peak_measured").
FP64_FMA_PER_SM_CLK = 2
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
DEFAULT_WORKLOAD = "plummer_eccentric_fp64"
# lines of the default run: (JSON key, workload); the first is the headline
DEFAULT_LINES = [("headline", "plummer_eccentric_fp64"), ("mixed", "plummer_eccentric_mixed"),
                 ("batch", "batch10_mixed")]


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
        elif builder == "progenitor_batch":
            kw["scale"] = n_override / 1.91e6
        else:
            kw["n"] = n_override
    wl = fn(**kw)
    wl.pos = _f32_exact(wl.pos)
    wl.vel = _f32_exact(wl.vel)
    return wl, precision


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


def _f32_exact(a):
    """float64 array holding float32-representable values (the mixed-precision
    state then equals the double-precision one exactly)."""
    import numpy as np
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def oracle_sample(wl):
    """Progenitors the oracle checks: all of a single cluster; for a batch the
    three smallest (a bounded, stated sample of the same launch)."""
    if wl.offsets is None:
        return [0]
    sizes = [int(wl.offsets[i + 1] - wl.offsets[i]) for i in range(len(wl.offsets) - 1)]
    return sorted(sorted(range(len(sizes)), key=lambda i: sizes[i])[:3])


def oracle_reference(wl):
    """The FP64 oracle on the sampled progenitors: the initial acceleration
    (untimed) and one leapfrog step from it (timed: the CPU baseline)."""
    import numpy as np
    import oracle
    host = oracle.host_struct(wl.host) if wl.host else None
    refs, n_done, secs, t_init = [], 0, 0.0, 0.0
    for p in oracle_sample(wl):
        if wl.offsets is None:
            lo, hi, b, com = 0, wl.n, wl.b, (wl.com if wl.host else np.zeros(6))
        else:
            lo, hi = int(wl.offsets[p]), int(wl.offsets[p + 1])
            b, com = float(wl.b_per_prog[p]), np.array(wl.com_per_prog[p])
        pos, vel = wl.pos[lo:hi], wl.vel[lo:hi]
        t0 = time.perf_counter()
        A0 = oracle.coeffs(pos, wl.nmax, wl.lmax, b, alpha=wl.alpha)
        acc0 = oracle.forces(pos, A0, wl.nmax, wl.lmax, b, com=com, host=host, alpha=wl.alpha)
        t1 = time.perf_counter()
        p1, v1, a1, c1, A1 = oracle.step(pos, vel, acc0, wl.nmax, wl.lmax, b, wl.dt, 1, com=com, host=host,
                                         alpha=wl.alpha)
        t2 = time.perf_counter()
        t_init += t1 - t0
        secs += t2 - t1
        n_done += hi - lo
        refs.append((p, lo, hi, acc0, p1, v1, a1, c1, A1))
    if wl.offsets is None:
        sample = (f"one full leapfrog step of the same workload (N={wl.n}) by the FP64 C oracle "
                  f"(OpenMP, {oracle.num_threads()} threads); the initial force evaluation ({t_init:.1f} s) not counted")
    else:
        ps = [r[0] for r in refs]
        sample = (f"one leapfrog step of progenitors {ps} of the batch (the three smallest, N={n_done} of {wl.n}) by "
                  f"the FP64 C oracle (OpenMP, {oracle.num_threads()} threads); initial force evaluation not counted")
    base = {"value": n_done / secs, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle", "sample": sample,
            "seconds": secs}
    return base, refs


def oracle_error(sim, wl, refs, dtype, torch, use_com):
    """Error of one GPU step against the oracle's step from the same state
    (positions, velocities, the oracle's initial accelerations, centres), on
    the sampled progenitors; the GPU steps the whole launch."""
    import numpy as np
    dev = sim.device
    p = torch.tensor(wl.pos, device=dev, dtype=dtype)
    v = torch.tensor(wl.vel, device=dev, dtype=dtype)
    coms = wl.com[None] if wl.com_per_prog is None else wl.com_per_prog
    c = torch.tensor(coms, device=dev, dtype=torch.float64)
    a = sim.forces(p, sim.coeffs(p), com=c if use_com is not None else None)
    for (_, lo, hi, acc0, *_rest) in refs:
        a[lo:hi] = torch.tensor(acc0, device=dev, dtype=dtype)
    sim.step(p, v, a, com=c if use_com is not None else None, nsteps=1)
    A = sim.last_coeffs().cpu().numpy()
    ag = a.cpu().double().numpy()
    pg = p.cpu().double().numpy()
    cg = c.cpu().numpy()
    coeff, rel_all, pos_err, com_err = 0.0, [], 0.0, 0.0
    for (prog, lo, hi, acc0, p1, v1, a1, c1, A1) in refs:
        coeff = max(coeff, float(np.max(np.abs(A[prog] - A1)) / np.max(np.abs(A1))))
        na = np.linalg.norm(a1[:, :3], axis=1)
        rel_all.append(np.linalg.norm(ag[lo:hi, :3] - a1[:, :3], axis=1) / np.maximum(na, 1e-6 * np.median(na)))
        pos_err = max(pos_err, float(np.max(np.abs(pg[lo:hi, :3] - p1[:, :3]))))
        if use_com is not None:
            com_err = max(com_err, float(np.max(np.abs(cg[prog] - c1) / np.maximum(np.abs(c1), 1e-300))))
    rel = np.concatenate(rel_all)
    out = {
        "coeff_max_rel": coeff, "accel_rel_median": float(np.median(rel)), "accel_rel_p99": float(np.quantile(rel, 0.99)),
        "accel_rel_max": float(np.max(rel)), "pos_max_abs": pos_err,
        "what": "one leapfrog step from the same state, GPU vs the FP64 oracle"
                + ("" if wl.offsets is None else f" (progenitors {[r[0] for r in refs]} of the batched launch)"),
    }
    if use_com is not None:
        out["centre_max_rel"] = com_err
    return out


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
    # time (at most 3 s a step); the per-particle cost is measured on a probe
    # of 20000 particles (one coefficient + force evaluation, as in a step)
    per_step = min(3.0, 120.0 / max(1, args.steps + args.warmup))
    n0 = min(wl.n, 20000)
    probe = wl.pos[:n0].copy()
    probe[:, 3] *= wl.n / n0
    t0 = time.perf_counter()
    A0 = oracle.coeffs(probe, wl.nmax, wl.lmax, wl.b, alpha=wl.alpha)
    oracle.forces(probe, A0, wl.nmax, wl.lmax, wl.b, com=com, host=host, alpha=wl.alpha)
    t_probe = time.perf_counter() - t0
    n = wl.n
    if t_probe * wl.n / n0 > per_step:
        n = max(1000, min(wl.n, int(n0 * per_step / t_probe)))
    pos, vel = wl.pos[:n].copy(), wl.vel[:n].copy()
    pos[:, 3] *= wl.n / n
    A0 = oracle.coeffs(pos, wl.nmax, wl.lmax, wl.b, alpha=wl.alpha)
    acc = oracle.forces(pos, A0, wl.nmax, wl.lmax, wl.b, com=com, host=host, alpha=wl.alpha)
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


def fma_peaks(torch, stream):
    """Measured FMA-chain rates (TFLOP/s) of the FP32 and FP64 pipes with the
    SM clocks sampled while they ran (scf_fma_peak)."""
    from paper_2602_13385_gb300 import _lib
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    f32, ms32 = _lib.scf_fma_peak(_lib.SCF_MIXED, 20000, stream.cuda_stream)
    f64, ms64 = _lib.scf_fma_peak(_lib.SCF_FP64, 400, stream.cuda_stream)
    clocks = sampler.stop()
    return {"fp32_tflops": f32 / 1e12, "fp64_tflops": f64 / 1e12, "ms": [ms32, ms64], "clocks": clocks,
            "what": "independent FMA chains (8 per thread, 2048 threads per SM, best of 3 launches) on the FP32 and "
                    "FP64 pipes (scf_fma_peak)"}


def run_line(name, args, steps, torch, barrier, world, rank, local, peaks, oracle_cache, timing_extras):
    """One bench line: the workload's timed leapfrog steps, end to end rate,
    roofline, and (rank 0, one GPU) the CPU baseline and oracle error."""
    from paper_2602_13385_gb300 import SCF, Config
    wl, precision = build_workload(name, args.n)
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
    if name in FF_WORKLOADS:
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

    def timed_steps(profile):
        # `steps` steps, L2 flushed before each, CUDA events on the handle's
        # stream around each step; with profile, per-kernel events too (plain
        # launches: the captured graph of a step holds no timing events)
        if profile:
            sim.profile(True)
            sim.profile_read()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        torch.cuda.synchronize()
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            sim.step(p, v, a, com=use_com, nsteps=1)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
        if not profile:
            return ms, None, None
        kms_, kcount_ = sim.profile_read()
        sim.profile(False)
        return ms, kms_, kcount_

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            flush.fill_(float(i))
            sim.step(p, v, a, com=use_com, nsteps=1)
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        # the step rate: one captured graph per step, as scf_step runs it
        ms_total, _, _ = timed_steps(False)
        # the kernels' durations: the same steps again with an event pair
        # around every kernel launch
        ms_prof, kms, kcount = timed_steps(True)
        clocks = sampler.stop()
    rc, st = sim.status()
    if rc != 0:
        raise RuntimeError(f"device status {st} after the timed steps of {name}")

    ms_max = max_over_ranks(ms_total, dev)
    value = whole_job_rate(wl.n, steps, world, ms_max)
    ms_step = ms_max / steps

    # end to end through the public API with the state in pinned host memory:
    # every step reads the state from host memory and writes it back there
    # (scf_step_host; on mapped page-locked memory the kernels move it over
    # the host link themselves, overlapped with their arithmetic)
    h_p, h_v, h_a = (t.cpu().pin_memory() for t in (p, v, a))
    h_c = c.cpu().pin_memory() if use_com is not None else None
    e2e_steps = max(3, steps // 2)
    chunks = 1
    with torch.cuda.stream(stream):
        sim.step_host(p, v, a, h_p, h_v, h_a, com=use_com, host_com=h_c, chunks=chunks)   # untimed
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(e2e_steps):
            sim.step_host(p, v, a, h_p, h_v, h_a, com=use_com, host_com=h_c, chunks=chunks)
        t1.record(stream)
        torch.cuda.synchronize()
    e2e_ms = t0.elapsed_time(t1)
    bytes_io = sum(t.numel() * t.element_size() for t in (h_p, h_v, h_a))
    bytes_io += 0 if h_c is None else h_c.numel() * h_c.element_size()
    e2e = {"value": whole_job_rate(wl.n, e2e_steps, world, max_over_ranks(e2e_ms, dev)), "unit": UNIT,
           "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io, "steps": e2e_steps,
           "ms_per_step": e2e_ms / e2e_steps,
           "what": "scf_step_host through the C ABI: the state lives in pinned (mapped) host buffers; every step "
                   "the kernels read it from host memory and write the new state back over the host link"}

    # roofline: ALU-bound (FP64 pipe in fp64 mode, FP32 pipe in mixed mode)
    k1f, k3f = per_particle_flops(wl.nmax, wl.lmax)
    elem = 8 if precision == "fp64" else 4
    k1b, k3b = per_particle_bytes(elem)
    per_k = [kms[i] / max(1, kcount[i]) for i in range(3)]
    dom = 2 if per_k[2] >= per_k[0] else 0
    avg_ms = per_k[dom]
    flops = wl.n * (k3f if dom == 2 else k1f)
    achieved = flops / (avg_ms * 1e-3) / 1e12
    clock = clocks.get("sm_max_mhz") or 2070.0
    is64 = precision == "fp64" and name not in FF_WORKLOADS
    fma = FP64_FMA_PER_SM_CLK if is64 else FP32_FMA_PER_SM_CLK
    peak = N_SM * fma * 2 * clock * 1e6 / 1e12
    meas = peaks.get("fp64_tflops" if is64 else "fp32_tflops") if peaks else None
    kname = "k3_forces" if dom == 2 else "k1_partials"
    step_flops = wl.n * (k1f + k3f)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic_for(kname, name),
                "kernel": kname, "kernel_avg_ms": avg_ms,
                "peak_basis": f"nominal: {'FP64' if is64 else 'FP32'} pipe, {N_SM} SMs x {fma} FMA/clk x 2 "
                              f"x {clock:.0f} MHz (max SM clock)",
                "peak_measured": meas, "frac_of_measured": (achieved / meas) if meas else None,
                "frac_at_sampled_clock": (achieved / (N_SM * fma * 2 * clocks["sm_mhz"] * 1e-6)
                                          if clocks.get("sm_mhz") else None),
                "algorithmic_flops_per_launch": flops,
                "algorithmic_bytes_per_launch": wl.n * (k3b if dom == 2 else k1b),
                "kernels_ms_per_step": {"k1_partials": per_k[0], "k2_reduce": per_k[1], "k3_forces": per_k[2]},
                "kernel_timing": f"a second timed pass of {steps} steps with a CUDA-event pair around every "
                                 f"kernel (plain launches, {ms_prof / steps:.4f} ms per step against "
                                 f"{ms_total / steps:.4f} ms with the captured graph)",
                "whole_step": {"achieved": step_flops / (ms_step * 1e-3) / 1e12, "peak": peak,
                               "frac": step_flops / (ms_step * 1e-3) / 1e12 / peak,
                               "algorithmic_flops_per_step": step_flops,
                               "what": "(kernel 1 + kernel 3 algorithmic flops) x N / ms_per_step"}}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f64 (kernels 1 and 3 in float-float)" if name in FF_WORKLOADS else "f64")
                 if precision == "fp64" else "f32+f64",
        "data": "synthetic (seeded sample, see config.workload)",
        "config": workload_config(wl, precision, name),
        "roofline": roofline, "e2e": e2e,
        # the step kernels of the timed pass (3 per step), plus the centre step
        # computed ahead on the side stream when there is a host
        "gpu_launches": int(sum(kcount)) * (4 if use_com is not None else 3) // 3, "clocks": clocks,
        "kernel_shapes": dict(sim.tiles(), autotuned=tuning is not None,
                              candidates_ms=None if tuning is None else tuning["ms"]),
        "src_hash": src_hash(),
    }
    if timing_extras and not args.no_escape:
        line["escape"] = escape_timing(sim, p, v, offsets, precision, clocks, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        key = (WORKLOADS[name][0], args.n)
        if key not in oracle_cache:
            oracle_cache[key] = oracle_reference(wl)
        base, refs = oracle_cache[key]
        line["cpu_baseline"] = dict(base)
        line["error_vs_oracle"] = oracle_error(sim, wl, refs, dtype, torch, use_com)
    if timing_extras and not args.no_escape:
        line["refresh"] = refresh_timing(sim, p, v, torch)
    sim.close()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=None,
                    help="run only this line (default: the headline plus the mixed and batch lines)")
    ap.add_argument("--extra-steps", type=int, default=100,
                    help="timed steps of the mixed and batch lines of the default run (at least --steps)")
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
    if args.impl == "reference" and args.workload is None:
        args.workload = DEFAULT_WORKLOAD

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

    lines = DEFAULT_LINES if args.workload is None else [("headline", args.workload)]
    peaks = fma_peaks(torch, torch.cuda.current_stream())
    oracle_cache = {}
    out = {}
    for key, name in lines:
        steps = args.steps if key == "headline" else max(args.steps, args.extra_steps)
        # escape-physics and refresh timings ride on the mixed line (or on a single chosen line)
        extras = key == "mixed" or args.workload is not None
        out[key] = run_line(name, args, steps, torch, barrier, world, rank, local, peaks, oracle_cache, extras)
    line = dict(out.pop("headline"))
    line["warmup"] = args.warmup
    line["peak_measured"] = peaks
    for key, sub in out.items():
        sub = dict(sub)
        sub["warmup"] = args.warmup
        line[key] = sub
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
