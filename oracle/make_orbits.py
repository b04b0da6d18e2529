"""Write ``workloads/orbit_ics.json``: the cluster-centre orbits of the workloads.

Run ``python -m oracle.make_orbits``.  The orbits are integrated in the host of
the multi-cluster workloads (NFW + Miyamoto-Nagai + Hernquist, App. A forms)
with the oracle's host acceleration, in kpc, km/s and G = 4.30091727e-6
kpc (km/s)^2 / Msun:

* ``circular_8kpc``: R = (8, 0, 0) kpc in the disk plane, V = (0, v_c, 0) with
  v_c = sqrt(R |a_R|).
* ``eccentric_5_20kpc``: starts at apocentre 20 kpc in the direction of the
  paper's "Eccentric Test" initial position (Table A3), moving along +y like
  that orbit; the speed is root-found so that the pericentre is 5 kpc.
* ``batch``: seeded orbits with pericentre ~ U(3, 20) kpc and apocentre ~
  U(max(peri, 10), 40) kpc in random orbital planes, root-found the same way.
"""
from __future__ import annotations

import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import workloads  # noqa: E402

G_KPC = workloads.G_PC_KMS2_MSUN * 1e-3   # kpc (km/s)^2 / Msun


def host():
    comps = [(k, M, a * 1e-3, b * 1e-3) for (k, M, a, b) in workloads.galaxy_host_physical()]
    return oracle.host_struct(comps, G=G_KPC)


def peri_apo(h, R, V, t_max=3.0, dt=2e-5):
    """Leapfrog the orbit (time unit kpc/(km/s) ~ 0.978 Gyr) and return the
    extreme radii reached within ``t_max``."""
    R = np.array(R, float)
    V = np.array(V, float)
    a, _ = oracle.host_accel(h, R)
    rmin = rmax = float(np.linalg.norm(R))
    for _ in range(int(t_max / dt)):
        V += 0.5 * dt * a
        R += dt * V
        a, _ = oracle.host_accel(h, R)
        V += 0.5 * dt * a
        r = float(np.linalg.norm(R))
        rmin = min(rmin, r)
        rmax = max(rmax, r)
    return rmin, rmax


def vcirc(h, R):
    a, _ = oracle.host_accel(h, np.array(R, float))
    rhat = np.array(R, float) / np.linalg.norm(R)
    return math.sqrt(np.linalg.norm(R) * abs(float(a @ rhat)))


def solve_speed(h, R, vdir, peri_target, t_max):
    """Bisection on the tangential speed at apocentre so that the pericentre
    equals ``peri_target``."""
    lo, hi = 1.0, vcirc(h, R)
    for _ in range(30):
        mid = 0.5 * (lo + hi)
        pmin, _ = peri_apo(h, R, mid * vdir, t_max=t_max, dt=1e-4)
        if pmin < peri_target:
            lo = mid
        else:
            hi = mid
    v = 0.5 * (lo + hi)
    pmin, pmax = peri_apo(h, R, v * vdir, t_max=t_max, dt=2e-5)
    return v, pmin, pmax


def main():
    h = host()
    out = {"units": "R in kpc, V in km/s, host frame", "host": "NFW(Mvir=1e12, rs=20 kpc) + MN(6.8e10, 3, 0.28) + "
           "Hernquist(5e9, 0.5); G = 4.30091727e-6 kpc (km/s)^2/Msun"}
    R = [8.0, 0.0, 0.0]
    out["circular_8kpc"] = {"R_kpc": R, "V_kms": [0.0, vcirc(h, R), 0.0]}

    d = np.array([4.04231677, 0.0, 19.58670971])   # Table A3, Eccentric Test position
    R = 20.0 * d / np.linalg.norm(d)
    v, pmin, pmax = solve_speed(h, R, np.array([0.0, 1.0, 0.0]), 5.0, t_max=1.0)
    out["eccentric_5_20kpc"] = {"R_kpc": R.tolist(), "V_kms": [0.0, v, 0.0], "peri_kpc": pmin, "apo_kpc": pmax}

    rng = np.random.default_rng(40)
    batch = []
    for _ in range(10):
        peri = rng.uniform(3.0, 20.0)
        apo = rng.uniform(max(peri, 10.0), 40.0)
        if apo < peri:
            apo = peri
        u = rng.normal(size=3)
        rhat = u / np.linalg.norm(u)
        w = rng.normal(size=3)
        w -= (w @ rhat) * rhat
        vdir = w / np.linalg.norm(w)
        Rb = apo * rhat
        v, pmin, pmax = solve_speed(h, Rb, vdir, peri, t_max=2.0)
        batch.append({"R_kpc": Rb.tolist(), "V_kms": (v * vdir).tolist(), "peri_target_kpc": peri,
                      "apo_target_kpc": apo, "peri_kpc": pmin, "apo_kpc": pmax})
    out["batch"] = batch
    path = os.path.join(os.path.dirname(HERE), "workloads", "orbit_ics.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
