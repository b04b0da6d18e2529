"""Per-progenitor diagnostics of a run's state, and a JSON-lines log of them.

The quantities the paper follows (Sec. 2.1-2.2, Sec. 3.1, Fig. 4):

* the energy in the cluster frame, K, W, U and their sum (``scf_energy``);
* the bound count and mass (``scf_bound``, the Sec. 2.2 energy test);
* the energy-based Lagrange radii r_x, the smallest radii enclosing the
  fraction x of the bound stars, and the bound radius r_b = r_100;
* the number of stars outside r_b;
* the tidal radius (Sec. 3.1 footnote) and the integration timestep
  (``scf_tidal``);
* the centre (R, V).

The energies, the boundedness test and the tidal scales run in the CUDA
kernels; the Lagrange radii are order statistics of the bound stars' radii,
taken on the host from the flags and positions (r^2 compared in double
precision, as the kernels do).
"""
from __future__ import annotations

import json
import math

import numpy as np

LAGRANGE_FRACTIONS = (0.01, 0.1, 0.3, 0.5, 0.7, 0.8, 0.9, 0.99)


def snapshot(sim, pos, vel, acc, com=None, t: float = 0.0, kin: float = 0.5, eta: float = 1.0 / 400.0,
             fractions=LAGRANGE_FRACTIONS) -> list[dict]:
    """One record per progenitor.  ``acc`` must hold the accelerations and
    potential at ``pos`` (as ``step`` and ``forces`` leave them)."""
    E = sim.energy(pos, vel, acc, com).cpu().numpy()
    bnd, _, st, _ = sim.bound(pos, vel, kin=kin, frac=1.0)
    has_host = len(sim.config.host) > 0
    tid = sim.tidal(com, M_c=st[:, 1].contiguous(), eta=eta).cpu().numpy() if has_host else None
    b = bnd.cpu().numpy().astype(bool)
    p = pos.detach().double().cpu().numpy()
    r2 = (p[:, 0] * p[:, 0] + p[:, 1] * p[:, 1]) + p[:, 2] * p[:, 2]
    st = st.cpu().numpy()
    c = None if com is None else com.detach().cpu().numpy()
    out = []
    for i in range(sim.n_prog):
        s = slice(sim.offsets[i], sim.offsets[i + 1])
        rb2 = np.sort(r2[s][b[s]])
        lag = {}
        for x in fractions:
            k = max(1, int(math.ceil(x * rb2.size))) if rb2.size else 0
            lag[f"{x:g}"] = float(math.sqrt(rb2[k - 1])) if k else 0.0
        r_b = float(st[i, 2])
        rec = {
            "t": float(t), "progenitor": i,
            "K": float(E[i, 0]), "W": float(E[i, 1]), "U": float(E[i, 2]), "E": float(E[i, 3]),
            "n_bound": int(st[i, 0]), "M_bound": float(st[i, 1]), "r_b": r_b,
            "n_outside_r_b": int(np.count_nonzero(r2[s] > r_b * r_b)) if rb2.size else int(r2[s].size),
            "lagrange_radii": lag,
        }
        if tid is not None:
            rec.update({"r_t": float(tid[i, 14]), "dt_int": float(tid[i, 15]),
                        "tidal_eigenvalues": [float(v) for v in tid[i, 9:12]]})
        if c is not None:
            rec.update({"R": [float(v) for v in c[i, :3]], "V": [float(v) for v in c[i, 3:]]})
        out.append(rec)
    return out


class JsonlLog:
    """Appends diagnostic records to a JSON-lines file, one record a line."""

    def __init__(self, path: str):
        self.path = path
        self._f = open(path, "a", encoding="utf-8")

    def write(self, records) -> None:
        for r in records:
            self._f.write(json.dumps(r) + "\n")
        self._f.flush()

    def close(self) -> None:
        self._f.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def read_jsonl(path: str) -> list[dict]:
    with open(path, encoding="utf-8") as f:
        return [json.loads(line) for line in f if line.strip()]
