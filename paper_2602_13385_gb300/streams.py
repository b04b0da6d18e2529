"""Stream statistics of Sec. 3.3, measured on a snapshot (host-side analysis).

This is post-processing of the particles a run leaves in device memory
(positions, velocities, the bound flags of ``scf_bound``), not a step of the
gravity solver: it copies them to the host and bins them with numpy.

* Great-circle frame of an observer at the galactic centre (Figs. 1-2): the
  pole is the progenitor's orbital angular momentum R x V, the first axis
  points at the progenitor (phi_1 = phi_2 = 0 there) and phi_1 grows along
  its motion; phi_2 is the angle out of the instantaneous orbital plane.
* Binning (Sec. 3.3): the unbound stars are binned in phi_1 from the
  progenitor outwards, leading (phi_1 > 0) and trailing (phi_1 < 0) tails
  separately, each bin closed once it holds at least ``min_count`` stars and
  spans at least ``min_width`` degrees; a remainder too small to close a bin
  joins the last bin of its tail.
* Per bin: the normalised density rho = n / (n_unbound dphi_1) (so the sum of
  rho dphi_1 over the bins is 1), the track (mean phi_2), the width (standard
  deviation of phi_2), the 1D velocity dispersion sigma = sqrt(tr Sigma / 3)
  of the host-frame velocities after removing a linear fit in phi_1 within
  the bin, and the mean cosine of the misalignment between each star's proper
  motion (as seen from the centre) and the tangent of the track, the track
  being a smoothing spline of the bin means of phi_2 against phi_1.
  The paper averages sigma over bootstrap draws of each bin; the plain
  estimate on all of the bin's stars is what those draws scatter about and is
  used here.
"""
from __future__ import annotations

import numpy as np


def great_circle_frame(R, V):
    """Orthonormal rows (e1, e2, e3): e1 = R / |R|, e3 along R x V, e2 = e3 x e1."""
    R = np.asarray(R, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    e1 = R / np.linalg.norm(R)
    L = np.cross(R, V)
    e3 = L / np.linalg.norm(L)
    e2 = np.cross(e3, e1)
    return np.stack([e1, e2, e3])


def sky_coords(X, R, V):
    """(phi_1, phi_2) in degrees of host-frame positions X (n, 3)."""
    E = great_circle_frame(R, V)
    q = np.asarray(X, dtype=np.float64) @ E.T
    phi1 = np.degrees(np.arctan2(q[:, 1], q[:, 0]))
    phi2 = np.degrees(np.arcsin(np.clip(q[:, 2] / np.linalg.norm(q, axis=1), -1.0, 1.0)))
    return phi1, phi2


def _tail_edges(a, min_count, min_width):
    """Bin edges in |phi_1| >= 0 for one tail (a = sorted |phi_1| values)."""
    edges = [0.0]
    i, n = 0, a.size
    while n - i >= min_count:
        hi = max(float(a[i + min_count - 1]), edges[-1] + min_width)
        j = int(np.searchsorted(a, hi, side="right"))     # stars a[i:j] lie in this bin
        if j >= n:                                        # it takes every remaining star
            edges.append(max(hi, float(a[-1])))
            return np.array(edges)
        edges.append(max(hi, 0.5 * float(a[j - 1] + a[j])))
        i = j
    if i < n:                          # a remainder too small for a bin of its own
        if len(edges) == 1:
            edges.append(max(float(a[-1]), min_width))
        else:
            edges[-1] = max(edges[-1], float(a[-1]))
    return np.array(edges)


def bin_edges(phi1, min_count=100, min_width=0.5):
    """Edges (ascending, degrees) of the Sec. 3.3 binning of ``phi1``: from 0
    outwards in each tail, each bin >= min_count stars and >= min_width wide."""
    phi1 = np.asarray(phi1, dtype=np.float64)
    lead = np.sort(phi1[phi1 >= 0.0])
    trail = np.sort(-phi1[phi1 < 0.0])
    el = _tail_edges(lead, min_count, min_width) if lead.size else np.array([0.0])
    et = _tail_edges(trail, min_count, min_width) if trail.size else np.array([0.0])
    return np.concatenate([-et[::-1], el[1:]]) if et.size > 1 else el


def _track_slope(c1, c2):
    """d phi_2 / d phi_1 of a smoothing spline through the bin means (c1
    ascending); a straight line below 5 bins."""
    if c1.size < 2:
        return lambda x: np.zeros_like(x)
    if c1.size < 5:
        k = np.polyfit(c1, c2, 1)[0]
        return lambda x: np.full_like(x, k)
    from scipy.interpolate import make_smoothing_spline
    spl = make_smoothing_spline(c1, c2)
    d = spl.derivative()
    return lambda x: d(np.clip(x, c1[0], c1[-1]))


def stream_stats(X, Vh, R, V, unbound, edges=None, min_count=100, min_width=0.5):
    """Statistics of the unbound stars per phi_1 bin.

    X, Vh: host-frame positions and velocities (n, 3); R, V: the progenitor's
    position and velocity; unbound: boolean (n,).  ``edges`` fixes the bins
    (e.g. those of another run) instead of the Sec. 3.3 rule.
    Returns a dict of arrays over bins: ``lo``, ``hi``, ``n``, ``rho``,
    ``track``, ``width``, ``sigma``, ``cos_mis``.
    """
    X = np.asarray(X, dtype=np.float64)[unbound]
    Vh = np.asarray(Vh, dtype=np.float64)[unbound]
    phi1, phi2 = sky_coords(X, R, V)
    if edges is None:
        edges = bin_edges(phi1, min_count, min_width)
    nb = len(edges) - 1
    out = {k: np.zeros(nb) for k in ("lo", "hi", "n", "rho", "track", "width", "sigma", "cos_mis", "phi1")}
    out["lo"], out["hi"] = edges[:-1].copy(), edges[1:].copy()
    which = np.searchsorted(edges, phi1, side="right") - 1
    # stars exactly on the last edge belong to the last bin
    which[phi1 == edges[-1]] = nb - 1
    inside = (which >= 0) & (which < nb)
    n_all = max(int(inside.sum()), 1)
    for k in range(nb):
        s = inside & (which == k)
        n = int(s.sum())
        out["n"][k] = n
        out["rho"][k] = n / (n_all * (edges[k + 1] - edges[k]))
        if n == 0:
            continue
        out["phi1"][k] = phi1[s].mean()
        out["track"][k] = phi2[s].mean()
        out["width"][k] = phi2[s].std()
        if n > 2:
            A = np.stack([np.ones(n), phi1[s] - out["phi1"][k]], axis=1)
            coef, *_ = np.linalg.lstsq(A, Vh[s], rcond=None)
            dv = Vh[s] - A @ coef
            cov = dv.T @ dv / (n - 1)
            out["sigma"][k] = np.sqrt(np.trace(cov) / 3.0)
    # misalignment of the proper motions with the track's tangent
    E = great_circle_frame(R, V)
    occupied = out["n"] > 0
    slope = _track_slope(out["phi1"][occupied], out["track"][occupied])
    p1, p2 = np.radians(phi1), np.radians(phi2)
    e_phi1 = (-np.sin(p1))[:, None] * E[0] + np.cos(p1)[:, None] * E[1]
    e_phi2 = ((-np.sin(p2) * np.cos(p1))[:, None] * E[0] + (-np.sin(p2) * np.sin(p1))[:, None] * E[1]
              + np.cos(p2)[:, None] * E[2])
    mu1 = np.sum(Vh * e_phi1, axis=1)
    mu2 = np.sum(Vh * e_phi2, axis=1)
    t1 = np.cos(p2)
    t2 = slope(phi1)
    norm = np.hypot(mu1, mu2) * np.hypot(t1, t2)
    cosm = np.where(norm > 0, (mu1 * t1 + mu2 * t2) / np.where(norm > 0, norm, 1.0), 0.0)
    for k in range(nb):
        s = inside & (which == k)
        if s.any():
            out["cos_mis"][k] = cosm[s].mean()
    return out


def compare(a, b, tol=0.01):
    """Largest relative differences between two stream_stats results on the
    same bins: density, width and sigma relative to run a, the track relative
    to run a's width, and the misalignment cosine absolutely.  Returns a dict
    and whether all are within ``tol``."""
    occ = a["n"] > 0
    def rel(x, y, s):
        return float(np.max(np.abs(x[occ] - y[occ]) / np.abs(s[occ]))) if occ.any() else 0.0
    d = {"rho": rel(a["rho"], b["rho"], a["rho"]),
         "track": rel(a["track"], b["track"], a["width"]),
         "width": rel(a["width"], b["width"], a["width"]),
         "sigma": rel(a["sigma"], b["sigma"], a["sigma"]),
         "cos_mis": float(np.max(np.abs(a["cos_mis"][occ] - b["cos_mis"][occ]))) if occ.any() else 0.0}
    return d, all(v <= tol for v in d.values())
