"""Pins of the stream statistics (paper_2602_13385_gb300.streams, Sec. 3.3) on
synthetic streams whose answers are known in closed form:

* the great-circle frame of a progenitor in the x-y plane moving along +y;
* the binning rule: bins start at the progenitor, every bin holds >= 100
  stars and spans >= 0.5 deg, the remainder joins the outermost bin;
* a stream with a known track offset, width, linear velocity gradient and
  isotropic dispersion: the estimators recover them (the detrending removes
  the gradient, which would otherwise inflate sigma), the density integrates
  to 1, and proper motions along the track give a misalignment cosine of 1
  while motions turned by 30 deg on the sky give cos 30 deg.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2602_13385_gb300 import streams  # noqa: E402


def test_frame_and_sky_coordinates():
    R, V = np.array([8.0, 0.0, 0.0]), np.array([0.0, 0.2, 0.0])
    E = streams.great_circle_frame(R, V)
    assert np.allclose(E, np.eye(3))
    X = np.array([[8.0, 0.0, 0.0], [0.0, 8.0, 0.0], [8.0, 0.0, 8.0], [-8.0, -1e-12, 0.0], [0.0, -3.0, 0.0]])
    p1, p2 = streams.sky_coords(X, R, V)
    assert np.allclose(p1, [0.0, 90.0, 0.0, -180.0, -90.0]) and np.allclose(p2, [0.0, 0.0, 45.0, 0.0, 0.0])
    # an inclined orbit: the progenitor is at (0, 0) and its velocity points to +phi_1
    R, V = np.array([3.0, 4.0, 1.0]), np.array([-1.0, 0.5, 2.0])
    p1, p2 = streams.sky_coords(np.stack([R, R + 1e-3 * V]), R, V)
    assert abs(p1[0]) < 1e-12 and abs(p2[0]) < 1e-12 and p1[1] > 0 and abs(p2[1]) < 1e-9


@pytest.mark.parametrize("seed", [1, 2])
def test_binning_rule(seed):
    rng = np.random.default_rng(seed)
    phi1 = np.concatenate([rng.exponential(6.0, 2345), -rng.exponential(2.0, 987), rng.uniform(0, 0.2, 50)])
    e = streams.bin_edges(phi1)
    assert np.all(np.diff(e) >= 0.5 - 1e-12)
    assert 0.0 in e
    h = np.histogram(phi1, e)[0]
    assert h.sum() == phi1.size and np.all(h >= 100)
    # from the progenitor outwards, every bin but the outermost of each tail is
    # closed as soon as both conditions hold: dropping its outermost star breaks one
    k0 = int(np.where(e == 0.0)[0][0])
    for k in range(k0, len(e) - 2):            # leading tail, inner bins
        s = np.sort(phi1[(phi1 >= e[k]) & (phi1 < e[k + 1])])
        assert s.size == 100 or s[-2] - e[k] < 0.5


def _synthetic_stream(n, track=0.3, width=0.2, sigma=5.0, grad=2.0, turn_deg=0.0, seed=3):
    """Stars on the great circle of a progenitor at (8, 0, 0) moving along +y,
    at phi_1 uniform in [-20, 20] deg and phi_2 ~ N(track, width) deg; host
    velocities = 200 along the track (turned by turn_deg on the sky) + a
    gradient grad * phi_1 along x + isotropic N(0, sigma)."""
    rng = np.random.default_rng(seed)
    p1 = np.radians(rng.uniform(-20, 20, n))
    p2 = np.radians(rng.normal(track, width, n))
    r = 8.0
    X = r * np.stack([np.cos(p2) * np.cos(p1), np.cos(p2) * np.sin(p1), np.sin(p2)], axis=1)
    e1 = np.stack([-np.sin(p1), np.cos(p1), np.zeros(n)], axis=1)
    e2 = np.stack([-np.sin(p2) * np.cos(p1), -np.sin(p2) * np.sin(p1), np.cos(p2)], axis=1)
    t = math.radians(turn_deg)
    Vh = 200.0 * (math.cos(t) * e1 + math.sin(t) * e2)
    Vt = Vh.copy()
    Vh = Vh + grad * np.degrees(p1)[:, None] * np.array([1.0, 0.0, 0.0]) + rng.normal(0, sigma, (n, 3))
    return X, Vh, Vt


def test_statistics_of_a_synthetic_stream():
    X, Vh, _ = _synthetic_stream(200_000, grad=20.0)
    R, V = np.array([8.0, 0.0, 0.0]), np.array([0.0, 200.0, 0.0])
    s = streams.stream_stats(X, Vh, R, V, np.ones(len(X), bool), min_count=5000, min_width=2.0)
    occ = s["n"] > 0
    assert occ.all() and s["n"].sum() == len(X)
    assert abs(np.sum(s["rho"] * (s["hi"] - s["lo"])) - 1.0) < 1e-12
    assert np.allclose(s["rho"], 1.0 / 40.0, rtol=0.1)
    assert np.allclose(s["track"], 0.3, atol=0.02)
    assert np.allclose(s["width"], 0.2, rtol=0.05)
    assert np.allclose(s["sigma"], 5.0, rtol=0.05)
    # without detrending, the gradient (20 km/s per degree over 2 degree bins) inflates sigma
    raw = [np.sqrt(np.trace(np.cov(Vh[(np.degrees(np.arctan2(X[:, 1], X[:, 0])) >= lo)
                                      & (np.degrees(np.arctan2(X[:, 1], X[:, 0])) < hi)].T)) / 3)
           for lo, hi in zip(s["lo"], s["hi"])]
    assert np.all(np.array(raw) > s["sigma"] * 1.3)


@pytest.mark.parametrize("turn", [0.0, 30.0])
def test_misalignment_angle(turn):
    X, _, Vt = _synthetic_stream(50_000, width=0.05, turn_deg=turn)
    R, V = np.array([8.0, 0.0, 0.0]), np.array([0.0, 200.0, 0.0])
    s = streams.stream_stats(X, Vt, R, V, np.ones(len(X), bool), min_count=2000)
    assert np.allclose(s["cos_mis"], math.cos(math.radians(turn)), atol=2e-3), s["cos_mis"]


def test_compare_on_identical_and_perturbed_runs():
    X, Vh, _ = _synthetic_stream(20_000)
    R, V = np.array([8.0, 0.0, 0.0]), np.array([0.0, 200.0, 0.0])
    u = np.ones(len(X), bool)
    a = streams.stream_stats(X, Vh, R, V, u)
    edges = np.concatenate([a["lo"], a["hi"][-1:]])
    d, ok = streams.compare(a, streams.stream_stats(X, Vh, R, V, u, edges=edges))
    assert ok and max(d.values()) == 0.0
    d, ok = streams.compare(a, streams.stream_stats(X, Vh * 1.05, R, V, u, edges=edges))
    assert not ok and abs(d["sigma"] - 0.05) < 1e-9
