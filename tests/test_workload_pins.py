"""Pins of the King (1966) sampler that generates the King-cluster workloads
(single cluster, the batch of progenitors, the differentiable run and the
paper's progenitors of Sec. 3).

* The depth W0 fixes the concentration c = log10(r_t / r_0) of the lowered
  isothermal model; King (1966) tabulates it (W0 = 3, 5, 6, 7, 9 give c =
  0.67, 1.03, 1.26, 1.53, 2.12, two decimals).  The sampler's Poisson
  integration must reproduce it.
* A sample is in Henon units: total energy E = K + U = -1/4 and virial ratio
  2K/|U| = 1 (both to sampling noise, U by direct summation), centred at the
  origin at rest.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

KING_1966_CONCENTRATION = {3.0: 0.67, 5.0: 1.03, 6.0: 1.26, 7.0: 1.53, 9.0: 2.12}


@pytest.mark.parametrize("W0", sorted(KING_1966_CONCENTRATION))
def test_king_concentration_matches_king_1966(W0):
    km = workloads.king_model(W0)
    assert math.log10(km.rt) == pytest.approx(KING_1966_CONCENTRATION[W0], abs=0.006)


@pytest.mark.parametrize("W0,seed", [(4.0, 1), (6.0, 2), (8.0, 3)])
def test_king_sample_is_in_henon_units(W0, seed):
    n = 20000
    pos, vel = workloads.king(n, W0, seed=seed)
    m = pos[:, 3]
    assert m.sum() == pytest.approx(1.0, rel=1e-12)
    K = 0.5 * float(np.sum(m * np.sum(vel[:, :3] ** 2, axis=1)))
    U = 0.5 * float(np.sum(m * oracle.direct(pos, pos)[:, 3]))
    # sampling noise of E and of the virial ratio at N = 2e4 is below 1%
    assert K + U == pytest.approx(-0.25, abs=0.005)
    assert 2 * K / abs(U) == pytest.approx(1.0, abs=0.015)
    assert np.max(np.abs(pos[:, :3].T @ m)) < 1e-14
    assert np.max(np.abs(vel[:, :3].T @ m)) < 1e-14


def test_king_speeds_stay_below_escape_speed():
    """The lowered isothermal DF has no stars with v^2/2 > W: every star is
    bound to the model (its speed below the local escape speed of the model's
    own potential, evaluated here by direct summation)."""
    pos, vel = workloads.king(4000, 6.0, seed=4)
    phi = oracle.direct(pos, pos)[:, 3]
    v2 = np.sum(vel[:, :3] ** 2, axis=1)
    # the sample's own potential is noisy at N = 4e3: allow 5% on phi
    assert np.all(0.5 * v2 < 1.05 * np.abs(phi))
