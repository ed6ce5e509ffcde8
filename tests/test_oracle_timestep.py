"""Pins of the oracle's synchronous time step (Sec. 2.1.1, Eq. (our_timestep)).

A_max is the supremum of |f_ij(r)| r^2 / M over r and the species pairs; the
oracle finds it by sampling its full (unsplit) laws. Worked out by hand from
Eq. (yukawa): the Newtonian factor is 1; the C = 1 Yukawa factor is
1 + a g(r) with g = (1 + r/l) e^{-r/l} running over (0, 1], so its largest
magnitude is max(1, |1 + a|); the pure Yukawa factor a g(r) peaks at |a|.
"""
import math

import numpy as np
import pytest

import oracle


def _params(G, law, ya, yl, eps=1e-3):
    D = len(G)
    return oracle.make_params(D, G, eps=eps, rs=0.02, rcut=0.09, law=law, ya=ya, yl=yl)


@pytest.mark.parametrize("law,a,want", [
    (oracle.NEWTON, 0.0, 1.0), (oracle.YUKAWA, 0.3, 1.3), (oracle.YUKAWA, -0.5, 1.0),
    (oracle.YUKAWA, -2.5, 1.5), (oracle.YUKAWA_PURE, 0.7, 0.7), (oracle.YUKAWA_PURE, -1.2, 1.2)])
def test_amax_closed_forms(law, a, want):
    p = _params([[2.0]], [[law]], [[a]], [[0.03]])
    assert oracle.law_amax(p) == pytest.approx(2.0 * want, rel=1e-9)


def test_amax_takes_the_largest_pair():
    G = [[1.0, 0.5], [0.5, 0.8]]
    p = _params(G, [[0, 1], [1, 2]], [[0, 1.0], [1.0, 3.0]], [[1, 0.05], [0.05, 0.02]])
    # pairs: 1 * 1, 0.5 * 2, 0.5 * 2, 0.8 * 3
    assert oracle.law_amax(p) == pytest.approx(2.4, rel=1e-9)


def test_timestep_formula():
    rng = np.random.Generator(np.random.PCG64(5))
    acc = rng.standard_normal((3, 1000)).astype(np.float32)
    p = _params([[1.5]], [[0]], [[0.0]], [[1.0]], eps=2e-3)
    eta, dt_max = 0.025, 1.0
    dt, amax = oracle.timestep(p, acc, eta, dt_max)
    assert amax == pytest.approx(np.linalg.norm(acc.astype(np.float64), axis=0).max(), rel=1e-6)
    assert dt == pytest.approx(math.sqrt(2 * eta * 2e-3 / (1.5 * amax)), rel=1e-12)
    # capped by dt_max, and dt_max when nothing accelerates
    assert oracle.timestep(p, acc, eta, 1e-4)[0] == 1e-4
    assert oracle.timestep(p, np.zeros((3, 10), np.float32), eta, 0.5)[0] == 0.5
    # dt scales as A_max^(-1/2)
    p4 = _params([[6.0]], [[0]], [[0.0]], [[1.0]], eps=2e-3)
    assert oracle.timestep(p4, acc, eta, dt_max)[0] == pytest.approx(0.5 * dt, rel=1e-12)
