"""Pins of the oracle's kick-drift-kick leapfrog (Sec. 2.1.1): exact time
reversibility, a circular two-body orbit against the analytic solution, and
free drift with periodic wrap."""
import math

import numpy as np
import pytest

import oracle
from paper_1502_07442_gb300 import inputs


def _p(D=1, rs=1e3, rcut=0.3, eps=1e-9):
    return oracle.make_params(D, np.ones((D, D)), eps=eps, rs=rs, rcut=rcut, theta=0.0)


def test_time_reversibility():
    rng = inputs.rng_for(31)
    n = 60
    pos = 0.4 + 0.2 * rng.random((3, n))
    vel = 0.01 * rng.standard_normal((3, n))
    typ = np.zeros(n, np.uint8)
    mass = np.full(n, 1.0 / n, np.float32)
    p = _p(eps=0.01)
    x1, v1, _ = oracle.kdk(p, pos, vel, typ, mass, 25, 2e-3)
    x2, v2, _ = oracle.kdk(p, x1, -v1, typ, mass, 25, 2e-3)
    np.testing.assert_allclose(x2, pos, atol=1e-12)
    np.testing.assert_allclose(-v2, vel, atol=1e-12)


def test_circular_two_body_orbit():
    d, M = 0.05, 1.0
    m = np.array([0.5, 0.5], np.float32)
    omega = math.sqrt(M / d ** 3)
    pos = np.array([[0.5 - d / 2, 0.5 + d / 2], [0.5, 0.5], [0.5, 0.5]])
    v = omega * d / 2
    vel = np.array([[0.0, 0.0], [-v, v], [0.0, 0.0]])
    period = 2 * math.pi / omega
    steps = 400
    dt = period / steps
    x, vv, _ = oracle.kdk(_p(), pos, vel, np.zeros(2, np.uint8), m, steps // 4, dt)
    # a quarter turn: body 0 (at -x, moving -y) ends at -y
    want0 = np.array([0.5, 0.5 - d / 2, 0.5])
    assert np.linalg.norm(x[:, 0] - want0) < 2e-3 * d
    # energy-like check: the separation stays d
    assert np.linalg.norm(x[:, 0] - x[:, 1]) == pytest.approx(d, rel=1e-4)


def test_free_drift_wraps():
    pos = np.array([[0.95], [0.02], [0.5]])
    vel = np.array([[1.0], [-1.0], [0.25]])
    x, v, a = oracle.kdk(_p(), pos, vel, np.zeros(1, np.uint8), np.ones(1, np.float32), 10, 0.01)
    np.testing.assert_allclose(x[:, 0], [0.05, 0.92, 0.525], atol=1e-12)
    assert np.all(a == 0.0)
