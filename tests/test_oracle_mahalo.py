"""Pins of the oracle's accumulator ("Mahalo") laws of Sec. 3.3, pure tree mode.

* The law: phi = -(2 M m / (pi r)) atan(r / a) is the potential of the cored
  density M a / (pi^2 (a^2 + r^2)^2) (radial quadrature of Poisson's
  equation), whose 3D transform is M e^{-a k} (quadrature), so two such
  objects attract with a = a_1 + a_2 (scales add under convolution; the
  remaining integral int e^{-a k} sin(kr)/k dk = atan(r/a) by quadrature).
  With a_i = m_i / (4 pi beta) this is Eq. (bambam). The force factor is the
  derivative of that potential (central difference) and tends to Newton far
  away.
* N_perp: a node of N_perp coincident bodies is represented exactly by its
  monopole when N_perp is used, and not when it is ignored.
* The Sec. 3.3 accuracy check: with two species (Newtonian, cored), the tree
  force with N_perp is many times more accurate against the direct sum than
  without, and about as accurate as the Newtonian-only tree.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from common import oracle_params
from metrics import rel_err
from paper_1502_07442_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


def _density(a, r):
    return a / (math.pi ** 2 * (a * a + r * r) ** 2)


def test_potential_of_the_cored_density():
    a = 0.03
    for r in (0.005, 0.03, 0.2):
        inner = integrate.quad(lambda x: 4 * math.pi * x * x * _density(a, x), 0, r,
                               epsabs=1e-14, epsrel=1e-12)[0]
        outer = integrate.quad(lambda x: 4 * math.pi * x * _density(a, x), r, np.inf,
                               epsabs=1e-14, epsrel=1e-12)[0]
        phi = -(inner / r + outer)
        assert phi == pytest.approx(-2 / (math.pi * r) * math.atan(r / a), rel=1e-9)
    total = integrate.quad(lambda x: 4 * math.pi * x * x * _density(a, x), 0, np.inf)[0]
    assert total == pytest.approx(1.0, rel=1e-10)


def test_scales_add_between_two_cored_objects():
    a1, a2 = 0.02, 0.05
    for k in (3.0, 20.0, 70.0):
        ft = integrate.quad(lambda x: 4 * math.pi * x * x * _density(a1, x) * math.sin(k * x) / (k * x),
                            0, np.inf, limit=400, epsabs=1e-13)[0]
        assert ft == pytest.approx(math.exp(-a1 * k), rel=1e-7, abs=1e-12)
    # mutual potential: -(2/pi) int_0^inf e^{-(a1+a2)k} sin(kr)/k dk / r
    for r in (0.01, 0.1, 0.4):
        I = integrate.quad(lambda k: math.exp(-(a1 + a2) * k) * math.sin(k * r) / k, 0, np.inf,
                           limit=400)[0]
        assert I == pytest.approx(math.atan(r / (a1 + a2)), rel=1e-9)
    # Eq. (bambam): a_i = m_i / (4 pi beta); the factor of the oracle is the
    # derivative of -(2/(pi r)) atan(4 pi beta r / (M + m)) times r^2
    beta, M, m = 1.3e-3, 2e-3, 5e-4
    V = lambda r: -2 / (math.pi * r) * math.atan(4 * math.pi * beta * r / (M + m))
    for r in (0.003, 0.05, 0.3):
        h = r * 1e-4
        dV = (V(r + h) - V(r - h)) / (2 * h)
        assert oracle.mahalo_factor(beta, M + m, r) / r ** 2 == pytest.approx(dV, rel=1e-6)
    # Newton far away; linear core near the centre
    for r in (1e2, 1e4):
        x = 4 * math.pi * beta * r / (M + m)       # atan(x) = pi/2 - 1/x + ...
        assert oracle.mahalo_factor(beta, M + m, r) == pytest.approx(1 - 4 / (math.pi * x), rel=1e-7)
    x = 1e-3
    r = x * (M + m) / (4 * math.pi * beta)
    assert oracle.mahalo_factor(beta, M + m, r) == pytest.approx(4 / (3 * math.pi) * x ** 3, rel=1e-5)


def _mahalo_params(beta, rcut=0.45, theta=0.5, leaf=8, ignore=0):
    return dict(D=2, G=[[1.0, 1.0], [1.0, 1.0]], law=[[0, 3], [3, 3]], ya=[[0, 0], [0, 0]],
                yl=[[1, 1], [1, 1]], box=1.0, eps=1e-5, rs=rcut / 4.5, rcut=rcut, theta=theta,
                pm_mesh=0, leaf_size=leaf, pure_tree=1, ignore_nperp=ignore, beta=beta)


def test_coincident_bodies_are_one_exact_monopole():
    # 50 cored bodies at one place (one level-20 leaf) and a distant target
    n = 51
    pos = np.zeros((3, n))
    pos[:, 1:] = np.array([0.45, 0.45, 0.45])[:, None]
    pos[:, 0] = [0.2, 0.25, 0.3]
    typ = np.ones(n, np.uint8)
    mass = np.full(n, 1e-3, np.float32)
    beta = 2e-3
    for ignore, exact in ((0, True), (1, False)):
        prm = _mahalo_params(beta, theta=0.9, leaf=8, ignore=ignore)
        t, c = oracle.tree_walk(oracle_params(prm), pos, typ, mass, tgt=np.array([0]))
        d = oracle.direct(oracle_params(prm), pos, typ, mass, tgt=np.array([0]), cells=False)
        assert c[0] == 1                       # one monopole term
        e = np.linalg.norm(t - d) / np.linalg.norm(d)
        assert (e < 1e-13) if exact else (e > 1e-2), e


def test_nperp_tracking_accuracy():
    rng = inputs.rng_for(91)
    n = 12000
    pos = inputs.clustered(n, rng, nspheres=8, a=0.02)
    typ = inputs.species_uniform(n, 2, rng)
    mass = np.full(n, 1.0 / n, np.float32)
    beta = (1.0 / n) / (4 * math.pi * 0.004)      # single-body core 0.004 L
    tgt = np.sort(rng.choice(n, 1500, replace=False))
    err = {}
    for ignore in (0, 1):
        prm = _mahalo_params(beta, ignore=ignore)
        op = oracle_params(prm)
        t, _ = oracle.tree_walk(op, pos, typ, mass, tgt=tgt)
        d = oracle.direct(op, pos, typ, mass, tgt=tgt)
        err[ignore] = rel_err(t, d)[0]
    newt = dict(_mahalo_params(beta), law=[[0, 0], [0, 0]])
    t, _ = oracle.tree_walk(oracle_params(newt), pos, typ, mass, tgt=tgt)
    d = oracle.direct(oracle_params(newt), pos, typ, mass, tgt=tgt)
    e_newton = rel_err(t, d)[0]
    assert np.median(err[1]) > 5 * np.median(err[0]), (np.median(err[1]), np.median(err[0]))
    assert np.median(err[0]) < 2 * np.median(e_newton), (np.median(err[0]), np.median(e_newton))
