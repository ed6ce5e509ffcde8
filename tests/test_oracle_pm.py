"""Pins of the oracle's PM long-range step (Sec. 2.4) and of the full TreePM
force. References: numpy's FFT, exact zero force of a uniform lattice, exact
momentum conservation of symmetric CIC + even Green's function, and the
textbook Ewald sum (itself pinned to the published lattice constant)."""
import math
import os

import numpy as np
import pytest

import ewald
import oracle
from paper_1502_07442_gb300 import inputs
from metrics import rel_err

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_test_side_ewald_matches_published_lattice_constant():
    assert ewald.lattice_constant() == pytest.approx(_golden("ewald_sc_lattice.txt")["xi"], abs=1e-8)


def test_fft_matches_numpy():
    rng = inputs.rng_for(21)
    x = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    np.testing.assert_allclose(oracle.fft1d(x, -1), np.fft.fft(x), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.fft1d(x, +1), np.fft.ifft(x) * 64, rtol=1e-12, atol=1e-12)
    m = rng.standard_normal((8, 8, 8))
    np.testing.assert_allclose(oracle.fft3d(m, -1), np.fft.fftn(m), rtol=1e-12, atol=1e-11)
    # Parseval
    F = oracle.fft3d(m, -1)
    assert (np.abs(F) ** 2).sum() / 512 == pytest.approx((m ** 2).sum(), rel=1e-12)


def _pm_params(D=1, G=None, mesh=16, law=None, ya=None, yl=None):
    rs = 1.25 / mesh
    G = np.ones((D, D)) if G is None else G
    return oracle.make_params(D, G, eps=0.0, rs=rs, rcut=4.5 * rs, theta=0.0, pm_mesh=mesh,
                              law=law, ya=ya, yl=yl)


def test_uniform_lattice_feels_no_force():
    mesh = 8
    g = (np.arange(mesh) + 0.0) / mesh
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), 0).reshape(3, -1)
    n = pos.shape[1]
    a = oracle.pm(_pm_params(mesh=mesh), pos, np.zeros(n, np.uint8), np.ones(n, np.float32))
    assert np.abs(a).max() < 1e-10


def test_pm_momentum_conservation():
    rng = inputs.rng_for(22)
    n, D = 300, 3
    pos = inputs.clustered(n, rng, nspheres=3, a=0.05)
    typ = inputs.species_uniform(n, D, rng)
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    c = inputs.yukawa_couplings(D, rng)
    p = _pm_params(D, c["G"], law=c["law"], ya=c["ya"], yl=c["yl"])
    a = oracle.pm(p, pos, typ, mass)
    m = mass.astype(np.float64)
    assert np.abs((a * m).sum(1)).max() <= 1e-11 * (np.abs(a) * m).sum()


def _two_body_errors(law=0, a=0.0, l=1.0, mesh=32, samples=40, seed=23):
    rng = inputs.rng_for(seed)
    p = _pm_params(1, mesh=mesh, law=[[law]], ya=[[a]], yl=[[l]])
    h = 1.0 / mesh
    errs, rr = [], []
    for s in range(samples):
        x1 = rng.random(3)
        dirn = rng.standard_normal(3)
        dirn /= np.linalg.norm(dirn)
        r = h * 10 ** rng.uniform(math.log10(0.3), math.log10(0.45 / h))
        x2 = np.mod(x1 + r * dirn, 1.0)
        pos = np.stack([x1, x2], 1)
        # a light test particle and a heavy source (Sec. 3.1 transition test)
        mass = np.array([1e-6, 1.0], np.float32)
        acc = oracle.force(p, pos, np.zeros(2, np.uint8), mass)[:, 0]
        want = ewald.accel(x1 - x2 - np.rint(x1 - x2))
        if law:
            want = want + ewald.yukawa_images(x1 - x2 - np.rint(x1 - x2), a, l)
        errs.append(np.linalg.norm(acc - want) / np.linalg.norm(want))
        rr.append(r)
    return np.array(errs), np.array(rr)


def test_treepm_two_body_matches_ewald():
    # the full short (direct) + long (PM) force against the textbook periodic
    # sum: a wrong sign, factor or missing window would be O(1) off
    err, r = _two_body_errors()
    assert np.sqrt(np.mean(err ** 2)) < 1e-2
    assert err.max() < 3e-2


def test_treepm_two_body_yukawa_matches_image_sum():
    err, r = _two_body_errors(law=1, a=0.3, l=0.05, seed=24)
    assert np.sqrt(np.mean(err ** 2)) < 1e-2
    assert err.max() < 3e-2


def test_species_reduction_in_pm():
    rng = inputs.rng_for(25)
    n = 200
    pos = inputs.uniform(n, rng)
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    a1 = oracle.pm(_pm_params(1, np.full((1, 1), 0.7)), pos, np.zeros(n, np.uint8), mass)
    typ = inputs.species_uniform(n, 4, rng)
    a4 = oracle.pm(_pm_params(4, np.full((4, 4), 0.7)), pos, typ, mass)
    np.testing.assert_allclose(a4, a1, rtol=1e-10, atol=1e-10 * np.abs(a1).max())
