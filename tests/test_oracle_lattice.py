"""Pins of the oracle's lattice corrections (Sec. 2.3, pure tree mode 2).

* The Newtonian correction (all images but the nearest, per unit G M)
  against an Ewald sum written here with another splitting parameter
  (alpha = 3 instead of 2: an Ewald sum does not depend on it), and two
  closed forms: zero at the origin, and -4/L^2 along x at (L/2, 0, 0), where
  the periodic force vanishes by symmetry and only the nearest image's
  -1/(L/2)^2 is left to cancel. Each component is odd in its own axis and
  even in the others.
* The Yukawa correction against the test-side image sum.
* The tabulated and interpolated pair force against the exact periodic
  force (nearest image + exact correction) at random separations.
* The stated use of the corrections: a consistency check of the Fourier
  (PM) computation. Pure tree mode 2 and TreePM give the same periodic force
  to the TreePM accuracy, for Newtonian and Yukawa laws.
* Tree at theta = 0 equals the direct sum; theta = 0.5 is sane.
"""
import math

import numpy as np
import pytest
from scipy.special import erfc

import ewald
import oracle
from common import oracle_params, small_clustered
from metrics import rel_err


def _ewald_alpha3(d):
    """Periodic acceleration toward a unit source and its images at offset
    d = source - target (L = 1), Ewald splitting alpha = 3."""
    al = 3.0
    g = np.arange(-3, 4)
    n = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(float)
    v = d[None, :] + n
    r = np.linalg.norm(v, axis=1)
    f = (erfc(al * r) + 2 * al * r / math.sqrt(math.pi) * np.exp(-al * al * r * r)) / r ** 3
    real = (f[:, None] * v).sum(0)
    g = np.arange(-10, 11)
    m = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(float)
    m = m[np.any(m != 0, axis=1)]
    k = 2 * math.pi * m
    k2 = (k * k).sum(1)
    w = 4 * math.pi / k2 * np.exp(-k2 / (4 * al * al)) * np.sin(k @ d)
    return real + (w[:, None] * k).sum(0)


def test_newton_correction_against_independent_ewald():
    rng = np.random.Generator(np.random.PCG64(11))
    for _ in range(20):
        d = rng.uniform(-0.5, 0.5, 3)
        got = oracle.lattice_correction(oracle.NEWTON, 0, 0, d)
        want = _ewald_alpha3(d) - d / np.linalg.norm(d) ** 3
        assert np.allclose(got, want, rtol=0, atol=1e-11), (got, want)
    assert np.allclose(oracle.lattice_correction(oracle.NEWTON, 0, 0, [0.5, 0, 0]), [-4, 0, 0],
                       atol=1e-12)
    assert np.allclose(oracle.lattice_correction(oracle.NEWTON, 0, 0, [0, 0, 0]), 0, atol=1e-12)
    d = np.array([0.13, -0.21, 0.34])
    c = oracle.lattice_correction(oracle.NEWTON, 0, 0, d)
    for axis in range(3):
        f = d.copy()
        f[axis] = -f[axis]
        cf = oracle.lattice_correction(oracle.NEWTON, 0, 0, f)
        sign = np.where(np.arange(3) == axis, -1.0, 1.0)
        assert np.allclose(cf, sign * c, atol=1e-13)


@pytest.mark.parametrize("law", [oracle.YUKAWA, oracle.YUKAWA_PURE])
def test_yukawa_correction_against_image_sum(law):
    rng = np.random.Generator(np.random.PCG64(12))
    a, l = 0.6, 0.08
    for _ in range(10):
        d = rng.uniform(-0.5, 0.5, 3)
        r = np.linalg.norm(d)
        near = a * (1 + r / l) * math.exp(-r / l) * d / r ** 3
        y = ewald.yukawa_images(-d, a, l, nmax=4)      # on the target, toward the source
        want = y - near
        if law == oracle.YUKAWA:
            want = want + oracle.lattice_correction(oracle.NEWTON, 0, 0, d)
        got = oracle.lattice_correction(law, a, l, d)
        assert np.allclose(got, want, rtol=1e-10, atol=1e-12)


def test_interpolated_pair_force():
    rng = np.random.Generator(np.random.PCG64(13))
    prm = dict(D=1, G=[[1.0]], law=[[0]], ya=[[0.0]], yl=[[1.0]], box=1.0, eps=1e-7, rs=0.05,
               rcut=0.2, theta=0.0, pm_mesh=0, leaf_size=8, pure_tree=2)
    errs = []
    for _ in range(200):
        pos = rng.random((3, 2))
        d = pos[:, 1] - pos[:, 0]
        d -= np.rint(d)
        got = oracle.direct(oracle_params(prm), pos, np.zeros(2, np.uint8),
                            np.array([0.0, 1.0], np.float32), tgt=np.array([0]), cells=False)[:, 0]
        want = ewald.accel(-d)                          # on the target, toward the source
        # in units of the nearest image's force (the periodic force itself
        # vanishes at the centres of the faces and at the corners of the cube)
        errs.append(np.linalg.norm(got - want) * (d @ d))
    # trilinear interpolation on a 64^3 grid over [0, L/2]^3: error ~ h^2 C''/8
    assert max(errs) <= 1e-4, max(errs)


@pytest.mark.parametrize("yukawa", [False, True], ids=["newton", "yukawa"])
def test_consistent_with_treepm(yukawa):
    w = small_clustered(4000, 2, 34 if yukawa else 33, mesh=64, yukawa=yukawa)
    prm = dict(w["params"], eps=1e-4)
    treepm = oracle.force(oracle_params(prm), w["pos"], w["type"], w["mass"])
    lattice = oracle.direct(oracle_params(dict(prm, pure_tree=2, pm_mesh=0, theta=0.0)),
                            w["pos"], w["type"], w["mass"])
    e, _ = rel_err(treepm, lattice)
    assert np.median(e) <= 5e-3 and np.percentile(e, 99) <= 3e-2, (np.median(e), np.percentile(e, 99))


def test_tree_in_lattice_mode():
    w = small_clustered(3000, 2, 35, mesh=64)
    prm = dict(w["params"], eps=1e-4, pure_tree=2, pm_mesh=0)
    direct = oracle.direct(oracle_params(dict(prm, theta=0.0)), w["pos"], w["type"], w["mass"])
    t0, _ = oracle.tree_walk(oracle_params(dict(prm, theta=0.0)), w["pos"], w["type"], w["mass"])
    assert rel_err(t0, direct)[0].max() < 1e-11
    t5, _ = oracle.tree_walk(oracle_params(dict(prm, theta=0.5)), w["pos"], w["type"], w["mass"])
    e, _ = rel_err(t5, direct)
    assert np.median(e) < 1e-2, np.median(e)
