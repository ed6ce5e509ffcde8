"""Pins of the oracle's TreePM split in the transition region (Sec. 3.2).

A massive source and test particles in shells of 1/r^3 density (intra-type
forces off, only test <- source on): the oracle's TreePM force (FP64 direct
short-range sum + FP64 PM) against the exact periodic force of the same law,
computed without the split: a textbook Ewald sum for the Newtonian law (the
Coulomb case) and a plain image sum for the pure Yukawa law (exponentially
convergent). Sec. 3.2 reports the rms error flat through the transition and
essentially the Coulomb one for the pure Yukawa interaction once the Yukawa
Green's function carries exp(-mu^2 r_s^2); without that factor the long-range
part is too large by exp(mu^2 r_s^2) (2.6x at y_m = 50 on a 64^3 mesh).

Bounds (binned rms of |dF|/|F|, bins logarithmic in r):
* r < r_s / 2, where the short-range part carries all but a tiny fraction of
  the force: <= 1e-3;
* every bin up to r = 0.05 L (past r_s, into the cut-off at 4.5 r_s = 0.088 L):
  <= 2e-2, the CIC + 4-point-gradient PM accuracy at 1.25 cells of
  smoothing; for the Newtonian and y_m = 10 laws every bin up to L/2;
* y_m = 10: largest transition-bin rms <= 1.5x the Coulomb one.
"""
import numpy as np
import pytest

import ewald
import oracle
from common import binned_rms, oracle_params, transition_case, transition_exact

MESH = 64
RS = 1.25 / MESH
EDGES = np.exp(np.linspace(np.log(0.1 * RS), np.log(0.5), 13))


def _stacked_errors(law, ym, seeds=(7, 8)):
    e_all, r_all = [], []
    for seed in seeds:
        w, d, r = transition_case(seed, 2000, MESH, law, ym)
        f = oracle.force(oracle_params(w["params"]), w["pos"], w["type"], w["mass"])[:, 1:].T
        ex = transition_exact(law, ym, d)
        e_all.append(np.linalg.norm(f - ex, axis=1) / np.linalg.norm(ex, axis=1))
        r_all.append(r)
    return np.concatenate(r_all), np.concatenate(e_all)


def test_yukawa_image_sum_is_converged_and_tends_to_the_pair_law():
    x = np.array([0.13, -0.07, 0.21])
    for l in (0.1, 0.02):
        a3 = ewald.yukawa_images(x, 1.0, l, nmax=3)
        a4 = ewald.yukawa_images(x, 1.0, l, nmax=4)
        assert np.allclose(a3, a4, rtol=1e-13, atol=0)
    # close to the source the nearest image is the whole force
    x = np.array([1e-3, 2e-3, -1e-3])
    r = np.linalg.norm(x)
    mu = 50.0
    pair = -(1 + mu * r) * np.exp(-mu * r) / r ** 2 * x / r
    assert np.allclose(ewald.yukawa_images(x, 1.0, 1 / mu, nmax=3), pair, rtol=1e-12)


@pytest.fixture(scope="module")
def errors():
    return {key: _stacked_errors(*key) for key in ((0, 10.0), (2, 10.0), (2, 50.0))}


@pytest.mark.parametrize("key", [(0, 10.0), (2, 10.0), (2, 50.0)],
                         ids=["coulomb", "yukawa_ym10", "yukawa_ym50"])
def test_transition_error_is_flat(errors, key):
    r, e = errors[key]
    rms = binned_rms(r, e, EDGES)
    lo = EDGES[1:] <= 0.5 * RS
    assert np.all(rms[lo] <= 1e-3), rms[lo]
    mid = EDGES[:-1] < 0.05
    assert np.all(rms[mid] <= 2e-2), rms[mid]
    if key[1] == 10.0:
        assert np.all(rms <= 2e-2), rms


def test_pure_yukawa_transition_matches_coulomb(errors):
    r0, e0 = errors[(0, 10.0)]
    r1, e1 = errors[(2, 10.0)]
    band = (EDGES[:-1] >= 0.5 * RS) & (EDGES[1:] <= 4.5 * RS)
    c = binned_rms(r0, e0, EDGES)[band]
    y = binned_rms(r1, e1, EDGES)[band]
    assert y.max() <= 1.5 * c.max(), (y, c)
