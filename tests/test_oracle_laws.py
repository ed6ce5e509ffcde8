"""Pins of the oracle's force laws (CPU only).

The oracle codes the short-range factors in closed form. These tests reach
the same quantity by another route: the paper's general-law construction of
Sec. 2.4.1, Eq. (short_pot)/(short_accel), where the long-range part is the
inverse Fourier transform of the Gaussian-filtered k-space potential and the
short-range part is what is left of the full law. The radial transforms are
done here by numerical quadrature (scipy), not by any formula of the oracle.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


def _long_accel(r, rs, phik_times_k):
    """Attractive long-range acceleration d(phi_long)/dr for a unit source.

    phi_long(r) = 1/(2 pi^2 r) int_0^inf k sin(kr) phi(k) e^{-k^2 rs^2} dk, with
    phik_times_k(k) = k phi(k) e^{-k^2 rs^2} (the filtered 3D transform times k).
    """
    kmax = 14.0 / rs
    I = integrate.quad(lambda k: math.sin(k * r) * phik_times_k(k), 0.0, kmax,
                       limit=800, epsabs=1e-14, epsrel=1e-12)[0]
    dI = integrate.quad(lambda k: k * math.cos(k * r) * phik_times_k(k), 0.0, kmax,
                        limit=800, epsabs=1e-14, epsrel=1e-12)[0]
    return -I / (2 * math.pi ** 2 * r * r) + dI / (2 * math.pi ** 2 * r)


def _newton_phik_k(rs):
    # phi(k) = -4 pi / k^2 for phi(r) = -1/r
    return lambda k: -4.0 * math.pi / k * math.exp(-k * k * rs * rs) if k > 0 else 0.0


def _yukawa_phik_k(rs, a, l):
    # phi(k) = -4 pi a / (k^2 + mu^2) for phi(r) = -a e^{-mu r}/r; the long-range
    # part carries the extra exp(-mu^2 rs^2) of Sec. 3.2
    mu = 1.0 / l
    return lambda k: (-4.0 * math.pi * a * k / (k * k + mu * mu)
                      * math.exp(-(k * k + mu * mu) * rs * rs))


@pytest.mark.parametrize("r_over_rs", [0.05, 0.3, 1.0, 2.0, 3.0, 4.4])
def test_newton_short_equals_full_minus_long(r_over_rs):
    rs = 0.01
    r = r_over_rs * rs
    full = 1.0 / r ** 2
    long_ = _long_accel(r, rs, _newton_phik_k(rs))
    short_quad = full - long_
    short_or = oracle.short_factor(oracle.NEWTON, 0.0, 1.0, rs, r) / r ** 2
    assert short_or == pytest.approx(short_quad, rel=2e-9, abs=1e-9 * full)


@pytest.mark.parametrize("a,l", [(0.3, 0.01), (-0.25, 0.05), (0.1, 0.003), (1.0, 0.02)])
@pytest.mark.parametrize("r_over_rs", [0.1, 0.7, 1.5, 3.0, 4.4])
def test_yukawa_short_equals_full_minus_long(a, l, r_over_rs):
    rs = 0.01
    r = r_over_rs * rs
    mu = 1.0 / l
    full_y = a * (1.0 + mu * r) * math.exp(-mu * r) / r ** 2
    long_y = _long_accel(r, rs, _yukawa_phik_k(rs, a, l))
    long_n = _long_accel(r, rs, _newton_phik_k(rs))
    short_quad = (1.0 / r ** 2 - long_n) + (full_y - long_y)
    short_or = oracle.short_factor(oracle.YUKAWA, a, l, rs, r) / r ** 2
    assert short_or == pytest.approx(short_quad, rel=2e-8, abs=1e-9 / r ** 2)


def test_full_factor_is_eq_yukawa_derivative():
    # F = G M m d/dr[(1 + a e^{-r/l})/r]: compare to a central difference of V
    a, l = 0.2, 0.04
    V = lambda r: -(1.0 + a * math.exp(-r / l)) / r
    for r in (0.005, 0.02, 0.1):
        h = r * 1e-5
        dV = (V(r + h) - V(r - h)) / (2 * h)
        assert oracle.full_factor(oracle.YUKAWA, a, l, r) / r ** 2 == pytest.approx(dV, rel=1e-8)
    assert oracle.full_factor(oracle.NEWTON, a, l, 0.3) == 1.0


def test_short_factor_limits():
    rs = 0.01
    # r -> 0: the long-range part is smooth, so the short part carries the whole law
    assert oracle.short_factor(oracle.NEWTON, 0, 1, rs, 1e-7) == pytest.approx(1.0, abs=1e-12)
    a, l = 0.3, 0.02
    assert oracle.short_factor(oracle.YUKAWA, a, l, rs, 1e-7) == pytest.approx(1.0 + a, abs=1e-9)
    # rs -> infinity: no long-range part at all, short part = full law
    for r in (0.01, 0.05):
        assert oracle.short_factor(oracle.YUKAWA, a, l, 1e6, r) == pytest.approx(
            oracle.full_factor(oracle.YUKAWA, a, l, r), rel=1e-6)
    # far beyond the split scale the short part vanishes
    assert abs(oracle.short_factor(oracle.YUKAWA, a, l, rs, 12 * rs)) < 1e-13


def test_newton_short_textbook_values():
    # erfc(u) + 2u/sqrt(pi) e^{-u^2} at u = 1/2, 1, 2 (Abramowitz & Stegun Table 7.1
    # gives erf(0.5) = 0.5204998778, erf(1) = 0.8427007929, erf(2) = 0.9953222650)
    rs = 0.5
    for u, erf in ((0.5, 0.5204998778), (1.0, 0.8427007929), (2.0, 0.9953222650)):
        want = (1 - erf) + 2 * u / math.sqrt(math.pi) * math.exp(-u * u)
        assert oracle.short_factor(oracle.NEWTON, 0, 1, rs, 2 * rs * u) == pytest.approx(want, abs=2e-10)


def test_long_kernel_is_filtered_greens_function():
    # the long-range kernel, transformed back with the radial quadrature above,
    # must give the same long-range force as the filtered potential
    rs, a, l = 0.01, 0.2, 0.03
    def phik_k(k):
        return -4 * math.pi * k * oracle.long_kernel(oracle.YUKAWA, a, l, rs, k * k) if k > 0 else 0.0
    ref_n, ref_y = _newton_phik_k(rs), _yukawa_phik_k(rs, a, l)
    for r in (0.5 * rs, 2 * rs, 5 * rs):
        got = _long_accel(r, rs, phik_k)
        want = _long_accel(r, rs, lambda k: ref_n(k) + ref_y(k))
        assert got == pytest.approx(want, rel=1e-10)
    assert oracle.long_kernel(oracle.YUKAWA, a, l, rs, 0.0) == 0.0


# --- the pure Yukawa law (C = 0 in Eq. (yukawa); Sec. 3.2 transition test)

@pytest.mark.parametrize("a,l", [(1.0, 0.1), (1.0, 0.02), (-0.5, 0.05)])
@pytest.mark.parametrize("r_over_rs", [0.1, 0.7, 1.5, 3.0, 4.4])
def test_pure_yukawa_short_equals_full_minus_long(a, l, r_over_rs):
    rs = 0.0195
    r = r_over_rs * rs
    mu = 1.0 / l
    full_y = a * (1.0 + mu * r) * math.exp(-mu * r) / r ** 2
    long_y = _long_accel(r, rs, _yukawa_phik_k(rs, a, l))
    short_or = oracle.short_factor(oracle.YUKAWA_PURE, a, l, rs, r) / r ** 2
    assert short_or == pytest.approx(full_y - long_y, rel=2e-8, abs=1e-9 * abs(full_y))


def test_pure_yukawa_limits_and_derivative():
    a, l, rs = 0.7, 0.05, 0.01
    # no Newtonian part: the full law is -d/dr of -a e^{-r/l}/r
    V = lambda r: -a * math.exp(-r / l) / r
    for r in (0.004, 0.02, 0.1):
        h = r * 1e-5
        dV = (V(r + h) - V(r - h)) / (2 * h)
        assert oracle.full_factor(oracle.YUKAWA_PURE, a, l, r) / r ** 2 == pytest.approx(dV, rel=1e-8)
    # r -> 0: the short part carries the whole law, whose factor tends to a
    assert oracle.short_factor(oracle.YUKAWA_PURE, a, l, rs, 1e-7) == pytest.approx(a, abs=1e-9)
    # rs -> infinity: no long-range part
    for r in (0.01, 0.05):
        assert oracle.short_factor(oracle.YUKAWA_PURE, a, l, 1e6, r) == pytest.approx(
            oracle.full_factor(oracle.YUKAWA_PURE, a, l, r), rel=1e-6)
    # Newtonian + pure Yukawa = the C = 1 law, term by term
    for r in (0.3 * rs, 2 * rs):
        assert (oracle.short_factor(oracle.NEWTON, 0, 1, rs, r)
                + oracle.short_factor(oracle.YUKAWA_PURE, a, l, rs, r)) == pytest.approx(
            oracle.short_factor(oracle.YUKAWA, a, l, rs, r), rel=1e-14)


def test_pure_yukawa_long_kernel_has_no_newtonian_part():
    rs, a, l = 0.01, 0.8, 0.03
    mu = 1.0 / l
    for k2 in (1.0, 400.0, 1e4):
        want = a * math.exp(-mu * mu * rs * rs) / (k2 + mu * mu) * math.exp(-k2 * rs * rs)
        assert oracle.long_kernel(oracle.YUKAWA_PURE, a, l, rs, k2) == pytest.approx(want, rel=1e-14)
    def phik_k(k):
        return -4 * math.pi * k * oracle.long_kernel(oracle.YUKAWA_PURE, a, l, rs, k * k) if k > 0 else 0.0
    ref = _yukawa_phik_k(rs, a, l)
    for r in (0.5 * rs, 2 * rs, 5 * rs):
        assert _long_accel(r, rs, phik_k) == pytest.approx(_long_accel(r, rs, ref), rel=1e-10)
