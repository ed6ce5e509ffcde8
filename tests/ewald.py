"""Textbook Ewald sums for a periodic unit box (test-side reference).

psi(r) = sum_n erfc(alpha|r_n|)/|r_n| + 4 pi sum_{k != 0} e^{-k^2/4 alpha^2} cos(k.r)/k^2
         - pi / alpha^2,   r_n = r - n (box side 1, neutralising background).
The gravitational acceleration toward a unit mass at the origin is grad psi.
Checked against the published lattice constant in tests/golden/."""
import math

import numpy as np
from scipy.special import erfc

ALPHA = 2.0
NR = 4
NK = 8


def _lattice(nmax):
    g = np.arange(-nmax, nmax + 1)
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)


_N = _lattice(NR)
_K = _lattice(NK)
_K = _K[np.any(_K != 0, axis=1)] * 2 * math.pi
_K2 = (_K ** 2).sum(1)
_KW = np.exp(-_K2 / (4 * ALPHA ** 2)) / _K2


def lattice_constant():
    n = _N[np.any(_N != 0, axis=1)]
    r = np.linalg.norm(n, axis=1)
    return (erfc(ALPHA * r) / r).sum() + 4 * math.pi * _KW.sum() - math.pi / ALPHA ** 2 \
        - 2 * ALPHA / math.sqrt(math.pi)


def accel(r):
    """Periodic Newtonian acceleration at offset r (3,) from a unit mass, G = 1."""
    rn = np.asarray(r, np.float64)[None, :] - _N
    d = np.linalg.norm(rn, axis=1)
    f = -(erfc(ALPHA * d) / d ** 2 + 2 * ALPHA / math.sqrt(math.pi) * np.exp(-ALPHA ** 2 * d ** 2) / d)
    real = (f[:, None] * rn / d[:, None]).sum(0)
    ks = -4 * math.pi * (_KW[:, None] * _K * np.sin(_K @ np.asarray(r, np.float64))[:, None]).sum(0)
    return real + ks


def yukawa_images(r, a, l, nmax=2):
    """Periodic sum of the Yukawa part a (1 + r/l) e^{-r/l} / r^2 (attractive)."""
    rn = np.asarray(r, np.float64)[None, :] - _lattice(nmax)
    d = np.linalg.norm(rn, axis=1)
    f = -a * (1 + d / l) * np.exp(-d / l) / d ** 2
    return (f[:, None] * rn / d[:, None]).sum(0)
