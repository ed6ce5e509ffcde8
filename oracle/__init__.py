"""FP64 CPU oracle for the multi-species TreePM force (arXiv:1502.07442).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product library
(``paper_1502_07442_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``ngravs_oracle.cpp`` (plain double precision, each
routine citing the paper passage it follows); this module only compiles it
with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ngravs_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NEWTON = 0
YUKAWA = 1
YUKAWA_PURE = 2
MAHALO = 3


class OrParams(ctypes.Structure):
    """Mirror of ``or_params`` in ngravs_oracle.cpp."""

    _fields_ = [
        ("D", ctypes.c_int32),
        ("leaf_size", ctypes.c_int32),
        ("pm_mesh", ctypes.c_int32),
        ("pad0", ctypes.c_int32),
        ("box", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("rs", ctypes.c_double),
        ("rcut", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("G", (ctypes.c_double * 6) * 6),
        ("law", (ctypes.c_int32 * 6) * 6),
        ("ya", (ctypes.c_double * 6) * 6),
        ("yl", (ctypes.c_double * 6) * 6),
        ("opening", ctypes.c_int32),
        ("pad1", ctypes.c_int32),
        ("alpha", ctypes.c_double),
        ("pure_tree", ctypes.c_int32),
        ("ignore_nperp", ctypes.c_int32),
        ("beta", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (FP64, OpenMP, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-o", tmp, _SRC]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        d, i64, vp = ctypes.c_double, ctypes.c_int64, ctypes.c_void_p
        P = ctypes.POINTER(OrParams)
        L.or_short_factor.argtypes = [ctypes.c_int, d, d, d, d]
        L.or_short_factor.restype = d
        L.or_full_factor.argtypes = [ctypes.c_int, d, d, d]
        L.or_full_factor.restype = d
        L.or_long_kernel.argtypes = [ctypes.c_int, d, d, d, d]
        L.or_long_kernel.restype = d
        L.or_mahalo_factor.argtypes = [d, d, d]
        L.or_mahalo_factor.restype = d
        L.or_lattice_correction.argtypes = [ctypes.c_int, d, d, ctypes.c_void_p, ctypes.c_void_p]
        L.or_lattice_correction.restype = None
        L.or_keys.argtypes = [i64, vp, vp, d, vp]
        L.or_sort_perm.argtypes = [i64, vp, vp]
        L.or_tree.argtypes = [P, i64, vp, vp, vp, i64] + [vp] * 9
        L.or_tree.restype = i64
        for f in ("or_direct", "or_direct_cells"):
            getattr(L, f).argtypes = [P, i64, vp, vp, vp, i64, vp, vp]
        L.or_direct_mag.argtypes = [P, i64, vp, vp, vp, i64, vp, vp, vp]
        L.or_tree_walk.argtypes = [P, i64, vp, vp, vp, i64, vp, vp, vp]
        L.or_tree_walk_timed.argtypes = [P, i64, vp, vp, vp, i64, vp, vp, vp, vp]
        L.or_tree_walk_aold.argtypes = [P, i64, vp, vp, vp, vp, i64, vp, vp, vp]
        L.or_fft1d.argtypes = [i64, vp, vp, ctypes.c_int]
        L.or_fft3d.argtypes = [i64, vp, vp, ctypes.c_int]
        L.or_pm.argtypes = [P, i64, vp, vp, vp, vp]
        L.or_force.argtypes = [P, i64, vp, vp, vp, vp]
        L.or_kdk.argtypes = [P, i64, vp, vp, vp, vp, ctypes.c_int, d, vp]
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_set_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int = 0) -> int:
    """Set (n > 0) and return the OpenMP thread count the oracle uses."""
    return lib().or_set_threads(int(n))


def make_params(D, G, *, box=1.0, eps, rs, rcut, theta=0.5, leaf_size=8, pm_mesh=0,
                law=None, ya=None, yl=None, opening=0, alpha=0.005, pure_tree=0,
                ignore_nperp=0, beta=0.0) -> OrParams:
    """Build the oracle's parameter block from plain numbers / nested lists.
    opening 0: geometric criterion (theta); 1: relative criterion (alpha, with
    the previous acceleration magnitudes given to tree_walk)."""
    p = OrParams()
    p.opening, p.alpha = int(opening), float(alpha)
    p.pure_tree, p.ignore_nperp, p.beta = int(pure_tree), int(ignore_nperp), float(beta)
    p.D, p.leaf_size, p.pm_mesh = int(D), int(leaf_size), int(pm_mesh)
    p.box, p.eps, p.rs, p.rcut, p.theta = float(box), float(eps), float(rs), float(rcut), float(theta)
    G = np.asarray(G, dtype=np.float64)
    law = np.zeros((D, D), np.int32) if law is None else np.asarray(law, np.int32)
    ya = np.zeros((D, D)) if ya is None else np.asarray(ya, np.float64)
    yl = np.ones((D, D)) if yl is None else np.asarray(yl, np.float64)
    for i in range(D):
        for j in range(D):
            p.G[i][j] = G[i, j]
            p.law[i][j] = int(law[i, j])
            p.ya[i][j] = ya[i, j]
            p.yl[i][j] = yl[i, j]
    return p


def _soa(pos):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    assert pos.ndim == 2 and pos.shape[0] == 3
    return pos


def short_factor(law, a, l, rs, rho):
    return lib().or_short_factor(int(law), float(a), float(l), float(rs), float(rho))


def lattice_correction(law, a, l_box, d):
    """Lattice correction (all images but the nearest) of law (kind, a, l) at
    offset d (source - target, box units, L = 1) per unit G M."""
    dd = np.ascontiguousarray(d, np.float64)
    out = np.zeros(3)
    lib().or_lattice_correction(int(law), float(a), float(l_box), _p(dd), _p(out))
    return out


def mahalo_factor(beta, scale, r):
    """|F| r^2 / (G M m) of the Sec. 3.3 law with core scale `scale`."""
    return lib().or_mahalo_factor(float(beta), float(scale), float(r))


def full_factor(law, a, l, r):
    return lib().or_full_factor(int(law), float(a), float(l), float(r))


def long_kernel(law, a, l, rs, k2):
    return lib().or_long_kernel(int(law), float(a), float(l), float(rs), float(k2))


def keys(pos, typ, box=1.0):
    pos = _soa(pos)
    typ = np.ascontiguousarray(typ, np.uint8)
    n = pos.shape[1]
    out = np.zeros(n, np.uint64)
    lib().or_keys(n, _p(pos), _p(typ), float(box), _p(out))
    return out


def sort_perm(k):
    k = np.ascontiguousarray(k, np.uint64)
    out = np.zeros(k.size, np.uint32)
    lib().or_sort_perm(k.size, _p(k), _p(out))
    return out


def tree(p: OrParams, pos, typ, mass):
    """Canonical octree; returns a dict of per-node arrays in canonical order."""
    pos = _soa(pos)
    typ = np.ascontiguousarray(typ, np.uint8)
    mass = np.ascontiguousarray(mass, np.float32)
    n = pos.shape[1]
    L = lib()
    nn = L.or_tree(ctypes.byref(p), n, _p(pos), _p(typ), _p(mass), 0, *([None] * 9))
    D = p.D
    out = dict(level=np.zeros(nn, np.int32), prefix=np.zeros(nn, np.uint64),
               first=np.zeros(nn, np.int64), count=np.zeros(nn, np.int64),
               child_first=np.zeros(nn, np.int64), nchild=np.zeros(nn, np.int32),
               cnt=np.zeros((nn, D), np.uint32), mass=np.zeros((nn, D)),
               com=np.zeros((nn, D, 3)))
    L.or_tree(ctypes.byref(p), n, _p(pos), _p(typ), _p(mass), nn,
              *[_p(out[k]) for k in ("level", "prefix", "first", "count", "child_first",
                                      "nchild", "cnt", "mass", "com")])
    return out


def _targets(n, tgt):
    return np.arange(n, dtype=np.int64) if tgt is None else np.ascontiguousarray(tgt, np.int64)


def direct(p: OrParams, pos, typ, mass, tgt=None, cells=True):
    """Short-range direct sum; returns acc [3][len(tgt)] in float64."""
    pos = _soa(pos)
    typ = np.ascontiguousarray(typ, np.uint8)
    mass = np.ascontiguousarray(mass, np.float32)
    n = pos.shape[1]
    t = _targets(n, tgt)
    acc = np.zeros((3, t.size))
    f = lib().or_direct_cells if cells else lib().or_direct
    f(ctypes.byref(p), n, _p(pos), _p(typ), _p(mass), t.size, _p(t), _p(acc))
    return acc


def direct_mag(p: OrParams, pos, typ, mass, tgt=None):
    """Brute-force direct sum and, per target, the sum of the term magnitudes."""
    pos = _soa(pos)
    typ = np.ascontiguousarray(typ, np.uint8)
    mass = np.ascontiguousarray(mass, np.float32)
    n = pos.shape[1]
    t = _targets(n, tgt)
    acc = np.zeros((3, t.size))
    mag = np.zeros(t.size)
    lib().or_direct_mag(ctypes.byref(p), n, _p(pos), _p(typ), _p(mass), t.size, _p(t), _p(acc),
                        _p(mag))
    return acc, mag


def tree_walk(p: OrParams, pos, typ, mass, tgt=None, aold=None):
    """Per-particle tree walk; returns (acc [3][len(tgt)], counts [len(tgt)]).
    aold (float32 [n], original order): previous acceleration magnitudes for
    the relative criterion (p.opening == 1); without it the walk is geometric."""
    pos = _soa(pos)
    typ = np.ascontiguousarray(typ, np.uint8)
    mass = np.ascontiguousarray(mass, np.float32)
    n = pos.shape[1]
    t = _targets(n, tgt)
    acc = np.zeros((3, t.size))
    cnt = np.zeros(t.size, np.int64)
    if aold is None:
        lib().or_tree_walk(ctypes.byref(p), n, _p(pos), _p(typ), _p(mass), t.size, _p(t),
                           _p(acc), _p(cnt))
    else:
        a = np.ascontiguousarray(aold, np.float32)
        assert a.shape == (n,)
        lib().or_tree_walk_aold(ctypes.byref(p), n, _p(pos), _p(typ), _p(mass), _p(a), t.size,
                                _p(t), _p(acc), _p(cnt))
    return acc, cnt


def tree_walk_timed(p: OrParams, pos, typ, mass, tgt):
    """Per-particle walk of the targets; returns (acc, counts, build_s, walk_s)."""
    pos = _soa(pos)
    typ = np.ascontiguousarray(typ, np.uint8)
    mass = np.ascontiguousarray(mass, np.float32)
    n = pos.shape[1]
    t = _targets(n, tgt)
    acc = np.zeros((3, t.size))
    cnt = np.zeros(t.size, np.int64)
    times = np.zeros(2)
    lib().or_tree_walk_timed(ctypes.byref(p), n, _p(pos), _p(typ), _p(mass), t.size, _p(t),
                             _p(acc), _p(cnt), _p(times))
    return acc, cnt, float(times[0]), float(times[1])


def fft1d(x, sign=-1):
    x = np.asarray(x, np.complex128)
    re = np.ascontiguousarray(x.real)
    im = np.ascontiguousarray(x.imag)
    lib().or_fft1d(x.size, _p(re), _p(im), int(sign))
    return re + 1j * im


def fft3d(x, sign=-1):
    x = np.asarray(x, np.complex128)
    N = x.shape[0]
    re = np.ascontiguousarray(x.real).copy()
    im = np.ascontiguousarray(x.imag).copy()
    lib().or_fft3d(N, _p(re), _p(im), int(sign))
    return re + 1j * im


def pm(p: OrParams, pos, typ, mass):
    pos = _soa(pos)
    typ = np.ascontiguousarray(typ, np.uint8)
    mass = np.ascontiguousarray(mass, np.float32)
    n = pos.shape[1]
    acc = np.zeros((3, n))
    lib().or_pm(ctypes.byref(p), n, _p(pos), _p(typ), _p(mass), _p(acc))
    return acc


def force(p: OrParams, pos, typ, mass):
    pos = _soa(pos)
    typ = np.ascontiguousarray(typ, np.uint8)
    mass = np.ascontiguousarray(mass, np.float32)
    n = pos.shape[1]
    acc = np.zeros((3, n))
    lib().or_force(ctypes.byref(p), n, _p(pos), _p(typ), _p(mass), _p(acc))
    return acc


def law_amax(p: OrParams, box=None):
    """A_max of Sec. 2.1.1 (the constant of Eq. (our_timestep)): the largest
    G_ij |f_ij(r)| r^2 / M over the species pairs, the supremum over r taken
    on a dense logarithmic grid of the full (unsplit) law from 1e-9 L to
    1e3 L (the laws are defined for every separation)."""
    L = p.box if box is None else box
    r = np.geomspace(1e-9 * L, 1e3 * L, 200001)
    A = 0.0
    for i in range(p.D):
        for j in range(p.D):
            f = np.array([abs(full_factor(p.law[i][j], p.ya[i][j], p.yl[i][j], x)) for x in r[::100]])
            k = int(np.argmax(f))
            lo, hi = max(0, 100 * k - 100), min(r.size, 100 * k + 101)
            fine = max(abs(full_factor(p.law[i][j], p.ya[i][j], p.yl[i][j], x)) for x in r[lo:hi])
            A = max(A, abs(p.G[i][j]) * max(f.max(), fine))
    return A


def timestep(p: OrParams, acc, eta, dt_max):
    """Synchronous step: the smallest per-particle step of Eq. (our_timestep),
    dt_i = min(dt_max, sqrt(2 eta eps / (A_max |a_i|))), with |a_i| formed in
    float32 as sqrt((x x + y y) + z z). Returns (dt, max |a|)."""
    a = np.ascontiguousarray(acc, np.float32)
    mag = np.sqrt((a[0] * a[0] + a[1] * a[1]) + a[2] * a[2]).astype(np.float32)
    A = law_amax(p)
    steps = [dt_max]
    for m in mag:
        if m > 0 and A > 0:
            steps.append(min(dt_max, math.sqrt(2.0 * eta * p.eps / (A * float(m)))))
    return min(steps), float(mag.max())


def kdk(p: OrParams, pos, vel, typ, mass, nsteps, dt):
    """Returns (pos, vel, acc) after nsteps kick-drift-kick steps."""
    pos = _soa(pos).copy()
    vel = np.ascontiguousarray(vel, np.float64).copy()
    typ = np.ascontiguousarray(typ, np.uint8)
    mass = np.ascontiguousarray(mass, np.float32)
    n = pos.shape[1]
    acc = np.zeros((3, n))
    lib().or_kdk(ctypes.byref(p), n, _p(pos), _p(vel), _p(typ), _p(mass), int(nsteps),
                 float(dt), _p(acc))
    return pos, vel, acc
