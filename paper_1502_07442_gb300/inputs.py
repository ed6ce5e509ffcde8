"""Seeded synthetic inputs for the multi-species TreePM force.

This module only draws random numbers (numpy's PCG64, identical on every
platform) and assembles plain parameter dictionaries. It holds none of the
method's arithmetic, so both the CUDA path and the FP64 oracle can be fed from
it.

The paper's own initial conditions (GADGET-2's packaged galaxy collision,
LambdaCDM and gas sphere files, Appendix A) are not available; the
generators below stand in for them with the shapes of the workloads the
library is measured on:

* ``uniform``: positions uniform in the periodic box.
* ``clustered``: a mixture of Plummer spheres (scale radius ``a``, centres
  uniform) holding ``1 - frac_uniform`` of the particles, plus a uniform
  background; radii follow r = a (u^(-2/3) - 1)^(-1/2), untruncated, then
  wrapped into the box.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["uniform", "clustered", "species_blocks", "species_uniform",
           "newton_couplings", "yukawa_couplings", "workload", "WORKLOADS"]


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform(n: int, rng: np.random.Generator, box: float = 1.0) -> np.ndarray:
    """Positions [3][n] uniform in [0, box)^3."""
    return rng.random((3, n)) * box


def clustered(n: int, rng: np.random.Generator, nspheres: int = 512, a: float = 0.005,
              frac_uniform: float = 0.3, box: float = 1.0) -> np.ndarray:
    """Positions [3][n]: Plummer spheres plus a uniform background, wrapped."""
    nu = int(round(frac_uniform * n))
    nc = n - nu
    pos = np.empty((3, n))
    pos[:, :nu] = rng.random((3, nu)) * box
    centres = rng.random((3, nspheres)) * box
    which = rng.integers(0, nspheres, nc)
    u = rng.random(nc)
    u = np.clip(u, 1e-12, 1.0 - 1e-12)
    r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    v = rng.standard_normal((3, nc))
    v /= np.linalg.norm(v, axis=0, keepdims=True)
    pos[:, nu:] = np.mod(centres[:, which] + r * v, box)
    # shuffle so that background and cluster bodies interleave in input order
    perm = rng.permutation(n)
    return np.ascontiguousarray(pos[:, perm])


def source_shells(ntest: int, rng: np.random.Generator, rmin: float, rmax: float,
                  box: float = 1.0) -> np.ndarray:
    """One source at a uniform random place followed by ntest test positions
    at separations log-uniform in [rmin, rmax] (number density falling as
    1/r^3, so every logarithmic shell holds about as many) in isotropic
    directions, wrapped into the box. Returns [3][ntest + 1]."""
    src = rng.random(3) * box
    r = np.exp(rng.uniform(np.log(rmin), np.log(rmax), ntest))
    v = rng.standard_normal((ntest, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    pos = np.mod(src[None, :] + r[:, None] * v, box)
    return np.ascontiguousarray(np.concatenate([src[None, :], pos]).T)


def species_blocks(n: int, D: int, rng: np.random.Generator) -> np.ndarray:
    """Species labels with n/D bodies of each species, in random order."""
    t = np.repeat(np.arange(D, dtype=np.uint8), -(-n // D))[:n]
    return rng.permutation(t).astype(np.uint8)


def species_uniform(n: int, D: int, rng: np.random.Generator) -> np.ndarray:
    """Species labels drawn uniformly per body."""
    return rng.integers(0, D, n).astype(np.uint8)


def _sym(rng, D, lo, hi):
    m = rng.uniform(lo, hi, (D, D))
    return np.triu(m) + np.triu(m, 1).T


def newton_couplings(D: int, rng: np.random.Generator, lo=0.5, hi=1.5) -> dict:
    return dict(G=_sym(rng, D, lo, hi), law=np.zeros((D, D), np.int32),
                ya=np.zeros((D, D)), yl=np.ones((D, D)))


def yukawa_couplings(D: int, rng: np.random.Generator) -> dict:
    """Symmetric G in [0.5,1.5], alpha in [-0.3,0.3], lambda in [0.01,0.1]."""
    return dict(G=_sym(rng, D, 0.5, 1.5), law=np.ones((D, D), np.int32),
                ya=_sym(rng, D, -0.3, 0.3), yl=_sym(rng, D, 0.01, 0.1))


def _params(D, coup, n, mesh, theta, box=1.0, asmth=1.25, rcut_over_rs=4.5, eps_coef=0.02,
            leaf_size=8):
    rs = asmth * box / mesh
    return dict(D=D, G=np.asarray(coup["G"], np.float64), law=np.asarray(coup["law"], np.int32),
                ya=np.asarray(coup["ya"], np.float64), yl=np.asarray(coup["yl"], np.float64),
                box=box, eps=eps_coef * box / n ** (1.0 / 3.0), rs=rs,
                rcut=rcut_over_rs * rs, theta=theta, pm_mesh=mesh, leaf_size=leaf_size)


def workload(name: str, n: int | None = None, seed: int | None = None,
             species: int | None = None) -> dict:
    """Inputs and parameters of a named workload (optionally at another N, or
    with another species count: couplings of the workload's kind drawn for
    that D, Newtonian ones where the workload fixes a 2 x 2 table).

    Returns dict(pos [3][n] f64, type [n] u8, mass [n] f32, vel [3][n] f32,
    params dict, steps, dt).
    """
    spec = WORKLOADS[name]
    n = spec["n"] if n is None else int(n)
    rng = rng_for(spec["seed"] if seed is None else seed)
    D = spec["D"] if species is None else int(species)
    if spec["gen"] == "uniform":
        pos = uniform(n, rng)
    else:
        pos = clustered(n, rng)
    typ = species_blocks(n, D, rng) if spec["species"] == "blocks" else species_uniform(n, D, rng)
    if spec["couplings"] == "cfg0" and D == 2:
        coup = dict(G=np.array([[1.0, 0.8], [0.8, 1.2]]), law=np.zeros((2, 2), np.int32),
                    ya=np.zeros((2, 2)), yl=np.ones((2, 2)))
    elif spec["couplings"] == "yukawa":
        coup = yukawa_couplings(D, rng)
    else:
        coup = newton_couplings(D, rng)
    mass = np.full(n, 1.0 / n, np.float32)
    params = _params(D, coup, n, spec["mesh"], spec["theta"])
    return dict(pos=pos, type=typ, mass=mass, vel=np.zeros((3, n), np.float32),
                params=params, steps=spec.get("steps", 1), dt=spec.get("dt", 1e-3),
                name=name if species is None else f"{name} with D={D}")


#: The measured workloads. Names state what each is.
WORKLOADS = {
    # N=4096, D=2 (2048 each), uniform, Newtonian G=[[1,.8],[.8,1.2]], PM 32^3
    "uniform4k_d2_newton": dict(n=4096, D=2, gen="uniform", species="blocks", couplings="cfg0",
                                mesh=32, theta=0.5, seed=1000),
    # N=2^21, D=2, 512 Plummer spheres + 30% uniform, couplings as above, PM 128^3
    "clustered2m_d2_newton": dict(n=1 << 21, D=2, gen="clustered", species="uniform",
                                  couplings="cfg0", mesh=128, theta=0.5, seed=1001),
    # N=2^24, D=4, clustered, Yukawa-modulated symmetric laws, PM 256^3, KDK dt=1e-3
    "clustered16m_d4_yukawa": dict(n=1 << 24, D=4, gen="clustered", species="uniform",
                                   couplings="yukawa", mesh=256, theta=0.5, seed=1002,
                                   steps=20, dt=1e-3),
}


def batch_specs(count: int = 64, seed: int = 1003, nmin_log2: int = 12, nmax_log2: int = 18,
                mesh: int = 64):
    """Independent simulations: N log-uniform, D uniform in 1..6, Newtonian
    symmetric couplings in [0.5, 1.5], clustered positions."""
    rng = rng_for(seed)
    out = []
    for sid in range(count):
        n = int(round(2.0 ** rng.uniform(nmin_log2, nmax_log2)))
        D = int(rng.integers(1, 7))
        sub = rng_for(seed * 1000 + sid)
        pos = clustered(n, sub)
        typ = species_uniform(n, D, sub)
        coup = newton_couplings(D, sub)
        mass = np.full(n, 1.0 / n, np.float32)
        out.append(dict(pos=pos, type=typ, mass=mass, vel=np.zeros((3, n), np.float32),
                        params=_params(D, coup, n, mesh, 0.5), steps=10, dt=1e-3))
    return out


def log_uniform_int(rng, lo_log2: float, hi_log2: float) -> int:
    return int(round(2.0 ** rng.uniform(lo_log2, hi_log2)))


def serve_mesh(n: int) -> int:
    """PM mesh for a request of n bodies: next power of two of n^(1/3),
    clamped to [32, 128]."""
    m = 1 << max(0, math.ceil(math.log2(max(1.0, n ** (1.0 / 3.0)))))
    return int(min(128, max(32, m)))
