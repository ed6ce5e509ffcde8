"""Shared helpers of the GPU parity tests: one parameter dict (from the
seeded input module) is turned into the oracle's parameter block and into
ng_params, and arrays are moved to cuda:0."""
import numpy as np

import oracle
from paper_1502_07442_gb300 import inputs


def oracle_params(prm, **over):
    q = dict(prm)
    q.update(over)
    return oracle.make_params(q["D"], q["G"], box=q["box"], eps=q["eps"], rs=q["rs"],
                              rcut=q["rcut"], theta=q["theta"], leaf_size=q.get("leaf_size", 8),
                              pm_mesh=q["pm_mesh"], law=q["law"], ya=q["ya"], yl=q["yl"],
                              opening=q.get("opening", 0), alpha=q.get("alpha", 0.005),
                              pure_tree=q.get("pure_tree", 0), ignore_nperp=q.get("ignore_nperp", 0),
                              beta=q.get("beta", 0.0))


def ng_params(prm, **over):
    from paper_1502_07442_gb300 import binding
    return binding.params_from_workload(prm, **over)


def device_arrays(w):
    import torch
    dev = torch.device("cuda:0")
    return (torch.from_numpy(np.ascontiguousarray(w["pos"])).to(dev),
            torch.from_numpy(np.ascontiguousarray(w["type"])).to(dev),
            torch.from_numpy(np.ascontiguousarray(w["mass"])).to(dev))


def small_clustered(n, D, seed, yukawa=False, mesh=32, theta=0.5, leaf=8):
    """Clustered bodies with config-like parameters scaled to n."""
    rng = inputs.rng_for(seed)
    pos = inputs.clustered(n, rng, nspheres=max(4, n // 4096), a=0.005)
    typ = inputs.species_uniform(n, D, rng)
    coup = inputs.yukawa_couplings(D, rng) if yukawa else inputs.newton_couplings(D, rng)
    mass = np.full(n, 1.0 / n, np.float32)
    rs = 1.25 / mesh
    prm = dict(D=D, G=coup["G"], law=coup["law"], ya=coup["ya"], yl=coup["yl"], box=1.0,
               eps=0.02 / n ** (1 / 3), rs=rs, rcut=4.5 * rs, theta=theta, pm_mesh=mesh,
               leaf_size=leaf)
    return dict(pos=pos, type=typ, mass=mass, params=prm, vel=np.zeros((3, n), np.float32))


def transition_case(seed, ntest=2000, mesh=64, law=0, ym=10.0):
    """Transition test of Sec. 3.2 (and of the Coulomb case before it): one
    massive source of species 0 and test particles of species 1 in shells of
    1/r^3 density from 0.1 r_s to L/2. Only the coupling of test particles to
    the source is on (intra-type forces off), with the given law (Newtonian,
    or pure Yukawa of field mass y_m in box units, mu = y_m / L)."""
    rng = inputs.rng_for(seed)
    rs = 1.25 / mesh
    pos = inputs.source_shells(ntest, rng, 0.1 * rs, 0.5)
    typ = np.concatenate([[0], np.ones(ntest)]).astype(np.uint8)
    mass = np.concatenate([[1.0], np.full(ntest, 1e-30)]).astype(np.float32)
    prm = dict(D=2, G=[[0.0, 0.0], [1.0, 0.0]], law=[[0, 0], [law, 0]],
               ya=[[0.0, 0.0], [1.0, 0.0]], yl=[[1.0, 1.0], [1.0 / ym, 1.0]], box=1.0,
               eps=1e-6, rs=rs, rcut=4.5 * rs, theta=0.5, pm_mesh=mesh, leaf_size=8)
    d = pos[:, 1:] - pos[:, :1]
    d -= np.rint(d)
    return dict(pos=pos, type=typ, mass=mass, params=prm), d.T, np.linalg.norm(d, axis=0)


def transition_exact(law, ym, d):
    """Exact periodic acceleration on test particles at offsets d (target -
    source) from a unit source: Ewald sum (Newtonian) or image sum (Yukawa)."""
    import ewald
    if law == 0:
        return np.array([ewald.accel(x) for x in d])
    return np.array([ewald.yukawa_images(x, 1.0, 1.0 / ym, nmax=3) for x in d])


def binned_rms(r, e, edges):
    """rms of e in each [edges[k], edges[k+1]) bin of r (nan for empty bins)."""
    idx = np.digitize(r, edges) - 1
    return np.array([np.sqrt(np.mean(e[idx == k] ** 2)) if np.any(idx == k) else np.nan
                     for k in range(len(edges) - 1)])
