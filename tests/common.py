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
                              opening=q.get("opening", 0), alpha=q.get("alpha", 0.005))


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
