"""Autotuner for the walk's leaf size and group-cell size.

For one workload (device arrays and a parameter dict) it times, through the
C ABI, the tree build plus the short-range walk for each candidate
(leaf_size, group_cell) and returns the fastest. The choice is made on time
to solution (build + walk), never on the interaction count, which itself
grows with the leaf size. Every candidate evaluates the same method: leaf and
group sizes change how much the walk opens, never the law or the criterion.
"""
from __future__ import annotations

import itertools

from . import binding as ng

LEAVES = (8, 16, 32)
GROUP_CELLS = (32, 64, 128, 256)


def tune(params: dict, pos, typ, mass, leaves=LEAVES, cells=GROUP_CELLS, repeats: int = 2,
         stream=None):
    """Returns (best dict(leaf_size, group_cell, ms), list of all trials)."""
    import torch
    n = typ.numel()
    acc = torch.empty((3, n), dtype=torch.float32, device=pos.device)
    trials = []
    for leaf, cell in itertools.product(leaves, cells):
        sim = ng.Simulation(ng.params_from_workload(params, leaf_size=leaf, group_cell=cell), stream)
        best = float("inf")
        for _ in range(repeats):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            ng.ng_build_tree(sim.ctx, pos, typ, mass)
            ng.ng_tree_force(sim.ctx, acc)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        sim.close()
        trials.append(dict(leaf_size=leaf, group_cell=cell, ms=best))
    return min(trials, key=lambda t: t["ms"]), trials


def tune_batch(params_list, state, shortlist, steps: int = 3, dt: float = 1e-3, stream=None):
    """Times batch steps (one captured graph per step, as ng_batch_step runs
    them) for each (leaf_size, group_cell) of the shortlist, on copies of the
    batch's arrays, and returns (best dict(leaf_size, group_cell, ms), trials).
    A batch mixes small and large simulations, so the leaf and group sizes
    that are fastest for its largest member alone need not be fastest for the
    batch."""
    import torch
    trials = []
    for leaf, cell in shortlist:
        cp = [{k: v.clone() for k, v in x.items()} for x in state]
        b = ng.ng_batch_create([ng.params_from_workload(p, leaf_size=leaf, group_cell=cell)
                                for p in params_list], stream)
        try:
            arrays = [[x[k] for x in cp] for k in ("pos", "vel", "typ", "mass", "acc")]
            ng.ng_batch_step(b, *arrays, False, 2, dt)     # sizes, captures, replays once
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            ng.ng_batch_step(b, *arrays, True, steps, dt)
            e1.record()
            torch.cuda.synchronize()
            trials.append(dict(leaf_size=leaf, group_cell=cell, ms=e0.elapsed_time(e1) / steps))
        finally:
            ng.ng_batch_destroy(b)
    return min(trials, key=lambda t: t["ms"]), trials
