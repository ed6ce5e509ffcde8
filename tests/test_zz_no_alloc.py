"""The allocation-free key sort (ng_sort_keys_noalloc) against ng_build_tree.

Callers that cannot allocate device memory (their allocator is owned by
another framework, or they may not stall on cudaMalloc) get the sorted keys
and permutation from a fixed device scratch array. Keys and permutation are
integers, so the comparison is exact. Calls in a row (different inputs, each
smaller than the one before, the last in a box of side 0.75 with bodies
outside it) check that the shared scratch carries nothing over and that the
general wrap and quantisation match. This file is named to be collected last."""
import numpy as np
import pytest

from common import device_arrays, ng_params, small_clustered
from paper_1502_07442_gb300 import inputs

pytestmark = pytest.mark.gpu

MAX_BODIES = 1 << 18


@pytest.fixture(scope="module")
def ng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1502_07442_gb300 import binding, build
    build.build()
    return binding


def _boxed(w, L, seed):
    """The same bodies in a box of side L, a tenth of them shifted outside it."""
    rng = inputs.rng_for(seed)
    n = w["type"].size
    shift = rng.choice([-1.0, 1.0, 2.0], size=n) * (rng.random(n) < 0.1)
    prm = w["params"]
    prm = dict(prm, box=L, eps=prm["eps"] * L, rs=prm["rs"] * L, rcut=prm["rcut"] * L)
    pos = np.ascontiguousarray(w["pos"] * L + shift[None, :] * L)
    return dict(w, pos=pos, params=prm)


def _reference(ng, w):
    import torch
    pos, typ, mass = device_arrays(w)
    n = typ.numel()
    sim = ng.Simulation(ng_params(w["params"]))
    keys = torch.empty(n, dtype=torch.int64, device=pos.device)
    perm = torch.empty(n, dtype=torch.int32, device=pos.device)
    ng.ng_build_tree(sim.ctx, pos, typ, mass, keys, perm)
    torch.cuda.synchronize()
    sim.close()
    return pos, typ, keys.cpu().numpy(), perm.cpu().numpy()


def test_noalloc_sort_matches_build_tree_twice(ng):
    import torch
    cases = [small_clustered(MAX_BODIES, 4, 91), small_clustered(70001, 2, 92)]
    cases[1]["pos"][:, 10:500] = cases[1]["pos"][:, 9:10]          # ties: stable order
    # a box that is not a power of two: the general FP64 wrap and quantisation
    cases.append(_boxed(small_clustered(50000, 3, 93), 0.75, 94))
    for w in cases:
        pos, typ, k_ref, p_ref = _reference(ng, w)
        n = typ.numel()
        keys = torch.full((n,), -1, dtype=torch.int64, device=pos.device)
        perm = torch.full((n,), -1, dtype=torch.int32, device=pos.device)
        assert ng.ng_sort_keys_noalloc(pos, typ, keys, perm, box=w["params"]["box"]) == ng.NG_OK
        torch.cuda.synchronize()
        assert np.array_equal(keys.cpu().numpy(), k_ref)
        assert np.array_equal(perm.cpu().numpy(), p_ref)


def test_noalloc_sort_rejects_too_many_bodies(ng):
    import torch
    w = inputs.workload("uniform4k_d2_newton")
    pos, typ, _ = device_arrays(w)
    keys = torch.empty(4096, dtype=torch.int64, device=pos.device)
    perm = torch.empty(4096, dtype=torch.int32, device=pos.device)
    big = torch.zeros(MAX_BODIES + 1, dtype=torch.uint8, device=pos.device)
    assert ng.ng_sort_keys_noalloc(pos, big, keys, perm) == ng.NG_EINVAL
    assert ng.ng_sort_keys_noalloc(pos, typ, keys, perm, box=0.0) == ng.NG_EINVAL
