"""GPU parity of the integer outputs (bit-exact) and the FP64 monopoles:
keys, permutation, canonical octree, N_perp counts, type-major order and
the per-particle interaction counts, through the C ABI against the oracle."""
import numpy as np
import pytest

import oracle
from common import device_arrays, ng_params, oracle_params, small_clustered
from paper_1502_07442_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1502_07442_gb300 import binding, build
    build.build()
    return binding


def _cases():
    yield "cfg0", inputs.workload("uniform4k_d2_newton")
    yield "clustered_d4", small_clustered(40000, 4, 41, yukawa=True)
    yield "tiny1", small_clustered(1, 1, 42)
    yield "tiny33", small_clustered(33, 3, 43)
    w = small_clustered(5000, 2, 44, leaf=1)
    w["pos"][:, 100:400] = w["pos"][:, 99:100]             # 300 duplicates: level-20 leaf
    yield "dups_leaf1", w


CASES = list(_cases())


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_keys_perm_tree_bit_exact(ng, name, w):
    import torch
    prm = w["params"]
    pos, typ, mass = device_arrays(w)
    n = typ.numel()
    sim = ng.Simulation(ng_params(prm))
    keys = torch.empty(n, dtype=torch.int64, device=pos.device)
    perm = torch.empty(n, dtype=torch.int32, device=pos.device)
    ng.ng_build_tree(sim.ctx, pos, typ, mass, keys, perm)
    torch.cuda.synchronize()
    k_ref = oracle.keys(w["pos"], w["type"])
    p_ref = oracle.sort_perm(k_ref)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), p_ref)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), k_ref[p_ref])
    T = ng.ng_tree_export(sim.ctx, prm["D"])
    R = oracle.tree(oracle_params(prm), w["pos"], w["type"], w["mass"])
    for f in ("level", "prefix", "first", "count", "nchild", "child_first", "cnt"):
        assert np.array_equal(T[f], R[f].astype(T[f].dtype)), f
    np.testing.assert_allclose(T["mass"], R["mass"], rtol=1e-12, atol=0)
    # centres of mass: the same FP64 sums of m x in another order (tree levels);
    # both round within (terms + 2) units of 2^-53 of the box size per coordinate
    dcom = np.abs(T["com"] - R["com"]).max(axis=2)
    bound = 2.0 ** -53 * 4 * (R["cnt"].astype(np.float64) + 2)
    assert np.all(dcom <= bound)
    sim.close()


@pytest.mark.parametrize("name,w", CASES[:2], ids=[c[0] for c in CASES[:2]])
def test_type_major_order(ng, name, w):
    import torch
    prm = w["params"]
    pos, typ, mass = device_arrays(w)
    n = typ.numel()
    sim = ng.Simulation(ng_params(prm))
    ng.ng_build_tree(sim.ctx, pos, typ, mass)
    order = torch.empty(n, dtype=torch.int32, device=pos.device)
    offs = ng.ng_type_order(sim.ctx, prm["D"], order)
    p_ref = oracle.sort_perm(oracle.keys(w["pos"], w["type"]))
    t_sorted = w["type"][p_ref]
    want = p_ref[np.argsort(t_sorted, kind="stable")]
    assert np.array_equal(order.cpu().numpy().view(np.uint32), want)
    counts = np.bincount(w["type"], minlength=prm["D"])
    assert np.array_equal(offs, np.concatenate([[0], np.cumsum(counts)]))
    sim.close()


@pytest.mark.parametrize("name,w,theta", [(CASES[0][0], CASES[0][1], 0.5),
                                          (CASES[1][0], CASES[1][1], 0.5),
                                          (CASES[1][0], CASES[1][1], 0.0),
                                          (CASES[4][0], CASES[4][1], 0.7)],
                         ids=["cfg0", "clustered_d4", "clustered_d4_direct", "dups_leaf1"])
def test_interaction_counts_bit_exact(ng, name, w, theta):
    import torch
    prm = dict(w["params"], theta=theta)
    pos, typ, mass = device_arrays(w)
    n = typ.numel()
    sim = ng.Simulation(ng_params(prm))
    ng.ng_build_tree(sim.ctx, pos, typ, mass)
    counts = torch.empty(n, dtype=torch.int64, device=pos.device)
    total = ng.ng_count_interactions(sim.ctx, counts)
    _, c_ref = oracle.tree_walk(oracle_params(prm), w["pos"], w["type"], w["mass"])
    got = counts.cpu().numpy()
    assert np.array_equal(got, c_ref)
    assert total == int(c_ref.sum())
    sim.close()


def test_tree_queries_after_single_steps(ng):
    """ng_step with nsteps = 1 takes the eager path and may then regrow the
    node arrays for the replayed steps; the tree left in the context must
    still be the tree of the current positions (this case triggers the
    regrow: 2551 nodes in the initial 4096-node capacity)."""
    import torch
    w = small_clustered(20000, 3, 91, leaf=32)
    prm = w["params"]
    pos, typ, mass = device_arrays(w)
    n = typ.numel()
    vel = torch.zeros((3, n), dtype=torch.float32, device=pos.device)
    acc = torch.empty((3, n), dtype=torch.float32, device=pos.device)
    sim = ng.Simulation(ng_params(prm))
    ng.ng_step(sim.ctx, pos, vel, typ, mass, acc, False, 1, 1e-3)
    ng.ng_step(sim.ctx, pos, vel, typ, mass, acc, True, 1, 1e-3)
    counts = torch.empty(n, dtype=torch.int64, device=pos.device)
    total = ng.ng_count_interactions(sim.ctx, counts)
    tree = ng.ng_tree_export(sim.ctx, prm["D"])
    fresh = ng.Simulation(ng_params(prm))
    ng.ng_build_tree(fresh.ctx, pos, typ, mass)
    counts_f = torch.empty(n, dtype=torch.int64, device=pos.device)
    total_f = ng.ng_count_interactions(fresh.ctx, counts_f)
    tree_f = ng.ng_tree_export(fresh.ctx, prm["D"])
    assert total == total_f
    assert torch.equal(counts, counts_f)
    for k in ("level", "prefix", "first", "count", "nchild", "child_first", "cnt"):
        assert np.array_equal(tree[k], tree_f[k]), k
    sim.close()
    fresh.close()


def _large(D, leaf, seed):
    w = small_clustered((1 << 20) + 777, D, seed, leaf=leaf)
    rng = inputs.rng_for(seed + 1)
    n = w["type"].size
    w["mass"] = (rng.uniform(0.5, 1.5, n) / n).astype(np.float32)   # unequal masses
    if leaf == 1:
        w["pos"][:, 1000:1400] = w["pos"][:, 999:1000]              # 400 duplicates: level-20 leaf
    return w


@pytest.mark.parametrize("D,leaf", [(6, 64), (1, 1)], ids=["d6_leaf64", "d1_leaf1"])
def test_binned_monopoles_large_trees(ng, D, leaf):
    """Trees of 2^20 bodies or more take the binned monopole order (leaves by
    body count up to the largest leaf size, one bin above it; internal nodes
    by level and child count): six species with 64-body leaves, and one
    species with 1-body leaves whose duplicates end in a level-20 leaf above
    the leaf size. The tree is bit-exact and the FP64 monopoles, with unequal
    masses, within the summation-order bound of the oracle's (Sec. 2.2)."""
    import torch
    w = _large(D, leaf, 61 + D)
    prm = w["params"]
    pos, typ, mass = device_arrays(w)
    sim = ng.Simulation(ng_params(prm))
    ng.ng_build_tree(sim.ctx, pos, typ, mass)
    torch.cuda.synchronize()
    T = ng.ng_tree_export(sim.ctx, D)
    sim.close()
    R = oracle.tree(oracle_params(prm), w["pos"], w["type"], w["mass"])
    for f in ("level", "prefix", "first", "count", "nchild", "child_first", "cnt"):
        assert np.array_equal(T[f], R[f].astype(T[f].dtype)), f
    leaf_counts = T["count"][T["nchild"] == 0]
    assert (leaf_counts > (32 if leaf == 64 else 1)).any()
    # FP64 sums of n terms in another order: n ulps of the sum of |terms|
    m = R["mass"]
    bound_m = 2.0 ** -53 * (R["cnt"].astype(np.float64) + 2) * m
    assert np.all(np.abs(T["mass"] - m) <= bound_m)
    dcom = np.abs(T["com"] - R["com"]).max(axis=2)
    bound = 2.0 ** -53 * 4 * (R["cnt"].astype(np.float64) + 2)
    assert np.all(dcom <= bound)
