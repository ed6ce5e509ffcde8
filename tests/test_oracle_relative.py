"""Pins of the oracle's relative opening criterion (Sec. 2.2: ngravs keeps
GADGET-2's Newtonian relative criterion, accept a node iff the target lies
outside the cube of side 1.2 l about its centre and G_max M l^2 <=
alpha |a_old| r^4).

* alpha -> 0 opens every node: the walk is the direct sum;
* a node at a known place: the acceptance threshold of a_old is the closed
  form G_max M l^2 / (alpha r^4) of that node's mass, side and distance;
* with |a_old| unbounded every node outside its enlarged cube is accepted:
  the walk's count equals an independent count over the tree's ancestor
  chains;
* only the product alpha |a_old| enters (exact for powers of two);
* with the exact |a| the force error falls with alpha and stays below it.
"""
import numpy as np

import oracle
from common import oracle_params, small_clustered
from metrics import rel_err


def _rel(prm, alpha):
    op = oracle_params(prm)
    op.opening = 1
    op.alpha = alpha
    return op


def test_alpha_to_zero_is_direct():
    w = small_clustered(6000, 3, 61)
    prm = w["params"]
    aold = np.ones(6000, np.float32)
    t, c = oracle.tree_walk(_rel(prm, 1e-300), w["pos"], w["type"], w["mass"], aold=aold)
    d = oracle.direct(oracle_params(prm), w["pos"], w["type"], w["mass"])
    e, _ = rel_err(t, d)
    assert e.max() < 1e-12
    _, c0 = oracle.tree_walk(oracle_params(prm, theta=0.0), w["pos"], w["type"], w["mass"])
    assert np.array_equal(c, c0)


def _cluster_case(m=0.1):
    """A lone target and 8 equal bodies, one in each octant of the level-6 cell
    [0.5, 0.5 + 1/64)^3 (leaf size 4: that cell is a node with 8 one-body
    leaves)."""
    h = 1.0 / 64
    corner = np.array([0.5, 0.5, 0.5])
    offs = np.array([[i, j, k] for i in (0.25, 0.75) for j in (0.25, 0.75) for k in (0.25, 0.75)])
    cl = corner[None, :] + offs * h
    tgt = np.array([[0.3, 0.31, 0.29]])
    pos = np.ascontiguousarray(np.concatenate([tgt, cl]).T)
    typ = np.zeros(9, np.uint8)
    mass = np.full(9, m, np.float32)
    prm = dict(D=1, G=[[1.5]], law=[[0]], ya=[[0.0]], yl=[[1.0]], box=1.0, eps=1e-6,
               rs=1.0, rcut=0.49, theta=0.5, pm_mesh=0, leaf_size=4)
    return pos, typ, mass, prm, cl, h


def test_threshold_is_the_closed_form():
    pos, typ, mass, prm, cl, h = _cluster_case()
    M = float(mass[1:].astype(np.float64).sum())
    com = cl.mean(axis=0)
    r = np.linalg.norm(com - pos[:, 0])
    alpha = 0.005
    a_star = 1.5 * M * h * h / (alpha * r ** 4)
    counts = []
    for f in (1.01, 0.99):
        aold = np.full(9, 1.0, np.float32)
        aold[0] = np.float32(f * a_star)
        _, c = oracle.tree_walk(_rel(prm, alpha), pos, typ, mass, tgt=np.array([0]), aold=aold)
        counts.append(int(c[0]))
    # above the threshold the cluster node is one monopole; below it the walk
    # opens it and meets its 8 one-body leaves (accepted or opened: 8 terms)
    assert counts == [1, 8]


def _node_geometry(level, prefix):
    ix = iy = iz = 0
    for b in range(int(level)):
        iz |= ((int(prefix) >> (3 * b)) & 1) << b
        iy |= ((int(prefix) >> (3 * b + 1)) & 1) << b
        ix |= ((int(prefix) >> (3 * b + 2)) & 1) << b
    s = 1.0 / (1 << int(level))
    return np.array([ix + 0.5, iy + 0.5, iz + 0.5]) * s, s


def test_unbounded_aold_accepts_every_node_outside_its_enlarged_cube():
    w = small_clustered(400, 2, 62, leaf=4)
    prm = dict(w["params"], rcut=0.3, leaf_size=4)
    n = 400
    aold = np.full(n, 1e30, np.float32)
    _, c = oracle.tree_walk(_rel(prm, 1.0), w["pos"], w["type"], w["mass"], aold=aold)
    T = oracle.tree(oracle_params(prm), w["pos"], w["type"], w["mass"])
    nn = len(T["level"])
    parent = np.full(nn, -1)
    for k in range(nn):
        for j in range(int(T["nchild"][k])):
            parent[T["child_first"][k] + j] = k
    geo = [_node_geometry(T["level"][k], T["prefix"][k]) for k in range(nn)]
    keys = oracle.keys(w["pos"], w["type"])
    perm = oracle.sort_perm(keys)
    rank = np.empty(n, np.int64)
    rank[perm] = np.arange(n)
    rc2 = prm["rcut"] ** 2
    for i in range(n):
        x = w["pos"][:, i]
        reach, accept = np.zeros(nn, bool), np.zeros(nn, bool)
        for k in range(nn):
            cen, side = geo[k]
            dc = cen - x
            dc -= np.rint(dc)
            gap = np.maximum(0.0, np.abs(dc) - 0.5 * side)
            reach[k] = (gap ** 2).sum() < rc2
            accept[k] = reach[k] and not np.all(np.abs(dc) < 0.6 * side)
        expect = 0
        for k in range(nn):
            a = parent[k]
            opened = True          # every ancestor reached and not accepted
            while a >= 0:
                if not reach[a] or accept[a]:
                    opened = False
                    break
                a = parent[a]
            if not opened or not reach[k]:
                continue
            if accept[k]:
                expect += int((T["mass"][k] > 0).sum())
            elif T["nchild"][k] == 0:
                f, cnt = T["first"][k], T["count"][k]
                expect += cnt - (1 if f <= rank[i] < f + cnt else 0)
        assert c[i] == expect, (i, c[i], expect)


def test_only_alpha_times_aold_enters():
    w = small_clustered(5000, 2, 63)
    prm = w["params"]
    rng = np.random.Generator(np.random.PCG64(64))
    aold = rng.uniform(0.5, 2.0, 5000).astype(np.float32)
    t1, c1 = oracle.tree_walk(_rel(prm, 0.005), w["pos"], w["type"], w["mass"], aold=aold)
    t2, c2 = oracle.tree_walk(_rel(prm, 0.02), w["pos"], w["type"], w["mass"],
                              aold=aold * np.float32(0.25))
    assert np.array_equal(c1, c2)
    assert np.array_equal(t1, t2)


def test_error_falls_with_alpha_and_stays_below_it():
    w = small_clustered(20000, 3, 65)
    prm = w["params"]
    d = oracle.direct(oracle_params(prm), w["pos"], w["type"], w["mass"])
    aold = np.linalg.norm(d, axis=0).astype(np.float32)
    p50, p90, p99, cnt = [], [], [], []
    for alpha in (0.02, 0.005, 0.00125):
        t, c = oracle.tree_walk(_rel(prm, alpha), w["pos"], w["type"], w["mass"], aold=aold)
        e, _ = rel_err(t, d)
        p50.append(np.percentile(e, 50))
        p90.append(np.percentile(e, 90))
        p99.append(np.percentile(e, 99))
        cnt.append(c.sum())
        assert p90[-1] < alpha and p99[-1] < 2 * alpha, (alpha, p90[-1], p99[-1])
    assert p50[0] > p50[1] > p50[2]
    assert cnt[0] < cnt[1] < cnt[2]
