"""Pins of the oracle's geometric opening criterion (Sec. 2.2, the Barnes-Hut
walk; the configurations fix the opening angle theta).

The oracle walks the canonical tree per target: a node is reached when the
gap between the target and the node cube is below r_cut, accepted as D
species monopoles when the target lies outside the cube and
side < theta * d (d the minimum-image distance to the node's all-species
centre of mass), and otherwise opened (a leaf into its bodies).

These tests recompute every target's interaction count from the exported
tree alone, without the walk: a node contributes iff every ancestor is
reached and not accepted, and it is itself reached; then it adds its species
with mass if accepted, or its bodies (the target excluded) if it is a leaf.
The recomputation is vectorised over nodes and targets in numpy and shares
nothing with the oracle's C++ walk. It covers theta 0.3, 0.5 and 0.8, leaf
sizes 1, 8 and 32, one and six species, uniform and clustered bodies.

Constructed cases pin the three places where a plausible slip would leave
random inputs nearly unchanged: the strict inequality (a node with
side == theta * d exactly), the target-inside-the-cell test (theta = 0.8,
where a cell holding the target can pass the angle test), and the minimum
image of d (a node across the periodic boundary). A force pin checks the
accepted monopoles against their closed form.
"""
import numpy as np
import pytest

import oracle
from common import oracle_params, small_clustered
from paper_1502_07442_gb300 import inputs


def _geometry(T, L):
    """Centres [nn, 3] and sides [nn] of the canonical nodes (physical units)."""
    lvl = T["level"].astype(np.int64)
    pre = T["prefix"].astype(np.uint64)
    ijk = np.zeros((lvl.size, 3), np.int64)
    for b in range(21):
        for axis, shift in ((0, 2), (1, 1), (2, 0)):
            bit = (pre >> np.uint64(3 * b + shift)) & np.uint64(1)
            ijk[:, axis] |= bit.astype(np.int64) << b
    side = L / (2.0 ** lvl)
    return (ijk + 0.5) * side[:, None], side


def _parents(T):
    nn = T["level"].size
    parent = np.full(nn, -1, np.int64)
    for k in np.nonzero(T["nchild"] > 0)[0]:
        parent[T["child_first"][k]:T["child_first"][k] + T["nchild"][k]] = k
    return parent


def independent_counts(prm, pos, typ, mass, targets):
    """Per-target counts of the geometric walk, from the exported tree."""
    op = oracle_params(prm)
    T = oracle.tree(op, pos, typ, mass)
    L = float(prm["box"])
    cen, side = _geometry(T, L)
    parent = _parents(T)
    M = T["mass"]                                   # [nn, D]
    mt = M.sum(axis=1)
    com_all = (M[:, :, None] * T["com"]).sum(axis=1) / np.where(mt > 0, mt, 1.0)[:, None]
    nspec = (M > 0).sum(axis=1)
    keys = oracle.keys(pos, typ, box=L)
    rank = np.empty(pos.shape[1], np.int64)
    rank[oracle.sort_perm(keys)] = np.arange(pos.shape[1])
    x = pos[:, targets].T                           # [nt, 3]
    dc = cen[None, :, :] - x[:, None, :]
    dc -= L * np.rint(dc / L)                       # minimum image
    gap = np.maximum(0.0, np.abs(dc) - 0.5 * side[None, :, None])
    reach = (gap ** 2).sum(axis=2) < float(prm["rcut"]) ** 2
    inside = np.all(np.abs(dc) <= 0.5 * side[None, :, None], axis=2)
    dm = com_all[None, :, :] - x[:, None, :]
    dm -= L * np.rint(dm / L)
    d = np.sqrt((dm ** 2).sum(axis=2))
    accept = reach & ~inside & (side[None, :] < float(prm["theta"]) * d)
    # a node is visited iff its parent was visited, reached and not accepted
    visited = np.zeros_like(reach)
    visited[:, 0] = True
    for lv in range(1, int(T["level"].max()) + 1):
        ks = np.nonzero(T["level"] == lv)[0]
        p = parent[ks]
        visited[:, ks] = visited[:, p] & reach[:, p] & ~accept[:, p]
    contrib = visited & reach
    leaf = T["nchild"] == 0
    first, count = T["first"], T["count"]
    out = np.zeros(len(targets), np.int64)
    out += (contrib & accept) @ nspec
    body_terms = contrib & ~accept & leaf[None, :]
    out += body_terms @ count
    own = (first[None, :] <= rank[targets][:, None]) & (rank[targets][:, None] < (first + count)[None, :])
    out -= (body_terms & own).sum(axis=1)
    return out


def _uniform(n, D, seed, leaf):
    w = small_clustered(n, D, seed, leaf=leaf)
    rng = inputs.rng_for(seed + 500)
    w["pos"] = rng.random((3, n))
    return w


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.8])
@pytest.mark.parametrize("leaf", [1, 8, 32])
@pytest.mark.parametrize("D", [1, 6])
@pytest.mark.parametrize("gen", ["uniform", "clustered"])
def test_counts_equal_ancestor_chain_recount(theta, leaf, D, gen):
    n = 4000
    seed = 3000 + 97 * leaf + 13 * D + int(100 * theta) + (0 if gen == "uniform" else 7)
    w = _uniform(n, D, seed, leaf) if gen == "uniform" else small_clustered(n, D, seed, leaf=leaf)
    # a cut-off close to L/2 reaches nodes far enough to pass the angle test
    # even at theta = 0.3 with leaves of 32 bodies
    prm = dict(w["params"], theta=theta, leaf_size=leaf, rcut=0.45, rs=0.1)
    tgt = np.arange(0, n, 7)
    _, cnt = oracle.tree_walk(oracle_params(prm), w["pos"], w["type"], w["mass"], tgt=tgt)
    want = independent_counts(prm, w["pos"], w["type"], w["mass"], tgt)
    assert np.array_equal(cnt, want), np.nonzero(cnt != want)[0][:10]
    # the criterion is active: accepting nodes changes targets' counts
    # (either way: an accepted node straddling the cut-off is one term even
    # where none of its bodies is within r_cut)
    _, c0 = oracle.tree_walk(oracle_params(dict(prm, theta=0.0)), w["pos"], w["type"], w["mass"],
                             tgt=tgt)
    assert (cnt != c0).sum() >= 5


def _boundary_case():
    """Target T = (9/64, 17/64, 17/64); three bodies of mass 1/4 on the x axis
    through C = T + (1/16, 0, 0) (at C and C -+ 1/256), inside the level-5
    cell [3/16, 7/32) x [1/4, 9/32)^2 (side 1/32), and two more bodies in the
    neighbouring level-5 cell of the same level-4 parent, so that the three
    form a leaf with leaf size 4. Every coordinate is dyadic, so the leaf's
    centre of mass is C exactly and d = 1/16: with theta = 0.5,
    side == theta * d."""
    t = np.array([9 / 64, 17 / 64, 17 / 64])
    c = t + np.array([1 / 16, 0.0, 0.0])
    h = 1 / 256
    three = [c - np.array([h, 0, 0]), c, c + np.array([h, 0, 0])]
    two = [np.array([15 / 64, 17 / 64, 17 / 64]), np.array([15 / 64, 35 / 128, 17 / 64])]
    pos = np.ascontiguousarray(np.array([t] + three + two).T)
    typ = np.zeros(6, np.uint8)
    mass = np.full(6, 0.25, np.float32)
    prm = dict(D=1, G=[[1.0]], law=[[0]], ya=[[0.0]], yl=[[1.0]], box=1.0, eps=1e-6, rs=0.1,
               rcut=0.45, theta=0.5, pm_mesh=0, leaf_size=4)
    return pos, typ, mass, prm


def test_strict_inequality_at_side_equal_theta_d():
    pos, typ, mass, prm = _boundary_case()
    T = oracle.tree(oracle_params(prm), pos, typ, mass)
    cen, side = _geometry(T, 1.0)
    # the three bodies form a leaf of side 1/32 whose centre of mass is exactly
    # 1/16 from the target: side == theta * d
    k = [i for i in range(T["level"].size) if T["nchild"][i] == 0 and T["count"][i] == 3]
    assert len(k) == 1 and side[k[0]] == 1 / 32
    assert np.allclose(T["com"][k[0], 0], pos[:, 0] + [1 / 16, 0, 0], rtol=0, atol=0)
    _, c = oracle.tree_walk(oracle_params(prm), pos, typ, mass, tgt=np.array([0]))
    # not accepted (strict <): its three bodies are opened; the other leaf
    # (two bodies, farther than twice its side) is one monopole
    assert int(c[0]) == 3 + 1
    assert int(independent_counts(prm, pos, typ, mass, np.array([0]))[0]) == 3 + 1
    # a hair larger angle accepts the leaf as one monopole
    _, c2 = oracle.tree_walk(oracle_params(dict(prm, theta=0.5 + 1e-9)), pos, typ, mass,
                             tgt=np.array([0]))
    assert int(c2[0]) == 1 + 1


def test_cell_holding_the_target_is_never_accepted():
    # theta = 0.8 lets a cell pass the angle test while holding the target:
    # the target sits in one corner of a level-3 cell (side 1/8) and 15 heavy
    # bodies in the opposite corner put the centre of mass ~1.6 sides away
    s = 1 / 8
    base = np.array([0.5, 0.5, 0.5])
    tgt = base + np.array([0.01, 0.01, 0.01]) * s
    far = [base + (0.97 - 0.01 * j) * s * np.ones(3) for j in range(15)]
    # two bodies in the neighbouring level-3 cell make the level-2 parent split
    filler = [np.array([0.7, 0.7, 0.7]), np.array([0.72, 0.7, 0.7]),
              np.array([0.1, 0.1, 0.1]), np.array([0.9, 0.1, 0.3])]
    pos = np.ascontiguousarray(np.array([tgt] + far + filler).T)
    n = pos.shape[1]
    typ = np.zeros(n, np.uint8)
    mass = np.ones(n, np.float32)
    prm = dict(D=1, G=[[1.0]], law=[[0]], ya=[[0.0]], yl=[[1.0]], box=1.0, eps=1e-6, rs=0.1,
               rcut=0.45, theta=0.8, pm_mesh=0, leaf_size=16)
    T = oracle.tree(oracle_params(prm), pos, typ, mass)
    cen, side = _geometry(T, 1.0)
    # the level-3 leaf holds the target and the 15 bodies; its centre of mass
    # is more than side / theta from the target
    k = [i for i in range(T["level"].size) if T["level"][i] == 3 and T["count"][i] == 16]
    assert len(k) == 1
    d = np.linalg.norm(T["com"][k[0], 0] - tgt)
    assert side[k[0]] < 0.8 * d
    _, c = oracle.tree_walk(oracle_params(prm), pos, typ, mass, tgt=np.array([0]))
    # the cell holding the target is opened: its 15 other bodies are terms
    assert int(c[0]) >= 15
    assert int(c[0]) == int(independent_counts(prm, pos, typ, mass, np.array([0]))[0])


def test_distance_uses_the_minimum_image():
    # four bodies just across the periodic boundary form a level-2 leaf (side
    # 1/4; a fifth body in the same level-1 cell makes that cell split). Their
    # centre of mass is 0.047 from the target through the boundary and 0.953
    # the other way: at the nearest image the leaf fails the angle test and
    # is opened (4 terms); at the raw offset it would be one monopole
    tgt = np.array([0.02, 0.6, 0.6])
    cl = [np.array([0.97 + 0.002 * j, 0.6, 0.6]) for j in range(4)]
    filler = [np.array([0.6, 0.6, 0.6])]
    pos = np.ascontiguousarray(np.array([tgt] + cl + filler).T)
    n = pos.shape[1]
    typ = np.zeros(n, np.uint8)
    mass = np.ones(n, np.float32)
    prm = dict(D=1, G=[[1.0]], law=[[0]], ya=[[0.0]], yl=[[1.0]], box=1.0, eps=1e-6, rs=0.1,
               rcut=0.45, theta=0.5, pm_mesh=0, leaf_size=4)
    T = oracle.tree(oracle_params(prm), pos, typ, mass)
    k = [i for i in range(T["level"].size) if T["nchild"][i] == 0 and T["count"][i] == 4]
    assert len(k) == 1 and T["level"][k[0]] == 2
    _, c = oracle.tree_walk(oracle_params(prm), pos, typ, mass, tgt=np.array([0]))
    # the cluster's 4 bodies plus the filler leaf (0.44 away: side 1/4 > theta d)
    assert int(c[0]) == 4 + 1
    assert int(c[0]) == int(independent_counts(prm, pos, typ, mass, np.array([0]))[0])


def test_accepted_monopoles_give_their_closed_form_force():
    # one target and, far from it, a compact group of two species whose
    # monopoles are known exactly; with r_s much larger than the separations
    # the short-range factor is 1 to within 1e-15, so the walk's force is
    # G_st M_t (c_t - x) / (r^2 + eps^2)^(3/2) summed over the two species
    tgt = np.array([0.3, 0.3, 0.3])
    a = np.array([0.5 + 1 / 64, 0.5 + 1 / 64, 0.5 + 1 / 64])
    h = 1 / 512
    bodies = [a + [h, 0, 0], a - [h, 0, 0], a + [0, h, 0], a - [0, h, 0]]
    # a massless body near them makes their cells split below level 1, so
    # that a node small enough for the angle test holds them (it adds nothing
    # to any monopole)
    filler = [np.array([0.55, 0.515625, 0.515625])]
    pos = np.ascontiguousarray(np.array([tgt] + bodies + filler).T)
    typ = np.array([0, 0, 0, 1, 1, 0], np.uint8)
    mass = np.array([1.0, 0.5, 0.5, 0.25, 0.75, 0.0], np.float32)
    G = [[1.2, 0.7], [0.7, 0.9]]
    eps = 1e-3
    prm = dict(D=2, G=G, law=[[0, 0], [0, 0]], ya=[[0.0] * 2] * 2, yl=[[1.0] * 2] * 2, box=1.0,
               eps=eps, rs=1e6, rcut=0.49, theta=0.5, pm_mesh=0, leaf_size=4)
    acc, c = oracle.tree_walk(oracle_params(prm), pos, typ, mass, tgt=np.array([0]))
    assert int(c[0]) == 2                  # one accepted node: one term per species
    want = np.zeros(3)
    for t, idx in ((0, [1, 2]), (1, [3, 4])):
        M = float(mass[idx].astype(np.float64).sum())
        com = (pos[:, idx] * mass[idx].astype(np.float64)).sum(axis=1) / M
        dv = com - tgt
        q = dv @ dv + eps * eps
        want += G[0][t] * M * dv / q ** 1.5
    np.testing.assert_allclose(acc[:, 0], want, rtol=1e-12)
