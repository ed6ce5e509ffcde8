"""Pins of the oracle's integer outputs: keys, permutation, canonical octree.

Each is checked against a brute-force route written here from the
definitions (cells found from positions, not from keys)."""
import numpy as np
import pytest

import oracle
from paper_1502_07442_gb300 import inputs


def _py_key(x, y, z, t, L=1.0):
    q = []
    for c in (x, y, z):
        w = c - L * np.floor(c / L)
        v = int(np.floor((w / L) * 1048576.0))
        q.append(min(max(v, 0), 1048575))
    m = 0
    for b in range(20):
        for axis, shift in ((0, 2), (1, 1), (2, 0)):
            m |= ((q[axis] >> b) & 1) << (3 * b + shift)
    return (m << 3) | int(t)


def test_keys_match_bit_loop_and_special_values():
    rng = inputs.rng_for(7)
    pos = rng.uniform(-1.5, 2.5, (3, 300))
    typ = rng.integers(0, 6, 300).astype(np.uint8)
    k = oracle.keys(pos, typ)
    for i in range(300):
        assert int(k[i]) == _py_key(*pos[:, i], typ[i])
    special = np.array([[0.0, 0.999999999, -1e-300, 0.5, 1.0],
                        [0.0, 0.999999999, 0.0, 0.5, 0.0],
                        [0.0, 0.999999999, 0.0, 0.5, 2.0]])
    ks = oracle.keys(special, np.array([3, 0, 1, 2, 5], np.uint8))
    assert int(ks[0]) == 3                               # origin: only the type
    assert int(ks[1]) == ((1 << 60) - 1) << 3            # every Morton bit set
    # x = -1e-300 wraps to 1 - tiny which rounds to 1.0: clamped to the last cell
    qx = 0
    for b in range(20):
        qx |= ((int(ks[2]) >> 3 >> (3 * b + 2)) & 1) << b
    assert qx == (1 << 20) - 1
    # centre of the box: x = y = z = 2^19 -> bits 57..59 set at level 1
    assert int(ks[3]) >> 3 == 0b111 << 57
    # 1.0 wraps to 0, 2.0 wraps to 0
    assert int(ks[4]) == 5


def test_sort_perm_is_stable_argsort():
    rng = inputs.rng_for(8)
    k = rng.integers(0, 40, 5000).astype(np.uint64)       # many ties
    perm = oracle.sort_perm(k)
    assert np.array_equal(perm, np.argsort(k, kind="stable").astype(np.uint32))


def _brute_tree(pos, typ, mass, D, leaf):
    """Canonical octree from positions: BFS over cells, children in octant order."""
    n = pos.shape[1]
    w = pos - np.floor(pos)
    q = np.minimum(np.floor(w * 1048576.0).astype(np.int64), 1048575)
    nodes = [(0, 0, 0, 0)]          # level, ix, iy, iz
    out = []
    idx = 0
    while idx < len(nodes):
        lev, ix, iy, iz = nodes[idx]
        sh = 20 - lev
        inside = ((q[0] >> sh) == ix) & ((q[1] >> sh) == iy) & ((q[2] >> sh) == iz)
        members = np.nonzero(inside)[0]
        cnt = np.array([(typ[members] == t).sum() for t in range(D)], np.uint32)
        msp = np.array([mass[members][typ[members] == t].astype(np.float64).sum() for t in range(D)])
        com = np.zeros((D, 3))
        for t in range(D):
            sel = members[typ[members] == t]
            if sel.size:
                com[t] = (w[:, sel] * mass[sel].astype(np.float64)).sum(axis=1) / msp[t]
        leaf_here = members.size <= leaf or lev == 20
        nch = 0
        if not leaf_here:
            for o in range(8):
                cx, cy, cz = 2 * ix + (o >> 2 & 1), 2 * iy + (o >> 1 & 1), 2 * iz + (o & 1)
                sh2 = 20 - (lev + 1)
                if np.any(((q[0] >> sh2) == cx) & ((q[1] >> sh2) == cy) & ((q[2] >> sh2) == cz)):
                    nodes.append((lev + 1, cx, cy, cz))
                    nch += 1
        prefix = 0
        for b in range(lev):
            prefix |= ((ix >> b) & 1) << (3 * b + 2) | ((iy >> b) & 1) << (3 * b + 1) | ((iz >> b) & 1) << (3 * b)
        out.append(dict(level=lev, prefix=prefix, count=members.size, nchild=nch, cnt=cnt,
                        mass=msp, com=com))
        idx += 1
    return out


@pytest.mark.parametrize("n,D,leaf,gen", [(1, 1, 8, "u"), (9, 2, 8, "u"), (200, 3, 4, "u"),
                                          (600, 2, 8, "c"), (300, 6, 1, "c")])
def test_tree_matches_brute_force_cells(n, D, leaf, gen):
    rng = inputs.rng_for(100 + n)
    pos = inputs.uniform(n, rng) if gen == "u" else inputs.clustered(n, rng, nspheres=4, a=0.002)
    typ = inputs.species_uniform(n, D, rng)
    mass = rng.uniform(0.5, 2.0, n).astype(np.float32)
    p = oracle.make_params(D, np.ones((D, D)), eps=1e-3, rs=0.05, rcut=0.2, leaf_size=leaf)
    T = oracle.tree(p, pos, typ, mass)
    B = _brute_tree(pos, typ, mass, D, leaf)
    assert len(B) == T["level"].size
    for k, b in enumerate(B):
        assert T["level"][k] == b["level"] and int(T["prefix"][k]) == b["prefix"]
        assert T["count"][k] == b["count"] and T["nchild"][k] == b["nchild"]
        assert np.array_equal(T["cnt"][k], b["cnt"])
        np.testing.assert_allclose(T["mass"][k], b["mass"], rtol=1e-12)
        np.testing.assert_allclose(T["com"][k], b["com"], rtol=1e-12, atol=1e-14)
    # children are contiguous and bodies partition the parent range
    for k in range(len(B)):
        if T["nchild"][k]:
            c0 = T["child_first"][k]
            ch = range(c0, c0 + T["nchild"][k])
            assert sum(T["count"][c] for c in ch) == T["count"][k]
            assert T["first"][c0] == T["first"][k]


def test_duplicate_positions_collapse_into_level20_leaf():
    pos = np.full((3, 40), 0.3)
    pos[:, 20:] = 0.7
    typ = np.zeros(40, np.uint8)
    mass = np.ones(40, np.float32)
    p = oracle.make_params(1, np.ones((1, 1)), eps=1e-3, rs=0.05, rcut=0.2, leaf_size=8)
    T = oracle.tree(p, pos, typ, mass)
    leaves = np.nonzero(T["nchild"] == 0)[0]
    assert sorted(T["count"][leaves].tolist()) == [20, 20]
    assert set(T["level"][leaves].tolist()) == {20}
