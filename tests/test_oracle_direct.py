"""Pins of the oracle's short-range sums: direct sum and per-particle tree walk.

Checked against physics the paper fixes (Sec. 2, Eq. (map); Sec. 2.2): the
passive/active index convention, momentum conservation for symmetric
couplings, reduction of D equal species to one species, translation
invariance of the periodic sum, the cut-off, exactness of the walk when every
node is opened, and brute-force interaction counts."""
import numpy as np
import pytest

import oracle
from paper_1502_07442_gb300 import inputs
from metrics import rel_err


def _params(D, G=None, theta=0.5, eps=1e-3, rs=0.02, rcut=None, leaf=8, law=None, ya=None, yl=None):
    G = np.ones((D, D)) if G is None else G
    return oracle.make_params(D, G, eps=eps, rs=rs, rcut=4.5 * rs if rcut is None else rcut,
                              theta=theta, leaf_size=leaf, law=law, ya=ya, yl=yl)


def test_passive_active_convention_two_bodies():
    G = np.array([[1.0, 2.0], [0.5, 1.0]])          # G[passive][active]
    p = _params(2, G, eps=0.0)
    pos = np.array([[0.40, 0.45], [0.5, 0.5], [0.5, 0.5]])
    typ = np.array([0, 1], np.uint8)
    mass = np.array([1.0, 3.0], np.float32)
    a = oracle.direct(p, pos, typ, mass, cells=False)
    r = 0.05
    T = oracle.short_factor(0, 0, 1, p.rs, r)
    # body 0 (species 0) feels G[0][1] * m1; body 1 feels G[1][0] * m0; both attractive
    assert a[0, 0] == pytest.approx(2.0 * 3.0 * T / r ** 2, rel=1e-12)
    assert a[0, 1] == pytest.approx(-0.5 * 1.0 * T / r ** 2, rel=1e-12)
    assert np.all(a[1:] == 0.0)


def test_cutoff_is_strict_on_softened_separation():
    # a term contributes iff sqrt(r^2 + eps^2) < r_cut
    p = _params(1, rcut=0.1, eps=0.01)
    typ = np.zeros(2, np.uint8)
    mass = np.ones(2, np.float32)
    r_in = np.sqrt(0.1 ** 2 - 0.01 ** 2) * (1 - 1e-9)
    r_out = np.sqrt(0.1 ** 2 - 0.01 ** 2) * (1 + 1e-9)
    inside = np.array([[0.5, 0.5 + r_in], [0.5, 0.5], [0.5, 0.5]])
    outside = np.array([[0.5, 0.5 + r_out], [0.5, 0.5], [0.5, 0.5]])
    assert oracle.direct(p, inside, typ, mass, cells=False)[0, 0] > 0
    assert np.all(oracle.direct(p, outside, typ, mass, cells=False) == 0.0)


def test_magnitude_sum_bounds_the_force():
    rng = inputs.rng_for(18)
    n = 300
    pos = inputs.clustered(n, rng, nspheres=3, a=0.01)
    typ = inputs.species_uniform(n, 2, rng)
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    p = _params(2, rs=0.03)
    a, mag = oracle.direct_mag(p, pos, typ, mass)
    np.testing.assert_allclose(a, oracle.direct(p, pos, typ, mass), rtol=1e-13, atol=0)
    assert np.all(np.linalg.norm(a, axis=0) <= mag * (1 + 1e-12))
    # one pair: the sum of magnitudes is the magnitude
    two = np.array([[0.5, 0.52], [0.5, 0.5], [0.5, 0.5]])
    a2, m2 = oracle.direct_mag(p, two, np.zeros(2, np.uint8), np.ones(2, np.float32))
    np.testing.assert_allclose(np.linalg.norm(a2, axis=0), m2, rtol=1e-14)


def test_periodic_minimum_image():
    p = _params(1, rcut=0.1, eps=0.0)
    typ = np.zeros(2, np.uint8)
    mass = np.ones(2, np.float32)
    pos = np.array([[0.01, 0.97], [0.5, 0.5], [0.5, 0.5]])    # 0.04 apart across x = 0
    a = oracle.direct(p, pos, typ, mass, cells=False)
    assert a[0, 0] < 0 and a[0, 1] > 0                        # pulled across the boundary


@pytest.mark.parametrize("gen", ["uniform", "clustered"])
def test_cell_list_equals_brute_force(gen):
    rng = inputs.rng_for(11)
    n, D = 700, 3
    pos = inputs.uniform(n, rng) if gen == "uniform" else inputs.clustered(n, rng, nspheres=5, a=0.01)
    typ = inputs.species_uniform(n, D, rng)
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    c = inputs.yukawa_couplings(D, rng)
    p = _params(D, c["G"], law=c["law"], ya=c["ya"], yl=c["yl"], rs=0.03)
    a1 = oracle.direct(p, pos, typ, mass, cells=False)
    a2 = oracle.direct(p, pos, typ, mass, cells=True)
    np.testing.assert_allclose(a2, a1, rtol=1e-11, atol=1e-11 * np.abs(a1).max())


def test_momentum_conservation_symmetric_couplings():
    rng = inputs.rng_for(12)
    n, D = 800, 4
    pos = inputs.clustered(n, rng, nspheres=6, a=0.01)
    typ = inputs.species_uniform(n, D, rng)
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    c = inputs.yukawa_couplings(D, rng)
    p = _params(D, c["G"], law=c["law"], ya=c["ya"], yl=c["yl"], rs=0.03)
    a = oracle.direct(p, pos, typ, mass)
    m = mass.astype(np.float64)
    tot = np.abs((a * m).sum(axis=1)).max()
    assert tot <= 1e-12 * (np.abs(a) * m).sum()


def test_equal_couplings_reduce_to_one_species():
    rng = inputs.rng_for(13)
    n = 600
    pos = inputs.clustered(n, rng, nspheres=4, a=0.01)
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    one = _params(1, np.full((1, 1), 1.3))
    a1 = oracle.direct(one, pos, np.zeros(n, np.uint8), mass)
    w1, _ = oracle.tree_walk(one, pos, np.zeros(n, np.uint8), mass)
    e1, _ = rel_err(w1, a1)
    for D in (2, 5):
        typ = inputs.species_uniform(n, D, rng)
        pD = _params(D, np.full((D, D), 1.3))
        aD = oracle.direct(pD, pos, typ, mass)
        np.testing.assert_allclose(aD, a1, rtol=1e-12, atol=1e-12 * np.abs(a1).max())
        wD, _ = oracle.tree_walk(pD, pos, typ, mass)
        # per-species monopoles describe the mass finer than one monopole, so
        # the tree error does not grow with D (Sec. 2.2, Sec. 3.1)
        err, _ = rel_err(wD, a1)
        assert np.median(err) <= np.median(e1)
        assert np.percentile(err, 99) <= 1.2 * np.percentile(e1, 99)


def test_translation_invariance():
    rng = inputs.rng_for(14)
    n, D = 500, 2
    pos = inputs.uniform(n, rng)
    typ = inputs.species_blocks(n, D, rng)
    mass = np.full(n, 1.0 / n, np.float32)
    p = _params(D, np.array([[1.0, 0.8], [0.8, 1.2]]), rs=0.04)
    a = oracle.direct(p, pos, typ, mass)
    shifted = np.mod(pos + np.array([[0.37], [0.11], [0.93]]), 1.0)
    b = oracle.direct(p, shifted, typ, mass)
    np.testing.assert_allclose(b, a, rtol=1e-9, atol=1e-9 * np.abs(a).max())


def test_walk_opening_everything_is_direct():
    rng = inputs.rng_for(15)
    n, D = 900, 3
    pos = inputs.clustered(n, rng, nspheres=4, a=0.01)
    typ = inputs.species_uniform(n, D, rng)
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    c = inputs.yukawa_couplings(D, rng)
    p = _params(D, c["G"], law=c["law"], ya=c["ya"], yl=c["yl"], rs=0.03, theta=0.0)
    w, _ = oracle.tree_walk(p, pos, typ, mass)
    d = oracle.direct(p, pos, typ, mass)
    np.testing.assert_allclose(w, d, rtol=1e-11, atol=1e-11 * np.abs(d).max())


def test_walk_error_is_tree_sized_and_shrinks_with_theta():
    rng = inputs.rng_for(16)
    n, D = 3000, 2
    pos = inputs.clustered(n, rng, nspheres=8, a=0.01)
    typ = inputs.species_uniform(n, D, rng)
    mass = np.full(n, 1.0 / n, np.float32)
    d = oracle.direct(_params(D, rs=0.03), pos, typ, mass)
    stats = []
    for th in (0.3, 0.5, 0.8):
        w, cnt = oracle.tree_walk(_params(D, rs=0.03, theta=th), pos, typ, mass)
        err, _ = rel_err(w, d)
        stats.append(np.percentile(err, [50, 90, 99]))
    stats = np.array(stats)
    for q in range(3):
        assert stats[0, q] < stats[1, q] < stats[2, q]
    # geometric Barnes-Hut at theta = 0.5: sub-percent typical error
    assert stats[1, 0] < 5e-3 and stats[1, 1] < 2e-2


def test_walk_counts_at_theta0_match_brute_force_leaves():
    rng = inputs.rng_for(17)
    n, D = 400, 2
    pos = inputs.uniform(n, rng)
    typ = inputs.species_uniform(n, D, rng)
    mass = np.ones(n, np.float32)
    p = _params(D, rs=0.02, theta=0.0, leaf=4)
    _, cnt = oracle.tree_walk(p, pos, typ, mass)
    T = oracle.tree(p, pos, typ, mass)
    leaves = np.nonzero(T["nchild"] == 0)[0]
    w = pos - np.floor(pos)
    want = np.zeros(n, np.int64)
    for k in leaves:
        lev, pre = int(T["level"][k]), int(T["prefix"][k])
        idx = [0, 0, 0]
        for b in range(lev):
            for ax, sh in ((0, 2), (1, 1), (2, 0)):
                idx[ax] |= ((pre >> (3 * b + sh)) & 1) << b
        side = 1.0 / (1 << lev)
        cen = (np.array(idx) + 0.5) * side
        dc = w - cen[:, None]
        dc -= np.rint(dc)
        gap = np.maximum(0.0, np.abs(dc) - side / 2)
        near = (gap ** 2).sum(axis=0) < p.rcut ** 2
        inside = np.all(np.abs(dc) <= side / 2, axis=0)
        want += near * int(T["count"][k]) - (near & inside)
    assert np.array_equal(cnt, want)
