"""Batched independent simulations: every simulation advanced inside a batch
(sort/tree/PM on worker streams, one walk launch for all species counts)
matches the same simulation advanced alone through ng_step, and, in direct
summation, the FP64 oracle's integration. The batch's walk reads the class's
law table (one row per distinct law of its members, its own segment count),
so batch and alone differ at the table's accuracy (~1e-5 of a force): 99 %
of bodies within 1e-4 of their displacement / velocity change, all within
1e-2."""
import numpy as np
import pytest

from common import ng_params, small_clustered
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


def _sims():
    # uneven N and D, one law and one mesh: one walk launch serves them all
    specs = [(5000, 2, 71), (20000, 2, 72), (3000, 1, 73), (12000, 4, 74), (1500, 6, 75),
             (777, 3, 76)]
    out = []
    for n, D, seed in specs:
        w = small_clustered(n, D, seed, mesh=32)
        rng = inputs.rng_for(seed + 100)
        w["vel"] = (0.01 * rng.standard_normal((3, n))).astype(np.float32)
        out.append(w)
    return out


def _dev(w):
    import torch
    d = torch.device("cuda:0")
    return dict(pos=torch.from_numpy(w["pos"].copy()).to(d), vel=torch.from_numpy(w["vel"].copy()).to(d),
                typ=torch.from_numpy(w["type"]).to(d), mass=torch.from_numpy(w["mass"]).to(d),
                acc=torch.zeros((3, w["type"].size), dtype=torch.float32, device=d))


def _rel_change(got, want, start):
    d = got - want
    d -= np.rint(d)
    m = want - start
    m -= np.rint(m)
    return np.linalg.norm(d, axis=0) / np.maximum(np.linalg.norm(m, axis=0), 1e-300)


@pytest.mark.parametrize("variant", [{}, {"opening": 1, "alpha": 0.005}, {"accumulate_fp64": 1}],
                         ids=["geometric", "relative", "fp64_accumulated"])
def test_batch_matches_each_simulation_alone(ng, variant):
    """Also with the relative criterion (|a_old| refreshed inside the captured
    batch step) and with the FP64-accumulated walk.

    A single simulation's walk evaluates its record lists in longer runs than
    the batch launch (up to 80-128 records per species list against 64), so
    each body's FP32 sum is grouped, and rounded, differently. With the
    relative criterion of Sec. 2.2 the opening decision depends on |a_old|,
    so a rounding-level difference there accepts other nodes for a few bodies
    and their steps differ by the walk's truncation error: that variant's
    99th percentile is held to 2e-4 instead of 1e-4."""
    import torch
    sims = _sims()
    for w in sims:
        w["params"] = dict(w["params"], **variant)
    steps, dt = 3, 1e-3
    alone = []
    for w in sims:
        a = _dev(w)
        s = ng.Simulation(ng_params(w["params"]))
        ng.ng_step(s.ctx, a["pos"], a["vel"], a["typ"], a["mass"], a["acc"], False, steps, dt)
        torch.cuda.synchronize()
        alone.append({k: v.cpu().numpy() for k, v in a.items()})
        s.close()
    b = ng.ng_batch_create([ng_params(w["params"]) for w in sims])
    assert ng.ng_batch_walk_launches(b) == 1           # every species count in one launch
    m = [_dev(w) for w in sims]
    ng.ng_batch_step(b, [x["pos"] for x in m], [x["vel"] for x in m], [x["typ"] for x in m],
                     [x["mass"] for x in m], [x["acc"] for x in m], False, steps, dt)
    torch.cuda.synchronize()
    for w, x, ref in zip(sims, m, alone):
        rx = _rel_change(x["pos"].cpu().numpy(), ref["pos"], w["pos"])
        rv = _rel_change(x["vel"].cpu().numpy().astype(np.float64), ref["vel"].astype(np.float64),
                         w["vel"].astype(np.float64))
        p99 = 2e-4 if variant.get("opening") else 1e-4
        assert np.percentile(rx, 99) <= p99 and rx.max() <= 1e-2, (np.percentile(rx, 99), rx.max())
        assert np.percentile(rv, 99) <= p99 and rv.max() <= 1e-2, (np.percentile(rv, 99), rv.max())
    # a second call replays the captured batch step
    ng.ng_batch_step(b, [x["pos"] for x in m], [x["vel"] for x in m], [x["typ"] for x in m],
                     [x["mass"] for x in m], [x["acc"] for x in m], True, 2, dt)
    torch.cuda.synchronize()
    for x in m:
        assert torch.isfinite(x["pos"]).all() and torch.isfinite(x["acc"]).all()
    ng.ng_batch_destroy(b)


def test_batch_rejects_bad_arguments(ng):
    import torch
    w = small_clustered(100, 1, 77)
    b = ng.ng_batch_create([ng_params(w["params"])])
    x = _dev(w)
    with pytest.raises(ng.NgError):
        ng.ng_batch_step(b, [x["pos"]], [x["vel"]], [x["typ"]], [x["mass"]], [x["acc"]], False, -1, 1e-3)
    ng.ng_batch_destroy(b)


def test_batch_members_match_the_oracle(ng):
    """Three simulations of D = 1, 3 and 6 in one batch, direct summation
    (theta = 0: the batch's group walk opens every leaf) plus PM, three KDK
    steps against the FP64 oracle's integration of each: velocity and
    position changes within 1e-4 of the oracle's for 99 % of bodies."""
    import torch
    import oracle
    from common import oracle_params
    sims = []
    for n, D, seed in [(3000, 1, 81), (2500, 3, 82), (2000, 6, 83)]:
        w = small_clustered(n, D, seed, mesh=32)
        w["params"] = dict(w["params"], theta=0.0)
        rng = inputs.rng_for(seed + 100)
        w["vel"] = (0.01 * rng.standard_normal((3, n))).astype(np.float32)
        sims.append(w)
    b = ng.ng_batch_create([ng_params(w["params"]) for w in sims])
    assert ng.ng_batch_walk_launches(b) == 1
    m = [_dev(w) for w in sims]
    ng.ng_batch_step(b, [x["pos"] for x in m], [x["vel"] for x in m], [x["typ"] for x in m],
                     [x["mass"] for x in m], [x["acc"] for x in m], False, 3, 1e-3)
    torch.cuda.synchronize()
    ng.ng_batch_destroy(b)
    for w, x in zip(sims, m):
        xo, vo, _ = oracle.kdk(oracle_params(w["params"]), w["pos"], w["vel"].astype(np.float64),
                               w["type"], w["mass"], 3, 1e-3)
        rx = _rel_change(x["pos"].cpu().numpy(), xo, w["pos"])
        rv = _rel_change(x["vel"].cpu().numpy().astype(np.float64), vo, w["vel"].astype(np.float64))
        assert np.percentile(rx, 99) <= 1e-4, np.percentile(rx, 99)
        assert np.percentile(rv, 99) <= 1e-4, np.percentile(rv, 99)


def _mixed_laws(theta):
    """Yukawa members (D = 3: six distinct laws; D = 2: three) and Newtonian
    members (one law, the same row for both): ten rows in one class table."""
    sims = []
    for n, D, seed, yuk in [(4000, 3, 91, True), (3000, 2, 92, True), (5000, 4, 93, False),
                            (2000, 1, 94, False)]:
        w = small_clustered(n, D, seed, yukawa=yuk, mesh=32)
        w["params"] = dict(w["params"], theta=theta)
        rng = inputs.rng_for(seed + 100)
        w["vel"] = (0.01 * rng.standard_normal((3, n))).astype(np.float32)
        sims.append(w)
    return sims


def test_batch_with_mixed_laws(ng):
    """Each member's species pairs map to the right rows of the shared table:
    in direct summation (theta = 0) three KDK steps of every member match the
    oracle's integration, and with the walk (theta = 0.5) every member matches
    the same simulation stepped alone."""
    import torch
    import oracle
    from common import oracle_params
    sims = _mixed_laws(0.0)
    b = ng.ng_batch_create([ng_params(w["params"]) for w in sims])
    assert ng.ng_batch_walk_launches(b) == 1
    m = [_dev(w) for w in sims]
    ng.ng_batch_step(b, [x["pos"] for x in m], [x["vel"] for x in m], [x["typ"] for x in m],
                     [x["mass"] for x in m], [x["acc"] for x in m], False, 3, 1e-3)
    torch.cuda.synchronize()
    ng.ng_batch_destroy(b)
    for w, x in zip(sims, m):
        xo, vo, _ = oracle.kdk(oracle_params(w["params"]), w["pos"], w["vel"].astype(np.float64),
                               w["type"], w["mass"], 3, 1e-3)
        rx = _rel_change(x["pos"].cpu().numpy(), xo, w["pos"])
        rv = _rel_change(x["vel"].cpu().numpy().astype(np.float64), vo, w["vel"].astype(np.float64))
        assert np.percentile(rx, 99) <= 1e-4, np.percentile(rx, 99)
        assert np.percentile(rv, 99) <= 1e-4, np.percentile(rv, 99)
    sims = _mixed_laws(0.5)
    alone = []
    for w in sims:
        a = _dev(w)
        s = ng.Simulation(ng_params(w["params"]))
        ng.ng_step(s.ctx, a["pos"], a["vel"], a["typ"], a["mass"], a["acc"], False, 3, 1e-3)
        torch.cuda.synchronize()
        alone.append({k: v.cpu().numpy() for k, v in a.items()})
        s.close()
    b = ng.ng_batch_create([ng_params(w["params"]) for w in sims])
    m = [_dev(w) for w in sims]
    ng.ng_batch_step(b, [x["pos"] for x in m], [x["vel"] for x in m], [x["typ"] for x in m],
                     [x["mass"] for x in m], [x["acc"] for x in m], False, 3, 1e-3)
    torch.cuda.synchronize()
    ng.ng_batch_destroy(b)
    for w, x, ref in zip(sims, m, alone):
        rv = _rel_change(x["vel"].cpu().numpy().astype(np.float64), ref["vel"].astype(np.float64),
                         w["vel"].astype(np.float64))
        assert np.percentile(rv, 99) <= 1e-4 and rv.max() <= 1e-2, (np.percentile(rv, 99), rv.max())
