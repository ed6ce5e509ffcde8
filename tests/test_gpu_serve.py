"""Serving: requests that run concurrently (continuous batching over slots
and streams) give the same results as each request served alone; admission
respects the byte budget; queued requests can be cancelled; malformed
requests are rejected on the host; bounded waits time out into a status.
Same-result tolerance: the walk is deterministic, the CIC atomics may add in
another order (99 % of bodies within 1e-5 relative, all within 1e-3)."""
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


def _workload(seed, count=10):
    rng = inputs.rng_for(seed)
    out = []
    for k in range(count):
        n = inputs.log_uniform_int(rng, 10, 14)
        D = int(rng.integers(1, 7))
        w = small_clustered(n, D, seed * 100 + k, mesh=inputs.serve_mesh(n))
        kind = int(k % 2)
        out.append(dict(w=w, kind=kind, nsteps=4 if kind else 0))
    return out


def _run(ng, items, slots, budget, cancel=None):
    reqs = (ng.NgRequest * len(items))()
    res = (ng.NgResult * len(items))()
    outs = []
    for i, it in enumerate(items):
        w = it["w"]
        n = w["type"].size
        acc = np.zeros((3, n), np.float32)
        pos = np.zeros((3, n))
        vel = np.zeros((3, n), np.float32)
        outs.append(dict(acc=acc, pos=pos, vel=vel))
        reqs[i] = ng.make_request(it["kind"], ng_params(w["params"]), w["pos"], w["type"], w["mass"],
                                  nsteps=it["nsteps"], dt=1e-3, pos_out=pos, vel_out=vel, acc_out=acc)
    s = ng.ng_serve_create(slots, budget)
    try:
        if cancel is None:
            ng.ng_serve(s, reqs, res, None, 300.0)
        else:
            ids = [ng.ng_serve_submit(s, reqs[i], res[i]) for i in range(len(items))]
            ng.ng_serve_cancel(s, ids[cancel])
            ng.ng_serve_wait(s, 300.0)
    finally:
        ng.ng_serve_destroy(s)
    return outs, res


def _close(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    rel = np.linalg.norm(a - b, axis=0) / np.maximum(np.linalg.norm(b, axis=0), 1e-30)
    return np.percentile(rel, 99) <= 1e-5 and rel.max() <= 1e-3


def test_mix_equals_alone(ng):
    items = _workload(81)
    mixed, res = _run(ng, items, slots=6, budget=8 << 30)
    assert all(r.status == 0 for r in res)
    # overlapping service: some request was admitted before an earlier one finished
    assert any(res[i].t_admit < res[i - 1].t_done for i in range(1, len(items)))
    for it, got in zip(items, mixed):
        alone, r1 = _run(ng, [it], slots=1, budget=8 << 30)
        assert r1[0].status == 0
        assert _close(got["acc"], alone[0]["acc"])
        if it["kind"]:
            w = it["w"]
            assert _close(got["vel"], alone[0]["vel"])
            moved = alone[0]["pos"] - w["pos"]
            d = got["pos"] - alone[0]["pos"]
            rel = np.linalg.norm(d - np.rint(d), axis=0) / np.maximum(
                np.linalg.norm(moved - np.rint(moved), axis=0), 1e-300)
            assert np.percentile(rel, 99) <= 1e-5 and rel.max() <= 1e-3


def test_tight_budget_holds_and_completes(ng):
    items = _workload(82, count=6)
    sizes = []
    for it in items:
        w = it["w"]
        sizes.append(ng.ng_serve_request_bytes(
            ng.make_request(it["kind"], ng_params(w["params"]), w["pos"], w["type"], w["mass"])))
    budget = int(1.2 * max(sizes))                 # at most one or two requests at once
    mixed, _ = _run(ng, items, slots=6, budget=8 << 30)
    tight, res = _run(ng, items, slots=6, budget=budget)
    assert all(r.status == 0 for r in res)
    # at every admission, the requests then running fit in the budget
    for i in range(len(items)):
        t = res[i].t_admit
        running = [j for j in range(len(items)) if res[j].t_admit <= t < res[j].t_done]
        assert sum(sizes[j] for j in running) <= budget
    for x, y in zip(mixed, tight):
        assert _close(x["acc"], y["acc"])


def test_cancel_and_reject(ng):
    items = _workload(83, count=4)
    outs, res = _run(ng, items, slots=1, budget=1 << 27, cancel=3)
    assert [r.status for r in res[:3]] == [0, 0, 0]
    assert res[3].status == ng.NG_ESTATE
    s = ng.ng_serve_create(2, 1 << 30)
    try:
        w = items[0]["w"]
        bad = ng.make_request(0, ng_params(w["params"]), w["pos"], w["type"], w["mass"])
        bad.n = 0
        with pytest.raises(ng.NgError) as e:
            ng.ng_serve_submit(s, bad, ng.NgResult())
        assert e.value.code == ng.NG_EINVAL
        p = ng_params(w["params"])
        p.D = 7
        with pytest.raises(ng.NgError) as e:
            ng.ng_serve_submit(s, ng.make_request(0, p, w["pos"], w["type"], w["mass"]), ng.NgResult())
        assert e.value.code == ng.NG_EINVAL
        big = ng.make_request(0, ng_params(w["params"]), w["pos"], w["type"], w["mass"])
        big.n = 1 << 30
        with pytest.raises(ng.NgError) as e:
            ng.ng_serve_submit(s, big, ng.NgResult())
        assert e.value.code == ng.NG_EBUSY
    finally:
        ng.ng_serve_destroy(s)


def test_bounded_wait_times_out_into_status(ng):
    w = small_clustered(60000, 3, 84, mesh=64)
    s = ng.ng_serve_create(1, 8 << 30)
    acc = np.zeros((3, 60000), np.float32)
    r = ng.make_request(1, ng_params(w["params"]), w["pos"], w["type"], w["mass"], nsteps=3,
                        dt=1e-3, acc_out=acc)
    res = ng.NgResult()
    try:
        ng.ng_serve_submit(s, r, res)
        with pytest.raises(ng.NgError) as e:
            ng.ng_serve_wait(s, 0.0)
        assert e.value.code == ng.NG_ETIMEOUT
        ng.ng_serve_wait(s, 300.0)                  # the context stays usable
        assert res.status == 0 and np.isfinite(acc).all()
    finally:
        ng.ng_serve_destroy(s)


def test_one_slot_serves_growing_species_count(ng):
    # a slot reused by a request with more species and fewer bodies must
    # regrow its per-species node arrays
    items = []
    for k, (n, D) in enumerate([(6000, 1), (2500, 6), (4000, 3)]):
        w = small_clustered(n, D, 850 + k, mesh=32)
        items.append(dict(w=w, kind=k % 2, nsteps=2 if k % 2 else 0))
    seq, res = _run(ng, items, slots=1, budget=8 << 30)
    assert all(r.status == 0 for r in res)
    for it, got in zip(items, seq):
        alone, r1 = _run(ng, [it], slots=1, budget=8 << 30)
        assert r1[0].status == 0
        assert _close(got["acc"], alone[0]["acc"])


def test_tree_regrow_is_budgeted(ng):
    # with leaf size 1 the clustered tree has more than n + 1024 nodes, so the
    # first try of each request overflows its slot's node capacity and the
    # request is rerun with a larger tree; the regrown slot is counted against
    # the budget (the rerun happens only if it fits)
    items = []
    for k, n in enumerate((3000, 3500)):
        w = small_clustered(n, 2, 860 + k, mesh=32, leaf=1)
        items.append(dict(w=w, kind=0, nsteps=0))
    sizes = [ng.ng_serve_request_bytes(ng.make_request(0, ng_params(it["w"]["params"]),
                                                       it["w"]["pos"], it["w"]["type"],
                                                       it["w"]["mass"])) for it in items]
    budget = 8 * max(sizes)
    reqs = (ng.NgRequest * len(items))()
    res = (ng.NgResult * len(items))()
    outs = []
    for i, it in enumerate(items):
        w = it["w"]
        acc = np.zeros((3, w["type"].size), np.float32)
        outs.append(acc)
        reqs[i] = ng.make_request(0, ng_params(w["params"]), w["pos"], w["type"], w["mass"],
                                  acc_out=acc)
    s = ng.ng_serve_create(2, budget)
    try:
        ng.ng_serve(s, reqs, res, None, 300.0)
        held, peak, retries, _ = ng.ng_serve_stats(s)
    finally:
        ng.ng_serve_destroy(s)
    assert all(r.status == 0 for r in res)
    assert retries >= 1
    assert peak <= budget and held <= budget
    # the rerun result is the plain solve of the same request
    import torch
    from common import device_arrays
    for it, got in zip(items, outs):
        w = it["w"]
        pos, typ, mass = device_arrays(w)
        sim = ng.Simulation(ng_params(w["params"]))
        acc = torch.zeros((3, typ.numel()), dtype=torch.float32, device=pos.device)
        vel = torch.zeros_like(acc)
        ng.ng_step(sim.ctx, pos, vel, typ, mass, acc, False, 0, 1e-3)
        torch.cuda.synchronize()
        sim.close()
        assert _close(got, acc.cpu().numpy())


def test_tree_regrow_beyond_budget_fails_cleanly(ng):
    # a budget that admits the first estimate but not the regrown tree: the
    # request fails with NG_ENOMEM and the slots never hold more than the budget
    w = small_clustered(3000, 2, 870, mesh=32, leaf=1)
    acc = np.zeros((3, 3000), np.float32)
    r = ng.make_request(0, ng_params(w["params"]), w["pos"], w["type"], w["mass"], acc_out=acc)
    budget = ng.ng_serve_request_bytes(r) + 1024
    s = ng.ng_serve_create(1, budget)
    res = ng.NgResult()
    try:
        ng.ng_serve_submit(s, r, res)
        ng.ng_serve_wait(s, 300.0)
        held, peak, retries, _ = ng.ng_serve_stats(s)
    finally:
        ng.ng_serve_destroy(s)
    assert res.status == ng.NG_ENOMEM
    assert retries == 0 and peak <= budget


def test_served_results_match_the_oracle(ng):
    # direct mode (theta = 0: FP64 pair sums) plus the PM part, so the served
    # force is held to the direct-mode and PM bounds against the FP64 oracle:
    # |dF| <= 2e-5 |F| + 2e-5 rms(F); a 3-step integration's velocity and
    # position changes within 1e-4 of the oracle's change for 99 % of bodies
    import oracle
    from common import oracle_params
    items = []
    for k, (n, D, yuk) in enumerate([(3000, 2, False), (2500, 3, True), (2000, 4, False)]):
        w = small_clustered(n, D, 880 + k, yukawa=yuk, mesh=32)
        w["params"] = dict(w["params"], theta=0.0)
        items.append(dict(w=w, kind=k % 2, nsteps=3 if k % 2 else 0))
    out, res = _run(ng, items, slots=3, budget=8 << 30)
    assert all(r.status == 0 for r in res)
    for it, got in zip(items, out):
        w = it["w"]
        op = oracle_params(w["params"])
        if it["kind"] == 0:
            ref = oracle.force(op, w["pos"], w["type"], w["mass"])
            dF = np.linalg.norm(got["acc"] - ref, axis=0)
            F = np.linalg.norm(ref, axis=0)
            rms = np.sqrt(np.mean(F ** 2))
            assert (dF <= 2e-5 * F + 2e-5 * rms).all(), (dF / (F + rms)).max()
        else:
            n = w["type"].size
            x, v, a = oracle.kdk(op, w["pos"], np.zeros((3, n)), w["type"], w["mass"], 3, 1e-3)
            for g, want, start in ((got["vel"], v, np.zeros((3, n))), (got["pos"], x, w["pos"])):
                d = g - want
                d -= np.rint(d)
                moved = want - start
                moved -= np.rint(moved)
                rel = np.linalg.norm(d, axis=0) / np.maximum(np.linalg.norm(moved, axis=0), 1e-300)
                assert np.percentile(rel, 99) <= 1e-4, np.percentile(rel, 99)


def test_relative_and_pure_tree_requests(ng):
    # requests that need the relative criterion's |a_old| buffer or the
    # exact-law walk: every buffer is sized on the admitting thread, so the
    # launch threads allocate nothing (a launch thread that did would fail its
    # request with NG_ESTATE)
    items = []
    w = small_clustered(4000, 2, 890, mesh=32)
    w["params"] = dict(w["params"], opening=1, alpha=0.005)
    items.append(dict(w=w, kind=1, nsteps=2))
    w = small_clustered(3000, 2, 891, mesh=32)
    w["params"] = dict(w["params"], pure_tree=1, pm_mesh=0, rs=0.01, rcut=0.045)
    items.append(dict(w=w, kind=0, nsteps=0))
    mixed, res = _run(ng, items, slots=2, budget=8 << 30)
    assert [r.status for r in res] == [0, 0]
    for it, got in zip(items, mixed):
        alone, r1 = _run(ng, [it], slots=1, budget=8 << 30)
        assert r1[0].status == 0
        assert _close(got["acc"], alone[0]["acc"])


def test_same_parameters_do_not_reconfigure(ng):
    # a slot's context is reconfigured only when a request's parameters
    # differ from the previous request's, defaults filled in on both sides
    # (comparing a request's raw parameters with the context's normalised ones
    # once reconfigured the slot for every request, from the launch thread)
    w = small_clustered(3000, 2, 895, mesh=32)
    p = ng_params(w["params"])
    assert p.group_cell == 0                     # a default the library fills in
    items = [dict(w=w, kind=k % 2, nsteps=2 if k % 2 else 0) for k in range(6)]
    reqs = (ng.NgRequest * len(items))()
    res = (ng.NgResult * len(items))()
    for i, it in enumerate(items):
        reqs[i] = ng.make_request(it["kind"], p, w["pos"], w["type"], w["mass"], nsteps=it["nsteps"],
                                  dt=1e-3)
    s = ng.ng_serve_create(1, 8 << 30)
    try:
        ng.ng_serve(s, reqs, res, None, 300.0)
        _, _, _, reconf = ng.ng_serve_stats(s)
    finally:
        ng.ng_serve_destroy(s)
    assert all(r.status == 0 for r in res)
    assert reconf == 1


def test_sixteen_slots_with_changing_sizes_and_species(ng):
    # the concurrent configuration of the serving benchmark, with small
    # requests: 16 slots, requests of varying N, D and mesh in a round-robin
    # order, so every slot serves a sequence of different parameters
    rng = inputs.rng_for(896)
    items = []
    for k in range(24):
        n = inputs.log_uniform_int(rng, 10, 14)
        D = int(rng.integers(1, 7))
        w = small_clustered(n, D, 8960 + k, mesh=inputs.serve_mesh(n))
        items.append(dict(w=w, kind=k % 2, nsteps=3 if k % 2 else 0))
    items = items * 4
    out, res = _run(ng, items, slots=16, budget=32 << 30)
    assert all(r.status == 0 for r in res), [r.status for r in res]
    # every repetition of a request gives the same result
    for k in range(24):
        for rep in (1, 2, 3):
            assert _close(out[k + 24 * rep]["acc"], out[k]["acc"])
