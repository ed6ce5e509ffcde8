"""GPU parity for boxes other than the unit box, with positions outside it.

Two boxes: L = 4 (a power of two: keys, wrap and drift take the exact
bit-level path) and L = 3.7 (the general FP64 path: wrap x - L floor(x/L)
and quantisation floor(x/L 2^20), each operation rounded). A tenth of the
bodies are shifted by -L, +L or +2L, so that the periodic wrap is exercised.
Keys, permutation, the canonical octree and the interaction counts are
compared bit for bit; forces in direct mode with the 2e-5 rule; the PM force
to 1e-5 of the rms; KDK steps to the tolerances of the unit-box step test.
"""
import numpy as np
import pytest

import oracle
from common import device_arrays, ng_params, oracle_params, small_clustered
from metrics import rel_err
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


def _boxed(L, seed, n=6000, D=3):
    w = small_clustered(n, D, seed, yukawa=True)
    rng = inputs.rng_for(seed + 1000)
    pos = w["pos"] * L
    shift = rng.choice([-1.0, 1.0, 2.0], size=n) * (rng.random(n) < 0.1)
    pos = pos + shift[None, :] * L
    prm = dict(w["params"], box=L, eps=w["params"]["eps"] * L, rs=w["params"]["rs"] * L,
               rcut=w["params"]["rcut"] * L, yl=np.asarray(w["params"]["yl"]) * L)
    return dict(pos=np.ascontiguousarray(pos), type=w["type"], mass=w["mass"], params=prm,
                vel=np.zeros((3, n), np.float32))


BOXES = [("pow2_L4", 4.0, 71), ("general_L3.7", 3.7, 72)]


@pytest.fixture(scope="module", params=BOXES, ids=[b[0] for b in BOXES])
def box(request):
    _, L, seed = request.param
    return L, _boxed(L, seed)


def test_keys_tree_counts_bit_exact(ng, box):
    import torch
    L, w = box
    prm = w["params"]
    pos, typ, mass = device_arrays(w)
    n = typ.numel()
    sim = ng.Simulation(ng_params(prm))
    keys = torch.empty(n, dtype=torch.int64, device=pos.device)
    perm = torch.empty(n, dtype=torch.int32, device=pos.device)
    ng.ng_build_tree(sim.ctx, pos, typ, mass, keys, perm)
    counts = torch.empty(n, dtype=torch.int64, device=pos.device)
    ng.ng_count_interactions(sim.ctx, counts)
    torch.cuda.synchronize()
    k_ref = oracle.keys(w["pos"], w["type"], box=L)
    p_ref = oracle.sort_perm(k_ref)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), p_ref)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), k_ref[p_ref])
    T = ng.ng_tree_export(sim.ctx, prm["D"])
    R = oracle.tree(oracle_params(prm), w["pos"], w["type"], w["mass"])
    for f in ("level", "prefix", "first", "count", "nchild", "child_first", "cnt"):
        assert np.array_equal(T[f], R[f].astype(T[f].dtype)), f
    np.testing.assert_allclose(T["mass"], R["mass"], rtol=1e-12, atol=0)
    _, c_ref = oracle.tree_walk(oracle_params(prm), w["pos"], w["type"], w["mass"])
    assert np.array_equal(counts.cpu().numpy(), c_ref)
    sim.close()


def test_direct_and_pm_forces(ng, box):
    import torch
    L, w = box
    prm = dict(w["params"], theta=0.0)
    pos, typ, mass = device_arrays(w)
    n = typ.numel()
    sim = ng.Simulation(ng_params(prm))
    ng.ng_build_tree(sim.ctx, pos, typ, mass)
    short = torch.empty((3, n), dtype=torch.float32, device=pos.device)
    ng.ng_tree_force(sim.ctx, short)
    long_ = torch.empty_like(short)
    ng.ng_pm_force(sim.ctx, long_)
    torch.cuda.synchronize()
    sim.close()
    op = oracle_params(prm)
    ref = oracle.direct(op, w["pos"], w["type"], w["mass"])
    got = short.cpu().numpy().astype(np.float64)
    dF = np.linalg.norm(got - ref, axis=0)
    F = np.linalg.norm(ref, axis=0)
    assert not (dF > 2e-5 * F).any()
    pm = oracle.pm(op, w["pos"], w["type"], w["mass"])
    rms = np.sqrt(np.mean(np.sum(pm ** 2, axis=0)))
    err = np.linalg.norm(long_.cpu().numpy().astype(np.float64) - pm, axis=0) / rms
    assert err.max() <= 1e-5, err.max()


def test_kdk_steps_wrap(ng, box):
    import torch
    L, w = box
    prm = dict(w["params"], theta=0.0)
    n = w["type"].size
    rng = inputs.rng_for(73)
    vel0 = (0.05 * L * rng.standard_normal((3, n))).astype(np.float32)
    pos, typ, mass = device_arrays(w)
    vel = torch.from_numpy(vel0.copy()).to(pos.device)
    acc = torch.empty((3, n), dtype=torch.float32, device=pos.device)
    sim = ng.Simulation(ng_params(prm))
    ng.ng_step(sim.ctx, pos, vel, typ, mass, acc, False, 3, 1e-3)
    torch.cuda.synchronize()
    sim.close()
    x_ref, v_ref, a_ref = oracle.kdk(oracle_params(prm), w["pos"], vel0.astype(np.float64),
                                     w["type"], w["mass"], 3, 1e-3)
    got = pos.cpu().numpy()
    assert got.min() >= 0.0 and got.max() < L       # wrapped into [0, L)
    d = (got - x_ref) / L
    d -= np.rint(d)
    moved = (x_ref - w["pos"]) / L
    moved -= np.rint(moved)
    rel = np.linalg.norm(d, axis=0) / np.maximum(np.linalg.norm(moved, axis=0), 1e-300)
    assert np.percentile(rel, 99) <= 1e-4 and rel.max() <= 1e-2, (np.percentile(rel, 99), rel.max())
    e, _ = rel_err(acc.cpu().numpy(), a_ref)
    assert np.percentile(e, 99) <= 1e-4
