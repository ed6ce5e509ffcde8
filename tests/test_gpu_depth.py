"""Captured steps build the tree only a few levels below the deepest level
seen before the capture. When the bodies later need a deeper tree, the
replayed build keeps the cells at the cap as leaves (a valid tree, not the
canonical one): every consumer walks, sums and groups leaves of any size, so
the step stays correct, and the next call captures again, deeper.

Here a captured step of uniform bodies (a shallow tree) is replayed on all
bodies packed into a cube of side 1e-3, whose canonical tree is about six
levels deeper: the capped leaf then holds the whole cube, which the walk opens
body by body. Sec. 2.1.1 (KDK) against the oracle's integration."""
import numpy as np
import pytest

import oracle
from common import oracle_params, ng_params
from metrics import rel_err
from paper_1502_07442_gb300 import inputs

pytestmark = pytest.mark.gpu

N = 4096


@pytest.fixture(scope="module")
def ng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1502_07442_gb300 import binding, build
    build.build()
    return binding


def _case(seed, theta):
    rng = inputs.rng_for(seed)
    coup = inputs.newton_couplings(2, rng)
    mesh = 32
    rs = 1.25 / mesh
    prm = dict(D=2, G=coup["G"], law=coup["law"], ya=coup["ya"], yl=coup["yl"], box=1.0,
               eps=1e-5, rs=rs, rcut=4.5 * rs, theta=theta, pm_mesh=mesh, leaf_size=8)
    uniform = rng.random((3, N))
    # inside one cell of side 2^-7 (the cap stays below level 8 for uniform bodies)
    cube = 0.3 + 1e-3 * (rng.random((3, N)) - 0.5)
    typ = inputs.species_uniform(N, 2, rng)
    mass = np.full(N, 1.0 / N, np.float32)
    return prm, uniform, cube, typ, mass


def _check(got, want, start, tol):
    d = got - want
    d -= np.rint(d)
    moved = want - start
    moved -= np.rint(moved)
    rel = np.linalg.norm(d, axis=0) / np.maximum(np.linalg.norm(moved, axis=0), 1e-300)
    assert np.percentile(rel, 99) <= tol, np.percentile(rel, 99)


@pytest.mark.parametrize("theta", [0.0, 0.5], ids=["direct", "walk"])
def test_replayed_tree_deeper_than_its_cap(ng, theta):
    import torch
    prm, uniform, cube, typ, mass = _case(71, theta)
    dev = torch.device("cuda:0")
    pos = torch.from_numpy(uniform.copy()).to(dev)
    vel = torch.zeros((3, N), dtype=torch.float32, device=dev)
    acc = torch.empty((3, N), dtype=torch.float32, device=dev)
    typ_d = torch.from_numpy(typ).to(dev)
    mass_d = torch.from_numpy(mass).to(dev)
    sim = ng.Simulation(ng_params(prm))
    dt = 1e-6
    # eager step, capture at the uniform bodies' depth, one replay
    ng.ng_step(sim.ctx, pos, vel, typ_d, mass_d, acc, False, 2, dt)
    # the same arrays now hold the cube; the acceleration there is the oracle's
    # direct TreePM force (the cube's capped leaf is walked body by body)
    op = oracle_params(prm, theta=0.0)
    a0 = oracle.force(op, cube, typ, mass)
    pos.copy_(torch.from_numpy(cube))
    vel.zero_()
    acc.copy_(torch.from_numpy(a0.astype(np.float32)))
    ng.ng_step(sim.ctx, pos, vel, typ_d, mass_d, acc, True, 1, dt)   # replayed, capped
    torch.cuda.synchronize()
    x1, _, a1 = oracle.kdk(op, cube, np.zeros((3, N)), typ, mass, 1, dt)
    _check(pos.cpu().numpy(), x1, cube, 1e-4)
    err, _ = rel_err(acc.cpu().numpy(), a1)
    assert np.percentile(err, 99) <= 1e-4, np.percentile(err, 99)
    # the next call captures again at the cube's depth: its final force
    # against the direct TreePM force at the final positions, within the
    # oracle walk's own error at this opening angle (tree-mode rule)
    ng.ng_step(sim.ctx, pos, vel, typ_d, mass_d, acc, True, 2, dt)
    torch.cuda.synchronize()
    xf = pos.cpu().numpy()
    ref = oracle.force(op, xf, typ, mass)
    err, _ = rel_err(acc.cpu().numpy(), ref)
    if theta == 0.0:
        assert np.percentile(err, 99) <= 1e-4, np.percentile(err, 99)
    else:
        tree, _ = rel_err(oracle.force(oracle_params(prm), xf, typ, mass), ref)
        assert np.percentile(err, 99) <= 1.1 * np.percentile(tree, 99) + 1e-5, (
            np.percentile(err, 99), np.percentile(tree, 99))
    sim.close()


def test_batch_replay_deeper_than_its_cap(ng):
    """The batch step's captured trees are capped the same way."""
    import torch
    prm, uniform, cube, typ, mass = _case(72, 0.0)
    dev = torch.device("cuda:0")
    pos = [torch.from_numpy(uniform.copy()).to(dev), torch.from_numpy(uniform[::-1].copy()).to(dev)]
    vel = [torch.zeros((3, N), dtype=torch.float32, device=dev) for _ in range(2)]
    acc = [torch.empty((3, N), dtype=torch.float32, device=dev) for _ in range(2)]
    typ_d = [torch.from_numpy(typ).to(dev) for _ in range(2)]
    mass_d = [torch.from_numpy(mass).to(dev) for _ in range(2)]
    b = ng.ng_batch_create([ng_params(prm), ng_params(prm)])
    dt = 1e-6
    ng.ng_batch_step(b, pos, vel, typ_d, mass_d, acc, False, 2, dt)
    # simulation 1 now holds the cube; simulation 0 goes on with uniform bodies
    op = oracle_params(prm)
    start0 = pos[0].cpu().numpy().astype(np.float64)
    v0 = vel[0].cpu().numpy().astype(np.float64)
    a_start0 = acc[0].cpu().numpy()
    a0 = oracle.force(op, cube, typ, mass)
    pos[1].copy_(torch.from_numpy(cube))
    vel[1].zero_()
    acc[1].copy_(torch.from_numpy(a0.astype(np.float32)))
    ng.ng_batch_step(b, pos, vel, typ_d, mass_d, acc, True, 1, dt)   # replayed, capped
    torch.cuda.synchronize()
    x1, _, a1 = oracle.kdk(op, cube, np.zeros((3, N)), typ, mass, 1, dt)
    _check(pos[1].cpu().numpy(), x1, cube, 1e-4)
    err, _ = rel_err(acc[1].cpu().numpy(), a1)
    assert np.percentile(err, 99) <= 1e-4, np.percentile(err, 99)
    # the uniform simulation is unaffected: one oracle step from its state
    _, _, a_ref0 = oracle.kdk(op, start0, v0, typ, mass, 1, dt)
    err, _ = rel_err(acc[0].cpu().numpy(), a_ref0)
    assert np.percentile(err, 99) <= 1e-4, np.percentile(err, 99)
    assert np.isfinite(a_start0).all()
    ng.ng_batch_step(b, pos, vel, typ_d, mass_d, acc, True, 1, dt)   # captured again
    torch.cuda.synchronize()
    assert np.isfinite(acc[1].cpu().numpy()).all()
    ng.ng_batch_destroy(b)


def test_capped_replay_large_tree_binned_monopoles(ng):
    """Trees of 2^20 bodies or more reduce their monopoles in an order binned
    by each node's work, with one bin for the leaves above the leaf size that
    a level cap leaves. A step captured on uniform bodies is replayed after
    8192 of them were packed into a cube of side 1e-4: the capped tree then
    holds a leaf far above the leaf size. Every node's species counts and
    masses are exact sums of its bodies (equal FP32 masses add exactly in
    FP64), and the replayed force on a sample of cube and background bodies
    meets the tree-mode rule against the direct TreePM force (Sec. 2.2,
    Sec. 2.4)."""
    import torch
    n = (1 << 20) + 8192
    rng = inputs.rng_for(73)
    coup = inputs.newton_couplings(2, rng)
    mesh = 32
    rs = 1.25 / mesh
    prm = dict(D=2, G=coup["G"], law=coup["law"], ya=coup["ya"], yl=coup["yl"], box=1.0,
               eps=1e-5, rs=rs, rcut=4.5 * rs, theta=0.5, pm_mesh=mesh, leaf_size=8)
    uniform = rng.random((3, n))
    packed = uniform.copy()
    packed[:, :8192] = 0.3 + 1e-4 * (rng.random((3, 8192)) - 0.5)
    typ = inputs.species_uniform(n, 2, rng)
    m32 = np.float32(1.0 / n)
    mass = np.full(n, m32, np.float32)
    dev = torch.device("cuda:0")
    pos = torch.from_numpy(uniform.copy()).to(dev)
    vel = torch.zeros((3, n), dtype=torch.float32, device=dev)
    acc = torch.zeros((3, n), dtype=torch.float32, device=dev)
    typ_d = torch.from_numpy(typ).to(dev)
    mass_d = torch.from_numpy(mass).to(dev)
    sim = ng.Simulation(ng_params(prm))
    dt = 1e-6
    ng.ng_step(sim.ctx, pos, vel, typ_d, mass_d, acc, False, 2, dt)   # captured on uniform bodies
    # at rest with a zero opening kick the drift leaves every position as it
    # is, so the replayed step's force is the force at the packed positions
    pos.copy_(torch.from_numpy(packed))
    vel.zero_()
    acc.zero_()
    ng.ng_step(sim.ctx, pos, vel, typ_d, mass_d, acc, True, 1, dt)    # replayed, capped
    torch.cuda.synchronize()
    assert np.array_equal(pos.cpu().numpy(), packed)
    T = ng.ng_tree_export(sim.ctx, 2)
    leaf = T["nchild"] == 0
    assert (T["count"][leaf] > 8).any()                # the cap kept an oversize leaf
    assert np.array_equal(T["cnt"].sum(axis=1), T["count"])
    assert np.array_equal(T["mass"], T["cnt"].astype(np.float64) * float(m32))
    assert np.array_equal(T["cnt"][0], np.bincount(typ, minlength=2))
    got = acc.cpu().numpy().astype(np.float64)
    sim.close()
    sample = np.concatenate([np.arange(0, 8192, 41), 8192 + rng.choice(n - 8192, 300, replace=False)])
    op = oracle_params(prm)
    long_ = oracle.pm(op, packed, typ, mass)[:, sample]
    ref = oracle.direct(op, packed, typ, mass, tgt=sample) + long_
    tree, _ = oracle.tree_walk(op, packed, typ, mass, tgt=sample)
    e_gpu, _ = rel_err(got[:, sample], ref)
    e_cpu, _ = rel_err(tree + long_, ref)
    assert np.percentile(e_gpu, 99) <= 1.1 * np.percentile(e_cpu, 99) + 1e-5, (
        np.percentile(e_gpu, 99), np.percentile(e_cpu, 99))
