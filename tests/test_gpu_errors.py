"""The single-simulation calls through the C ABI reject what the header says
they reject, before any launch, and leave the context usable: empty and
oversized inputs (n outside [1, 2^31)), NULL arrays, negative step counts and
non-finite time steps (NG_EINVAL); forces before a tree and a PM force without
a mesh (NG_ESTATE)."""
import ctypes

import numpy as np
import pytest

from common import ng_params, small_clustered

pytestmark = pytest.mark.gpu

EINVAL, ESTATE = -1, -6


@pytest.fixture(scope="module")
def ng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1502_07442_gb300 import binding, build
    build.build()
    return binding


def _dev(w):
    import torch
    d = torch.device("cuda:0")
    return (torch.from_numpy(w["pos"].copy()).to(d), torch.from_numpy(w["type"]).to(d),
            torch.from_numpy(w["mass"]).to(d))


def _code(fn):
    from paper_1502_07442_gb300 import binding
    with pytest.raises(binding.NgError) as e:
        fn()
    return e.value.code


def test_calls_reject_bad_arguments_and_stay_usable(ng):
    import torch
    w = small_clustered(300, 2, 91)
    pos, typ, mass = _dev(w)
    n = typ.numel()
    dev = pos.device
    acc = torch.zeros((3, n), dtype=torch.float32, device=dev)
    vel = torch.zeros((3, n), dtype=torch.float32, device=dev)
    sim = ng.Simulation(ng_params(w["params"]))
    # forces before any tree
    assert _code(lambda: ng.ng_tree_force(sim.ctx, acc)) == ESTATE
    assert _code(lambda: ng.ng_pm_force(sim.ctx, acc)) == ESTATE
    assert _code(lambda: ng.ng_force(sim.ctx, acc)) == ESTATE
    # empty input
    e3 = torch.empty((3, 0), dtype=torch.float64, device=dev)
    e1 = torch.empty(0, dtype=torch.uint8, device=dev)
    ef = torch.empty(0, dtype=torch.float32, device=dev)
    assert _code(lambda: ng.ng_build_tree(sim.ctx, e3, e1, ef)) == EINVAL
    assert _code(lambda: ng.ng_step(sim.ctx, e3, e3.float(), e1, ef, e3.float(), False, 1, 1e-3)) == EINVAL
    # oversized input: rejected on n alone (the arrays are never read)
    L = ng.lib()
    p = ctypes.c_void_p
    assert L.ng_build_tree(sim.ctx, 1 << 31, p(pos.data_ptr()), p(typ.data_ptr()), p(mass.data_ptr()),
                           None, None) == EINVAL
    # NULL arrays, bad step counts and steps
    assert L.ng_build_tree(sim.ctx, n, None, p(typ.data_ptr()), p(mass.data_ptr()), None, None) == EINVAL
    assert _code(lambda: ng.ng_step(sim.ctx, pos, vel, typ, mass, acc, False, -1, 1e-3)) == EINVAL
    assert _code(lambda: ng.ng_step(sim.ctx, pos, vel, typ, mass, acc, False, 1, float("nan"))) == EINVAL
    # the context still works: a tree, both forces, their sum in the library
    ng.ng_build_tree(sim.ctx, pos, typ, mass)
    short = torch.empty_like(acc)
    long_ = torch.empty_like(acc)
    ng.ng_tree_force(sim.ctx, short)
    ng.ng_pm_force(sim.ctx, long_)
    ng.ng_force(sim.ctx, acc)
    torch.cuda.synchronize()
    s, l_, a = (t.cpu().numpy().astype(np.float64) for t in (short, long_, acc))
    assert np.isfinite(a).all()
    np.testing.assert_allclose(a, s + l_, rtol=1e-5, atol=1e-6 * np.abs(a).max())
    # and a step from the unchanged positions
    ng.ng_step(sim.ctx, pos, vel, typ, mass, acc, False, 1, 1e-4)
    torch.cuda.synchronize()
    assert torch.isfinite(pos).all() and torch.isfinite(acc).all()
    sim.close()


def test_pm_force_without_mesh_is_a_state_error(ng):
    import torch
    w = small_clustered(200, 1, 92)
    prm = dict(w["params"], pm_mesh=0)
    pos, typ, mass = _dev(w)
    sim = ng.Simulation(ng_params(prm))
    ng.ng_build_tree(sim.ctx, pos, typ, mass)
    acc = torch.zeros((3, typ.numel()), dtype=torch.float32, device=pos.device)
    assert _code(lambda: ng.ng_pm_force(sim.ctx, acc)) == ESTATE
    ng.ng_tree_force(sim.ctx, acc)                       # the short-range force alone still runs
    torch.cuda.synchronize()
    assert torch.isfinite(acc).all()
    sim.close()
