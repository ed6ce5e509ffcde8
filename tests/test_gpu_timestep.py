"""GPU parity of the synchronous time step of Eq. (our_timestep) through the
C ABI: the largest |a| (FP32, the same rounding on both sides) bit for bit,
and dt against the oracle's (its A_max found by sampling the full laws, the
library's from the closed forms) to 1e-9 relative."""
import numpy as np
import pytest

import oracle
from common import ng_params, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1502_07442_gb300 import binding, build
    build.build()
    return binding


@pytest.mark.parametrize("law,ya", [([[0, 1, 2], [1, 0, 1], [2, 1, 1]], 0.4),
                                    ([[2, 2, 2], [2, 2, 2], [2, 2, 2]], -1.7)],
                         ids=["mixed", "pure_yukawa"])
def test_timestep_matches_oracle(ng, law, ya):
    import torch
    rng = np.random.Generator(np.random.PCG64(17))
    G = [[1.0, 0.7, 0.4], [0.7, 1.3, 0.9], [0.4, 0.9, 0.6]]
    prm = dict(D=3, G=G, law=law, ya=[[ya] * 3] * 3, yl=[[0.02] * 3] * 3, box=1.0, eps=1.5e-3,
               rs=1.25 / 32, rcut=4.5 * 1.25 / 32, theta=0.5, pm_mesh=32, leaf_size=8)
    acc = (rng.standard_normal((3, 100003)) * rng.lognormal(0, 2, 100003)).astype(np.float32)
    sim = ng.Simulation(ng_params(prm))
    dacc = torch.from_numpy(acc).cuda()
    for eta, dt_max in ((0.025, 1.0), (0.025, 1e-5)):
        dt, amax = ng.ng_timestep(sim.ctx, dacc, eta, dt_max)
        want, amax_ref = oracle.timestep(oracle_params(prm), acc, eta, dt_max)
        assert np.float32(amax) == np.float32(amax_ref)
        assert dt == pytest.approx(want, rel=1e-9)
    dt0, a0 = ng.ng_timestep(sim.ctx, torch.zeros((3, 50), device="cuda"), 0.025, 0.3)
    assert dt0 == 0.3 and a0 == 0.0
    sim.close()
