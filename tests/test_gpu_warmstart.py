"""The GPU's non-iterative reconstruction (ei_single_shot_fbp) against the
oracle's (moment retrieval, shift integration, Ram-Lak FBP), and as a warm
start of the solver.  Tolerance: relative L2 <= 1e-4 per channel (the
moments and the running sum are accumulated in FP64 on the GPU too)."""
import numpy as np
import pytest

import oracle
from paper_2202_08627_gb300 import inputs
from tests.problems import gpu_geometry, measured, oracle_geometry, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build
    build.build()


@pytest.mark.parametrize("shape", [(64, 90, 96, 7), (128, 180, 192, 5), (37, 23, 61, 3)])
def test_single_shot_matches_oracle(shape):
    from paper_2202_08627_gb300 import ei
    spec = inputs.make_slice(12, *shape)
    geom = oracle_geometry(spec)
    if shape[0] == 37:
        geom.m_o = inputs.uniform_noise(geom.n_theta, 60, -0.02, 0.02)
        geom.m_r = inputs.uniform_noise(geom.n_det, 61, -0.02, 0.02)
    s_exp = measured(spec, geom)
    G = gpu_geometry([spec], [geom])
    out = G.empty("vol")
    ei.ei_single_shot_fbp(G, G.pack_meas([s_exp]), out)
    got = G.unpack_volume(out)[0]
    ref = oracle.single_shot(s_exp, geom)
    for c in range(3):
        assert rel_l2(got[c], ref[c]) <= 1e-4, (c, rel_l2(got[c], ref[c]))


def test_single_shot_uneven_batch():
    from paper_2202_08627_gb300 import ei
    shapes = [(64, 90, 96, 5), (37, 23, 61, 5), (20, 7, 131, 5)]
    probs = []
    for i, sh in enumerate(shapes):
        spec = inputs.make_slice(70 + i, *sh)
        geom = oracle_geometry(spec)
        probs.append((spec, geom, measured(spec, geom)))
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    out = G.empty("vol")
    ei.ei_single_shot_fbp(G, G.pack_meas(meas), out)
    got = G.unpack_volume(out)
    for i in range(3):
        ref = oracle.single_shot(meas[i], geoms[i])
        for c in range(3):
            assert rel_l2(got[i][c], ref[c]) <= 1e-4


def test_warm_start_lowers_the_initial_cost():
    """The single-shot volume is a better start than zero: the objective at
    it is below the objective at x0 = 0."""
    from paper_2202_08627_gb300 import ei
    spec = inputs.make_slice(3, 128, 180, 192, 7)
    geom = oracle_geometry(spec)
    s_exp = measured(spec, geom)
    G = gpu_geometry([spec], [geom])
    meas = G.pack_meas([s_exp])
    x_ss = G.empty("vol")
    ei.ei_single_shot_fbp(G, meas, x_ss)
    S = torch.zeros(2, dtype=torch.float64, device="cuda")
    ei.ei_objective_grad(G, G.empty("vol"), meas, S[0:1], None)
    ei.ei_objective_grad(G, x_ss, meas, S[1:2], None)
    assert S[1].item() < S[0].item()
