"""The paper's single-shot retrieval (Eq. 3) on the GPU against the FP64
oracle: per-slice DFT kernels of 1 / (1 + i q a), circular convolution along
t, -ln, ramp filter and FBP, on an uneven batch of linked phantoms."""
import numpy as np
import pytest

import oracle
from paper_2202_08627_gb300 import inputs
from tests.problems import gpu_geometry, oracle_geometry, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GAMMA = 5e-6
SHAPES = [(64, 90, 96, 7), (37, 23, 61, 7), (128, 180, 192, 7), (20, 7, 131, 7)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build
    build.build()


def _linked(shapes, seed0):
    probs = []
    for i, sh in enumerate(shapes):
        spec = inputs.make_slice(seed0 + i, *sh)
        geom = oracle_geometry(spec)
        Ph = spec.P_exact[0]
        P = np.stack([Ph, GAMMA * Ph, np.zeros_like(Ph)])
        probs.append((spec, geom, inputs.poisson_noise(oracle.ic_model(P, geom), spec.seed)))
    return probs


@pytest.mark.parametrize("m_index", [1, 5])
def test_eq3_matches_oracle(m_index):
    from paper_2202_08627_gb300 import ei
    probs = _linked(SHAPES, 1000)
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    vol = G.empty("vol")
    ei.ei_single_shot_eq3(G, G.pack_meas(meas), m_index, GAMMA, vol)
    out = G.unpack_volume(vol)
    for (spec, geom, s_exp), v in zip(probs, out):
        _, h_ref = oracle.single_shot_eq3(s_exp, geom, m_index, GAMMA)
        assert rel_l2(v[0], h_ref) <= 1e-4, (spec.n, rel_l2(v[0], h_ref))
        assert rel_l2(v[1], GAMMA * h_ref) <= 1e-4
        assert not np.any(v[2])


def test_eq3_rejects_bad_arguments():
    from paper_2202_08627_gb300 import ei
    probs = _linked(SHAPES[:1], 1100)
    G = gpu_geometry([probs[0][0]], [probs[0][1]])
    meas = G.pack_meas([probs[0][2]])
    for m_index, gamma in [(-1, GAMMA), (7, GAMMA), (1, -1.0), (1, float("nan"))]:
        with pytest.raises(ei.EIError):
            ei.ei_single_shot_eq3(G, meas, m_index, gamma, G.empty("vol"))
