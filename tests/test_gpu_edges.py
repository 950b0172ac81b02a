"""Edge cases of the hot path on the GPU against the FP64 oracle: degenerate
slices (one voxel, one angle, one detector pixel, one mask position), alone
and together in one uneven batch, and the largest sizes the boundary accepts
(EI_MAX_NDET detector pixels, EI_MAX_NM mask positions)."""
import numpy as np
import pytest

import oracle
from paper_2202_08627_gb300 import inputs
from tests.problems import gpu_geometry, measured, oracle_geometry, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (n, n_theta, n_det, n_m)
DEGENERATE = [(1, 1, 1, 1), (2, 3, 1, 1), (1, 4, 5, 2), (5, 1, 3, 3), (3, 2, 2, 1)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build
    build.build()


def _check(specs, geoms, meas, xs, G):
    from paper_2202_08627_gb300 import ei
    vol = G.pack_volume(xs)
    S = torch.zeros(G.n_slices, dtype=torch.float64, device="cuda")
    grad = G.empty("vol")
    ei.ei_objective_grad(G, vol, G.pack_meas(meas), S, grad)
    s_mod = G.empty("meas")
    ei.ei_forward(G, vol, s_mod)
    torch.cuda.synchronize()
    gs, sm = G.unpack_volume(grad), G.unpack_meas(s_mod)
    for i, (spec, geom, s_exp, x) in enumerate(zip(specs, geoms, meas, xs)):
        S_ref, g_ref = oracle.objective_grad(x, s_exp, geom)
        assert abs(S[i].item() - S_ref) <= 1e-5 * abs(S_ref), (spec.n, S[i].item(), S_ref)
        for c in range(3):
            assert rel_l2(gs[i][c], g_ref[c]) <= 1e-4, (spec.n, c, rel_l2(gs[i][c], g_ref[c]))
        assert rel_l2(sm[i], oracle.forward(x, geom)) <= 1e-5, spec.n


@pytest.mark.parametrize("shape", DEGENERATE)
def test_degenerate_slice_matches_oracle(shape):
    spec = inputs.make_slice(21, *shape)
    geom = oracle_geometry(spec)
    G = gpu_geometry([spec], [geom])
    _check([spec], [geom], [measured(spec, geom)], [spec.truth * 0.9], G)


def test_degenerate_slices_in_one_uneven_batch():
    """Slices of different sizes share n_m: the batch takes the shapes with
    M = 1, each with its own geometry, in one launch per kernel."""
    shapes = [s for s in DEGENERATE if s[3] == 1] + [(4, 3, 6, 1)]
    specs = [inputs.make_slice(30 + i, *sh) for i, sh in enumerate(shapes)]
    geoms = [oracle_geometry(sp) for sp in specs]
    G = gpu_geometry(specs, geoms, uneven=True)
    _check(specs, geoms, [measured(sp, g) for sp, g in zip(specs, geoms)],
           [sp.truth * 1.1 for sp in specs], G)


def test_maximum_detector_width_and_mask_positions():
    from paper_2202_08627_gb300 import ei
    spec = inputs.make_slice(40, 48, 5, ei.EI_MAX_NDET, ei.EI_MAX_NM)
    geom = oracle_geometry(spec)
    G = gpu_geometry([spec], [geom])
    meas = [measured(spec, geom)]
    _check([spec], [geom], meas, [spec.truth * 0.95], G)
    # and the flat (zero volume): every channel's projection is zero
    _check([spec], [geom], meas, [np.zeros_like(spec.truth)], G)
