"""The no-allocation entry point against the regular one.

ei_objective_grad_noalloc serves callers that cannot allocate GPU memory —
code running while a stream is captured into a CUDA graph, frameworks that
keep all device memory in their own pool, loops that cannot pay cudaMalloc's
synchronisation.  It keeps every intermediate in one static device array, so
two calls in a row must each reproduce ei_objective_grad on their own input
(the second call must not see the first call's leftovers).  This file is
collected last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

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


def _args(geom):
    return dict(n=geom.n, n_theta=geom.n_theta, n_det=geom.n_det, pitch_cm=geom.pitch,
                n_m=geom.n_m, m=geom.m, z_cm=geom.z_cm, period_cm=geom.period_cm,
                kappa_sigma=geom.kappa, flat_A=geom.flat_A, flat_c=geom.flat_c,
                flat_w=geom.flat_w, lam=geom.lam, scale=geom.scale, theta=geom.theta,
                m_o=geom.m_o, m_r=geom.m_r)


@pytest.mark.parametrize("shape", [(64, 90, 96, 7), (256, 720, 384, 7), (37, 23, 61, 3)])
def test_noalloc_matches_objective_grad_twice(shape):
    from paper_2202_08627_gb300 import ei
    spec = inputs.make_slice(11, *shape)
    geom = oracle_geometry(spec)
    if shape[0] == 37:
        geom.m_o = inputs.uniform_noise(geom.n_theta, 40, -0.03, 0.03)
        geom.m_r = inputs.uniform_noise(geom.n_det, 41, -0.03, 0.03)
    s_exp = measured(spec, geom)
    G = gpu_geometry([spec], [geom])
    meas = G.pack_meas([s_exp])
    for call, factor in enumerate((0.9, 1.1)):          # two calls in a row, different inputs
        vol = G.pack_volume([spec.truth * factor])
        S_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        g_ref = G.empty("vol")
        ei.ei_objective_grad(G, vol, meas, S_ref, g_ref)
        S = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = torch.full_like(g_ref, float("nan"))
        ei.ei_objective_grad_noalloc(vol=vol, s_exp=meas, S_out=S, grad=g, **_args(geom))
        torch.cuda.synchronize()
        assert abs(S.item() - S_ref.item()) <= 1e-5 * abs(S_ref.item()), (call, S.item(), S_ref.item())
        a, b = G.unpack_volume(g)[0], G.unpack_volume(g_ref)[0]
        for c in range(3):
            assert rel_l2(a[c], b[c]) <= 1e-4, (call, c, rel_l2(a[c], b[c]))


def test_noalloc_rejects_slices_beyond_the_scratch():
    from paper_2202_08627_gb300 import ei
    spec = inputs.make_slice(0, 64, 8, 96, 3)
    geom = oracle_geometry(spec)
    args = _args(geom)
    args.update(n=2048, n_theta=1800, n_det=3000, pitch_cm=0.32 / 2048, theta=None,
                flat_A=np.ones(3000), flat_c=np.zeros(3000), flat_w=np.full(3000, 0.25))
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    S = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ei.EIError) as err:
        ei.ei_objective_grad_noalloc(vol=dummy, s_exp=dummy, S_out=S, **args)
    assert err.value.status == ei.EI_ERR_ARG
