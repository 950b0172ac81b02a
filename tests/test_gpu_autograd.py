"""torch.autograd wrappers (EIObjective, EIProject) against the FP64 oracle.

The 128x128 slice, 180 angles, 192 pixels, M = 5: the gradient obtained by
autograd through EIObjective is compared with the oracle's analytic gradient
(relative L2 <= 1e-4) and with central finite differences of the FP64 oracle
objective (h = 1e-6 in the solver's scaled variables) on 64 random voxels per
channel.  EIProject's backward must be the oracle's R^T.
"""
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


def _setup(seed=3, shape=(128, 180, 192, 5)):
    spec = inputs.make_slice(seed, *shape)
    geom = oracle_geometry(spec)
    s_exp = measured(spec, geom)
    G = gpu_geometry([spec], [geom])
    return spec, geom, s_exp, G


def test_objective_autograd_matches_oracle_gradient():
    from paper_2202_08627_gb300.autograd import objective
    spec, geom, s_exp, G = _setup()
    x = spec.truth * 0.85
    vol = G.pack_volume([x]).requires_grad_(True)
    S = objective(vol, G, G.pack_meas([s_exp]))
    S.sum().backward()
    S_ref, g_ref = oracle.objective_grad(x, s_exp, geom)
    assert abs(S.item() - S_ref) <= 1e-5 * S_ref
    g = G.unpack_volume(vol.grad)[0]
    for c in range(3):
        assert rel_l2(g[c], g_ref[c]) <= 1e-4, (c, rel_l2(g[c], g_ref[c]))
    assert torch.all(vol.grad[:, 3] == 0)


def test_objective_autograd_against_finite_differences():
    from paper_2202_08627_gb300.autograd import objective
    spec, geom, s_exp, G = _setup()
    scale = np.asarray(geom.scale)[:, None, None]
    u = spec.truth / scale * 0.85
    vol = G.pack_volume([u * scale]).requires_grad_(True)
    objective(vol, G, G.pack_meas([s_exp])).sum().backward()
    g_u = G.unpack_volume(vol.grad)[0].astype(np.float64) * scale     # chain rule to u
    rng = np.random.Generator(np.random.PCG64(17))
    h = 1e-6
    for c in range(3):
        idx = rng.choice(geom.n * geom.n, size=64, replace=False)
        fd = np.empty(64)
        for k, flat in enumerate(idx):
            r, cc = divmod(int(flat), geom.n)
            du = np.zeros_like(u)
            du[c, r, cc] = h
            Sp, _ = oracle.objective_grad(u + du, s_exp, geom, want_grad=False, scaled=True)
            Sm, _ = oracle.objective_grad(u - du, s_exp, geom, want_grad=False, scaled=True)
            fd[k] = (Sp - Sm) / (2 * h)
        got = g_u[c].reshape(-1)[idx]
        assert rel_l2(got, fd) <= 1e-4, (c, rel_l2(got, fd))


def test_objective_autograd_scales_per_slice():
    from paper_2202_08627_gb300.autograd import objective
    spec, geom, s_exp, _ = _setup(shape=(64, 90, 96, 7))
    G2 = gpu_geometry([spec, spec], [geom, geom])
    x = spec.truth * 0.9
    vol = G2.pack_volume([x, x]).requires_grad_(True)
    S = objective(vol, G2, G2.pack_meas([s_exp, s_exp]))
    (S * torch.tensor([2.0, -3.0], dtype=torch.float64, device="cuda")).sum().backward()
    g = G2.unpack_volume(vol.grad)
    _, g_ref = oracle.objective_grad(x, s_exp, geom)
    for c in range(3):
        assert rel_l2(g[0][c], 2.0 * g_ref[c]) <= 1e-4
        assert rel_l2(g[1][c], -3.0 * g_ref[c]) <= 1e-4


def test_project_autograd_backward_is_transpose():
    from paper_2202_08627_gb300.autograd import project
    spec, geom, _, G = _setup(shape=(37, 23, 61, 3))
    x = inputs.uniform_noise((3, 37, 37), 50)
    y = inputs.uniform_noise((3, geom.n_theta, geom.n_det), 51)
    vol = G.pack_volume([x]).requires_grad_(True)
    proj = project(vol, G)
    for c in range(3):
        assert rel_l2(G.unpack_proj(proj.detach())[0][c], oracle.project(x[c], geom)) <= 1e-5
    (proj * G.pack_proj([y])).sum().backward()
    g = G.unpack_volume(vol.grad)[0]
    for c in range(3):
        assert rel_l2(g[c], oracle.backproject(y[c], geom)) <= 1e-5
