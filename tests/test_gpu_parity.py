"""GPU (libei.so through its C ABI) against the FP64 oracle, element by element
on the same seeded inputs.

Tolerances (FP32 path against FP64): projections, s_mod and the forward
model within 1e-5 relative L2; the objective within 1e-5 relative; the
gradient within 1e-4 relative L2; the adjoint identity of the GPU pair within
1e-5.
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


def ei():
    from paper_2202_08627_gb300 import ei as _ei
    return _ei


# (n, n_theta, n_det, n_m): the small-slice and the autograd-check shapes, a
# ragged one (odd n, detector not a multiple of 4, more pixels than a tile)
SHAPES = [(64, 90, 96, 7), (128, 180, 192, 5), (37, 23, 61, 3), (20, 7, 131, 2)]


def _problem(seed, n, n_theta, n_det, n_m, noise=True, **kw):
    spec = inputs.make_slice(seed, n, n_theta, n_det, n_m)
    geom = oracle_geometry(spec, **kw)
    return spec, geom, measured(spec, geom, noise)


@pytest.mark.parametrize("shape", SHAPES)
def test_project_matches_oracle(shape):
    spec, geom, _ = _problem(1, *shape)
    G = gpu_geometry([spec], [geom])
    vol = G.pack_volume([spec.truth])
    proj = G.empty("proj")
    ei().ei_project(G, vol, proj)
    got = G.unpack_proj(proj)[0]
    for c in range(3):
        ref = oracle.project(spec.truth[c], geom)
        assert rel_l2(got[c], ref) <= 1e-5, (c, rel_l2(got[c], ref))


def test_project_random_angles_and_padding():
    spec, geom, _ = _problem(2, 33, 17, 50, 3)
    geom.theta = inputs.uniform_noise(17, 5, 0.0, 2 * np.pi)
    G = gpu_geometry([spec], [geom])
    x = inputs.uniform_noise((3, 33, 33), 6)
    vol = G.pack_volume([x])
    proj = torch.full((G.proj_count,), 7.0, device="cuda")
    ei().ei_project(G, vol, proj)
    got = G.unpack_proj(proj)[0]
    for c in range(3):
        assert rel_l2(got[c], oracle.project(x[c], geom)) <= 1e-5
    # padding pixels are written as zero
    sl = G.slices[0]
    raw = proj.cpu().numpy()[:sl.proj_count].reshape(3, sl.n_theta, sl.n_dp)
    assert np.all(raw[:, :, sl.n_det:] == 0)


@pytest.mark.parametrize("shape", SHAPES)
def test_backproject_matches_oracle(shape):
    spec, geom, _ = _problem(3, *shape)
    G = gpu_geometry([spec], [geom])
    y = inputs.uniform_noise((3, geom.n_theta, geom.n_det), 7)
    out = G.empty("vol")
    ei().ei_backproject(G, G.pack_sino4([y]), out)
    got = G.unpack_volume(out)[0]
    for c in range(3):
        assert rel_l2(got[c], oracle.backproject(y[c], geom)) <= 1e-5


@pytest.mark.parametrize("shape", [(64, 90, 96, 7), (256, 720, 384, 7), (37, 23, 61, 3)])
@pytest.mark.parametrize("signed", [False, True])
def test_gpu_adjoint_identity(shape, signed):
    """<R x, y> = <x, R^T y> for the GPU pair.  Non-negative vectors: within
    1e-5 of <R x, y>.  Signed vectors, whose inner products cancel: within
    1e-5 of |R x| |y| (the Cauchy-Schwarz scale of the products)."""
    spec, geom, _ = _problem(4, *shape)
    G = gpu_geometry([spec], [geom])
    lo = -1.0 if signed else 0.0
    x = inputs.uniform_noise((3, geom.n, geom.n), 8, lo, 1.0)
    y = inputs.uniform_noise((3, geom.n_theta, geom.n_det), 9, lo, 1.0)
    proj = G.empty("proj")
    ei().ei_project(G, G.pack_volume([x]), proj)
    back = G.empty("vol")
    ei().ei_backproject(G, G.pack_sino4([y]), back)
    Ax = G.unpack_proj(proj)[0].astype(np.float64)
    ATy = G.unpack_volume(back)[0].astype(np.float64)
    for c in range(3):
        lhs, rhs = np.vdot(Ax[c], y[c]), np.vdot(x[c], ATy[c])
        ref = np.linalg.norm(Ax[c]) * np.linalg.norm(y[c]) if signed else abs(lhs)
        assert abs(lhs - rhs) <= 1e-5 * ref, (c, lhs, rhs)


@pytest.mark.parametrize("shape", SHAPES)
def test_ic_model_matches_oracle(shape):
    spec, geom, _ = _problem(5, *shape)
    geom.m_o = inputs.uniform_noise(geom.n_theta, 10, -0.03, 0.03)
    geom.m_r = inputs.uniform_noise(geom.n_det, 11, -0.03, 0.03)
    G = gpu_geometry([spec], [geom])
    s_mod = G.empty("meas")
    ei().ei_ic_model(G, G.pack_proj([spec.P_exact]), s_mod)
    got = G.unpack_meas(s_mod)[0]
    ref = oracle.ic_model(spec.P_exact, geom)
    assert rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_forward_matches_oracle(shape):
    spec, geom, _ = _problem(6, *shape)
    G = gpu_geometry([spec], [geom])
    s_mod = G.empty("meas")
    ei().ei_forward(G, G.pack_volume([spec.truth]), s_mod)
    assert rel_l2(G.unpack_meas(s_mod)[0], oracle.forward(spec.truth, geom)) <= 1e-5


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("offsets", [False, True])
def test_objective_and_gradient_match_oracle(shape, offsets):
    spec, geom, s_exp = _problem(7, *shape)
    if offsets:
        geom.m_o = inputs.uniform_noise(geom.n_theta, 12, -0.03, 0.03)
        geom.m_r = inputs.uniform_noise(geom.n_det, 13, -0.03, 0.03)
    x = spec.truth * 0.85 + 0.02 * inputs.uniform_noise(spec.truth.shape, 14) * \
        np.array(inputs.SCALE)[:, None, None]
    G = gpu_geometry([spec], [geom])
    S = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = G.empty("vol")
    ei().ei_objective_grad(G, G.pack_volume([x]), G.pack_meas([s_exp]), S, grad)
    S_ref, g_ref = oracle.objective_grad(x, s_exp, geom)
    assert abs(S.item() - S_ref) <= 1e-5 * abs(S_ref), (S.item(), S_ref)
    g = G.unpack_volume(grad)[0]
    for c in range(3):
        assert rel_l2(g[c], g_ref[c]) <= 1e-4, (c, rel_l2(g[c], g_ref[c]))


def test_objective_host_output_and_objective_only():
    spec, geom, s_exp = _problem(8, 64, 90, 96, 7)
    G = gpu_geometry([spec], [geom])
    S = torch.zeros(1, dtype=torch.float64)          # host memory
    ei().ei_objective_grad(G, G.pack_volume([spec.truth]), G.pack_meas([s_exp]), S, None)
    S_ref, _ = oracle.objective_grad(spec.truth, s_exp, geom, want_grad=False)
    assert abs(S.item() - S_ref) <= 1e-5 * S_ref


def test_uneven_batch_matches_per_slice_oracle():
    shapes = [(64, 90, 96, 5), (37, 23, 61, 5), (128, 180, 192, 5), (20, 7, 131, 5)]
    probs = [_problem(20 + i, *sh) for i, sh in enumerate(shapes)]
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    xs = [sp.truth * 0.9 for sp in specs]
    S = torch.zeros(len(shapes), dtype=torch.float64, device="cuda")
    grad = G.empty("vol")
    ei().ei_objective_grad(G, G.pack_volume(xs), G.pack_meas(meas), S, grad)
    gs = G.unpack_volume(grad)
    for i in range(len(shapes)):
        S_ref, g_ref = oracle.objective_grad(xs[i], meas[i], geoms[i])
        assert abs(S[i].item() - S_ref) <= 1e-5 * abs(S_ref)
        for c in range(3):
            assert rel_l2(gs[i][c], g_ref[c]) <= 1e-4


def test_domain_guard_and_nonfinite():
    spec, geom, s_exp = _problem(9, 37, 23, 61, 3)
    G = gpu_geometry([spec, spec], [geom, geom])
    x = np.zeros((3, 37, 37))
    x_bad = x.copy()
    x_bad[2] = -50.0                                  # V below 0.01 w^2
    meas = [s_exp, s_exp.copy()]
    meas[1][0, 0, 0] = np.nan
    S = torch.zeros(2, dtype=torch.float64, device="cuda")
    ei().ei_objective_grad(G, G.pack_volume([x_bad, x]), G.pack_meas(meas), S, G.empty("vol"))
    assert S[0].item() == float("inf")
    assert np.isnan(S[1].item())


def test_reconstruct_matches_oracle_trajectory():
    """20 L-BFGS iterations from x0 = 0 on the 64^2 slice: the final objective
    agrees with the FP64 oracle's within 1e-4 relative."""
    spec, geom, s_exp = _problem(0, 64, 90, 96, 7)
    G = gpu_geometry([spec], [geom])
    vol = G.empty("vol")
    rep = ei().ei_reconstruct(G, G.pack_meas([s_exp]), vol, tol=0.0, max_iter=20)
    x_ref, rep_ref = oracle.reconstruct(s_exp, geom, opts=oracle.SolveOptions(tol=0.0, max_iter=20))
    assert rep.iterations[0] == rep_ref.iterations == 20
    assert abs(rep.f_final[0] - rep_ref.f_history[-1]) <= 1e-4 * rep_ref.f_history[-1], \
        (rep.f_final[0], rep_ref.f_history[-1])
    assert abs(rep.f_initial[0] - rep_ref.f_history[0]) <= 1e-5 * rep_ref.f_history[0]
