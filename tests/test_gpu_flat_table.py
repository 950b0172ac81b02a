"""The sampled flat IC (ei_set_flat_table: f(t, m) tabulated at K mask
positions over one period, periodic Catmull-Rom in m, as the paper's flat
scan measures it) on the GPU against the FP64 oracle: forward model, cost and
gradient, the offsets' gradient, the linked solver's trajectory, and the
switch back to the Gaussian flat."""
import numpy as np
import pytest

import oracle
from paper_2202_08627_gb300 import inputs
from tests.problems import gpu_geometry, oracle_geometry, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GAMMA = 5e-7
K_STEPS = 33                       # mask positions of one flat scan
SHAPES = [(64, 90, 96, 5), (37, 23, 61, 5), (128, 180, 192, 5), (20, 7, 131, 5)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build
    build.build()


def flat_table(geom, K, seed):
    """A flat IC sampled at m = k / K: the periodised Gaussian of the geometry's
    (A, c, w) with a seeded per-pixel asymmetry, so the table is not a Gaussian."""
    m = np.arange(K) / K
    d = m[None, :] - geom.flat_c[:, None]
    g = sum(np.exp(-(d + j) ** 2 / (2 * geom.flat_w[:, None] ** 2)) for j in range(-3, 4))
    a = 0.15 * inputs.uniform_noise(geom.n_det, seed, -1.0, 1.0)
    return geom.flat_A[:, None] * g * (1.0 + a[:, None] * np.sin(2 * np.pi * d))


def _problems(shapes, seed0, linked=False, offsets=True):
    probs = []
    for i, sh in enumerate(shapes):
        spec = inputs.make_slice(seed0 + i, *sh)
        kw = {}
        if offsets:
            kw = dict(m_o=inputs.uniform_noise(spec.n_theta, seed0 + 100 + i, -0.03, 0.03),
                      m_r=inputs.uniform_noise(spec.n_det, seed0 + 200 + i, -0.03, 0.03))
        geom = oracle_geometry(spec, **kw)
        geom.flat_table = flat_table(geom, K_STEPS, seed0 + 300 + i)
        P = spec.P_exact
        if linked:
            P = np.stack([P[0], GAMMA * P[0], np.zeros_like(P[0])])
        s_exp = inputs.poisson_noise(oracle.ic_model(P, geom), spec.seed)
        probs.append((spec, geom, s_exp))
    return probs


def _gpu(probs):
    from paper_2202_08627_gb300 import ei
    specs, geoms, _ = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    ei.ei_set_flat_table(G, np.concatenate([g.flat_table for g in geoms]).astype(np.float32))
    return G


@pytest.mark.parametrize("ic_variant", [0, 1])
def test_model_cost_and_gradient_match_oracle(ic_variant):
    """Three channels; the sigma lane has no effect (gradient 0).  The
    persistent IC variant is requested too: a table runs the per-row kernel."""
    from paper_2202_08627_gb300 import ei
    probs = _problems(SHAPES, 1100)
    G = _gpu(probs)
    ei.ei_set_ic_variant(G, ic_variant)
    xs = [p[0].truth * 0.9 for p in probs]
    vol = G.pack_volume(xs)
    meas = G.pack_meas([p[2] for p in probs])
    S = torch.zeros(G.n_slices, dtype=torch.float64, device="cuda")
    grad = G.empty("vol")
    ei.ei_objective_grad(G, vol, meas, S, grad)
    s_mod = G.empty("meas")
    ei.ei_forward(G, vol, s_mod)
    g_mo, g_mr = ei.ei_offset_grad(G, vol, meas)
    torch.cuda.synchronize()
    gs, sm = G.unpack_volume(grad), G.unpack_meas(s_mod)
    g_mo, g_mr = g_mo.cpu().numpy(), g_mr.cpu().numpy()
    o_th = o_px = 0
    for i, ((spec, geom, s_exp), x) in enumerate(zip(probs, xs)):
        assert rel_l2(sm[i], oracle.forward(x, geom)) <= 1e-5, i
        S_ref, g_ref = oracle.objective_grad(x, s_exp, geom)
        assert abs(S[i].item() - S_ref) <= 1e-5 * abs(S_ref), (i, S[i].item(), S_ref)
        # sigma's gradient is the regulariser's alone (the data term ignores it)
        for ch in range(3):
            assert rel_l2(gs[i][ch], g_ref[ch]) <= 1e-4, (i, ch, rel_l2(gs[i][ch], g_ref[ch]))
        r_mo, r_mr = oracle.offset_grads(x, s_exp, geom)
        assert rel_l2(g_mo[o_th:o_th + spec.n_theta], r_mo) <= 1e-4, (i, "m_o")
        assert rel_l2(g_mr[o_px:o_px + spec.n_det], r_mr) <= 1e-4, (i, "m_r")
        o_th += spec.n_theta
        o_px += spec.n_det


def test_linked_reconstruct_matches_oracle_trajectory():
    """The paper's setting: the linked unknown h with the measured flat.  20
    L-BFGS iterations from h = 0 agree with the FP64 oracle's."""
    from paper_2202_08627_gb300 import ei
    probs = _problems([(64, 90, 96, 7)], 1200, linked=True)
    (spec, geom, s_exp), = probs
    G = _gpu(probs)
    ei.ei_set_linked(G, GAMMA)
    vol = G.empty("vol")
    rep = ei.ei_reconstruct(G, G.pack_meas([s_exp]), vol, tol=0.0, max_iter=20)

    def fun(u):
        return oracle.objective_grad_linked(u, s_exp, geom, GAMMA, scaled=True)

    u_ref, rep_ref = oracle.lbfgs(fun, np.zeros((64, 64)), oracle.SolveOptions(tol=0.0, max_iter=20))
    assert rep.iterations[0] == rep_ref.iterations == 20
    assert abs(rep.f_initial[0] - rep_ref.f_history[0]) <= 1e-5 * rep_ref.f_history[0]
    assert abs(rep.f_final[0] - rep_ref.f_history[-1]) <= 1e-4 * rep_ref.f_history[-1], \
        (rep.f_final[0], rep_ref.f_history[-1])
    h = G.unpack_volume(vol)[0][0]
    s_mu = float(np.asarray(geom.scale)[0])
    assert rel_l2(h, u_ref * s_mu) <= 2e-2


def test_clearing_the_table_restores_the_gaussian_flat():
    from paper_2202_08627_gb300 import ei
    probs = _problems(SHAPES[:2], 1300)
    G = _gpu(probs)
    vol = G.pack_volume([p[0].truth for p in probs])
    a, b = G.empty("meas"), G.empty("meas")
    ei.ei_set_flat_table(G, None)
    ei.ei_forward(G, vol, a)
    G2 = gpu_geometry([p[0] for p in probs], [p[1] for p in probs])     # never had a table
    ei.ei_forward(G2, vol, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    # a device-resident table gives the same model as the host copy
    tab = np.concatenate([p[1].flat_table for p in probs]).astype(np.float32)
    ei.ei_set_flat_table(G, torch.from_numpy(tab).cuda())
    ei.ei_forward(G, vol, a)
    ei.ei_set_flat_table(G2, tab)
    ei.ei_forward(G2, vol, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_set_flat_table_rejects_bad_sizes():
    from paper_2202_08627_gb300 import ei
    probs = _problems([(16, 8, 24, 3)], 1400, offsets=False)
    G = _gpu(probs)
    with pytest.raises(ei.EIError):
        ei.ei_set_flat_table(G, np.ones((24, 3), np.float32))
    with pytest.raises(ei.EIError):
        ei.ei_set_flat_table(G, np.ones((24, 65537), np.float32))
    with pytest.raises(ValueError):
        ei.ei_set_flat_table(G, np.ones((23, 33), np.float32))
