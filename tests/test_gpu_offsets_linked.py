"""The terms of Eq. 4 beyond the three-channel model on the GPU, against the
FP64 oracle: the gradient with respect to the drift m_o(theta) and the ring
term m_r(t) (ei_offset_grad), the gauge ambiguity the paper points out for
them, the linked single unknown h (mu = h, delta = gamma h, sigma = 0;
ei_set_linked) through ei_forward, ei_objective_grad and ei_reconstruct, and
the offsets as unknowns of the solver (ei_set_offset_unknowns)."""
import numpy as np
import pytest

import oracle
from paper_2202_08627_gb300 import inputs
from tests.problems import gpu_geometry, measured, oracle_geometry, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GAMMA = 5e-7          # delta / mu in cm: mu in [0, 2] / cm gives delta in [0, 1e-6]
SHAPES = [(64, 90, 96, 5), (37, 23, 61, 5), (128, 180, 192, 5), (20, 7, 131, 5)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build
    build.build()


def _with_offsets(shapes, seed0, shift=0.0):
    probs = []
    for i, sh in enumerate(shapes):
        spec = inputs.make_slice(seed0 + i, *sh)
        m_o = inputs.uniform_noise(spec.n_theta, seed0 + 100 + i, -0.04, 0.04) + shift
        m_r = inputs.uniform_noise(spec.n_det, seed0 + 200 + i, -0.04, 0.04) - shift
        geom = oracle_geometry(spec, m_o=m_o, m_r=m_r)
        probs.append((spec, geom, measured(spec, geom)))
    return probs


def test_offset_gradients_match_oracle():
    from paper_2202_08627_gb300 import ei
    probs = _with_offsets(SHAPES, 300)
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    xs = [sp.truth * 0.9 for sp in specs]
    g_mo, g_mr = ei.ei_offset_grad(G, G.pack_volume(xs), G.pack_meas(meas))
    g_mo, g_mr = g_mo.cpu().numpy(), g_mr.cpu().numpy()
    o_th = o_px = 0
    for (spec, geom, s_exp), x in zip(probs, xs):
        r_mo, r_mr = oracle.offset_grads(x, s_exp, geom)
        assert rel_l2(g_mo[o_th:o_th + spec.n_theta], r_mo) <= 1e-4, (spec.n, "m_o")
        assert rel_l2(g_mr[o_px:o_px + spec.n_det], r_mr) <= 1e-4, (spec.n, "m_r")
        o_th += spec.n_theta
        o_px += spec.n_det


def test_gauge_ambiguity_on_the_gpu():
    """(m_o + a, m_r - a) leaves S unchanged, and the two gradients have the
    same sum (the derivative of that invariance)."""
    from paper_2202_08627_gb300 import ei
    a, b = _with_offsets(SHAPES[:2], 400), _with_offsets(SHAPES[:2], 400, shift=0.0371)
    Ga = gpu_geometry([p[0] for p in a], [p[1] for p in a])
    Gb = gpu_geometry([p[0] for p in b], [p[1] for p in b])
    xs = [p[0].truth * 1.05 for p in a]
    meas = [p[2] for p in a]                     # the same measured data for both
    S = torch.zeros(2, 2, dtype=torch.float64, device="cuda")
    ei.ei_objective_grad(Ga, Ga.pack_volume(xs), Ga.pack_meas(meas), S[0], None)
    ei.ei_objective_grad(Gb, Gb.pack_volume(xs), Gb.pack_meas(meas), S[1], None)
    S = S.cpu().numpy()
    np.testing.assert_allclose(S[1], S[0], rtol=1e-6)
    g_mo, g_mr = ei.ei_offset_grad(Ga, Ga.pack_volume(xs), Ga.pack_meas(meas))
    g_mo, g_mr = g_mo.cpu().numpy().astype(np.float64), g_mr.cpu().numpy().astype(np.float64)
    o_th = o_px = 0
    for spec, _, _ in a:
        s_mo, s_mr = g_mo[o_th:o_th + spec.n_theta].sum(), g_mr[o_px:o_px + spec.n_det].sum()
        assert abs(s_mo - s_mr) <= 1e-4 * np.abs(g_mo[o_th:o_th + spec.n_theta]).sum()
        o_th += spec.n_theta
        o_px += spec.n_det


def _linked_problems(shapes, seed0):
    """Measured ICs of a linked phantom: P = (R h, gamma R h, 0) from the exact
    line integrals of the attenuation phantom h."""
    probs = []
    for i, sh in enumerate(shapes):
        spec = inputs.make_slice(seed0 + i, *sh)
        geom = oracle_geometry(spec, m_o=inputs.uniform_noise(spec.n_theta, seed0 + 7 + i, -0.02, 0.02))
        Ph = spec.P_exact[0]
        P = np.stack([Ph, GAMMA * Ph, np.zeros_like(Ph)])
        s_exp = inputs.poisson_noise(oracle.ic_model(P, geom), spec.seed)
        probs.append((spec, geom, s_exp))
    return probs


def test_linked_objective_gradient_and_forward_match_oracle():
    from paper_2202_08627_gb300 import ei
    probs = _linked_problems(SHAPES, 500)
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    ei.ei_set_linked(G, GAMMA)
    hs = [sp.truth[0] * 0.9 for sp in specs]
    # the delta and sigma lanes are ignored in linked mode
    vols = [np.stack([h, np.full_like(h, 123.0), np.full_like(h, -7.0)]) for h in hs]
    vol = G.pack_volume(vols)
    S = torch.zeros(G.n_slices, dtype=torch.float64, device="cuda")
    grad = G.empty("vol")
    ei.ei_objective_grad(G, vol, G.pack_meas(meas), S, grad)
    s_mod = G.empty("meas")
    ei.ei_forward(G, vol, s_mod)
    torch.cuda.synchronize()
    gv = grad.cpu().numpy()
    gs = G.unpack_volume(grad)
    sm = G.unpack_meas(s_mod)
    for i, ((spec, geom, s_exp), h) in enumerate(zip(probs, hs)):
        S_ref, g_ref = oracle.objective_grad_linked(h, s_exp, geom, GAMMA)
        assert abs(S[i].item() - S_ref) <= 1e-5 * abs(S_ref), (i, S[i].item(), S_ref)
        assert rel_l2(gs[i][0], g_ref) <= 1e-4, (i, rel_l2(gs[i][0], g_ref))
        assert not np.any(gs[i][1:]), i
        x = np.stack([h, GAMMA * h, np.zeros_like(h)])
        assert rel_l2(sm[i], oracle.forward(x, geom)) <= 1e-5
    assert not np.any(gv[:, 3])


@pytest.mark.parametrize("adj_variant", [0, 3, 5, 6, 7])
def test_linked_kernels_agree_with_the_three_channel_path(adj_variant):
    """The single-channel linked kernels against the three-channel ones on the
    same model (lambda = 0, so only the data term): S(h) = S(h, gamma h, 0),
    dS/dh = dS/dmu + gamma dS/ddelta, and the forward ICs agree; both paths in
    FP32 with different summation orders.  Adjoint variants: rows of 8 voxels,
    2 x 4 sub-patches, voxel pairs along rows and on 4 x 4 sub-patches."""
    from paper_2202_08627_gb300 import ei
    probs = _linked_problems(SHAPES, 550)
    specs = [p[0] for p in probs]
    geoms = [oracle_geometry(sp, lam=(0.0, 0.0, 0.0), m_o=p[1].m_o) for sp, p in zip(specs, probs)]
    meas = [p[2] for p in probs]
    G = gpu_geometry(specs, geoms)
    ei.ei_set_variant(G, 8, adj_variant, False)
    hs = [sp.truth[0] * 0.8 for sp in specs]
    m = G.pack_meas(meas)
    out = {}
    for mode in ("three", "linked"):
        if mode == "linked":
            ei.ei_set_linked(G, GAMMA)
            vol = G.pack_volume([np.stack([h, np.zeros_like(h), np.zeros_like(h)]) for h in hs])
        else:
            ei.ei_set_linked(G, 0.0)
            vol = G.pack_volume([np.stack([h, GAMMA * h, np.zeros_like(h)]) for h in hs])
        S = torch.zeros(G.n_slices, dtype=torch.float64, device="cuda")
        grad = G.empty("vol")
        ei.ei_objective_grad(G, vol, m, S, grad)
        s_mod = G.empty("meas")
        ei.ei_forward(G, vol, s_mod)
        torch.cuda.synchronize()
        out[mode] = (S.cpu().numpy(), G.unpack_volume(grad), G.unpack_meas(s_mod))
    S3, g3, f3 = out["three"]
    S1, g1, f1 = out["linked"]
    np.testing.assert_allclose(S1, S3, rtol=2e-6)
    for i in range(len(specs)):
        ref = g3[i][0] + GAMMA * g3[i][1]
        assert rel_l2(g1[i][0], ref) <= 2e-5, (i, rel_l2(g1[i][0], ref))
        assert rel_l2(f1[i], f3[i]) <= 1e-6, i


def test_linked_reconstruct_matches_oracle_trajectory():
    """20 L-BFGS iterations on the linked unknown from h = 0: the final
    objective agrees with the FP64 oracle's within 1e-4 relative, and the
    solution keeps the delta and sigma lanes at zero."""
    from paper_2202_08627_gb300 import ei
    (spec, geom, s_exp), = _linked_problems([(64, 90, 96, 7)], 600)
    G = gpu_geometry([spec], [geom])
    ei.ei_set_linked(G, GAMMA)
    vol = G.pack_volume([np.stack([np.zeros((64, 64)), np.full((64, 64), 5.0), np.ones((64, 64))])])
    rep = ei.ei_reconstruct(G, G.pack_meas([s_exp]), vol, tol=0.0, max_iter=20)

    def fun(u):
        return oracle.objective_grad_linked(u, s_exp, geom, GAMMA, scaled=True)

    u_ref, rep_ref = oracle.lbfgs(fun, np.zeros((64, 64)), oracle.SolveOptions(tol=0.0, max_iter=20))
    assert rep.iterations[0] == rep_ref.iterations == 20
    assert abs(rep.f_initial[0] - rep_ref.f_history[0]) <= 1e-5 * rep_ref.f_history[0]
    assert abs(rep.f_final[0] - rep_ref.f_history[-1]) <= 1e-4 * rep_ref.f_history[-1], \
        (rep.f_final[0], rep_ref.f_history[-1])
    out = G.unpack_volume(vol)[0]
    assert not np.any(out[1:])
    assert rep.f_final[0] < rep.f_initial[0]


def test_set_linked_rejects_bad_gamma():
    from paper_2202_08627_gb300 import ei
    (spec, geom, _), = _linked_problems([(16, 8, 24, 3)], 700)
    G = gpu_geometry([spec], [geom])
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(ei.EIError):
            ei.ei_set_linked(G, bad)
    ei.ei_set_linked(G, 0.0)


def test_get_offsets_returns_the_setup_values():
    from paper_2202_08627_gb300 import ei
    probs = _with_offsets(SHAPES, 800)
    specs, geoms, _ = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    m_o, m_r = ei.ei_get_offsets(G)
    np.testing.assert_array_equal(m_o, np.concatenate([g.m_o for g in geoms]).astype(np.float32))
    np.testing.assert_array_equal(m_r, np.concatenate([g.m_r for g in geoms]).astype(np.float32))


def test_joint_offsets_match_oracle_trajectory():
    """m_o and m_r among the unknowns (the paper's joint minimisation of Eq. 5
    over the volume and Eq. 4's offsets), with the gauge fixed by keeping the
    mean of m_r: 20 L-BFGS iterations from zero volume and zero offsets agree
    with the FP64 oracle running the same algorithm on the same vector
    [u_volume, m_o / 0.01, m_r / 0.01]."""
    from paper_2202_08627_gb300 import ei
    spec = inputs.make_slice(900, 64, 90, 96, 7)
    truth_geom = oracle_geometry(spec, m_o=inputs.uniform_noise(90, 901, -0.05, 0.05),
                                 m_r=inputs.uniform_noise(96, 902, -0.03, 0.03))
    s_exp = measured(spec, truth_geom)
    geom = oracle_geometry(spec)                          # offsets start at 0
    G = gpu_geometry([spec], [geom])
    ei.ei_set_offset_unknowns(G, ei.EI_OFFSET_MO | ei.EI_OFFSET_MR, 0.01)
    vol = G.empty("vol")
    rep = ei.ei_reconstruct(G, G.pack_meas([s_exp]), vol, tol=0.0, max_iter=20)
    m_o, m_r = ei.ei_get_offsets(G)

    n, sc, osc = 64, np.asarray(geom.scale)[:, None, None], 0.01
    nv = 3 * n * n

    def fun(w):
        u = w[:nv].reshape(3, n, n)
        geom.m_o = w[nv:nv + 90] * osc
        geom.m_r = w[nv + 90:] * osc
        S, gu = oracle.objective_grad(u, s_exp, geom, scaled=True)
        g_mo, g_mr = oracle.offset_grads(u * sc, s_exp, geom)
        g_mr = g_mr - g_mr.mean()                       # the gauge: mean of m_r fixed
        return S, np.concatenate([gu.ravel(), osc * g_mo, osc * g_mr])

    w_ref, rep_ref = oracle.lbfgs(fun, np.zeros(nv + 90 + 96), oracle.SolveOptions(tol=0.0, max_iter=20))
    assert rep.iterations[0] == rep_ref.iterations == 20
    assert abs(rep.f_initial[0] - rep_ref.f_history[0]) <= 1e-5 * rep_ref.f_history[0]
    assert abs(rep.f_final[0] - rep_ref.f_history[-1]) <= 1e-4 * rep_ref.f_history[-1], \
        (rep.f_final[0], rep_ref.f_history[-1])
    assert rel_l2(m_o, w_ref[nv:nv + 90] * osc) <= 2e-2
    assert rel_l2(m_r, w_ref[nv + 90:] * osc) <= 2e-2
    assert abs(float(m_r.mean())) <= 1e-6
    # the joint solve fits the data better than the volume alone from the same start
    G2 = gpu_geometry([spec], [oracle_geometry(spec)])
    rep2 = ei.ei_reconstruct(G2, G2.pack_meas([s_exp]), G2.empty("vol"), tol=0.0, max_iter=20)
    assert rep.f_final[0] < rep2.f_final[0]
