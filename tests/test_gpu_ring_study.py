"""The synthetic ring-artefact study through the library (the paper's
"Experimental improvements" section: flat ICs from noisy flat scans leave
per-pixel errors that become rings; the ring term m_r(t) of Eq. 4 absorbs
them).  A small case of the study's setup: three granules, one mask position
on the IC slope, the homogeneous-sample model (mu = h, delta = gamma h), the
flat IC fitted per pixel to one noisy flat scan.  The reconstruction solves
for h and m_r together, with m_r restricted to ring frequencies (its steps
orthogonal to the lowest DCT-II modes across the detector); over its first
ten iterations it must follow the FP64 oracle running the same algorithm,
keep m_r free of those modes, and give the study's measures.
"""
import numpy as np
import pytest

import oracle
from paper_2202_08627_gb300 import inputs, metrics, ring_study
from tests.problems import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build
    build.build()


def _case(n=64, n_theta=60, seed=5):
    theta = inputs.angles(n_theta)
    pitch = inputs.pitch_for(n)
    A, c, w = inputs.flat_ic(seed, n)

    def geom(flat, m_r=None):
        return oracle.Geometry(n=n, n_theta=n_theta, n_det=n, pitch=pitch, theta=theta,
                               m=np.array([ring_study.SLOPE_M]), z_cm=inputs.Z_CM,
                               period_cm=inputs.PERIOD_CM, kappa=inputs.KAPPA, flat_A=flat[0],
                               flat_c=flat[1], flat_w=flat[2], lam=np.full(3, inputs.LAMBDA),
                               scale=np.array(inputs.SCALE), m_r=m_r)

    P = inputs.ellipse_line_integrals(ring_study.phantom(), theta, n, pitch)
    s_exp = inputs.poisson_noise(oracle.ic_model(P, geom((A, c, w))), seed)
    flat = ring_study.estimate_flat(ring_study.flat_scans(A, c, w, 1, seed + 1))
    return theta, flat, s_exp, geom


ITERS = 10     # the FP64 objective still falls by > 8e-7 relative per iteration here,
               # within what the FP32 objective resolves (after ~12 it falls by < 1e-7)


@pytest.mark.parametrize("K", [4, 1])
def test_ring_restricted_m_r_follows_the_oracle(K):
    from paper_2202_08627_gb300 import ei
    n, n_theta, osc, gam = 64, 60, 0.01, ring_study.GAMMA
    theta, flat, s_exp, geom = _case(n, n_theta)
    G = ring_study.geometry(n, theta, *flat)
    ei.ei_set_linked(G, gam)
    ei.ei_set_offset_unknowns(G, ei.EI_OFFSET_MR, osc)
    ei.ei_set_ring_modes(G, K)
    vol = G.empty("vol")
    rep = ei.ei_reconstruct(G, G.pack_meas([s_exp]), vol, tol=0.0, max_iter=ITERS)
    _, m_r = ei.ei_get_offsets(G)

    og = geom(flat)
    s_mu = inputs.SCALE[0]
    nv = n * n

    def fun(wv):
        h = wv[:nv].reshape(n, n)
        og.m_r = wv[nv:] * osc
        S, gh = oracle.objective_grad_linked(h, s_exp, og, gam, scaled=True)
        x = np.stack([h * s_mu, gam * h * s_mu, np.zeros_like(h)])
        _, g_mr = oracle.offset_grads(x, s_exp, og)
        return S, np.concatenate([gh.ravel(), osc * oracle.ring_project(g_mr, K)])

    w_ref, rep_ref = oracle.lbfgs(fun, np.zeros(nv + n), oracle.SolveOptions(tol=0.0, max_iter=ITERS))
    assert rep.iterations[0] == rep_ref.iterations == ITERS
    assert abs(rep.f_initial[0] - rep_ref.f_history[0]) <= 1e-5 * rep_ref.f_history[0]
    assert abs(rep.f_final[0] - rep_ref.f_history[-1]) <= 1e-4 * rep_ref.f_history[-1], \
        (rep.f_final[0], rep_ref.f_history[-1])
    assert rel_l2(m_r, w_ref[nv:] * osc) <= 2e-2
    # m_r started at 0 and keeps no component along the K lowest modes
    from scipy.fft import dct
    coeffs = dct(np.asarray(m_r, dtype=np.float64), type=2, norm="ortho")
    assert np.all(np.abs(coeffs[:K]) <= 1e-5 * np.linalg.norm(coeffs)), coeffs[:K]
    # the study's measures of the reconstruction
    h = G.unpack_volume(vol)[0][0]
    half = 0.5 * n
    masks = [metrics.disc_mask(n, half - y * half, half + x * half, 0.6 * r * half)
             for (x, y, r, _) in ring_study.GRANULES]
    assert np.isfinite(metrics.cnr(h, masks[0], masks[2]))
    G.close()


def test_ring_modes_argument_checks():
    from paper_2202_08627_gb300 import ei
    theta, flat, _, _ = _case(32, 16)
    G = ring_study.geometry(32, theta, *flat)
    for bad in (-1, 33, 1025):
        with pytest.raises(ei.EIError) as err:
            ei.ei_set_ring_modes(G, bad)
        assert err.value.status == ei.EI_ERR_ARG
    ei.ei_set_ring_modes(G, 32)
    ei.ei_set_ring_modes(G, 0)
    G.close()
