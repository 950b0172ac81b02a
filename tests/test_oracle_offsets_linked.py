"""Oracle pins for the terms of Eq. 4 beyond the three-channel model: the
gradient with respect to the drift m_o(theta) and the ring term m_r(t), and
the linked single unknown h (mu = h, delta = gamma h, no scatter).

Pins: central differences of S in m_o, m_r and h on tiny inputs; the identity
sum_theta dS/dm_o = sum_t dS/dm_r, which is the derivative of the gauge
invariance S(m_o + a, m_r - a) = S(m_o, m_r) the paper points out for Eq. 4;
and the linked cost against the three-channel cost at (h, gamma h, 0), whose
own pins (flat IC at zero volume, Beer-Lambert, moments, differences) live in
test_oracle_model.py."""
import numpy as np
import pytest

from paper_2202_08627_gb300 import inputs
from tests.problems import small_problem

GAMMA = 5e-7          # delta / mu in cm: mu in [0, 2] / cm gives delta in [0, 1e-6]


def _offsets(geom, seed):
    geom.m_o = inputs.uniform_noise(geom.n_theta, seed, -0.04, 0.04)
    geom.m_r = inputs.uniform_noise(geom.n_det, seed + 1, -0.04, 0.04)


def test_offset_gradients_central_differences(oracle):
    spec, geom, s_exp = small_problem(seed=11, n=8, n_theta=6, n_det=12, n_m=3)
    _offsets(geom, 40)
    x = spec.truth * 0.85
    g_mo, g_mr = oracle.offset_grads(x, s_exp, geom)
    h = 1e-6
    fd_mo, fd_mr = np.zeros(geom.n_theta), np.zeros(geom.n_det)
    base_mo, base_mr = geom.m_o.copy(), geom.m_r.copy()
    for a in range(geom.n_theta):
        for sgn in (1, -1):
            geom.m_o = base_mo.copy()
            geom.m_o[a] += sgn * h
            fd_mo[a] += sgn * oracle.objective_grad(x, s_exp, geom, want_grad=False)[0] / (2 * h)
    geom.m_o = base_mo
    for t in range(geom.n_det):
        for sgn in (1, -1):
            geom.m_r = base_mr.copy()
            geom.m_r[t] += sgn * h
            fd_mr[t] += sgn * oracle.objective_grad(x, s_exp, geom, want_grad=False)[0] / (2 * h)
    geom.m_r = base_mr
    assert np.linalg.norm(g_mo - fd_mo) <= 1e-6 * np.linalg.norm(fd_mo)
    assert np.linalg.norm(g_mr - fd_mr) <= 1e-6 * np.linalg.norm(fd_mr)


def test_offset_gradient_sums_agree(oracle):
    """d/da S(m_o + a, m_r - a) = 0 at every point: sum dS/dm_o = sum dS/dm_r."""
    spec, geom, s_exp = small_problem(seed=12, n=16, n_theta=20, n_det=24, n_m=5)
    _offsets(geom, 50)
    g_mo, g_mr = oracle.offset_grads(spec.truth * 1.1, s_exp, geom)
    assert abs(g_mo.sum() - g_mr.sum()) <= 1e-12 * np.abs(g_mo).sum()
    assert np.abs(g_mo).max() > 0


@pytest.mark.parametrize("scaled", [True, False])
def test_linked_gradient_central_differences(oracle, scaled):
    spec, geom, s_exp = small_problem(seed=13, n=8, n_theta=6, n_det=12, n_m=3)
    _offsets(geom, 60)
    hvol = spec.truth[0] * 0.9 + 0.05 * inputs.uniform_noise((geom.n, geom.n), 61)
    S, g = oracle.objective_grad_linked(hvol, s_exp, geom, GAMMA, scaled=scaled)
    step = 1e-6
    fd = np.zeros_like(hvol)
    for idx in np.ndindex(*hvol.shape):
        d = np.zeros_like(hvol)
        d[idx] = step
        Sp = oracle.objective_grad_linked(hvol + d, s_exp, geom, GAMMA, want_grad=False, scaled=scaled)[0]
        Sm = oracle.objective_grad_linked(hvol - d, s_exp, geom, GAMMA, want_grad=False, scaled=scaled)[0]
        fd[idx] = (Sp - Sm) / (2 * step)
    assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(fd)


def test_linked_cost_is_three_channel_cost_at_linked_volume(oracle):
    """S_linked(h) = S(h, gamma h, 0) minus the delta channel's regulariser
    (the paper regularises only h)."""
    spec, geom, s_exp = small_problem(seed=14, n=16, n_theta=12, n_det=24, n_m=5)
    _offsets(geom, 70)
    hvol = spec.truth[0]
    S_l, _ = oracle.objective_grad_linked(hvol, s_exp, geom, GAMMA, want_grad=False)
    x = np.stack([hvol, GAMMA * hvol, np.zeros_like(hvol)])
    S3, _ = oracle.objective_grad(x, s_exp, geom, want_grad=False)
    reg_delta = geom.lam[1] * np.sum((GAMMA * hvol / geom.scale[1]) ** 2)
    assert abs(S_l - (S3 - reg_delta)) <= 1e-12 * abs(S_l)
    # zero volume: only the data term of the (shifted) flat IC remains
    S0, _ = oracle.objective_grad_linked(np.zeros_like(hvol), s_exp, geom, GAMMA, want_grad=False)
    S30, _ = oracle.objective_grad(np.zeros_like(x), s_exp, geom, want_grad=False)
    assert abs(S0 - S30) <= 1e-12 * abs(S30)


def test_ring_projection_keeps_ring_frequencies_only(oracle):
    """The restriction of m_r to ring frequencies is the orthogonal projector
    onto the complement of the K lowest cosine modes: built here from the
    textbook DCT-II vectors b_k(j) = sqrt((2 - [k = 0]) / N) cos(pi k (j + 1/2) / N),
    it maps b_k (k < K) to 0 and b_k (k >= K) to itself, is symmetric and
    idempotent, and K = 1 is the zero-mean gauge of the joint solve."""
    N, K = 48, 6
    j = np.arange(N)
    B = np.stack([np.sqrt((2.0 - (k == 0)) / N) * np.cos(np.pi * k * (j + 0.5) / N) for k in range(N)])
    np.testing.assert_allclose(B @ B.T, np.eye(N), atol=1e-12)
    Pm = np.stack([oracle.ring_project(e, K) for e in np.eye(N)])      # the projector's matrix
    for k in range(N):
        want = np.zeros(N) if k < K else B[k]
        np.testing.assert_allclose(oracle.ring_project(B[k], K), want, atol=1e-12)
    np.testing.assert_allclose(Pm, Pm.T, atol=1e-12)
    np.testing.assert_allclose(Pm @ Pm, Pm, atol=1e-12)
    g = inputs.uniform_noise(N, 77)
    np.testing.assert_allclose(oracle.ring_project(g, 1), g - g.mean(), atol=1e-12)
    np.testing.assert_array_equal(oracle.ring_project(g, 0), g)
