"""Pins for the oracle's finite-difference derivative D, the IC model (Eq. 2
with the Eq. 4 offsets and the scatter broadening) and the cost S of Eq. 5
with its gradient.

Anchors: exactness of the central difference on quadratics, an explicit dense
D, the reduction of the model to the flat IC when the sample is absent, the
Beer-Lambert factor alone, the conserved IC area and the IC's first and second
moments (which fix the refraction shift and the broadening), the gauge
invariance of Eq. 4 under (m_o + a, m_r - a), and central finite differences
of S for the gradient.
"""
import numpy as np
import pytest

from paper_2202_08627_gb300 import inputs
from tests.problems import oracle_geometry, small_problem


# ----------------------------------------------------------------- D, D^T
def test_deriv_exact_on_quadratics(oracle):
    pitch = 0.013
    t = np.arange(17) * pitch
    p = 0.3 - 2.0 * t + 5.0 * t * t
    d = oracle.deriv(p[None, :], pitch)[0]
    np.testing.assert_allclose(d[1:-1], -2.0 + 10.0 * t[1:-1], rtol=1e-12)
    lin = 0.7 + 3.0 * t
    dl = oracle.deriv(lin[None, :], pitch)[0]
    np.testing.assert_allclose(dl, np.full(17, 3.0), rtol=1e-12)


@pytest.mark.parametrize("nd", [1, 2, 3, 7])
def test_deriv_transpose_dense(oracle, nd):
    pitch = 0.5
    D = np.stack([oracle.deriv(np.eye(nd)[k][None, :], pitch)[0] for k in range(nd)], axis=1)
    g = inputs.uniform_noise((3, nd), 11)
    np.testing.assert_allclose(oracle.deriv_T(g, pitch), g @ D, rtol=0, atol=1e-13)
    x = inputs.uniform_noise((3, nd), 12)
    assert abs(np.vdot(oracle.deriv(x, pitch), g) - np.vdot(x, oracle.deriv_T(g, pitch))) < 1e-12


# ----------------------------------------------------------------- IC model
def _flat(geom):
    """The flat IC f(t, m) = A exp(-(m - c)^2 / (2 w^2)), [M][n_det]."""
    m = geom.m[:, None]
    return geom.flat_A[None, :] * np.exp(-(m - geom.flat_c[None, :]) ** 2 / (2 * geom.flat_w[None, :] ** 2))


def test_no_sample_gives_flat_ic(oracle):
    spec, geom, _ = small_problem(n_m=5)
    s = oracle.ic_model(np.zeros((3, geom.n_theta, geom.n_det)), geom)
    f = _flat(geom)
    for a in range(geom.n_theta):
        np.testing.assert_array_equal(s[:, a, :], f)


def test_attenuation_only_is_beer_lambert(oracle):
    spec, geom, _ = small_problem(n_m=5)
    P = np.zeros((3, geom.n_theta, geom.n_det))
    P[0] = inputs.uniform_noise((geom.n_theta, geom.n_det), 13, 0.0, 2.0)
    s = oracle.ic_model(P, geom)
    np.testing.assert_allclose(s, np.exp(-P[0])[None] * _flat(geom)[:, None, :], rtol=1e-14)


def _dense_m_geometry(spec, kappa=inputs.KAPPA):
    geom = oracle_geometry(spec, kappa=kappa)
    geom.m = np.linspace(-4.0, 4.0, 8001)
    return geom


def test_ic_area_and_moments(oracle):
    """With dense m, the IC's area is exp(-R mu) A w sqrt(2 pi) whatever the
    refraction and scatter; its centroid is c + (z/period) dR[delta]/dt and its
    variance w^2 + kappa R[sigma]."""
    spec = inputs.make_slice(5, 8, 2, 9, 3)
    geom = _dense_m_geometry(spec)
    t = (np.arange(9) - 4) * spec.pitch
    P = np.zeros((3, 2, 9))
    P[0] = 0.4
    slope = 2.0e-6                      # R[delta] linear in t -> constant derivative
    P[1] = slope * t[None, :]
    P[2] = 0.3
    s = oracle.ic_model(P, geom)        # [M][2][9]
    dm = geom.m[1] - geom.m[0]
    area = s.sum(axis=0) * dm
    np.testing.assert_allclose(area, np.exp(-0.4) * spec.flat_A * spec.flat_w * np.sqrt(2 * np.pi) *
                               np.ones((2, 1)), rtol=1e-8)
    mean = (geom.m[:, None, None] * s).sum(axis=0) * dm / area
    shift = geom.z_over_p * slope
    np.testing.assert_allclose(mean, (spec.flat_c + shift) * np.ones((2, 1)), rtol=0, atol=1e-9)
    var = ((geom.m[:, None, None] - mean[None]) ** 2 * s).sum(axis=0) * dm / area
    np.testing.assert_allclose(var, (spec.flat_w ** 2 + geom.kappa * 0.3) * np.ones((2, 1)), rtol=1e-8)


def test_drift_and_ring_shift_the_ic(oracle):
    """m_o(theta) and m_r(t) of Eq. 4 move the IC centroid by m_o + m_r."""
    spec = inputs.make_slice(6, 8, 3, 7, 3)
    geom = _dense_m_geometry(spec)
    geom.m_o = np.array([0.05, -0.1, 0.0])
    geom.m_r = np.linspace(-0.03, 0.04, 7)
    s = oracle.ic_model(np.zeros((3, 3, 7)), geom)
    mean = (geom.m[:, None, None] * s).sum(axis=0) / s.sum(axis=0)
    ref = spec.flat_c[None, :] + geom.m_o[:, None] + geom.m_r[None, :]
    np.testing.assert_allclose(mean, ref, rtol=0, atol=1e-9)


def test_gauge_invariance_of_offsets(oracle):
    """S is unchanged under (m_o + a, m_r - a), the ambiguity the paper points
    out for Eq. 4."""
    spec, geom, s_exp = small_problem(seed=2)
    x = spec.truth * 0.9
    geom.m_o = inputs.uniform_noise(geom.n_theta, 20, -0.05, 0.05)
    geom.m_r = inputs.uniform_noise(geom.n_det, 21, -0.05, 0.05)
    S1, _ = oracle.objective_grad(x, s_exp, geom, want_grad=False)
    geom.m_o = geom.m_o + 0.0371
    geom.m_r = geom.m_r - 0.0371
    S2, _ = oracle.objective_grad(x, s_exp, geom, want_grad=False)
    assert abs(S1 - S2) <= 1e-12 * abs(S1)


def test_variance_domain_guard(oracle):
    spec, geom, s_exp = small_problem()
    x = np.zeros((3, geom.n, geom.n))
    x[2] = -50.0                               # drives V below 0.01 w^2
    S, _ = oracle.objective_grad(x, s_exp, geom, want_grad=False)
    assert S == np.inf


# ----------------------------------------------------------------- S and grad S
def test_objective_is_regulariser_on_exact_data(oracle):
    spec, geom, _ = small_problem()
    x = spec.truth
    s_exp = oracle.forward(x, geom)
    S, _ = oracle.objective_grad(x, s_exp, geom, want_grad=False)
    reg = sum(geom.lam[c] * np.sum((x[c] / geom.scale[c]) ** 2) for c in range(3))
    assert abs(S - reg) <= 1e-12 * reg


def test_objective_residual_value(oracle):
    """S - regulariser equals the plain sum of squared residuals of Eq. 5."""
    spec, geom, s_exp = small_problem(seed=4)
    x = spec.truth * 1.1
    S, _ = oracle.objective_grad(x, s_exp, geom, want_grad=False)
    reg = sum(geom.lam[c] * np.sum((x[c] / geom.scale[c]) ** 2) for c in range(3))
    resid = np.sum((oracle.forward(x, geom) - s_exp) ** 2)
    assert abs((S - reg) - resid) <= 1e-12 * resid


@pytest.mark.parametrize("scaled", [True, False])
def test_gradient_central_differences(oracle, scaled):
    """Every coordinate of grad S against (S(u + h e) - S(u - h e)) / 2h,
    h = 1e-6 in the solver's scaled variables, on a tiny problem."""
    spec, geom, s_exp = small_problem(seed=1, n=8, n_theta=6, n_det=12, n_m=3)
    geom.m_o = inputs.uniform_noise(geom.n_theta, 30, -0.02, 0.02)
    geom.m_r = inputs.uniform_noise(geom.n_det, 31, -0.02, 0.02)
    scale = geom.scale[:, None, None]
    u = spec.truth / scale * 0.8 + 0.05 * inputs.uniform_noise(spec.truth.shape, 32)
    x = u if scaled else u * scale
    S, g = oracle.objective_grad(x, s_exp, geom, scaled=scaled)
    h = 1e-6
    fd = np.zeros_like(u)
    for idx in np.ndindex(*u.shape):
        du = np.zeros_like(u)
        du[idx] = h
        step = du if scaled else du * scale
        Sp, _ = oracle.objective_grad(x + step, s_exp, geom, want_grad=False, scaled=scaled)
        Sm, _ = oracle.objective_grad(x - step, s_exp, geom, want_grad=False, scaled=scaled)
        fd[idx] = (Sp - Sm) / (2 * h)
    gu = g if scaled else g * scale            # chain rule to the scaled variables
    err = np.linalg.norm(gu - fd) / np.linalg.norm(fd)
    assert err <= 1e-6, err


def test_ic_gradient_against_projection_differences(oracle):
    """dS/dP from ic_objective_grad against central differences in P."""
    spec, geom, s_exp = small_problem(seed=3, n_m=4)
    P = spec.P_exact * 0.9
    S, gP = oracle.ic_objective_grad(P, s_exp, geom)
    rng_idx = [(c, a, j) for c in range(3) for a in (0, 3) for j in (0, 1, 5, 11)]
    for (c, a, j) in rng_idx:
        h = 1e-6 * (1e-6 if c == 1 else 1.0)
        dP = np.zeros_like(P)
        dP[c, a, j] = h
        Sp, _ = oracle.ic_objective_grad(P + dP, s_exp, geom, want_grad=False)
        Sm, _ = oracle.ic_objective_grad(P - dP, s_exp, geom, want_grad=False)
        fd = (Sp - Sm) / (2 * h)
        assert abs(gP[c, a, j] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gP[c]).max()), (c, a, j)
