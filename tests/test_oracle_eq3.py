"""Oracle pins for the paper's single-shot retrieval (Eq. 3), read as the
exact inverse of Eq. 4 linearised at one mask position:
s / f = (1 + a d/dt) T with a = (z/period) gamma f'(m) / f(m).

Pins: without phase (gamma = 0) the retrieval is Beer-Lambert exactly; for a
smooth transmission profile T(t) and y = T + a T' written with the analytic
derivative, the Fourier division returns T to spectral accuracy (a wrong sign
of a, q or the transform convention fails it); a against a central difference
of the pixel-averaged flat IC in m."""
import numpy as np

from paper_2202_08627_gb300 import inputs
from tests.problems import oracle_geometry


def _geom(n=32, n_theta=12, n_det=256, n_m=7, seed=3, uniform=True):
    spec = inputs.make_slice(seed, n, n_theta, n_det, n_m)
    geom = oracle_geometry(spec)
    if uniform:                                   # one flat IC for every pixel
        geom.flat_A = np.full(n_det, 1e4)
        geom.flat_c = np.zeros(n_det)
        geom.flat_w = np.full(n_det, 0.25)
    return spec, geom


def test_without_phase_it_is_beer_lambert(oracle):
    spec, geom = _geom(uniform=False)
    P_true = spec.P_exact[0]
    s_exp = oracle.ic_model(np.stack([P_true, np.zeros_like(P_true), np.zeros_like(P_true)]), geom)
    P, h = oracle.single_shot_eq3(s_exp, geom, 2, 0.0)
    np.testing.assert_allclose(P, P_true, rtol=0, atol=1e-12)
    np.testing.assert_allclose(h, oracle.fbp(P_true[None], geom)[0], rtol=0, atol=1e-10)


def test_fourier_division_inverts_one_plus_a_derivative(oracle):
    spec, geom = _geom()
    k, gamma = 1, 5e-6                              # m = -1/3: on the slope of the IC
    a = oracle.eq3_slope(geom, k, gamma)
    assert 3 * geom.pitch < abs(a) < 30 * geom.pitch
    nd = geom.n_det
    t = (np.arange(nd) - (nd - 1) / 2.0) * geom.pitch
    rows = []
    for t0, amp, sig in [(0.0, 0.3, 8.0), (-0.3, 0.5, 12.0), (0.45, 0.2, 6.0)]:
        sg = sig * geom.pitch
        g = np.exp(-(t - t0) ** 2 / (2 * sg * sg))
        T = 1.0 - amp * g
        dT = amp * g * (t - t0) / (sg * sg)
        rows.append((T, T + a * dT))
    f = oracle.flat_at_masks(geom)[k]
    s_exp = np.zeros((geom.n_m, len(rows), nd))
    s_exp[k] = np.stack([y for _, y in rows]) * f[None, :]
    geom.n_theta = len(rows)
    geom.theta = geom.theta[:len(rows)]
    P, _ = oracle.single_shot_eq3(s_exp, geom, k, gamma)
    for (T, _), p in zip(rows, P):
        np.testing.assert_allclose(np.exp(-p), T, rtol=0, atol=1e-9)


def test_slope_length_against_differences_of_the_flat(oracle):
    spec, geom = _geom(uniform=False)
    k, gamma, h = 1, 3e-7, 1e-5
    m = geom.m[k]

    def fbar(mm):
        return np.mean(geom.flat_A * np.exp(-(mm - geom.flat_c) ** 2 / (2 * geom.flat_w ** 2)))
    ref = geom.z_over_p * gamma * (fbar(m + h) - fbar(m - h)) / (2 * h) / fbar(m)
    assert abs(oracle.eq3_slope(geom, k, gamma) - ref) <= 1e-7 * abs(ref)
