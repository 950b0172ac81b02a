"""Pins for the oracle's non-iterative reconstruction (moment retrieval of
the three projections, integration of the refraction shift, Ram-Lak FBP).

Anchors: with a dense, wide set of mask positions the IC moments return the
model's projections exactly (area -> attenuation, centroid -> shift,
variance -> broadening); summing a finite difference recovers the function;
the ramp filter's discrete frequency response is close to |omega| at low
frequencies; FBP of the exact projections of a disk gives the disk; the
whole single-shot chain returns three disks, one per channel, each with its
value in its own channel.
"""
import numpy as np

import oracle
from paper_2202_08627_gb300 import inputs
from tests.problems import oracle_geometry


def test_moments_recover_projections_with_dense_m():
    spec = inputs.make_slice(4, 16, 6, 40, 3)
    geom = oracle_geometry(spec)
    geom.m = np.linspace(-4.0, 4.0, 4001)
    t = (np.arange(40) - 19.5) * spec.pitch
    P = np.zeros((3, 6, 40))
    P[0] = 0.3 + 0.2 * np.sin(np.arange(40) / 7.0)[None, :]
    P[1] = 1e-6 * np.exp(-(t / 0.05) ** 2)[None, :] * (1 + np.arange(6)[:, None] / 10)
    P[2] = 0.2 + 0.1 * np.cos(np.arange(40) / 5.0)[None, :]
    s = oracle.ic_model(P, geom)
    P_mu, shift, P_sigma = oracle.retrieve_moments(s, geom)
    np.testing.assert_allclose(P_mu, P[0], rtol=0, atol=1e-9)
    np.testing.assert_allclose(shift, geom.z_over_p * oracle.deriv(P[1], geom.pitch), rtol=0, atol=1e-9)
    np.testing.assert_allclose(P_sigma, P[2], rtol=0, atol=1e-7)


def test_integrating_the_shift_recovers_the_projection():
    spec = inputs.make_slice(4, 16, 3, 400, 3)
    geom = oracle_geometry(spec)
    t = (np.arange(400) - 199.5) * spec.pitch
    p = 1e-6 * np.exp(-(t / (60 * spec.pitch)) ** 2)
    shift = geom.z_over_p * oracle.deriv(p[None, :], geom.pitch)
    rec = oracle.integrate_shift(shift, geom)[0]
    assert np.max(np.abs(rec - p)) <= 0.02 * p.max()


def test_ramp_filter_frequency_response():
    """Filtering a sampled cosine of frequency w (cycles per pixel) scales the
    middle of the row by ~|w| / pitch, the ramp, for w well below Nyquist."""
    pitch = 0.01
    n = 512
    j = np.arange(n)
    for w in (0.02, 0.05, 0.1):
        p = np.cos(2 * np.pi * w * j)
        q = oracle.ramp_filter(p[None, :], pitch)[0]
        mid = slice(n // 4, 3 * n // 4)
        gain = np.dot(q[mid], p[mid]) / np.dot(p[mid], p[mid])
        assert abs(gain - w / pitch) <= 0.03 * w / pitch, (w, gain, w / pitch)


def test_fbp_of_a_disk():
    n, n_theta, n_det = 128, 180, 192
    spec = inputs.make_slice(0, n, n_theta, n_det, 3)
    geom = oracle_geometry(spec)
    rho, R = 1.5, 0.1
    disk = [inputs.Ellipse(0.0, 0.0, R, R, 0.0, np.array([rho, 0.0, 0.0]))]
    P = inputs.ellipse_line_integrals(disk, spec.theta, n_det, spec.pitch)
    rec = oracle.fbp(P[:1], geom)[0]
    c = (np.arange(n) - (n - 1) / 2) * spec.pitch
    r = np.hypot(c[None, :], c[:, None])
    assert abs(rec[r < 0.8 * R].mean() - rho) <= 0.02 * rho
    assert abs(rec[(r > 1.2 * R) & (r < 0.14)].mean()) <= 0.02 * rho


def test_single_shot_reconstructs_phantom_roughly():
    """Noise-free data of the small slice: the attenuation channel of the
    single-shot reconstruction correlates strongly with the phantom."""
    spec = inputs.make_slice(7, 64, 90, 96, 7)
    geom = oracle_geometry(spec)
    s = oracle.ic_model(spec.P_exact, geom)
    rec = oracle.single_shot(s, geom)
    corr = np.corrcoef(rec[0].ravel(), spec.truth[0].ravel())[0, 1]
    assert corr > 0.9, corr


def test_single_shot_recovers_each_channel_of_disks():
    """Noise-free data of three disks, one per channel at different places
    (mu 1.2 / cm left, delta 8e-7 right, sigma 1.5 at the top), measured at
    801 mask positions over +-4 periods, where the IC moments are exact: the
    composed single-shot reconstruction (moments, shift integration, Ram-Lak
    FBP) returns each disk's value inside it in its own channel and about 0
    in the other two channels there, so the channel order and every channel's
    scale are pinned, not only the correlation with the phantom."""
    n, n_theta, n_det = 96, 120, 144
    spec = inputs.make_slice(0, n, n_theta, n_det, 3)
    geom = oracle_geometry(spec)
    geom.m = np.linspace(-4.0, 4.0, 801)
    R = 0.045
    where = [(-0.08, 0.0), (0.08, 0.0), (0.0, 0.08)]
    value = [1.2, 8e-7, 1.5]
    disks = []
    for c in range(3):
        rho = np.zeros(3)
        rho[c] = value[c]
        disks.append(inputs.Ellipse(where[c][0], where[c][1], R, R, 0.0, rho))
    P = inputs.ellipse_line_integrals(disks, spec.theta, n_det, spec.pitch)
    rec = oracle.single_shot(oracle.ic_model(P, geom), geom)
    xc = (np.arange(n) - (n - 1) / 2) * spec.pitch
    X, Y = xc[None, :], xc[::-1][:, None]          # x to the right, y up (row 0 at the top)
    for c in range(3):
        inside = np.hypot(X - where[c][0], Y - where[c][1]) < 0.6 * R
        for k in range(3):
            got = rec[k][inside].mean()
            if k == c:
                assert abs(got - value[c]) <= 0.01 * value[c], (c, got, value[c])
            else:
                assert abs(got) <= 0.01 * value[k], (c, k, got, value[k])
