"""Pins for the image-quality measures (CNR of Eq. 7, FRC of Eq. 6)."""
import numpy as np

from paper_2202_08627_gb300 import inputs, metrics


def test_cnr_of_two_noisy_plateaus():
    n = 64
    m1 = metrics.disc_mask(n, 20, 20, 8)
    m2 = metrics.disc_mask(n, 44, 40, 8)
    noise = inputs.uniform_noise((n, n), 5, -1.0, 1.0) * np.sqrt(3.0) * 0.1   # std 0.1
    img = noise.copy()
    img[m1] += 1.0
    img[m2] += 0.5
    a, b = img[m1], img[m2]
    ref = abs(a.mean() - b.mean()) / np.sqrt(a.std() ** 2 + b.std() ** 2)
    assert abs(metrics.cnr(img, m1, m2) - ref) <= 1e-12 * ref
    assert 2.5 < metrics.cnr(img, m1, m2) < 4.5          # 0.5 / (0.1 sqrt 2) = 3.5


def test_frc_of_identical_images_is_one():
    img = inputs.uniform_noise((48, 48), 6)
    np.testing.assert_allclose(metrics.frc(img, img), 1.0, atol=1e-12)


def test_frc_of_independent_noise_is_small():
    n = 128
    a = inputs.uniform_noise((n, n), 7)
    b = inputs.uniform_noise((n, n), 8)
    c = metrics.frc(a, b)
    rings = np.arange(len(c))
    counts = np.maximum(2 * np.pi * rings, 1)
    assert np.all(np.abs(c[4:]) < 5.0 / np.sqrt(counts[4:]))
    assert abs(c[4:].mean()) < 0.02


def test_frc_resolution_of_a_blurred_object():
    """Two noisy copies of a smooth object: the FRC stays near 1 where the
    object's spectrum dominates the noise and drops where the noise takes
    over; stronger noise lowers the resolution (more pixels per period)."""
    n = 128
    y, x = np.mgrid[0:n, 0:n] - n / 2
    obj = np.exp(-(x ** 2 + y ** 2) / (2 * 6.0 ** 2))
    res = []
    for amp in (1e-4, 1e-2):
        a = obj + amp * inputs.uniform_noise((n, n), 9)
        b = obj + amp * inputs.uniform_noise((n, n), 10)
        res.append(metrics.frc_resolution(metrics.frc(a, b), n))
    assert 2.0 <= res[0] < res[1]
