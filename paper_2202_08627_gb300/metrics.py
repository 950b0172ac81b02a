"""Image-quality measures of the paper's evaluation ("Experimental
improvements" and results sections), for the synthetic studies.

* ``cnr`` — contrast-to-noise ratio between two regions (Eq. 7): the absolute
  difference of the region means over the root of the summed variances.
* ``frc`` — Fourier ring correlation of two images of the same object with
  independent noise (Eq. 6, read with the sums over each ring of frequencies
  and the magnitudes in the normalisation that its printed form leaves out):
  FRC(r) = Re sum_{|k| in ring r} F1(k) F2(k)* /
           sqrt(sum_ring |F1(k)|^2 sum_ring |F2(k)|^2).
* ``frc_resolution`` — the resolution (in pixels) where a Gaussian-smoothed
  FRC curve first drops below a cutoff (the paper uses 0.5): N / r for the
  first ring r below the cutoff, the period of that spatial frequency.

NumPy on the host: these run once per study on reconstructed slices.
"""
from __future__ import annotations

import numpy as np


def disc_mask(n: int, cy: float, cx: float, radius: float) -> np.ndarray:
    """Pixels of an n x n image whose centres lie within `radius` of (cy, cx)."""
    y, x = np.mgrid[0:n, 0:n]
    return (y - cy) ** 2 + (x - cx) ** 2 <= radius * radius


def cnr(img: np.ndarray, mask1: np.ndarray, mask2: np.ndarray) -> float:
    """Eq. 7: |mean_1 - mean_2| / sqrt(std_1^2 + std_2^2) over two regions."""
    a, b = img[mask1], img[mask2]
    return float(abs(a.mean() - b.mean()) / np.sqrt(a.var() + b.var()))


def frc(img1: np.ndarray, img2: np.ndarray) -> np.ndarray:
    """FRC for integer ring radii r = 0 .. n/2 - 1 of two square images."""
    n = img1.shape[0]
    if img1.shape != (n, n) or img2.shape != (n, n):
        raise ValueError("frc needs two square images of the same size")
    F1, F2 = np.fft.fft2(img1), np.fft.fft2(img2)
    k = np.fft.fftfreq(n) * n
    r = np.rint(np.hypot(k[:, None], k[None, :])).astype(int)
    nr = n // 2
    sel = r < nr
    num = np.bincount(r[sel], weights=np.real(F1 * np.conj(F2))[sel], minlength=nr)
    d1 = np.bincount(r[sel], weights=(np.abs(F1) ** 2)[sel], minlength=nr)
    d2 = np.bincount(r[sel], weights=(np.abs(F2) ** 2)[sel], minlength=nr)
    return num / np.sqrt(np.maximum(d1 * d2, 1e-300))


def frc_resolution(curve: np.ndarray, n: int, cutoff: float = 0.5, smooth: float = 2.0) -> float:
    """Pixels per period at the first ring (after ring 0) where the FRC,
    smoothed by a Gaussian of `smooth` rings, falls below `cutoff`; the
    Nyquist period (2 pixels) if it never does."""
    r = np.arange(len(curve))
    if smooth > 0:
        w = np.exp(-0.5 * ((r[:, None] - r[None, :]) / smooth) ** 2)
        curve = (w @ curve) / w.sum(axis=1)
    below = np.nonzero(curve[1:] < cutoff)[0]
    if len(below) == 0:
        return 2.0
    return float(n / (below[0] + 1))
