"""Seeded synthetic inputs shaped like the paper's edge-illumination scans.

This module is shared by the tests (which feed the FP64 oracle) and by the CUDA
path's benchmark; it holds none of the reconstruction method's arithmetic — no
projector, no illumination-curve model, no cost.  It draws:

* random-ellipse phantoms for the three channels (mu attenuation 1/cm, delta
  refractive decrement, sigma scatter), their voxelisation by 4 x 4
  supersampled coverage, and their exact (analytic) parallel-beam line
  integrals, the textbook ellipse projection (Kak & Slaney, cited for Eq. 1) —
  the measured data are built from these, not from the discrete model, so the
  reconstruction never sees its own discretisation;
* per-pixel Gaussian flat illumination curves (amplitude, centre, width);
* mask positions and projection angles;
* Poisson counting noise, given the expected normalised intensities.

Conventions (shared by value with the oracle and the CUDA library):
voxel (r, c) of an n x n slice is centred at x = (c - (n-1)/2) pitch,
y = ((n-1)/2 - r) pitch; detector pixel j at t_j = (j - (n_det-1)/2) pitch;
angle a at theta_a = a pi / n_theta; the ray (theta, t) is
{x cos theta + y sin theta = t}.  The field of view is FOV_CM = 0.32 cm for
every slice size, so pitch = FOV_CM / n.  Intensities are normalised by the
nominal flat amplitude A_REF = 1e4 counts.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

FOV_CM = 0.32          # field of view of every slice (cm)
A_REF = 1.0e4          # nominal flat-field counts; intensities are divided by it
Z_CM = 20.0            # sample-detector distance (paper, "Experimental improvements")
PERIOD_CM = 48e-4      # detector-mask pitch used as the IC period (same section)
KAPPA = 0.1            # IC variance (period^2) added per unit of R[sigma]
LAMBDA = 1e-2          # regulariser weight (paper: lambda = 1e-2)
SCALE = (1.0, 1e-6, 1.0)   # variable scaling u = x / scale per channel

MU_RANGE = (0.0, 2.0)      # 1/cm
DELTA_RANGE = (0.0, 1e-6)
SIGMA_RANGE = (0.0, 2.0)

_PURPOSE_PHANTOM, _PURPOSE_FLAT, _PURPOSE_NOISE, _PURPOSE_MISC = 1, 2, 3, 4


def _rng(seed: int, purpose: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), purpose]))


@dataclass
class Ellipse:
    x0: float
    y0: float
    a: float
    b: float
    phi: float
    values: np.ndarray   # [3] (mu, delta, sigma)


def angles(n_theta: int) -> np.ndarray:
    """theta_a = a pi / n_theta, a = 0..n_theta-1 (180 degrees)."""
    return np.arange(n_theta, dtype=np.float64) * np.pi / n_theta


def mask_positions(n_m: int) -> np.ndarray:
    """M mask positions spread over one IC period: -0.5 + k / (M - 1)."""
    if n_m == 1:
        return np.zeros(1)
    return -0.5 + np.arange(n_m, dtype=np.float64) / (n_m - 1)


def pitch_for(n: int) -> float:
    return FOV_CM / n


def round_up4(n: int) -> int:
    return (n + 3) // 4 * 4


def random_ellipses(seed: int, n_ellipses: int = 8, fov: float = FOV_CM,
                    ranges: Sequence = (MU_RANGE, DELTA_RANGE, SIGMA_RANGE)) -> List[Ellipse]:
    """8 ellipses: centre |c| <= 0.45 fov/2, semi-axes in [0.05, 0.35] fov/2,
    rotation in [0, pi), values uniform per channel; redrawn until inside the
    inscribed disk."""
    rng = _rng(seed, _PURPOSE_PHANTOM)
    R = 0.5 * fov
    out = []
    while len(out) < n_ellipses:
        rad = 0.45 * R * np.sqrt(rng.uniform())
        ang = rng.uniform(0.0, 2.0 * np.pi)
        x0, y0 = rad * np.cos(ang), rad * np.sin(ang)
        a, b = rng.uniform(0.05 * R, 0.35 * R, size=2)
        phi = rng.uniform(0.0, np.pi)
        vals = np.array([rng.uniform(lo, hi) for (lo, hi) in ranges])
        if np.hypot(x0, y0) + max(a, b) > R:
            continue
        out.append(Ellipse(float(x0), float(y0), float(a), float(b), float(phi), vals))
    return out


def voxelize(ellipses: Sequence[Ellipse], n: int, fov: float = FOV_CM,
             supersample: int = 4) -> np.ndarray:
    """[3][n][n] voxel values: ellipse values times the fraction of
    supersample^2 sub-points of each voxel that fall inside; overlaps add."""
    pitch = fov / n
    sub = (np.arange(supersample) + 0.5) / supersample - 0.5     # offsets in voxel units
    idx = np.arange(n) - 0.5 * (n - 1)
    # sub-point grid: x depends on (c, sc), y on (r, sr); y = -(r - (n-1)/2) pitch
    Xg = ((idx[:, None] + sub[None, :]) * pitch).reshape(1, n, 1, supersample)
    Y = (-(idx[:, None] + sub[None, :]) * pitch).reshape(n, 1, supersample, 1)
    out = np.zeros((3, n, n))
    for e in ellipses:
        dx, dy = Xg - e.x0, Y - e.y0
        cp, sp = np.cos(e.phi), np.sin(e.phi)
        xr = dx * cp + dy * sp
        yr = -dx * sp + dy * cp
        inside = (xr / e.a) ** 2 + (yr / e.b) ** 2 <= 1.0
        frac = inside.mean(axis=(2, 3))
        out += e.values[:, None, None] * frac[None]
    return out


def ellipse_line_integrals(ellipses: Sequence[Ellipse], theta: np.ndarray,
                           n_det: int, pitch: float) -> np.ndarray:
    """Exact line integrals [3][n_theta][n_det] of the ellipse phantom at the
    detector-pixel centres: 2 rho a b sqrt(a2 - t'^2) / a2 with
    a2 = a^2 cos^2(theta - phi) + b^2 sin^2(theta - phi) and
    t' = t - (x0 cos theta + y0 sin theta)."""
    t = (np.arange(n_det) - 0.5 * (n_det - 1)) * pitch
    th = np.asarray(theta, dtype=np.float64)[:, None]
    out = np.zeros((3, len(theta), n_det))
    for e in ellipses:
        al = th - e.phi
        a2 = (e.a * np.cos(al)) ** 2 + (e.b * np.sin(al)) ** 2
        tp = t[None, :] - (e.x0 * np.cos(th) + e.y0 * np.sin(th))
        rad = np.clip(a2 - tp * tp, 0.0, None)
        chord = 2.0 * e.a * e.b * np.sqrt(rad) / a2
        out += e.values[:, None, None] * chord[None]
    return out


def flat_ic(seed: int, n_det: int):
    """Per-pixel Gaussian flat IC, amplitude normalised by A_REF:
    A = 1 + 0.05 U[-1,1], centre c = 0.1 U[-1,1] period,
    width (std) w = 0.25 + 0.02 U[-1,1] period."""
    rng = _rng(seed, _PURPOSE_FLAT)
    A = 1.0 + 0.05 * rng.uniform(-1.0, 1.0, n_det)
    c = 0.1 * rng.uniform(-1.0, 1.0, n_det)
    w = 0.25 + 0.02 * rng.uniform(-1.0, 1.0, n_det)
    return A, c, w


def poisson_noise(expected: np.ndarray, seed: int, a_ref: float = A_REF) -> np.ndarray:
    """Counts ~ Poisson(a_ref * expected), returned divided by a_ref."""
    rng = _rng(seed, _PURPOSE_NOISE)
    lam = np.clip(np.asarray(expected, dtype=np.float64) * a_ref, 0.0, None)
    return rng.poisson(lam).astype(np.float64) / a_ref


def uniform_noise(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Plain uniform draws for test vectors (adjoint checks, random points)."""
    return _rng(seed, _PURPOSE_MISC).uniform(lo, hi, size=shape)


@dataclass
class SliceSpec:
    """Everything about one synthetic slice except the measured ICs (those
    need the IC model, which lives on the oracle or the CUDA side)."""
    seed: int
    n: int
    n_theta: int
    n_det: int
    n_m: int
    pitch: float
    theta: np.ndarray
    m: np.ndarray
    flat_A: np.ndarray
    flat_c: np.ndarray
    flat_w: np.ndarray
    ellipses: List[Ellipse]
    truth: np.ndarray          # [3][n][n] voxelised phantom
    P_exact: np.ndarray        # [3][n_theta][n_det] analytic projections


def make_slice(seed: int, n: int, n_theta: int, n_det: int, n_m: int,
               flat_seed: int | None = None) -> SliceSpec:
    pitch = pitch_for(n)
    th = angles(n_theta)
    ell = random_ellipses(seed)
    A, c, w = flat_ic(seed if flat_seed is None else flat_seed, n_det)
    return SliceSpec(seed, n, n_theta, n_det, n_m, pitch, th, mask_positions(n_m),
                     A, c, w, ell, voxelize(ell, n), ellipse_line_integrals(ell, th, n_det, pitch))


# ---------------------------------------------------------------------------
# Device versions (PyTorch on the GPU) of the same draws, for workloads too
# large to generate on the host.  Same formulas as above; the ellipse
# parameters and flat ICs still come from the seeded host draws.
# ---------------------------------------------------------------------------
def voxelize_torch(ellipses: Sequence[Ellipse], n: int, device, fov: float = FOV_CM,
                   supersample: int = 4):
    """[3][n][n] float32 tensor, as ``voxelize``."""
    import torch
    pitch = fov / n
    sub = (torch.arange(supersample, device=device, dtype=torch.float64) + 0.5) / supersample - 0.5
    idx = torch.arange(n, device=device, dtype=torch.float64) - 0.5 * (n - 1)
    xs = ((idx[:, None] + sub[None, :]) * pitch).reshape(-1)          # (c, sc)
    ys = (-(idx[:, None] + sub[None, :]) * pitch).reshape(-1)         # (r, sr)
    out = torch.zeros((3, n, n), device=device, dtype=torch.float32)
    for e in ellipses:
        cp, sp = np.cos(e.phi), np.sin(e.phi)
        dx = (xs - e.x0)[None, :]
        dy = (ys - e.y0)[:, None]
        xr = dx * cp + dy * sp
        yr = -dx * sp + dy * cp
        inside = ((xr / e.a) ** 2 + (yr / e.b) ** 2 <= 1.0).to(torch.float32)
        frac = inside.reshape(n, supersample, n, supersample).mean(dim=(1, 3))
        out += torch.tensor(e.values, device=device, dtype=torch.float32)[:, None, None] * frac[None]
    return out


def ellipse_line_integrals_torch(ellipses: Sequence[Ellipse], theta: np.ndarray, n_det: int,
                                 pitch: float, device):
    """[3][n_theta][n_det] float32 tensor, as ``ellipse_line_integrals``."""
    import torch
    t = (torch.arange(n_det, device=device, dtype=torch.float64) - 0.5 * (n_det - 1)) * pitch
    th = torch.as_tensor(np.asarray(theta, dtype=np.float64), device=device)[:, None]
    out = torch.zeros((3, th.shape[0], n_det), device=device, dtype=torch.float64)
    for e in ellipses:
        al = th - e.phi
        a2 = (e.a * torch.cos(al)) ** 2 + (e.b * torch.sin(al)) ** 2
        tp = t[None, :] - (e.x0 * torch.cos(th) + e.y0 * torch.sin(th))
        rad = torch.clamp(a2 - tp * tp, min=0.0)
        chord = 2.0 * e.a * e.b * torch.sqrt(rad) / a2
        out += torch.as_tensor(e.values, device=device)[:, None, None] * chord[None]
    return out.to(torch.float32)


def poisson_noise_torch(expected, seed: int, a_ref: float = A_REF):
    """Counts ~ Poisson(a_ref * expected) drawn on the expected tensor's device
    with a seeded generator, returned divided by a_ref (float32)."""
    import torch
    gen = torch.Generator(device=expected.device)
    gen.manual_seed(int(seed) * 1000003 + _PURPOSE_NOISE)
    lam = torch.clamp(expected.to(torch.float32) * a_ref, min=0.0)
    return torch.poisson(lam, generator=gen) / a_ref
