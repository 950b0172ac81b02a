"""Synthetic ring-artifact and resolution study after the paper's
"Experimental improvements" and results sections.

Setup (the paper's acquisition, synthetic): three homogeneous "granules"
(discs of different attenuation, delta = gamma mu) in an N x N slice;
n_theta angles, one mask position on the slope of the IC (m = -0.24
periods); the sample scan is taken with the true per-pixel flat IC and
Poisson noise.  The flat IC the reconstruction uses is estimated from flat
scans: the mask stepped over one period in 33 positions, `repeats` scans
averaged (the paper compares 1 and 20), Poisson counts, and per pixel a
Gaussian fitted to the averaged curve (weighted least squares on log f, exact
for noise-free data).  Errors of the estimated flat are fixed per detector
pixel and become ring artifacts; the ring term m_r(t) of Eq. 4, solved for
together with h, absorbs the shift part of them.

With --asym a > 0 the true flat is not a Gaussian: the periodised Gaussian
times (1 + a sin 2 pi (m - c)), so the Gaussian fit has a model error.

Reconstructions: the iterative method (linked unknown h, relative change
1e-6) with m_r fixed at 0, among the unknowns ("iter_mr"), or among the
unknowns restricted to ring frequencies ("iter_mr_ring": its steps orthogonal
to the n/16 lowest DCT-II modes across the detector, ei_set_ring_modes), the
iterative method with the averaged flat scans themselves as a sampled flat
(no fit, "iter_tab"), the iterative method with the true flat
("iter_true_flat", the bound), and the single-shot retrieval of Eq. 3 + FBP.
The regulariser weight is the paper's lambda = 1e-2 unless --lam is given:
with intensities normalised by the flat amplitude, the paper's value makes
the regulariser at the true object several times the noise part of the cost,
so the study can also run at smaller values.  Measures: the CNR of Eq. 7
between every pair of granules over discs of 0.6 granule radius; the FRC of Eq. 6 between the
reconstructions of the odd and of the even angles (independent noise), over
the central 140/220 of the slice, with the 0.5 cutoff.

    python -m paper_2202_08627_gb300.ring_study --n 256 --n-theta 400 [--asym 0.15] [--lam 1e-3]
"""
from __future__ import annotations

import argparse
import json
import time
from typing import Sequence

import numpy as np

from . import ei, inputs, metrics

GAMMA = 5e-7                 # delta / mu (cm)
SLOPE_M = -0.24              # mask position on the slope of the IC (periods)
FLAT_STEPS = 33              # mask positions of a flat scan over one period
FLAT_COUNTS = 1000.0         # expected counts at the IC peak per flat exposure
FRC_CROP = 140 / 220         # central part of the slice the FRC compares (140 of 220 voxels)
# granules: (x0, y0, radius) as fractions of the half field of view, attenuation (1/cm)
GRANULES = [(-0.40, 0.30, 0.28, 0.50), (0.40, 0.30, 0.28, 0.55), (0.0, -0.40, 0.28, 0.70)]


def phantom():
    R = 0.5 * inputs.FOV_CM
    return [inputs.Ellipse(x * R, y * R, r * R, r * R, 0.0, np.array([mu, GAMMA * mu, 0.0]))
            for (x, y, r, mu) in GRANULES]


def flat_positions():
    """Mask positions of a flat scan: FLAT_STEPS steps from -0.5 to 0.5 periods
    (the two ends are the same phase)."""
    return -0.5 + np.arange(FLAT_STEPS) / (FLAT_STEPS - 1)


def true_flat(A, c, w, asym: float, m):
    """The true flat IC f_t(m), [len(m)][n_det]: the Gaussian (A, c, w) for
    asym = 0, else the Gaussian summed over its periodic images times
    (1 + asym sin 2 pi (m - c)), an asymmetric, periodic curve that no
    Gaussian fits exactly."""
    m = np.asarray(m, dtype=np.float64)[:, None]
    if asym == 0.0:
        return A[None, :] * np.exp(-(m - c[None, :]) ** 2 / (2 * w[None, :] ** 2))
    d = m - c[None, :]
    g = sum(np.exp(-(d + j) ** 2 / (2 * w[None, :] ** 2)) for j in range(-3, 4))
    return A[None, :] * g * (1.0 + asym * np.sin(2 * np.pi * d))


def flat_scans(A, c, w, repeats: int, seed: int, asym: float = 0.0):
    """`repeats` flat scans with Poisson counts, averaged: [steps][n_det] counts."""
    rng = np.random.Generator(np.random.PCG64([seed, 91]))
    lam = FLAT_COUNTS * true_flat(A, c, w, asym, flat_positions())
    return rng.poisson(lam[None].repeat(repeats, 0)).mean(axis=0)


def flat_table(f):
    """The averaged scans as a sampled flat over one period, [n_det][K] with
    K = FLAT_STEPS - 1 samples at phase k / K (the duplicated end phase
    averaged), normalised like the model's intensities."""
    K = FLAT_STEPS - 1
    steps = f / FLAT_COUNTS
    per = steps[:K].copy()
    per[0] = 0.5 * (steps[0] + steps[K])
    phase = np.rint((flat_positions()[:K] % 1.0) * K).astype(int) % K
    table = np.empty((f.shape[1], K))
    table[:, phase] = per.T
    return table


def estimate_flat(f):
    """Per-pixel Gaussian (A, c, w) fitted to averaged flat scans f [steps][n_det]."""
    m = flat_positions()
    # weighted least squares of log f = a0 + a1 m + a2 m^2, weights f (Poisson variance of log f ~ 1/f)
    X = np.stack([np.ones_like(m), m, m * m], axis=1)
    A_e, c_e, w_e = (np.empty(f.shape[1]) for _ in range(3))
    for j in range(f.shape[1]):
        wt = f[:, j]
        ok = wt > 0
        Xw = X[ok] * wt[ok, None]
        coef = np.linalg.lstsq(Xw.T @ X[ok], Xw.T @ np.log(wt[ok]), rcond=None)[0]
        w2 = -0.5 / coef[2]
        c_e[j] = coef[1] * w2
        w_e[j] = np.sqrt(w2)
        A_e[j] = np.exp(coef[0] + c_e[j] ** 2 / (2 * w2)) / FLAT_COUNTS
    return A_e, c_e, w_e


def geometry(n, theta, A, c, w, lam: float = inputs.LAMBDA):
    return ei.ei_setup_geometry(
        n_m=1, m=[SLOPE_M], z_cm=inputs.Z_CM, period_cm=inputs.PERIOD_CM, kappa_sigma=inputs.KAPPA,
        flat_A=A, flat_c=c, flat_w=w, n=n, n_theta=len(theta), n_det=n,
        pitch_cm=inputs.pitch_for(n), n_slices=1, theta=theta, lam=(lam,) * 3,
        scale=inputs.SCALE)


def ring_modes(n_det: int) -> int:
    """DCT-II modes kept out of m_r in "iter_mr_ring": periods above 32 pixels."""
    return max(1, n_det // 16)


def measure(n, theta, A, c, w, seed, device="cuda", asym: float = 0.0):
    """Sample scan with the true flat: exact line integrals of the granules,
    the library's IC model (for asym > 0 with the true flat tabulated at 512
    steps), Poisson noise."""
    G = geometry(n, theta, A, c, w)
    if asym != 0.0:
        ei.ei_set_flat_table(G, true_flat(A, c, w, asym, np.arange(512) / 512).T.astype(np.float32))
    P = inputs.ellipse_line_integrals_torch(phantom(), theta, n, inputs.pitch_for(n), device)
    proj = G.empty("proj", device)
    proj.view(3, len(theta), G.slices[0].n_dp)[:, :, :n] = P
    clean = G.empty("meas", device)
    ei.ei_ic_model(G, proj, clean)
    G.close()
    return inputs.poisson_noise_torch(clean, seed=seed)


def reconstruct(n, theta, flat, s_exp, mode: str, tol: float = 1e-6, max_iter: int = 300,
                table=None, lam: float = inputs.LAMBDA):
    """h [n][n] from one of: "iter" (m_r = 0), "iter_mr" (m_r among the
    unknowns), "iter_mr_ring" (m_r among the unknowns, restricted to ring
    frequencies), "eq3" (single shot), with the flat IC `flat` = (A, c, w) or,
    for the iterative modes when `table` ([n_det][K]) is given, that sampled
    flat."""
    G = geometry(n, theta, *flat, lam=lam)
    if table is not None and mode != "eq3":
        ei.ei_set_flat_table(G, np.ascontiguousarray(table, dtype=np.float32))
    vol = G.empty("vol", s_exp.device)
    info = {}
    if mode == "eq3":
        ei.ei_single_shot_eq3(G, s_exp, 0, GAMMA, vol)
    else:
        ei.ei_set_linked(G, GAMMA)
        if mode in ("iter_mr", "iter_mr_ring"):
            ei.ei_set_offset_unknowns(G, ei.EI_OFFSET_MR, 0.01)
        if mode == "iter_mr_ring":
            ei.ei_set_ring_modes(G, ring_modes(n))
        rep = ei.ei_reconstruct(G, s_exp, vol, tol=tol, max_iter=max_iter, raise_on_error=False)
        info = {"iterations": int(rep.iterations[0]), "converged": bool(rep.converged[0])}
    h = G.unpack_volume(vol)[0][0]
    G.close()
    return h, info


def subset(s_exp, n_theta, n_dp, idx, device):
    import torch
    return s_exp.view(1, n_theta, n_dp)[:, torch.as_tensor(idx, device=device)].contiguous().view(-1)


def run(n: int = 256, n_theta: int = 400, repeats: Sequence[int] = (1, 20), seed: int = 3,
        device="cuda", asym: float = 0.0, lam: float = inputs.LAMBDA,
        modes: Sequence[str] = ("eq3", "iter", "iter_mr", "iter_mr_ring")):
    import torch
    theta = inputs.angles(n_theta)
    A, c, w = inputs.flat_ic(seed, n)
    s_exp = measure(n, theta, A, c, w, seed, device, asym)
    n_dp = inputs.round_up4(n)
    half = 0.5 * n
    centres = [(half - y * half, half + x * half, r * half) for (x, y, r, _) in GRANULES]
    masks = [metrics.disc_mask(n, cy, cx, 0.6 * r) for (cy, cx, r) in centres]
    pairs = [(0, 1), (0, 2), (1, 2)]
    crop = slice(int(n * (0.5 - FRC_CROP / 2)), int(n * (0.5 + FRC_CROP / 2)))
    rows = []
    odd, even = np.arange(1, n_theta, 2), np.arange(0, n_theta, 2)
    truth = (A, c, w), (None if asym == 0.0 else true_flat(A, c, w, asym, np.arange(512) / 512).T)

    def study(R, method, mode, flat, table, err):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h, info = reconstruct(n, theta, flat, s_exp, mode, table=table, lam=lam)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        h_odd, _ = reconstruct(n, theta[odd], flat, subset(s_exp, n_theta, n_dp, odd, device), mode,
                               table=table, lam=lam)
        h_even, _ = reconstruct(n, theta[even], flat, subset(s_exp, n_theta, n_dp, even, device),
                                mode, table=table, lam=lam)
        curve = metrics.frc(h_odd[crop, crop], h_even[crop, crop])
        row = {"flat_scans": R, "method": method, "seconds": dt, **info,
               "cnr": {"%d-%d" % p: metrics.cnr(h, masks[p[0]], masks[p[1]]) for p in pairs},
               "frc_resolution_px": metrics.frc_resolution(curve, crop.stop - crop.start),
               "flat_error": err}
        rows.append(row)
        print(json.dumps(row), flush=True)

    study(0, "iter_true_flat", "iter", truth[0], truth[1], {})
    for R in repeats:
        scans = flat_scans(A, c, w, R, seed + R, asym)
        flat = estimate_flat(scans)
        err = {"c_rms": float(np.sqrt(np.mean((flat[1] - c) ** 2))),
               "w_rel_rms": float(np.sqrt(np.mean((flat[2] / w - 1) ** 2))),
               "A_rel_rms": float(np.sqrt(np.mean((flat[0] / A - 1) ** 2)))}
        for mode in modes:
            if mode != "iter_tab":
                study(R, mode, mode, flat, None, err)
        if "iter_tab" in modes or asym != 0.0:
            study(R, "iter_tab", "iter", flat, flat_table(scans), err)
    return {"n": n, "n_theta": n_theta, "gamma_cm": GAMMA, "m": SLOPE_M, "asym": asym, "lam": lam,
            "ring_modes": ring_modes(n), "rows": rows}


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--n-theta", type=int, default=400)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--asym", type=float, default=0.0,
                    help="asymmetry of the true flat IC (0: Gaussian)")
    ap.add_argument("--lam", type=float, default=inputs.LAMBDA, help="regulariser weight")
    ap.add_argument("--modes", default="eq3,iter,iter_mr,iter_mr_ring,iter_tab",
                    help="comma-separated reconstructions")
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)
    print(json.dumps(run(args.n, args.n_theta, seed=args.seed, asym=args.asym, lam=args.lam,
                         modes=tuple(args.modes.split(",")))))


if __name__ == "__main__":
    main()
