"""Synthetic problems on the device, shaped like the paper's scans.

build_problem makes a geometry for a list of slices and their measured ICs:
seeded ellipse phantoms (inputs.py), their exact line integrals on the
device, the library's IC model (ei_ic_model) and seeded Poisson noise.  The
IC model is the library's own; nothing here reimplements the method.
"""
from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np

from . import ei, inputs


def build_problem(slices: Sequence[Tuple[int, int, int]], n_m: int, seeds: Sequence[int],
                  device, noise_seed: int, m: Sequence[float] | None = None,
                  linked_gamma: float | None = None):
    """(geometry, measured ICs as a device tensor) for slices (n, n_theta, n_det).
    m: mask positions (default inputs.mask_positions(n_m)).  linked_gamma: the
    measured data come from the homogeneous-sample model mu = h, delta =
    gamma h, sigma = 0, with h the phantom's attenuation channel."""
    import torch
    fA, fc, fw, th = [], [], [], []
    for s, (n, nth, nd) in enumerate(slices):
        A, c, w = inputs.flat_ic(seeds[s], nd)
        fA.append(A), fc.append(c), fw.append(w), th.append(inputs.angles(nth))
    m = inputs.mask_positions(n_m) if m is None else np.asarray(m, dtype=np.float64)
    G = ei.ei_setup_geometry(
        n_m=n_m, m=m, z_cm=inputs.Z_CM, period_cm=inputs.PERIOD_CM,
        kappa_sigma=inputs.KAPPA, flat_A=np.concatenate(fA), flat_c=np.concatenate(fc),
        flat_w=np.concatenate(fw), lam=(inputs.LAMBDA,) * 3, scale=inputs.SCALE,
        per_slice=[(n, nth, nd, inputs.pitch_for(n)) for (n, nth, nd) in slices],
        theta=np.concatenate(th))
    proj = G.empty("proj", device)
    for s, (n, nth, nd) in enumerate(slices):
        sl = G.slices[s]
        P = inputs.ellipse_line_integrals_torch(inputs.random_ellipses(seeds[s]), th[s], nd,
                                                inputs.pitch_for(n), device)
        if linked_gamma is not None:
            P = torch.stack([P[0], linked_gamma * P[0], torch.zeros_like(P[0])])
        proj[sl.proj_offset:sl.proj_offset + sl.proj_count].view(3, nth, sl.n_dp)[:, :, :nd] = P
    clean = G.empty("meas", device)
    ei.ei_ic_model(G, proj, clean)
    del proj
    s_exp = inputs.poisson_noise_torch(clean, seed=noise_seed)
    del clean
    torch.cuda.synchronize()
    return G, s_exp
