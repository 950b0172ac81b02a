"""Test-side helpers: build the oracle's view of a synthetic slice and its
measured ICs.  The measured data are the oracle's IC model applied to the
analytic (exact) line integrals, plus seeded Poisson noise."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2202_08627_gb300 import inputs


def oracle_geometry(spec: inputs.SliceSpec, lam=None, scale=None, m_o=None, m_r=None,
                    kappa=inputs.KAPPA) -> oracle.Geometry:
    return oracle.Geometry(
        n=spec.n, n_theta=spec.n_theta, n_det=spec.n_det, pitch=spec.pitch,
        theta=spec.theta, m=spec.m, z_cm=inputs.Z_CM, period_cm=inputs.PERIOD_CM,
        kappa=kappa, flat_A=spec.flat_A, flat_c=spec.flat_c, flat_w=spec.flat_w,
        lam=np.full(3, inputs.LAMBDA) if lam is None else np.asarray(lam, float),
        scale=np.array(inputs.SCALE) if scale is None else np.asarray(scale, float),
        m_o=m_o, m_r=m_r)


def measured(spec: inputs.SliceSpec, geom: oracle.Geometry, noise: bool = True) -> np.ndarray:
    clean = oracle.ic_model(spec.P_exact, geom)
    if not noise:
        return clean
    return inputs.poisson_noise(clean, spec.seed)


def small_problem(seed=0, n=8, n_theta=6, n_det=12, n_m=3, noise=True, **kw):
    spec = inputs.make_slice(seed, n, n_theta, n_det, n_m)
    geom = oracle_geometry(spec, **kw)
    return spec, geom, measured(spec, geom, noise)


# ---------------------------------------------------------------- GPU side
def gpu_geometry(specs, geoms, uneven=None):
    """libei geometry for a list of slices (SliceSpec + oracle Geometry each).
    All slices share n_m, z, period, kappa, lambda and scale."""
    from paper_2202_08627_gb300 import ei
    g0 = geoms[0]
    same = all((s.n, s.n_theta, s.n_det) == (specs[0].n, specs[0].n_theta, specs[0].n_det)
               and np.array_equal(g.flat_A, g0.flat_A) and np.array_equal(g.theta, g0.theta)
               for s, g in zip(specs, geoms))
    if uneven is None:
        uneven = not same
    kw = dict(n_m=g0.n_m, m=g0.m, z_cm=g0.z_cm, period_cm=g0.period_cm, kappa_sigma=g0.kappa,
              lam=g0.lam, scale=g0.scale)
    if not uneven:
        return ei.ei_setup_geometry(
            flat_A=g0.flat_A, flat_c=g0.flat_c, flat_w=g0.flat_w, n=g0.n, n_theta=g0.n_theta,
            n_det=g0.n_det, pitch_cm=g0.pitch, n_slices=len(specs), theta=g0.theta,
            m_o=g0.m_o, m_r=g0.m_r, **kw)
    cat = lambda name: np.concatenate([getattr(g, name) for g in geoms])
    m_o = None if g0.m_o is None else cat("m_o")
    m_r = None if g0.m_r is None else cat("m_r")
    return ei.ei_setup_geometry(
        flat_A=cat("flat_A"), flat_c=cat("flat_c"), flat_w=cat("flat_w"),
        per_slice=[(g.n, g.n_theta, g.n_det, g.pitch) for g in geoms], theta=cat("theta"),
        m_o=m_o, m_r=m_r, **kw)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
