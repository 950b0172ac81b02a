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
