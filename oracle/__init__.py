"""FP64 CPU oracle for model-based iterative reconstruction in x-ray
edge-illumination (EI) tomography, after Modregger et al., arXiv:2202.08627.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The CUDA library and its
Python binding never import it and share no code with it; the only thing both
sides consume is the seeded input generator, which holds none of the method's
arithmetic.

What it computes, in the paper's order and notation:

* ``project`` / ``backproject`` — the Radon transform R of Eq. 1 (a line
  integral, computed by ray-driven linear interpolation, see ``ei_oracle.c``)
  and its transpose, which the analytic gradient of Eq. 5 needs.
* ``deriv`` / ``deriv_T`` — the finite-difference detector derivative d/dt of
  Eq. 2 / Eq. 4 (the "Experimental improvements" section says the derivative is
  implemented as finite differences) and its transpose.
* ``ic_model`` — the illumination-curve model of Eq. 2: attenuation
  exp(-R[mu]) times the flat IC f(t, m) shifted by z d/dt R[delta] (shift in
  mask periods: z/period), extended by the drift m_o(theta) and ring term
  m_r(t) of Eq. 4 and by a scatter broadening: the Gaussian flat IC
  f(t, m) = A_t exp(-(m - c_t)^2 / (2 w_t^2)) is convolved with a Gaussian of
  variance kappa R[sigma], which keeps its area.
* ``table_interp`` and the table branches of ``ic_model``,
  ``ic_objective_grad`` and ``shift_gradient`` — the flat IC taken as the
  samples of a mask scan over one period (the "Experimental improvements"
  section measures it in 33 steps) instead of its Gaussian fit, interpolated
  in m by periodic cubic Catmull-Rom splines: s = exp(-R[mu]) f_t(m - shift).
* ``objective_grad`` — the cost S of Eq. 5 (sum of squared residuals plus an
  L2 regulariser) and its analytic gradient.
* ``objective_grad_linked`` — the same cost for the single unknown h of Eq. 4
  (mu = h, delta = gamma h, no scatter) and its gradient with respect to h.
* ``offset_grads`` — the gradient of S with respect to the drift m_o(theta)
  and the ring term m_r(t) of Eq. 4; ``ring_project`` restricts m_r's steps
  to ring (pixel-to-pixel) frequencies.
* ``single_shot`` / ``single_shot_eq3`` — non-iterative reconstructions: the
  three-channel moment retrieval used as the warm-start input, and the
  paper's single-shot retrieval of Eq. 3 for the linked unknown.
* ``lbfgs`` / ``reconstruct`` — the L-BFGS minimisation the paper uses
  ("Theoretical basis" section, [Byrd 1995] via SciPy), written out.

Parity: every function here is pinned by the ``-m "not gpu"`` tests against
closed forms, invariants or brute force (see tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        for name in ("eio_project", "eio_backproject"):
            fn = getattr(lib, name)
            fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                           dp, dp, dp]
            fn.restype = None
        for name in ("eio_deriv", "eio_deriv_T"):
            fn = getattr(lib, name)
            fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
            fn.restype = None
        lib.eio_num_threads.restype = ctypes.c_int
        lib.eio_set_num_threads.argtypes = [ctypes.c_int]
        _LIB = lib
    return _LIB


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    return _lib().eio_num_threads()


def set_num_threads(t: int) -> None:
    _lib().eio_set_num_threads(int(t))


# --------------------------------------------------------------------------
# Problem description
# --------------------------------------------------------------------------
@dataclass
class Geometry:
    """One slice's acquisition geometry and model constants (FP64).

    n            slice is n x n voxels
    n_theta      projection angles, ``theta`` [n_theta] in rad
    n_det        detector pixels; voxel pitch = detector pitch = ``pitch`` (cm)
    m            [M] mask positions in IC periods
    z_cm         sample-detector distance; ``period_cm`` the mask period the
                 IC shift is measured in (shift = (z/period) d/dt R[delta])
    kappa        IC variance added per unit R[sigma] (period^2 / unit)
    flat_A/c/w   [n_det] Gaussian flat IC per pixel: amplitude, centre, width
    lam, scale   per channel (mu, delta, sigma): regulariser weight and the
                 variable scaling u = x / scale the solver works in
    m_o, m_r     optional drift [n_theta] and ring [n_det] offsets (Eq. 4)
    flat_table   optional sampled flat IC [n_det][K]: f(t, k / K) over one period
                 (periodic in m with period 1); when given it replaces the
                 Gaussian (flat_A/c/w) in the model, interpolated in m by
                 periodic Catmull-Rom splines, and the scatter channel has no
                 effect
    """
    n: int
    n_theta: int
    n_det: int
    pitch: float
    theta: np.ndarray
    m: np.ndarray
    z_cm: float
    period_cm: float
    kappa: float
    flat_A: np.ndarray
    flat_c: np.ndarray
    flat_w: np.ndarray
    lam: np.ndarray = field(default_factory=lambda: np.full(3, 1e-2))
    scale: np.ndarray = field(default_factory=lambda: np.array([1.0, 1e-6, 1.0]))
    m_o: Optional[np.ndarray] = None
    m_r: Optional[np.ndarray] = None
    flat_table: Optional[np.ndarray] = None

    @property
    def n_m(self) -> int:
        return int(len(self.m))

    @property
    def z_over_p(self) -> float:
        return self.z_cm / self.period_cm


# --------------------------------------------------------------------------
# Linear operators (C core)
# --------------------------------------------------------------------------
def project(x: np.ndarray, geom: Geometry) -> np.ndarray:
    """R[x](t_j, theta_a) for one channel (Eq. 1).  x: [n][n] -> [n_theta][n_det]."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert x.shape == (geom.n, geom.n)
    th = np.ascontiguousarray(geom.theta, dtype=np.float64)
    p = np.empty((geom.n_theta, geom.n_det))
    _lib().eio_project(geom.n, geom.n_theta, geom.n_det, float(geom.pitch),
                       _ptr(th), _ptr(x), _ptr(p))
    return p


def backproject(g: np.ndarray, geom: Geometry) -> np.ndarray:
    """R^T g for one channel.  g: [n_theta][n_det] -> [n][n]."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    assert g.shape == (geom.n_theta, geom.n_det)
    th = np.ascontiguousarray(geom.theta, dtype=np.float64)
    x = np.empty((geom.n, geom.n))
    _lib().eio_backproject(geom.n, geom.n_theta, geom.n_det, float(geom.pitch),
                           _ptr(th), _ptr(g), _ptr(x))
    return x


def deriv(p: np.ndarray, pitch: float) -> np.ndarray:
    """Finite-difference d/dt along the last axis (rows of a sinogram)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    rows, nd = (1, p.shape[0]) if p.ndim == 1 else p.shape
    out = np.empty_like(p)
    _lib().eio_deriv(rows, nd, float(pitch), _ptr(p), _ptr(out))
    return out


def deriv_T(g: np.ndarray, pitch: float) -> np.ndarray:
    """Transpose of ``deriv``."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    rows, nd = (1, g.shape[0]) if g.ndim == 1 else g.shape
    out = np.empty_like(g)
    _lib().eio_deriv_T(rows, nd, float(pitch), _ptr(g), _ptr(out))
    return out


# --------------------------------------------------------------------------
# IC model (Eq. 2, Eq. 4) and cost (Eq. 5)
# --------------------------------------------------------------------------
def _shift_terms(geom: Geometry, P_delta: np.ndarray) -> np.ndarray:
    """Total IC shift in periods: m_o(theta) + m_r(t) + (z/period) d/dt R[delta]."""
    shift = geom.z_over_p * deriv(P_delta, geom.pitch)
    if geom.m_o is not None:
        shift = shift + np.asarray(geom.m_o, dtype=np.float64)[:, None]
    if geom.m_r is not None:
        shift = shift + np.asarray(geom.m_r, dtype=np.float64)[None, :]
    return shift


def table_interp(table: np.ndarray, x: np.ndarray):
    """Periodic Catmull-Rom interpolation of per-pixel samples table[t][k] at
    m = k / K, evaluated at x[..., t] (periods); returns (f, df/dm).  With
    u = x K = i + s: f = sum_{d=-1..2} table[(i + d) mod K] c_d(s), the cubic
    Hermite weights with slopes (p_{i+1} - p_{i-1}) / 2."""
    K = table.shape[1]
    u = np.asarray(x, dtype=np.float64) * K
    i = np.floor(u).astype(np.int64)
    s = u - i
    cols = np.arange(table.shape[0])
    p = [table[cols, np.mod(i + d, K)] for d in (-1, 0, 1, 2)]
    s2, s3 = s * s, s * s * s
    f = 0.5 * ((-s3 + 2 * s2 - s) * p[0] + (3 * s3 - 5 * s2 + 2) * p[1] +
               (-3 * s3 + 4 * s2 + s) * p[2] + (s3 - s2) * p[3])
    df = 0.5 * ((-3 * s2 + 4 * s - 1) * p[0] + (9 * s2 - 10 * s) * p[1] +
                (-9 * s2 + 8 * s + 1) * p[2] + (3 * s2 - 2 * s) * p[3]) * K
    return f, df


def ic_model(P: np.ndarray, geom: Geometry) -> np.ndarray:
    """s_mod(t, theta, m) from the three projections P = [R mu, R delta, R sigma].

    P: [3][n_theta][n_det] -> [M][n_theta][n_det].
      s = exp(-R[mu]) * A (w / sqrt(V)) exp(-(m - c - shift)^2 / (2 V)),
      V = w^2 + kappa R[sigma].
    """
    P_mu, P_delta, P_sigma = P
    shift = _shift_terms(geom, P_delta)
    out = np.empty((geom.n_m,) + P_mu.shape)
    if geom.flat_table is not None:                 # sampled flat IC: s = T f_t(m - shift)
        for k, mk in enumerate(geom.m):
            out[k] = np.exp(-P_mu) * table_interp(geom.flat_table, mk - shift)[0]
        return out
    A, c, w = geom.flat_A[None, :], geom.flat_c[None, :], geom.flat_w[None, :]
    V = w * w + geom.kappa * P_sigma
    for k, mk in enumerate(geom.m):
        q = mk - c - shift
        out[k] = np.exp(-P_mu) * A * (w / np.sqrt(V)) * np.exp(-q * q / (2.0 * V))
    return out


def ic_objective_grad(P: np.ndarray, s_exp: np.ndarray, geom: Geometry,
                      want_grad: bool = True):
    """Data term of Eq. 5 and its gradient with respect to the projections.

    Returns (S_data, dS/dP [3][n_theta][n_det] or None).  S_data is +inf when
    the broadened variance leaves its domain (V <= 0.01 w^2 anywhere).
      e = s_mod - s_exp,  q = m - c - shift
      dS/dR[mu]    = sum_m 2 e (-s)
      dS/dR[delta] = (z/period) D^T sum_m 2 e s q / V
      dS/dR[sigma] = kappa sum_m 2 e s (q^2 - V) / (2 V^2)
    """
    P_mu, P_delta, P_sigma = P
    shift = _shift_terms(geom, P_delta)
    if geom.flat_table is not None:
        # s = T f_t(m - shift): dS/dR[mu] = sum 2 e (-s), dS/dshift = sum 2 e (-T f')
        T = np.exp(-P_mu)
        S, G_mu, G_shift = 0.0, np.zeros_like(P_mu), np.zeros_like(P_mu)
        for k, mk in enumerate(geom.m):
            f, df = table_interp(geom.flat_table, mk - shift)
            s = T * f
            e = s - s_exp[k]
            S += float(np.sum(e * e))
            G_mu += 2.0 * e * (-s)
            G_shift += 2.0 * e * (-T * df)
        if not want_grad:
            return S, None
        g = np.zeros_like(P)
        g[0] = G_mu
        g[1] = geom.z_over_p * deriv_T(G_shift, geom.pitch)
        return S, g
    A, c, w = geom.flat_A[None, :], geom.flat_c[None, :], geom.flat_w[None, :]
    V = w * w + geom.kappa * P_sigma
    if np.any(V <= 0.01 * w * w):
        return np.inf, (np.zeros_like(P) if want_grad else None)
    S = 0.0
    G_mu = np.zeros_like(P_mu)
    G_shift = np.zeros_like(P_mu)
    G_V = np.zeros_like(P_mu)
    for k, mk in enumerate(geom.m):
        q = mk - c - shift
        s = np.exp(-P_mu) * A * (w / np.sqrt(V)) * np.exp(-q * q / (2.0 * V))
        e = s - s_exp[k]
        S += float(np.sum(e * e))
        if want_grad:
            G_mu += 2.0 * e * (-s)
            G_shift += 2.0 * e * s * q / V
            G_V += 2.0 * e * s * (q * q - V) / (2.0 * V * V)
    if not want_grad:
        return S, None
    g = np.empty_like(P)
    g[0] = G_mu
    g[1] = geom.z_over_p * deriv_T(G_shift, geom.pitch)
    g[2] = geom.kappa * G_V
    return S, g


def shift_gradient(P: np.ndarray, s_exp: np.ndarray, geom: Geometry) -> np.ndarray:
    """dS/d(shift) per pixel, [n_theta][n_det]: sum_m 2 e s q / V (the shift
    enters the model only through q = m - c - shift).  Zero where the model
    leaves its domain."""
    P_mu, P_delta, P_sigma = P
    shift = _shift_terms(geom, P_delta)
    G = np.zeros_like(P_mu)
    if geom.flat_table is not None:
        T = np.exp(-P_mu)
        for k, mk in enumerate(geom.m):
            f, df = table_interp(geom.flat_table, mk - shift)
            G += 2.0 * (T * f - s_exp[k]) * (-T * df)
        return G
    A, c, w = geom.flat_A[None, :], geom.flat_c[None, :], geom.flat_w[None, :]
    V = w * w + geom.kappa * P_sigma
    if np.any(V <= 0.01 * w * w):
        return np.zeros_like(P_mu)
    for k, mk in enumerate(geom.m):
        q = mk - c - shift
        s = np.exp(-P_mu) * A * (w / np.sqrt(V)) * np.exp(-q * q / (2.0 * V))
        G += 2.0 * (s - s_exp[k]) * s * q / V
    return G


def offset_grads(x: np.ndarray, s_exp: np.ndarray, geom: Geometry):
    """Gradients of S with respect to the drift m_o(theta) and the ring term
    m_r(t) of Eq. 4, for a physical volume x [3][n][n].  Both enter only the
    shift of pixel (theta, t), with coefficient 1, so
      dS/dm_o(theta) = sum_t dS/dshift(theta, t),
      dS/dm_r(t)     = sum_theta dS/dshift(theta, t)."""
    P = np.stack([project(np.asarray(x[ch], dtype=np.float64), geom) for ch in range(3)])
    G = shift_gradient(P, s_exp, geom)
    return G.sum(axis=1), G.sum(axis=0)


def ring_project(g: np.ndarray, K: int) -> np.ndarray:
    """The ring term m_r(t) of Eq. 4 restricted to pixel-to-pixel (ring)
    frequencies: the orthogonal projection of a per-pixel vector g [n_det]
    onto the complement of the K lowest orthonormal DCT-II modes across the
    detector (K = 0: g unchanged; K = 1: g minus its mean).  A ring artefact is
    a per-pixel error of the flat IC, present at every frequency, while the
    shift that the object's angle-averaged projection causes varies slowly
    across the detector; restricting m_r's steps to this subspace keeps it
    from absorbing the latter.  The restriction is a reading: the paper leaves
    m_r unconstrained.  The orthonormal DCT-II (scipy) serves as the change of
    basis."""
    from scipy.fft import dct, idct
    g = np.asarray(g, dtype=np.float64)
    if K <= 0:
        return g.copy()
    c = dct(g, type=2, norm="ortho")
    c[:K] = 0.0
    return idct(c, type=2, norm="ortho")


def objective_grad_linked(h: np.ndarray, s_exp: np.ndarray, geom: Geometry, gamma: float,
                          want_grad: bool = True, scaled: bool = False):
    """S of Eq. 5 for the single unknown of Eq. 4: mu = h, delta = gamma h,
    sigma = 0, with the regulariser lam_mu ||h / scale_mu||^2 (the paper's
    lambda ||h||^2).  h [n][n] physical (scaled=False) or h / scale_mu
    (scaled=True); the gradient is with respect to the same variable.
    Chain rule through the linear R:
      dS/dh = R^T (dS/dR[mu] + gamma dS/dR[delta]) + regulariser."""
    s_mu = float(np.asarray(geom.scale, dtype=np.float64)[0])
    lam = float(np.asarray(geom.lam, dtype=np.float64)[0])
    h = np.asarray(h, dtype=np.float64)
    u = h if scaled else h / s_mu
    hp = u * s_mu
    Ph = project(hp, geom)
    P = np.stack([Ph, gamma * Ph, np.zeros_like(Ph)])
    S_data, gP = ic_objective_grad(P, s_exp, geom, want_grad)
    S = S_data + lam * float(np.sum(u * u))
    if not want_grad:
        return S, None
    gh = backproject(gP[0] + gamma * gP[1], geom)
    if scaled:
        return S, s_mu * gh + 2.0 * lam * u
    return S, gh + 2.0 * lam * u / s_mu


def forward(x: np.ndarray, geom: Geometry) -> np.ndarray:
    """s_mod for a physical volume x [3][n][n] (mu, delta, sigma)."""
    P = np.stack([project(x[ch], geom) for ch in range(3)])
    return ic_model(P, geom)


def objective_grad(x: np.ndarray, s_exp: np.ndarray, geom: Geometry,
                   want_grad: bool = True, scaled: bool = False):
    """S of Eq. 5 and its gradient for one slice.

    scaled=False: x is the physical volume [3][n][n]; S = data + sum_c lam_c
    ||x_c / scale_c||^2 and the gradient is with respect to x.
    scaled=True: x holds u = x_phys / scale (what the solver iterates on); same
    S, gradient with respect to u.
    """
    scale = np.asarray(geom.scale, dtype=np.float64)
    lam = np.asarray(geom.lam, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    u = x if scaled else x / scale[:, None, None]
    xp = u * scale[:, None, None]
    P = np.stack([project(xp[ch], geom) for ch in range(3)])
    S_data, gP = ic_objective_grad(P, s_exp, geom, want_grad)
    S = S_data + float(np.sum(lam * np.sum(u * u, axis=(1, 2))))
    if not want_grad:
        return S, None
    grad_x = np.stack([backproject(gP[ch], geom) for ch in range(3)])
    if scaled:
        grad = scale[:, None, None] * grad_x + 2.0 * lam[:, None, None] * u
    else:
        grad = grad_x + 2.0 * lam[:, None, None] * u / scale[:, None, None]
    return S, grad


# --------------------------------------------------------------------------
# L-BFGS (the paper minimises S with SciPy's L-BFGS implementation)
# --------------------------------------------------------------------------
@dataclass
class SolveOptions:
    tol: float = 1e-6          # stop when the relative decrease of f is below tol
    max_iter: int = 100
    lbfgs_m: int = 10          # pairs kept (SciPy's default maxcor)
    c1: float = 1e-4           # Armijo sufficient-decrease constant
    max_trials: int = 20       # step halvings per line search
    curv_eps: float = 1e-10    # keep (s, y) only if s.y > curv_eps |s| |y|


@dataclass
class SolveReport:
    iterations: int
    f_history: list
    status: str                # "converged", "max_iter", "linesearch", "nonfinite"
    evaluations: int


def lbfgs(fun: Callable[[np.ndarray], tuple], u0: np.ndarray,
          opts: SolveOptions = SolveOptions()):
    """Minimise fun (returning (f, grad)) from u0.

    Steps per iteration k:
      1. d = -H g by the two-loop recursion over the kept (s_i, y_i) pairs, with
         H_0 = (s.y / y.y) I of the newest pair (I when none is kept);
      2. Armijo backtracking from alpha = 1/|g| when no pair is kept, else 1:
         accept the first alpha with f(u + alpha d) <= f + c1 alpha g.d, else
         halve, at most max_trials times;
      3. s = alpha d, y = g_new - g; keep the pair if s.y > curv_eps |s| |y|
         (oldest dropped beyond lbfgs_m);
      4. stop when (f - f_new) / max(|f|, |f_new|, 1) < tol, or after max_iter
         accepted steps.
    Returns (u, SolveReport).
    """
    u = np.array(u0, dtype=np.float64, copy=True)
    f, g = fun(u)
    n_eval = 1
    hist = [f]
    if not np.isfinite(f):
        return u, SolveReport(0, hist, "nonfinite", n_eval)
    S_mem, Y_mem = [], []
    k = 0
    while k < opts.max_iter:
        # 1. two-loop recursion
        q = g.copy()
        alphas = []
        for s_i, y_i in reversed(list(zip(S_mem, Y_mem))):
            rho = 1.0 / float(np.vdot(y_i, s_i))
            a_i = rho * float(np.vdot(s_i, q))
            q = q - a_i * y_i
            alphas.append((rho, a_i))
        if S_mem:
            gamma = float(np.vdot(S_mem[-1], Y_mem[-1])) / float(np.vdot(Y_mem[-1], Y_mem[-1]))
        else:
            gamma = 1.0
        r = gamma * q
        for (s_i, y_i), (rho, a_i) in zip(zip(S_mem, Y_mem), reversed(alphas)):
            b = rho * float(np.vdot(y_i, r))
            r = r + (a_i - b) * s_i
        d = -r
        gd = float(np.vdot(g, d))
        if not gd < 0.0:
            # no descent (g == 0 or a broken memory): restart from steepest descent
            S_mem, Y_mem = [], []
            d = -g
            gd = float(np.vdot(g, d))
            if gd == 0.0:
                return u, SolveReport(k, hist, "converged", n_eval)
        # 2. Armijo backtracking
        gnorm = float(np.sqrt(np.vdot(g, g)))
        alpha = 1.0 / gnorm if not S_mem else 1.0
        accepted = False
        for _ in range(opts.max_trials):
            u_new = u + alpha * d
            f_new, g_new = fun(u_new)
            n_eval += 1
            if np.isfinite(f_new) and f_new <= f + opts.c1 * alpha * gd:
                accepted = True
                break
            alpha *= 0.5
        if not accepted:
            return u, SolveReport(k, hist, "linesearch", n_eval)
        # 3. memory update
        s_new = u_new - u
        y_new = g_new - g
        sy = float(np.vdot(s_new, y_new))
        if sy > opts.curv_eps * float(np.linalg.norm(s_new)) * float(np.linalg.norm(y_new)):
            S_mem.append(s_new)
            Y_mem.append(y_new)
            if len(S_mem) > opts.lbfgs_m:
                S_mem.pop(0)
                Y_mem.pop(0)
        rel = (f - f_new) / max(abs(f), abs(f_new), 1.0)
        u, f, g = u_new, f_new, g_new
        hist.append(f)
        k += 1
        # 4. stop rule
        if rel < opts.tol:
            return u, SolveReport(k, hist, "converged", n_eval)
    return u, SolveReport(k, hist, "max_iter", n_eval)


def reconstruct(s_exp: np.ndarray, geom: Geometry, x0: Optional[np.ndarray] = None,
                opts: SolveOptions = SolveOptions()):
    """Minimise Eq. 5 for one slice; returns (x_phys [3][n][n], SolveReport)."""
    scale = np.asarray(geom.scale, dtype=np.float64)[:, None, None]
    if x0 is None:
        x0 = np.zeros((3, geom.n, geom.n))
    u0 = np.asarray(x0, dtype=np.float64) / scale

    def fun(u):
        return objective_grad(u, s_exp, geom, want_grad=True, scaled=True)

    u, rep = lbfgs(fun, u0, opts)
    return u * scale, rep


# --------------------------------------------------------------------------
# Single-shot retrieval and filtered back-projection (the non-iterative
# reconstruction of the paper's Eq. 3 + inverse Radon, generalised to three
# channels through the moments of the IC): the warm-start input.
# --------------------------------------------------------------------------
def flat_at_masks(geom: Geometry) -> np.ndarray:
    """f(t, m_k) of the Gaussian flat IC, [M][n_det]."""
    m = np.asarray(geom.m, dtype=np.float64)[:, None]
    return geom.flat_A[None, :] * np.exp(-(m - geom.flat_c[None, :]) ** 2 /
                                         (2.0 * geom.flat_w[None, :] ** 2))


def retrieve_moments(s_exp: np.ndarray, geom: Geometry):
    """Per pixel, from the zeroth, first and second moments over m of the
    measured IC and of the flat IC:
      T     = sum s / sum f                      (transmission, exp(-R[mu]))
      shift = mean_m(s) - mean_m(f) - m_o - m_r   (IC shift in periods)
      dv    = max(0, var_m(s) - var_m(f))         (IC broadening)
    Returns (P_mu = -ln T, shift, P_sigma = dv / kappa), each [n_theta][n_det].
    With moments over a dense, wide set of m these are exact for the model
    of ic_model; with a few positions over one period they are estimates."""
    m = np.asarray(geom.m, dtype=np.float64)[:, None, None]
    s = np.asarray(s_exp, dtype=np.float64)
    f = flat_at_masks(geom)[:, None, :]
    S0, S1, S2 = s.sum(0), (m * s).sum(0), (m * m * s).sum(0)
    F0, F1, F2 = f.sum(0), (m * f).sum(0), (m * m * f).sum(0)
    T = S0 / F0
    cs = S1 / np.where(S0 != 0.0, S0, 1.0)
    cf = F1 / F0
    shift = cs - cf
    if geom.m_o is not None:
        shift = shift - np.asarray(geom.m_o, dtype=np.float64)[:, None]
    if geom.m_r is not None:
        shift = shift - np.asarray(geom.m_r, dtype=np.float64)[None, :]
    vs = S2 / np.where(S0 != 0.0, S0, 1.0) - cs * cs
    vf = F2 / F0 - cf * cf
    dv = np.maximum(vs - vf, 0.0)
    P_mu = -np.log(np.maximum(T, 1e-6))
    P_sigma = dv / geom.kappa if geom.kappa > 0 else np.zeros_like(dv)
    return P_mu, shift, P_sigma


def integrate_shift(shift: np.ndarray, geom: Geometry) -> np.ndarray:
    """R[delta] from its detector derivative: shift = (z/period) dR/dt, so
    R(t_j) = (period/z) pitch sum_{j' <= j} shift_j' (running sum from the
    first pixel), then the straight line through 0 before the first pixel and
    the last running sum is removed, so that R vanishes outside the object at
    both ends of every row."""
    cum = np.cumsum(shift, axis=-1) * geom.pitch / geom.z_over_p
    nd = shift.shape[-1]
    ramp = (np.arange(nd) + 1.0) / nd
    return cum - cum[..., -1:] * ramp


def ramp_filter(p: np.ndarray, pitch: float) -> np.ndarray:
    """Ram-Lak filtering along t (Kak & Slaney's spatial kernel for the inverse
    Radon transform): q_j = pitch sum_k h(j - k) p_k with h(0) = 1/(4 pitch^2),
    h(d) = -1/(pi^2 d^2 pitch^2) for odd d, 0 for even d != 0, over the row."""
    p = np.asarray(p, dtype=np.float64)
    nd = p.shape[-1]
    d = np.arange(-(nd - 1), nd)
    h = np.zeros(d.shape)
    h[d == 0] = 0.25
    odd = (d % 2) != 0
    h[odd] = -1.0 / (np.pi ** 2 * d[odd].astype(np.float64) ** 2)
    h = h / pitch ** 2
    out = np.empty_like(p)
    for idx in np.ndindex(*p.shape[:-1]):
        out[idx] = pitch * np.convolve(p[idx], h, mode="full")[nd - 1:2 * nd - 1]
    return out


def fbp(P: np.ndarray, geom: Geometry) -> np.ndarray:
    """Filtered back-projection of projections P [c][n_theta][n_det] over
    180 degrees: x = (pi / n_theta) (1/pitch) R^T (ramp-filtered P), per channel
    (R^T carries one pitch per angle, hence the 1/pitch)."""
    scale = np.pi / geom.n_theta / geom.pitch
    return np.stack([scale * backproject(ramp_filter(P[c], geom.pitch), geom)
                     for c in range(P.shape[0])])


def eq3_slope(geom: Geometry, m_index: int, gamma: float) -> float:
    """The length a (cm) of the single-shot retrieval of Eq. 3: linearising
    Eq. 4 at one mask position m, f(m - shift) ~ f(m) - f'(m) shift with
    shift = (z/period) gamma dR[h]/dt and dT/dt = -T dR[h]/dt, gives
    s / f = (1 + a d/dt) T with a = (z/period) gamma f'(m) / f(m), where f is the
    flat IC averaged over the pixels (the paper's f(m)) and f' its derivative
    in m."""
    m = float(geom.m[m_index])
    A, c, w = geom.flat_A, geom.flat_c, geom.flat_w
    f = A * np.exp(-(m - c) ** 2 / (2.0 * w * w))
    df = -f * (m - c) / (w * w)
    return geom.z_over_p * gamma * float(df.mean()) / float(f.mean())


def single_shot_eq3(s_exp: np.ndarray, geom: Geometry, m_index: int, gamma: float):
    """The paper's single-shot retrieval (Eq. 3) from one mask position and its
    filtered back-projection, for the homogeneous-sample model mu = h,
    delta = gamma h (gamma in cm).  Per sinogram row: y = s(t, m) / f(t, m),
    T = Re F^-1[F[y] / (1 + i q a)] (DFT along t, q = 2 pi x the DFT frequencies
    / (n_det pitch), the e^{-iqt} convention, a from eq3_slope), R[h] = -ln T
    (T clamped at 1e-6); then h = FBP of R[h].  The offsets m_o, m_r of Eq. 4
    are not part of this model.  Returns (R[h] [n_theta][n_det], h [n][n])."""
    a = eq3_slope(geom, m_index, gamma)
    f = flat_at_masks(geom)[m_index]
    y = np.asarray(s_exp, dtype=np.float64)[m_index] / f[None, :]
    q = 2.0 * np.pi * np.fft.fftfreq(geom.n_det, d=geom.pitch)
    T = np.real(np.fft.ifft(np.fft.fft(y, axis=1) / (1.0 + 1j * a * q[None, :]), axis=1))
    P = -np.log(np.maximum(T, 1e-6))
    return P, fbp(P[None], geom)[0]


def single_shot(s_exp: np.ndarray, geom: Geometry) -> np.ndarray:
    """Non-iterative reconstruction [3][n][n] (physical units): moment
    retrieval of the three projections, integration of the shift, FBP."""
    P_mu, shift, P_sigma = retrieve_moments(s_exp, geom)
    P = np.stack([P_mu, integrate_shift(shift, geom), P_sigma])
    return fbp(P, geom)
