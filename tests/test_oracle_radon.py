"""Pins for the oracle's Radon transform R (Eq. 1) and its transpose.

Independent anchors: the textbook closed-form projection of an ellipse
(Kak & Slaney, the reference the paper cites for Eq. 1), column and row sums
at theta = 0 and pi/2, the exact chord through a constant slice, an explicit
dense matrix built in physical coordinates, and the adjoint identity.
"""
import numpy as np
import pytest

from paper_2202_08627_gb300 import inputs
from tests.problems import oracle_geometry


def _geom(oracle, n, n_theta, n_det, theta=None, pitch=None):
    spec = inputs.make_slice(0, n, n_theta, n_det, 3)
    g = oracle_geometry(spec)
    if theta is not None:
        g.theta = np.asarray(theta, dtype=np.float64)
        g.n_theta = len(theta)
    if pitch is not None:
        g.pitch = pitch
    return g


@pytest.mark.parametrize("n,n_theta,n_det", [(8, 6, 12), (17, 11, 25), (32, 45, 40), (5, 7, 3)])
def test_adjoint_identity(oracle, n, n_theta, n_det):
    g = _geom(oracle, n, n_theta, n_det)
    x = inputs.uniform_noise((n, n), 1)
    y = inputs.uniform_noise((n_theta, n_det), 2)
    lhs = np.vdot(oracle.project(x, g), y)
    rhs = np.vdot(x, oracle.backproject(y, g))
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), 1e-30)


def test_adjoint_identity_random_angles(oracle):
    th = inputs.uniform_noise(13, 3, 0.0, 2 * np.pi)
    g = _geom(oracle, 12, 13, 19, theta=th)
    x = inputs.uniform_noise((12, 12), 4)
    y = inputs.uniform_noise((13, 19), 5)
    lhs = np.vdot(oracle.project(x, g), y)
    rhs = np.vdot(x, oracle.backproject(y, g))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_dense_matrix_brute_force(oracle):
    """Every matrix entry built from the ray-driven description in physical
    coordinates (cm): a ray of angle th through t samples the voxel rows (or
    columns) at their crossing points; voxel (r, c) gets the linear-
    interpolation weight of that sample times the path length per row."""
    n, n_theta, n_det = 8, 6, 12
    th = np.array([0.0, 0.3, np.pi / 4, 1.2, np.pi / 2, 2.9])
    pitch = 0.04
    g = _geom(oracle, n, n_theta, n_det, theta=th, pitch=pitch)
    A = np.zeros((n_theta * n_det, n * n))
    for a in range(n_theta):
        ct, st = np.cos(th[a]), np.sin(th[a])
        for j in range(n_det):
            t = (j - (n_det - 1) / 2) * pitch
            if abs(ct) >= abs(st):
                for r in range(n):
                    y = ((n - 1) / 2 - r) * pitch
                    xc = (t - y * st) / ct            # crossing point of row r
                    for c in range(n):
                        x = (c - (n - 1) / 2) * pitch
                        A[a * n_det + j, r * n + c] += (pitch / abs(ct)) * max(0.0, 1 - abs(x - xc) / pitch)
            else:
                for c in range(n):
                    x = (c - (n - 1) / 2) * pitch
                    yc = (t - x * ct) / st            # crossing point of column c
                    for r in range(n):
                        y = ((n - 1) / 2 - r) * pitch
                        A[a * n_det + j, r * n + c] += (pitch / abs(st)) * max(0.0, 1 - abs(y - yc) / pitch)
    xs = inputs.uniform_noise((n, n), 7)
    ys = inputs.uniform_noise((n_theta, n_det), 8)
    np.testing.assert_allclose(oracle.project(xs, g).ravel(), A @ xs.ravel(), rtol=0, atol=1e-13)
    np.testing.assert_allclose(oracle.backproject(ys, g).ravel(), A.T @ ys.ravel(), rtol=0, atol=1e-13)


def test_special_angles_are_column_and_row_sums(oracle):
    """theta = 0 integrates along y (column sums), theta = pi/2 along x
    (row sums, top row at the far end of the detector)."""
    n, n_det, pitch = 8, 12, 0.05
    g = _geom(oracle, n, 2, n_det, theta=[0.0, np.pi / 2], pitch=pitch)
    x = inputs.uniform_noise((n, n), 9)
    p = oracle.project(x, g)
    off = (n_det - n) // 2
    col = np.zeros(n_det)
    col[off:off + n] = pitch * x.sum(axis=0)
    row = np.zeros(n_det)
    row[off:off + n] = pitch * x.sum(axis=1)[::-1]
    np.testing.assert_allclose(p[0], col, rtol=0, atol=1e-13)
    np.testing.assert_allclose(p[1], row, rtol=0, atol=1e-13)


def test_constant_square_chord(oracle):
    """For a constant slice, a ray that stays inside the square on every row
    (column) integrates to the exact chord length n pitch / max(|cos|, |sin|)."""
    n, n_theta, n_det = 24, 19, 40
    g = _geom(oracle, n, n_theta, n_det)
    x = np.ones((n, n))
    p = oracle.project(x, g)
    hn, hd = (n - 1) / 2, (n_det - 1) / 2
    checked = 0
    for a, th in enumerate(g.theta):
        ct, st = np.cos(th), np.sin(th)
        for j in range(n_det):
            t = j - hd
            if abs(ct) >= abs(st):
                cross = [(t - (hn - r) * st) / ct + hn for r in range(n)]
            else:
                cross = [hn - (t - (c - hn) * ct) / st for c in range(n)]
            if min(cross) >= 0 and max(cross) <= n - 1:
                ref = n * g.pitch / max(abs(ct), abs(st))
                assert abs(p[a, j] - ref) <= 1e-12 * ref
                checked += 1
    assert checked > n_theta * 4


def test_ellipse_closed_form_convergence(oracle):
    """R of the voxelised phantom approaches the exact ellipse line integrals:
    the relative L2 error falls as n doubles and is below 2% at n = 256."""
    errs = []
    for n in (32, 64, 128, 256):
        spec = inputs.make_slice(3, n, 32, int(1.5 * n), 3)
        g = oracle_geometry(spec)
        p = oracle.project(spec.truth[0], g)
        ref = spec.P_exact[0]
        errs.append(np.linalg.norm(p - ref) / np.linalg.norm(ref))
    for e0, e1 in zip(errs, errs[1:]):
        assert e1 < 0.7 * e0, errs
    assert errs[-1] < 0.02, errs


def test_ellipse_closed_form_single_disk(oracle):
    """A centred disk of radius R projects to 2 rho sqrt(R^2 - t^2) at every angle."""
    n = 128
    spec = inputs.make_slice(0, n, 8, 160, 3)
    g = oracle_geometry(spec)
    disk = [inputs.Ellipse(0.0, 0.0, 0.1, 0.1, 0.0, np.array([1.5, 0.0, 0.0]))]
    x = inputs.voxelize(disk, n)[0]
    p = oracle.project(x, g)
    t = (np.arange(160) - 79.5) * g.pitch
    ref = 2 * 1.5 * np.sqrt(np.clip(0.01 - t * t, 0, None))
    for a in range(8):
        assert np.linalg.norm(p[a] - ref) / np.linalg.norm(ref) < 0.01
