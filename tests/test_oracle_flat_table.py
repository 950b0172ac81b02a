"""Oracle pins for the sampled flat IC (f(t, m) tabulated at K mask
positions over one period, periodic Catmull-Rom interpolation in m): exact at
the samples, periodic, third-order accurate on a smooth curve, reducing to
the Gaussian model when the table samples the Gaussian densely, and its cost
gradient against central differences."""
import numpy as np

from paper_2202_08627_gb300 import inputs
from tests.problems import small_problem


def _smooth_table(n_det, K, seed=1):
    c = 0.1 * inputs.uniform_noise(n_det, seed)
    m = np.arange(K) / K
    return 1.0 + 0.5 * np.cos(2 * np.pi * (m[None, :] - c[:, None])), c


def test_interpolation_is_exact_at_samples_and_periodic(oracle):
    table, _ = _smooth_table(5, 16)
    for k in range(16):
        x = np.full((1, 5), k / 16)
        f, df = oracle.table_interp(table, x)
        np.testing.assert_allclose(f[0], table[:, k], rtol=0, atol=1e-14)
        ref = 16 * (table[:, (k + 1) % 16] - table[:, (k - 1) % 16]) / 2
        np.testing.assert_allclose(df[0], ref, rtol=0, atol=1e-12)
    x = inputs.uniform_noise((3, 5), 2)
    np.testing.assert_allclose(oracle.table_interp(table, x)[0],
                               oracle.table_interp(table, x + 1.0)[0], rtol=0, atol=1e-13)


def test_third_order_convergence(oracle):
    x = inputs.uniform_noise((64, 4), 3)
    errs = []
    for K in (32, 64):
        table, c = _smooth_table(4, K)
        f, _ = oracle.table_interp(table, x)
        exact = 1.0 + 0.5 * np.cos(2 * np.pi * (x - c[None, :]))
        errs.append(np.abs(f - exact).max())
    assert errs[0] / errs[1] > 6.0, errs


def test_dense_gaussian_table_reproduces_the_gaussian_model(oracle):
    """A dense table of the periodised Gaussian flat gives the sum of the
    Gaussian model over the flat's periodic images (c + j, j = -2..2) to the
    Catmull-Rom error, O(K^-3)."""
    spec, geom, _ = small_problem(seed=4, n=8, n_theta=6, n_det=12, n_m=5)
    P = spec.P_exact.copy()
    P[2] = 0.0                                       # no scatter in the table model
    c0 = geom.flat_c.copy()
    ref = 0.0
    for j in range(-2, 3):
        geom.flat_c = c0 + j
        ref = ref + oracle.ic_model(P, geom)
    geom.flat_c = c0
    K = 4096
    m = np.arange(K) / K
    d = m[None, :] - c0[:, None]
    geom.flat_table = sum(geom.flat_A[:, None] * np.exp(-(d + j) ** 2 / (2 * geom.flat_w[:, None] ** 2))
                          for j in range(-3, 4))
    got = oracle.ic_model(P, geom)
    assert np.abs(got - ref).max() <= 1e-7 * np.abs(ref).max()


def test_gradient_central_differences(oracle):
    spec, geom, s_exp = small_problem(seed=5, n=8, n_theta=6, n_det=12, n_m=3)
    geom.flat_table, _ = _smooth_table(12, 32, seed=6)
    geom.m_r = inputs.uniform_noise(12, 7, -0.02, 0.02)
    scale = geom.scale[:, None, None]
    u = spec.truth / scale * 0.8 + 0.05 * inputs.uniform_noise(spec.truth.shape, 8)
    S, g = oracle.objective_grad(u, s_exp, geom, scaled=True)
    h = 1e-6
    fd = np.zeros_like(u)
    for idx in np.ndindex(*u.shape):
        du = np.zeros_like(u)
        du[idx] = h
        fd[idx] = (oracle.objective_grad(u + du, s_exp, geom, want_grad=False, scaled=True)[0] -
                   oracle.objective_grad(u - du, s_exp, geom, want_grad=False, scaled=True)[0]) / (2 * h)
    assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(fd)
    # the offsets' gradient in table mode
    g_mo, g_mr = oracle.offset_grads(u * scale, s_exp, geom)
    base = geom.m_r.copy()
    for t in (0, 5, 11):
        geom.m_r = base.copy(); geom.m_r[t] += h
        Sp = oracle.objective_grad(u, s_exp, geom, want_grad=False, scaled=True)[0]
        geom.m_r = base.copy(); geom.m_r[t] -= h
        Sm = oracle.objective_grad(u, s_exp, geom, want_grad=False, scaled=True)[0]
        assert abs(g_mr[t] - (Sp - Sm) / (2 * h)) <= 1e-6 * np.abs(g_mr).max()
