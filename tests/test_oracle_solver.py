"""Pins for the oracle's L-BFGS minimiser (the paper minimises Eq. 5 with
SciPy's L-BFGS) and for a whole reconstruction.

Anchors: the minimiser of a strictly convex quadratic is the solution of a
linear system (numpy.linalg.solve); the Rosenbrock function's minimiser is
(1, 1); a direction that is not a descent direction must end in a line-search
failure; on a small slice the cost decreases monotonically and the
reconstruction moves towards the phantom; the trial points of the first
iterations on a 2-D quadratic equal those of the matrix form of the
limited-memory update in exact rational arithmetic; a pair without curvature
is dropped.
"""
import numpy as np

from paper_2202_08627_gb300 import inputs
from tests.problems import small_problem


def test_quadratic_minimiser(oracle):
    n = 30
    Q = inputs.uniform_noise((n, n), 40)
    H = Q @ Q.T + 0.5 * np.eye(n)
    b = inputs.uniform_noise(n, 41)

    def fun(u):
        return 0.5 * u @ H @ u - b @ u, H @ u - b

    opts = oracle.SolveOptions(tol=1e-15, max_iter=500)
    u, rep = oracle.lbfgs(fun, np.zeros(n), opts)
    ref = np.linalg.solve(H, b)
    assert np.linalg.norm(u - ref) <= 1e-6 * np.linalg.norm(ref), rep
    assert all(f1 <= f0 for f0, f1 in zip(rep.f_history, rep.f_history[1:]))


def test_rosenbrock(oracle):
    def fun(u):
        x, y = u
        f = (1 - x) ** 2 + 100 * (y - x * x) ** 2
        g = np.array([-2 * (1 - x) - 400 * x * (y - x * x), 200 * (y - x * x)])
        return f, g

    u, rep = oracle.lbfgs(fun, np.array([-1.2, 1.0]), oracle.SolveOptions(tol=1e-16, max_iter=500))
    np.testing.assert_allclose(u, [1.0, 1.0], atol=1e-5)
    assert rep.f_history[-1] < 1e-10


def test_linesearch_failure_is_reported(oracle):
    """A gradient that points the wrong way can never satisfy Armijo."""
    def fun(u):
        return float(u @ u), -2.0 * u

    u, rep = oracle.lbfgs(fun, np.ones(4), oracle.SolveOptions(max_trials=5))
    assert rep.status == "linesearch"


def test_reconstruction_descends_towards_phantom(oracle):
    spec, geom, s_exp = small_problem(seed=7, n=16, n_theta=24, n_det=24, n_m=5, noise=False)
    x, rep = oracle.reconstruct(s_exp, geom, opts=oracle.SolveOptions(tol=1e-9, max_iter=60))
    h = rep.f_history
    assert all(f1 <= f0 for f0, f1 in zip(h, h[1:]))
    # a minimiser cannot cost more than the phantom itself
    S_truth, _ = oracle.objective_grad(spec.truth, s_exp, geom, want_grad=False)
    assert h[-1] <= S_truth < h[0]
    # attenuation channel moves towards the phantom from x0 = 0
    err0 = np.linalg.norm(spec.truth[0])
    err = np.linalg.norm(x[0] - spec.truth[0])
    assert err < 0.8 * err0


# ---------------------------------------------------------------- trajectories by hand
from fractions import Fraction as Fr   # noqa: E402


def _recording(fun):
    points = []

    def wrapped(u):
        points.append(np.array(u, dtype=np.float64))
        return fun(u)
    return wrapped, points


def test_lbfgs_trajectory_on_a_2d_quadratic_by_hand(oracle):
    """Three iterations on f(u) = (u1^2 + 2 u2^2) / 2 from (3, 2), whose first
    gradient (3, 4) has norm 5, so every trial point is rational.  The expected
    trial points come from exact rational arithmetic on the matrix form of the
    limited-memory inverse Hessian (Nocedal & Wright, eq. 7.19): H0 = (s.y /
    y.y) I of the newest pair, then H <- V^T H V + rho s s^T with
    V = I - rho y s^T for every kept pair, oldest first; d = -H g.  The oracle
    runs the two-loop recursion instead, so this pins H0's scaling, the first
    step 1/|g| (here 1/5), the later first trial 1 and the Armijo halving
    against an independent route."""
    A = ((Fr(1), Fr(0)), (Fr(0), Fr(2)))
    c1 = Fr(1, 10000)

    def grad(u):
        return [A[0][0] * u[0] + A[0][1] * u[1], A[1][0] * u[0] + A[1][1] * u[1]]

    def f(u):
        g = grad(u)
        return (u[0] * g[0] + u[1] * g[1]) / 2

    dot = lambda a, b: a[0] * b[0] + a[1] * b[1]

    def matmul(P, Q):
        return [[sum(P[i][k] * Q[k][j] for k in range(2)) for j in range(2)] for i in range(2)]

    u = [Fr(3), Fr(2)]
    g, fu = grad(u), f(u)
    assert dot(g, g) == 25
    pairs, expected = [], []
    for it in range(3):
        if pairs:
            s_n, y_n = pairs[-1]
            gam = dot(s_n, y_n) / dot(y_n, y_n)
            H = [[gam, Fr(0)], [Fr(0), gam]]
            for s_i, y_i in pairs:
                rho = 1 / dot(y_i, s_i)
                V = [[(1 if i == j else 0) - rho * y_i[i] * s_i[j] for j in range(2)] for i in range(2)]
                VT = [[V[j][i] for j in range(2)] for i in range(2)]
                H = matmul(matmul(VT, H), V)
                H = [[H[i][j] + rho * s_i[i] * s_i[j] for j in range(2)] for i in range(2)]
            d = [-(H[0][0] * g[0] + H[0][1] * g[1]), -(H[1][0] * g[0] + H[1][1] * g[1])]
            alpha = Fr(1)
        else:
            d = [-g[0], -g[1]]
            alpha = Fr(1, 5)                    # 1 / |g| with |g| = 5
        gd = dot(g, d)
        while True:
            x = [u[0] + alpha * d[0], u[1] + alpha * d[1]]
            expected.append(x)
            if f(x) <= fu + c1 * alpha * gd:
                break
            alpha /= 2
        s = [x[0] - u[0], x[1] - u[1]]
        gx = grad(x)
        y = [gx[0] - g[0], gx[1] - g[1]]
        if dot(s, y) > 0:
            pairs.append((s, y))
        u, g, fu = x, gx, f(x)

    def fun(v):
        return 0.5 * (v[0] ** 2 + 2.0 * v[1] ** 2), np.array([v[0], 2.0 * v[1]])

    wrapped, points = _recording(fun)
    oracle.lbfgs(wrapped, np.array([3.0, 2.0]), oracle.SolveOptions(tol=0.0, max_iter=3))
    assert len(points) == 1 + len(expected)
    np.testing.assert_array_equal(points[0], [3.0, 2.0])
    np.testing.assert_allclose(points[1], [2.4, 1.2], rtol=0, atol=1e-15)   # u0 - g0 / 5
    for got, want in zip(points[1:], expected):
        np.testing.assert_allclose(got, [float(w) for w in want], rtol=1e-13, atol=1e-15)


def test_lbfgs_skips_a_pair_without_curvature(oracle):
    """f(u) = cos u from u = 0.1, where f is concave: the first step has length
    1 (alpha = 1/|g|, d = -g), lands at 1.1 where s.y < 0, so the pair is not
    kept and the second step is again the normalised steepest descent (length
    1, to 2.1), not a quasi-Newton step; s.y > 0 there, and the third
    iteration's direction is the one-dimensional secant step -(s / y) g, with
    Armijo halving computed here from the definition."""
    def fun(v):
        return float(np.cos(v[0])), np.array([-np.sin(v[0])])

    wrapped, points = _recording(fun)
    oracle.lbfgs(wrapped, np.array([0.1]), oracle.SolveOptions(tol=0.0, max_iter=3))
    x = [p[0] for p in points]
    assert abs(x[1] - 1.1) <= 1e-14 and abs(x[2] - 2.1) <= 1e-14, x[:3]
    assert (-np.sin(1.1) + np.sin(0.1)) * 1.0 < 0 < (-np.sin(2.1) + np.sin(1.1)) * 1.0
    s, y = 2.1 - 1.1, -np.sin(2.1) + np.sin(1.1)
    g2 = -np.sin(2.1)
    d = -(s / y) * g2
    alpha, want = 1.0, []
    while True:
        want.append(2.1 + alpha * d)
        if np.cos(2.1 + alpha * d) <= np.cos(2.1) + 1e-4 * alpha * g2 * d:
            break
        alpha *= 0.5
    np.testing.assert_allclose(x[3:], want, rtol=1e-12, atol=1e-12)
