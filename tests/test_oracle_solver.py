"""Pins for the oracle's L-BFGS minimiser (the paper minimises Eq. 5 with
SciPy's L-BFGS) and for a whole reconstruction.

Anchors: the minimiser of a strictly convex quadratic is the solution of a
linear system (numpy.linalg.solve); the Rosenbrock function's minimiser is
(1, 1); a direction that is not a descent direction must end in a line-search
failure; on a small slice the cost decreases monotonically and the
reconstruction moves towards the phantom.
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
