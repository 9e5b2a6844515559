"""Pins of the oracle's Newton-CG (paper Sec. 3: the truncated-Newton fit)
and of the whole oracle through toy-fit recovery of the generating parameters."""
import numpy as np
import pytest

import oracle
from oracle import newton_cg as ncg
from paper_2403_09225_b300 import workload as W


def test_inner_cg_solves_a_spd_system_in_n_steps():
    """CG on an SPD system reaches the solution in at most n steps (up to
    round-off) when its tolerance is zero."""
    rng = np.random.default_rng(2)
    n = 12
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + n * np.eye(n)
    g = rng.standard_normal(n)
    p, nh = ncg.inner_cg(lambda d: A @ d, g, 1e-12 * np.linalg.norm(g), 10 * n)
    assert np.allclose(p, np.linalg.solve(A, -g), rtol=0, atol=1e-10)
    assert nh <= n + 2


def test_inner_cg_exits_on_negative_curvature():
    A = np.diag([1.0, -1.0, 2.0])
    g = np.array([1.0, 1.0, 1.0])
    p, nh = ncg.inner_cg(lambda d: A @ d, g, 1e-12, 10)
    assert g @ p < 0  # still a descent direction


def test_newton_cg_minimises_a_quadratic():
    rng = np.random.default_rng(4)
    n = 12
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + n * np.eye(n)
    b = rng.standard_normal(n)
    fg = lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b)
    res = ncg.newton_cg(fg, lambda x, v: A @ v, np.zeros(n), xtol=1e-12)
    assert res.status == ncg.CONVERGED_XTOL
    assert np.allclose(res.x, np.linalg.solve(A, b), rtol=0, atol=1e-10)


@pytest.mark.parametrize("n", [2, 6])
def test_newton_cg_reaches_the_rosenbrock_minimum(n):
    def fg(x):
        f = np.sum(100 * (x[1:] - x[:-1] ** 2) ** 2 + (1 - x[:-1]) ** 2)
        g = np.zeros_like(x)
        g[:-1] = -400 * x[:-1] * (x[1:] - x[:-1] ** 2) - 2 * (1 - x[:-1])
        g[1:] += 200 * (x[1:] - x[:-1] ** 2)
        return f, g

    def hp(x, v):
        H = np.zeros((n, n))
        for i in range(n - 1):
            H[i, i] += 1200 * x[i] ** 2 - 400 * x[i + 1] + 2
            H[i, i + 1] += -400 * x[i]
            H[i + 1, i] += -400 * x[i]
            H[i + 1, i + 1] += 200
        return H @ v

    # classic start for n = 2; for the chained n = 6 function the classic start
    # leads to its known local minimum near (-1, 1, ..., 1), so start at 0
    x0 = np.array([-1.2, 1.0]) if n == 2 else np.zeros(n)
    res = ncg.newton_cg(fg, hp, x0, xtol=1e-10, maxiter=500)
    assert np.allclose(res.x, np.ones(n), atol=1e-6), res


def test_fit_recovers_generating_parameters_with_unit_pulls():
    """Toy recovery: data drawn from I(theta_true), fitted from theta_true;
    pulls (fit - true)/sigma over many toys are consistent with N(0, 1).
    A large shared MC sample keeps the normalisation error below the data's."""
    from oracle import toys
    n_toys = 48
    statuses, pulls = toys.toy_pulls("tiny", n_toys, n_data=1500, n_mc=60_000)
    assert all(s in ncg.CONVERGED for s in statuses), statuses
    # per-parameter mean within 4 standard errors, overall width near 1
    se = 1.0 / np.sqrt(n_toys)
    assert np.all(np.abs(pulls.mean(axis=0)) < 4 * se), pulls.mean(axis=0)
    sd = pulls.std()
    assert 0.8 < sd < 1.2, sd
