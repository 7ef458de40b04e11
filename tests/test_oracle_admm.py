"""Pins of the ADMM + L-BFGS benchmark oracle (Section 5.1, Algorithms 1-3).

CPU only.  Each check ties the oracle to something other than itself: the
two-loop recursion to the textbook BFGS inverse-Hessian update applied pair by
pair, the shrinkage to a brute-force minimisation, the gradient of the
augmented Lagrangian to central differences of it, the line search to the
Wolfe conditions it promises, and the ADMM loop to descent and feasibility."""
import numpy as np
import pytest

import phantoms
from oracle import acoustic, admm, optics


def test_two_loop_recursion_equals_bfgs_inverse_update():
    """Algorithm 1 applies H_k = V^T H_(k-1) V + rho s s^T (V = I - rho y s^T),
    oldest pair first from H_0 = (s^T y / y^T y) I of the newest pair."""
    rng = np.random.default_rng(0)
    n, m = 12, 5
    A = rng.normal(size=(n, n))
    A = A @ A.T + n * np.eye(n)                 # SPD: every y^T s > 0
    S = [rng.normal(size=n) for _ in range(m)]
    Y = [A @ s for s in S]
    g = rng.normal(size=n)
    H = float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1]) * np.eye(n)
    for s, y in zip(S, Y):
        rho = 1.0 / float(y @ s)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    np.testing.assert_allclose(admm.lbfgs_direction(g, S, Y), -H @ g, rtol=1e-12, atol=1e-12 * np.abs(H @ g).max())
    # no pairs: the identity
    np.testing.assert_array_equal(admm.lbfgs_direction(g, [], []), -g)
    # the secant condition of the newest pair: H y = s
    np.testing.assert_allclose(-admm.lbfgs_direction(Y[-1], S, Y), S[-1], rtol=1e-10)


def test_shrinkage_is_the_minimiser_of_the_l1_penalty():
    nu = 0.3
    grid = np.linspace(-3, 3, 60001)
    for v in (-2.0, -0.31, -0.1, 0.0, 0.25, 0.3, 1.7):
        brute = grid[np.argmin(0.5 * (v - grid) ** 2 + nu * np.abs(grid))]
        assert abs(admm.shrink(np.array(v), nu) - brute) <= 1e-4


def test_projection_lands_in_the_box():
    rng = np.random.default_rng(1)
    x = rng.uniform(0.5, 1.5, size=50)
    d = rng.normal(size=50) * 3
    p = admm.project_direction(x, d, 0.2, 2.0)
    assert np.all(x + p >= 0.2 - 1e-15) and np.all(x + p <= 2.0 + 1e-15)
    inside = (x + d > 0.2) & (x + d < 2.0)
    np.testing.assert_allclose(p[inside], d[inside], rtol=0, atol=1e-15 * np.abs(x).max() * 4)
    np.testing.assert_allclose((x + p)[x + d <= 0.2], 0.2)


@pytest.mark.parametrize("scale", [1.0, 30.0])
def test_line_search_meets_the_wolfe_conditions(scale):
    rng = np.random.default_rng(2)
    n = 8
    A = rng.normal(size=(n, n))
    A = A @ A.T + np.eye(n)
    b = rng.normal(size=n)
    f_and_g = lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b)
    x = rng.normal(size=n)
    f0, g0 = f_and_g(x)
    d = -scale * g0                           # scale 30: alpha = 1 is far too long
    prm = admm.ADMMParams()
    alpha, f, g = admm.line_search(f_and_g, x, f0, g0, d, prm)
    assert f <= f0 + prm.c1 * alpha * (g0 @ d)
    assert g @ d >= prm.c2 * (g0 @ d)
    assert alpha in [prm.tau ** k for k in range(prm.ls_max)]
    if scale > 1:
        assert alpha < 1.0


def _problem(joint, n=8, nt=24, illums=(1, 4), seed=3):
    w = phantoms.small(n=n, pml=4, nt=nt, n_sensors=12, seed=seed)
    S = acoustic.setup_from_workload(w)
    kappa = phantoms.optical_diffusion(w)
    mu_true = phantoms.optical_absorption(w)
    P = [acoustic.forward(S, optics.heating(mu_true, kappa, S.dx, q)) for q in illums]
    mu0 = np.full(w.interior_shape, w.mu_bg)
    kappa0 = 1.2 * kappa if joint else None
    return admm.Problem(S, kappa, illums, P, mu0, kappa0, edge=0.1), mu_true, w


@pytest.mark.parametrize("joint", [False, True])
def test_augmented_lagrangian_gradient_matches_central_differences(joint):
    prob, _, w = _problem(joint)
    rng = np.random.default_rng(4)
    prm = admm.ADMMParams(rho=0.7, nu=1e-2)
    x = prob.x0() * (1.0 + 0.1 * rng.normal(size=prob.shape))
    W = 0.05 * rng.normal(size=prob.Dx(x).shape)
    Uw = 0.05 * rng.normal(size=W.shape)
    Up = [0.1 * np.abs(p).max() * rng.normal(size=p.shape) for p in prob.P]
    g = prob.gradient(x, W, Uw, Up, prm)
    t = 1e-5
    for _ in range(3):
        v = rng.normal(size=prob.shape)
        fd = (prob.value(x + t * v, W, Uw, Up, prm) - prob.value(x - t * v, W, Uw, Up, prm)) / (2 * t)
        assert abs(fd - float(np.sum(g * v))) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("joint", [False, True])
def test_admm_descends_and_stays_in_the_box(joint):
    prob, mu_true, w = _problem(joint)
    prm = admm.ADMMParams(k_max=3, j_max=3, lower=0.05, upper=20.0, tol_out=0.0)
    x, hist = admm.admm(prob, prm)
    assert len(hist["inner"]) == 3 and all(i >= 1 for i in hist["inner"])
    assert hist["eps"][-1] < 0.5 * hist["eps"][0]
    assert np.all(x >= prm.lower) and np.all(x <= prm.upper)
    _, mu = prob.coeffs(x)
    mu0 = prob.mu0
    assert np.linalg.norm(mu - mu_true) < np.linalg.norm(mu0 - mu_true)


def test_inner_minimisation_decreases_the_augmented_lagrangian():
    prob, _, w = _problem(False)
    prm = admm.ADMMParams(j_max=4)
    x0 = prob.x0()
    W = admm.shrink(prob.Dx(x0), prm.nu)
    Uw = np.zeros_like(W)
    Up = [np.zeros_like(p) for p in prob.P]

    def f_and_g(xx):
        H = prob.series(xx)
        return prob.value(xx, W, Uw, Up, prm, H), prob.gradient(xx, W, Uw, Up, prm, H)
    f0, _ = f_and_g(x0)
    x, f, g, it = admm.lbfgs_minimise(f_and_g, x0, prm)
    assert it >= 2 and f < f0
    assert float(np.linalg.norm(g)) < float(np.linalg.norm(prob.gradient(x0, W, Uw, Up, prm)))
