"""Pins of the LD reconstruction oracle (Section 5.2.1, Algorithms 4 and 5).

CPU only.  Each check ties the oracle to something other than itself: the TV
operator to finite differences of the smoothed TV functional, the gradient
and the Gauss-Newton Hessian to finite differences of the forward map, and
the PCG of Algorithm 4 to a dense textbook solve and its closed-form first
step."""
import numpy as np
import pytest

import phantoms
from oracle import acoustic, ld, optics


def _problem(n=8, nt=30, illums=(1, 4), seed=3):
    w = phantoms.small(n=n, pml=4, nt=nt, n_sensors=12, seed=seed)
    S = acoustic.setup_from_workload(w)
    kappa = phantoms.optical_diffusion(w)
    mu_true = phantoms.optical_absorption(w)
    P = [acoustic.forward(S, optics.heating(mu_true, kappa, S.dx, q)) for q in illums]
    mu0 = np.full(w.interior_shape, w.mu_bg)
    return ld.Problem(S, kappa, illums, P, mu0), mu_true, w


@pytest.mark.parametrize("beta", [1e-2, 2e-5])
def test_tv_gradient_is_M_times_xbar(beta):
    rng = np.random.default_rng(0)
    xbar = rng.normal(size=(7, 9)) * 0.3
    edge, t = 0.1, 1e-6
    g = ld.tv_matrix(xbar, edge, beta) @ xbar.ravel()
    for k in range(6):
        v = rng.normal(size=xbar.shape)
        fd = (ld.tv_functional(xbar + t * v, edge, beta) - ld.tv_functional(xbar - t * v, edge, beta)) / (2 * t)
        assert abs(fd - g @ v.ravel()) <= 1e-6 * max(1.0, abs(fd))


def test_tv_matrix_structure_3d():
    rng = np.random.default_rng(1)
    xbar = rng.normal(size=(4, 5, 6))
    M = ld.tv_matrix(xbar, 0.01, 2e-5).toarray()
    assert np.allclose(M, M.T, rtol=0, atol=1e-12 * abs(M).max())
    assert np.allclose(M @ np.ones(M.shape[0]), 0.0, atol=1e-10 * abs(M).max())
    assert np.linalg.eigvalsh(M).min() >= -1e-10 * abs(M).max()
    # one face per neighbouring pair: 3 * 4*5*6 - (5*6 + 4*6 + 4*5) faces
    D = ld.tv_difference(xbar.shape, 1.0)
    assert D.shape[0] == 3 * 120 - (30 + 24 + 20)
    Mg = ld.m_gamma(xbar, 0.01, 2e-5, 1e-6)
    assert np.allclose(Mg @ np.ones(Mg.shape[0]), 1e-6, rtol=1e-6)


def test_gradient_matches_central_differences():
    prob, _, w = _problem()
    rng = np.random.default_rng(2)
    xbar = 0.2 * rng.normal(size=w.interior_shape)
    g = prob.gradient(xbar)
    t = 1e-4
    for k in range(3):
        v = rng.normal(size=w.interior_shape)
        fd = (prob.misfit(xbar + t * v) - prob.misfit(xbar - t * v)) / (2 * t)
        assert abs(fd - np.sum(g * v)) <= 1e-6 * abs(fd)


def test_gauss_newton_product_is_the_gram_form():
    prob, _, w = _problem()
    rng = np.random.default_rng(3)
    xbar = 0.2 * rng.normal(size=w.interior_shape)
    v, u = rng.normal(size=w.interior_shape), rng.normal(size=w.interior_shape)
    Hv, Hu = prob.gn_product(xbar, v), prob.gn_product(xbar, u)
    assert abs(np.sum(Hv * u) - np.sum(v * Hu)) <= 1e-12 * abs(np.sum(Hv * u))
    # <H v, u> = sum_q <(J S) v, (J S) u>, with (J S) v by central differences
    # of H_q[mu0 exp(Xbar)] along v
    t = 1e-5

    def jsv(d, q):
        return (prob.forward(prob.mu(xbar + t * d), q) - prob.forward(prob.mu(xbar - t * d), q)) / (2 * t)

    gram = sum(np.sum(jsv(v, q) * jsv(u, q)) for q in range(2))
    assert abs(gram - np.sum(Hv * u)) <= 1e-6 * abs(gram)


def test_pcg_is_a_textbook_solve():
    rng = np.random.default_rng(4)
    n = 12
    B = rng.normal(size=(n, n))
    A = B @ B.T + n * np.eye(n)
    P = np.diag(rng.uniform(1, 3, n)) + 0.1 * np.ones((n, n))
    b = rng.normal(size=n)
    x, i, rz = ld.pcg(lambda d: A @ d, b, lambda r: np.linalg.solve(P, r), i_max=n, i_m=n, tol_in=0.0)
    assert i == n
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-12)
    # first step: x1 = (r.z / z.A z) z with z = P^-1 b
    z = np.linalg.solve(P, b)
    x1, i1, _ = ld.pcg(lambda d: A @ d, b, lambda r: np.linalg.solve(P, r), i_max=1, i_m=5, tol_in=0.0)
    assert i1 == 1
    assert np.allclose(x1, (b @ z) / (z @ A @ z) * z, rtol=1e-13)


def test_pcg_stopping_rule():
    rng = np.random.default_rng(5)
    n = 40
    B = rng.normal(size=(n, n))
    A = B @ B.T + 0.1 * np.eye(n)
    b = rng.normal(size=n)
    for i_m, tol in ((2, 0.9), (3, 0.5), (5, 0.0)):
        x, i, rz = ld.pcg(lambda d: A @ d, b, lambda r: r, i_max=30, i_m=i_m, tol_in=tol)
        assert i == 30 or (i >= i_m and 1.0 - rz[i] / rz[i - i_m] <= tol)
        for j in range(i_m, i):
            assert 1.0 - rz[j] / rz[j - i_m] > tol


def test_pcg_zero_rhs_returns_zero():
    x, i, rz = ld.pcg(lambda d: 2 * d, np.zeros(5), lambda r: r, i_max=10, i_m=2, tol_in=0.0)
    assert i == 0 and not np.any(x)


def test_ld_newton_decreases_the_misfit_and_the_error():
    prob, mu_true, w = _problem(n=8, nt=30)
    prm = ld.LDParams(k_max=3, i_max=8, i_m=3, tol_in=0.0, tol_out=0.0, gamma=1e-6, beta=2e-5,
                      edge=w.dx / phantoms.MM)
    mu, xbar, eps, inner = ld.ld_newton(prob, prm)
    assert len(eps) == 4 and len(inner) == 3
    assert all(eps[k + 1] < eps[k] for k in range(3))
    assert eps[-1] < 0.2 * eps[0]
    assert np.linalg.norm(mu - mu_true) < np.linalg.norm(prob.mu0 - mu_true)
    assert np.allclose(mu, prob.mu0 * np.exp(xbar))


def _joint_problem(n=8, nt=30, illums=(1, 4, 2, 8), seed=3):
    w = phantoms.small(n=n, pml=4, nt=nt, n_sensors=12, seed=seed)
    S = acoustic.setup_from_workload(w)
    rng = np.random.default_rng(seed)
    kappa_true = phantoms.optical_diffusion(w) * np.exp(0.3 * rng.standard_normal(w.interior_shape))
    mu_true = phantoms.optical_absorption(w)
    P = [acoustic.forward(S, optics.heating(mu_true, kappa_true, S.dx, q)) for q in illums]
    mu0 = np.full(w.interior_shape, w.mu_bg)
    kappa0 = phantoms.optical_diffusion(w)
    return ld.JointProblem(S, illums, P, mu0, kappa0), (kappa_true, mu_true), w


def test_joint_gradient_matches_central_differences():
    prob, _, w = _joint_problem(illums=(1, 4))
    rng = np.random.default_rng(6)
    xbar = 0.2 * rng.normal(size=prob.shape)
    g = prob.gradient(xbar)
    t = 1e-4
    for k in range(3):
        v = rng.normal(size=prob.shape)
        fd = (prob.misfit(xbar + t * v) - prob.misfit(xbar - t * v)) / (2 * t)
        assert abs(fd - np.sum(g * v)) <= 1e-6 * abs(fd)


def test_joint_gauss_newton_product_is_the_gram_form():
    prob, _, w = _joint_problem(illums=(1, 4))
    rng = np.random.default_rng(7)
    xbar = 0.2 * rng.normal(size=prob.shape)
    v, u = rng.normal(size=prob.shape), rng.normal(size=prob.shape)
    Hv, Hu = prob.gn_product(xbar, v), prob.gn_product(xbar, u)
    assert abs(np.sum(Hv * u) - np.sum(v * Hu)) <= 1e-12 * abs(np.sum(Hv * u))
    t = 1e-5

    def jsv(d, q):
        kp, mp = prob.coeffs(xbar + t * d)
        km, mm = prob.coeffs(xbar - t * d)
        return (prob.forward(kp, mp, q) - prob.forward(km, mm, q)) / (2 * t)

    gram = sum(np.sum(jsv(v, q) * jsv(u, q)) for q in range(2))
    assert abs(gram - np.sum(Hv * u)) <= 1e-6 * abs(gram)


def test_joint_ld_newton_decreases_the_misfit():
    prob, (kappa_true, mu_true), w = _joint_problem()
    prm = ld.LDParams(k_max=3, i_max=4, i_m=4, tol_in=0.0, tol_out=0.0, edge=w.dx / phantoms.MM)
    (kappa, mu), xbar, eps, inner = ld.ld_newton(prob, prm)
    assert len(eps) == 4 and inner == [4, 4, 4]
    assert all(eps[k + 1] < eps[k] for k in range(3))
    assert np.allclose(mu, prob.mu0 * np.exp(xbar[1])) and np.allclose(kappa, prob.kappa0 * np.exp(xbar[0]))


# ---- Algorithm 6 (PD-IPM) ----------------------------------------------------------
def test_pd_preconditioner_without_dual_is_the_lagged_diffusivity_one():
    rng = np.random.default_rng(20)
    d = rng.normal(size=(6, 7)) * 0.3
    nf = ld.tv_difference(d.shape, 0.1).shape[0]
    A = ld.pd_matrix(d, np.zeros(nf), 0.1, 1e-6, 1e-4).toarray()
    B = ld.m_gamma(d, 0.1, 1e-6, 1e-4).toarray()
    assert np.allclose(A, B, rtol=1e-14, atol=0)


def test_pd_dual_direction_is_the_derivative_of_the_central_path():
    """On the central path chi = C[d] D d the dual direction of eq. dw is the
    derivative of d -> C[d] D d along the primal step (central differences),
    and a full step from any feasible chi with a zero primal step lands on the
    path."""
    rng = np.random.default_rng(21)
    edge, beta = 0.1, 1e-3
    d = rng.normal(size=(6, 7)) * 0.3
    dd = rng.normal(size=d.shape)
    D = ld.tv_difference(d.shape, edge)

    def chi_of(x):
        g = D @ x.ravel()
        return g / np.sqrt(g * g + beta)

    chi = chi_of(d)
    D_, g, c, wf = ld.pd_weights(d, chi, edge, beta)
    t = 1e-6
    fd = (chi_of(d + t * dd) - chi_of(d - t * dd)) / (2 * t)
    assert np.allclose(wf * (D @ dd.ravel()), fd, rtol=1e-6, atol=1e-9)
    chi0 = rng.uniform(-0.9, 0.9, size=chi.shape)
    assert np.allclose(ld.pd_dual_step(d, np.zeros_like(d), chi0, edge, beta), chi, rtol=1e-12, atol=1e-14)


def test_pd_dual_step_stays_feasible():
    rng = np.random.default_rng(22)
    d = rng.normal(size=(6, 7))
    chi = rng.uniform(-1, 1, size=ld.tv_difference(d.shape, 0.1).shape[0])
    for _ in range(5):
        dd = 50 * rng.normal(size=d.shape)
        chi = ld.pd_dual_step(d, dd, chi, 0.1, 1e-6)
        assert np.max(np.abs(chi)) <= 1.0 + 1e-12
        d = d + dd


def test_pdipm_first_step_equals_ld_and_descends():
    prob, mu_true, w = _problem()
    edge = w.dx / phantoms.MM
    one = ld.pdipm_newton(prob, ld.PDParams(k_max=1, i_max=2, i_m=2, tol_out=0.0, kp_max=1, gamma=1e-2,
                                            beta=1e-6, edge=edge))
    ref = ld.ld_newton(prob, ld.LDParams(k_max=1, i_max=2, i_m=2, tol_out=0.0, gamma=1e-2, beta=1e-6, edge=edge))
    assert np.allclose(one[0], ref[0], rtol=1e-13)
    mu, xbar, eps, inner = ld.pdipm_newton(prob, ld.PDParams(k_max=2, i_max=2, i_m=2, tol_out=0.0, kp_max=2,
                                                             tol_med=-1.0, gamma=1e-2, beta=1e-6, edge=edge))
    assert inner == [[2, 2], [2, 2]]
    assert eps[2] < eps[1] < eps[0]
    assert np.linalg.norm(mu - mu_true) < np.linalg.norm(prob.mu0 - mu_true)
