"""Pins of the FP64 diffusion-approximation oracle (Section 2.1, eq. DA;
Lemma 1) against facts fixed outside it: manufactured exact solutions with
second-order convergence, conservation, symmetry, a dense library solve, the
maximum principle, and central finite differences for the derivative."""
import math

import numpy as np
import pytest

from oracle import optics


def _exact_currents(shape, h, kappa, gam, phi, grad):
    """I on each boundary face from the Robin condition of eq. DA,
    I = gamma phi + (kappa / 2) d phi / dn, evaluated at the face centres."""
    dim = len(shape)
    n = shape[0]
    L = n * h
    centres = (np.arange(n) + 0.5) * h - L / 2
    out = []
    for i in range(dim):
        for side in (0, 1):
            xs = []
            for j in range(dim):          # physical axes other than i
                if j == i:
                    continue
                xs.append(centres)
            grids = np.meshgrid(*xs[::-1], indexing="ij")[::-1] if xs else []
            pts = []
            it = iter(grids)
            for j in range(dim):
                if j == i:
                    pts.append(np.full(grids[0].shape if grids else (), -L / 2 if side == 0 else L / 2))
                else:
                    pts.append(next(it))
            nrm = -1.0 if side == 0 else 1.0
            out.append(gam * phi(*pts) + 0.5 * kappa * nrm * grad(i, *pts))
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_manufactured_solution_second_order(dim):
    """phi = exp(lambda a.r) with |a| = 1, lambda = sqrt(mu / kappa) solves
    -kappa lap phi + mu phi = 0 exactly; feeding its Robin data as the boundary
    current, the cell-centred solution converges at second order."""
    kappa, mu = 0.4e-3, 20.0
    lam = math.sqrt(mu / kappa)
    a = np.array([0.6, 0.8, 0.0]) if dim == 2 else np.array([0.48, 0.6, 0.64])
    a = a[:dim] / np.linalg.norm(a[:dim])
    gam = optics.gamma_d(dim)

    def phi(*x):
        return np.exp(lam * sum(a[i] * x[i] for i in range(dim)) * 0.25)

    def grad(i, *x):
        return lam * 0.25 * a[i] * phi(*x)

    # lambda scaled by 1/4 in phi: use mu_eff so the PDE still holds exactly
    mu_eff = kappa * (lam * 0.25) ** 2
    errs = []
    sizes = [8, 16, 32] if dim == 2 else [6, 12, 24]
    L = 4e-3
    for n in sizes:
        h = L / n
        shape = (n,) * dim
        c = (np.arange(n) + 0.5) * h - L / 2
        grids = np.meshgrid(*([c] * dim), indexing="ij")[::-1]
        cur = _exact_currents(shape, h, kappa, gam, phi, grad)
        A, b = optics.assemble(np.full(shape, mu_eff), np.full(shape, kappa), h, cur)
        sol = optics.solve(A, b).reshape(shape)
        ex = phi(*grids)
        errs.append(np.sqrt(np.mean((sol - ex) ** 2)) / np.sqrt(np.mean(ex ** 2)))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]
    assert min(rates) > 1.8, (errs, rates)
    assert errs[-1] < 2e-3


def test_conservation_symmetry_and_dense_solve():
    rng = np.random.default_rng(0)
    n, h = 12, 1e-4
    mu = rng.uniform(5, 50, size=(n, n))
    kappa = rng.uniform(3e-4, 6e-4, size=(n, n))
    A, b = optics.assemble(mu, kappa, h, optics.boundary_current((n, n), 0b0101))
    Ad = A.toarray()
    np.testing.assert_allclose(Ad, Ad.T, rtol=0, atol=0)
    assert np.linalg.eigvalsh(Ad).min() > 0
    phi = optics.solve(A, b)
    np.testing.assert_allclose(phi, np.linalg.solve(Ad, b), rtol=1e-10)
    # absorbed power mu phi h^2 equals the net boundary inflow
    # 2 kappa (I - gamma phi) h / (gamma h + kappa) (interior fluxes cancel)
    gam = optics.gamma_d(2)
    absorbed = np.sum(mu.ravel() * phi * h * h)
    P = phi.reshape(n, n)
    cur = optics.boundary_current((n, n), 0b0101)
    inflow = 0.0
    for s, (sl, I) in enumerate(zip([(slice(None), 0), (slice(None), -1), (0, slice(None)), (-1, slice(None))], cur)):
        k = kappa[sl]
        inflow += np.sum(2 * k * (I - gam * P[sl]) * h / (gam * h + k))
    assert absorbed == pytest.approx(inflow, rel=1e-10)
    # maximum principle: a non-negative source gives a positive fluence
    assert phi.min() > 0


def test_single_side_illumination_decays_away_from_source():
    n, h = 32, 1e-4
    mu = np.full((n, n), 10.0)
    kappa = np.full((n, n), 1.0 / (2 * (10.0 + 1000.0)))
    phi = optics.fluence(mu, kappa, h, 0b0001)    # side 0 = low x
    prof = phi.mean(axis=0)
    assert np.all(np.diff(prof) < 0)


def test_jvp_matches_central_differences():
    rng = np.random.default_rng(1)
    n, h = 10, 1e-4
    mu = rng.uniform(5, 50, size=(n, n))
    kappa = np.full((n, n), 4.9e-4)
    H0 = lambda m: optics.heating(m, kappa, h, 0b0010)
    for k in range(5):
        v = rng.standard_normal((n, n))
        eps = 1e-4 * np.linalg.norm(mu) / np.linalg.norm(v)
        fd = (H0(mu + eps * v) - H0(mu - eps * v)) / (2 * eps)
        jv = optics.jvp(mu, kappa, h, 0b0010, v)
        assert np.linalg.norm(fd - jv) <= 1e-7 * np.linalg.norm(jv)


def test_vjp_is_transpose_of_jvp_brute_force():
    rng = np.random.default_rng(2)
    n, h = 6, 1e-4
    mu = rng.uniform(5, 50, size=(n, n))
    kappa = rng.uniform(3e-4, 6e-4, size=(n, n))
    J = np.zeros((n * n, n * n))
    for j in range(n * n):
        e = np.zeros(n * n)
        e[j] = 1
        J[:, j] = optics.jvp(mu, kappa, h, 0b1000, e.reshape(n, n)).ravel()
    w = rng.standard_normal((n, n))
    np.testing.assert_allclose(optics.vjp(mu, kappa, h, 0b1000, w).ravel(), J.T @ w.ravel(),
                               rtol=1e-10, atol=1e-14)


# ---- kappa derivatives (Lemma 1, delta-kappa rows) -------------------------------
@pytest.mark.parametrize("dim,mask", [(2, 0b0001), (2, 0b0110), (3, 0b010001)])
def test_kappa_jvp_matches_central_differences(dim, mask):
    rng = np.random.default_rng(11 + dim)
    n = 9 if dim == 2 else 6
    shape = (n,) * dim
    h = 1e-4
    mu = rng.uniform(5, 50, size=shape)
    kappa = rng.uniform(3e-4, 6e-4, size=shape)
    for k in range(3):
        v = rng.standard_normal(shape) * kappa
        t = 1e-6
        fd = (optics.heating(mu, kappa + t * v, h, mask) - optics.heating(mu, kappa - t * v, h, mask)) / (2 * t)
        jv = optics.jvp_kappa(mu, kappa, h, mask, v)
        assert np.linalg.norm(fd - jv) <= 1e-6 * np.linalg.norm(jv)


def test_kappa_vjp_is_transpose_brute_force():
    rng = np.random.default_rng(13)
    n, h = 5, 1e-4
    mu = rng.uniform(5, 50, size=(n, n))
    kappa = rng.uniform(3e-4, 6e-4, size=(n, n))
    J = np.zeros((n * n, n * n))
    for j in range(n * n):
        e = np.zeros(n * n)
        e[j] = 1
        J[:, j] = optics.jvp_kappa(mu, kappa, h, 0b0101, e.reshape(n, n)).ravel()
    w = rng.standard_normal((n, n))
    np.testing.assert_allclose(optics.vjp_kappa(mu, kappa, h, 0b0101, w).ravel(), J.T @ w.ravel(),
                               rtol=1e-10, atol=1e-14 * np.abs(J).max())


def test_kappa_derivative_of_a_homogeneous_scaling():
    """Scaling kappa and mu together by s with h fixed maps Phi to a problem
    whose heating changes only through the Robin terms; a check independent
    of the face formulas: d/ds heating(s mu, s kappa) at s = 1 equals
    J_mu mu + J_kappa kappa."""
    rng = np.random.default_rng(14)
    n, h = 8, 1e-4
    mu = rng.uniform(5, 50, size=(n, n))
    kappa = rng.uniform(3e-4, 6e-4, size=(n, n))
    t = 1e-6
    fd = (optics.heating((1 + t) * mu, (1 + t) * kappa, h, 0b0011)
          - optics.heating((1 - t) * mu, (1 - t) * kappa, h, 0b0011)) / (2 * t)
    both = optics.jvp(mu, kappa, h, 0b0011, mu) + optics.jvp_kappa(mu, kappa, h, 0b0011, kappa)
    assert np.linalg.norm(fd - both) <= 1e-6 * np.linalg.norm(both)
