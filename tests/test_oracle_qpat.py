"""Pins of the composite oracle maps (eqs. com_des, J_des): the Jacobian by
brute-force central differences over every unit vector on a 16 x 16 interior,
and the dot-product test of J against J^*."""
import numpy as np

import phantoms
from oracle import acoustic, optics, qpat


def _problem(n=16, nt=24, pml=4, seed=21):
    w = phantoms.small(n=n, pml=pml, nt=nt, n_sensors=10, seed=seed)
    S = acoustic.setup_from_workload(w)
    mu = phantoms.optical_absorption(w)
    kappa = phantoms.optical_diffusion(w)
    return w, S, mu, kappa


def test_full_jacobian_by_central_differences():
    w, S, mu, kappa = _problem()
    N = w.n * w.n
    # H_a is linear: build its matrix once, then difference only the optics
    Ha = np.zeros((w.nt * w.n_sensors, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        Ha[:, j] = acoustic.forward(S, e.reshape(w.n, w.n)).ravel()
    H = lambda m: Ha @ optics.heating(m, kappa, w.dx, 0b0001).ravel()
    # the composite forward equals the matrix form
    np.testing.assert_allclose(qpat.forward(S, mu, kappa, 0b0001).ravel(), H(mu), rtol=1e-10,
                               atol=1e-12 * np.abs(H(mu)).max())
    worst = 0.0
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        eps = 1e-4 * mu.ravel()[j]
        fd = (H(mu + eps * e.reshape(mu.shape)) - H(mu - eps * e.reshape(mu.shape))) / (2 * eps)
        jv = qpat.jvp(S, mu, kappa, 0b0001, e.reshape(mu.shape)).ravel() if j % 37 == 0 else \
            Ha @ optics.jvp(mu, kappa, w.dx, 0b0001, e.reshape(mu.shape)).ravel()
        worst = max(worst, np.linalg.norm(fd - jv) / np.linalg.norm(jv))
    assert worst < 1e-6


def test_composite_dot_product():
    w, S, mu, kappa = _problem(n=20, nt=40, seed=4)
    v = phantoms.random_field(w.interior_shape, 5)
    W = phantoms.random_field((w.nt, w.n_sensors), 6)
    lhs = np.sum(qpat.jvp(S, mu, kappa, 0b0100, v) * W)
    rhs = np.sum(v * qpat.vjp(S, mu, kappa, 0b0100, W))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
