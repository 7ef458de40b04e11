"""Pins of the FP64 oracle of the medium derivatives (sound speed c and
density rho of the discretised acoustic map).

* the discrete closed form of the homogeneous lossless periodic scheme,
  differentiated by hand in c;
* central finite differences of the pinned forward map, heterogeneous, with
  PML, with and without absorption, 2D and 3D;
* the transpose identity between the tangent and the adjoint loops;
* the exact invariance of the data under a uniform scaling of rho.
"""
import math

import numpy as np
import pytest

import phantoms
from oracle import acoustic, medium


def _all_node_sensors(n, dx):
    """One sensor on every node of an n x n grid, in C order (y rows, x fastest)."""
    x = (np.arange(n) - (n - 1) / 2.0) * dx
    Y, X = np.meshgrid(x, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def test_uniform_sound_speed_closed_form():
    """Homogeneous, lossless, periodic: p_n = F^-1{P0 cos(n theta)} for n >= 1
    with cos theta = 1 - (c |k| kappa dt)^2 / 2, kappa = sinc(c_ref |k| dt / 2)
    and c_ref held fixed, and p_0 = P0 / 2.  So along a uniform dc = 1,
    dp_n = F^-1{-P0 n sin(n theta) dtheta/dc}, dtheta/dc = c (|k| kappa dt)^2 / sin theta,
    and dp_0 = 0."""
    n, dx, c, nt = 16, 1e-4, 1500.0, 24
    dt = 0.3 * dx / c
    S = acoustic.make_setup(np.full((n, n), c), np.full((n, n), 1000.0), None, 1.5, dx, dt, nt, 0,
                            _all_node_sensors(n, dx), lossless=True)
    P0 = np.random.default_rng(4).standard_normal(S.shape)
    dP = medium.jvp_medium(S, 1.5, P0, np.ones(S.shape), np.zeros(S.shape))
    k = acoustic.wavenumbers(n, dx)
    K = np.sqrt(k[None, :] ** 2 + k[:, None] ** 2)
    kap = np.sinc(c * K * dt / 2.0 / math.pi)
    theta = np.arccos(1.0 - (c * K * kap * dt) ** 2 / 2.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        dtheta = np.where(K > 0, c * (K * kap * dt) ** 2 / np.sin(theta), 0.0)
    F0 = np.fft.fftn(P0)
    scale = np.abs(dP).max()
    assert scale > 0
    np.testing.assert_allclose(dP[0], 0.0, atol=1e-13 * scale)
    for m in range(1, nt):
        expect = np.real(np.fft.ifftn(-F0 * m * np.sin(m * theta) * dtheta))
        np.testing.assert_allclose(dP[m].reshape(n, n), expect, atol=1e-10 * scale)


def _problem(dim, lossless, seed):
    if dim == 2:
        w = phantoms.small(n=14, pml=4, nt=28, lossless=lossless, seed=seed, n_sensors=10)
    else:
        w = phantoms.small(n=8, pml=2, nt=14, dim=3, lossless=lossless, seed=seed, n_sensors=6)
    c, rho, alpha = phantoms.acoustic_medium(w)
    dt = phantoms.time_step(w, c)

    def setup(cc, rr):
        return acoustic.make_setup(cc, rr, None if lossless else alpha, w.y, w.dx, dt, w.nt, w.pml,
                                   phantoms.sensor_positions(w), c_ref=float(c.max()), lossless=lossless)
    S = setup(c, rho)
    rng = np.random.default_rng(seed + 100)
    P0 = acoustic.embed(S, phantoms.smooth_p0(w, seed))
    dc = c * rng.standard_normal(S.shape) * 0.05
    drho = rho * rng.standard_normal(S.shape) * 0.05
    W = rng.standard_normal((w.nt, w.n_sensors))
    return w, c, rho, S, setup, P0, dc, drho, W


CASES = [(2, False), (2, True), (3, False)]


@pytest.mark.parametrize("dim,lossless", CASES)
def test_tangent_matches_central_differences(dim, lossless):
    w, c, rho, S, setup, P0, dc, drho, _ = _problem(dim, lossless, 21)
    for a, b in ((dc, 0 * drho), (0 * dc, drho)):
        eps = 1e-4
        fd = (acoustic.forward_full(setup(c + eps * a, rho + eps * b), P0)
              - acoustic.forward_full(setup(c - eps * a, rho - eps * b), P0)) / (2 * eps)
        an = medium.jvp_medium(S, w.y, P0, a, b)
        assert np.linalg.norm(an) > 0
        assert np.linalg.norm(an - fd) <= 1e-7 * np.linalg.norm(an)


@pytest.mark.parametrize("dim,lossless", CASES)
def test_adjoint_is_the_transpose_of_the_tangent(dim, lossless):
    w, c, rho, S, setup, P0, dc, drho, W = _problem(dim, lossless, 33)
    lhs = np.sum(medium.jvp_medium(S, w.y, P0, dc, drho) * W)
    g_c, g_rho = medium.vjp_medium(S, w.y, P0, W)
    rhs = np.sum(g_c * dc) + np.sum(g_rho * drho)
    assert abs(lhs - rhs) <= 1e-12 * (abs(np.sum(g_c * dc)) + abs(np.sum(g_rho * drho)))


@pytest.mark.parametrize("lossless", [False, True])
def test_density_scaling_leaves_the_data_unchanged(lossless):
    """rho -> s rho scales v by 1/s and leaves rho_i and p unchanged, PML and
    absorption included; so the derivative along drho = rho vanishes."""
    w, c, rho, S, setup, P0, dc, drho, W = _problem(2, lossless, 45)
    along = medium.jvp_medium(S, w.y, P0, 0 * dc, rho)
    other = medium.jvp_medium(S, w.y, P0, 0 * dc, drho)
    assert np.linalg.norm(along) <= 1e-12 * np.linalg.norm(other) * np.linalg.norm(rho) / np.linalg.norm(drho)
    _, g_rho = medium.vjp_medium(S, w.y, P0, W)
    assert abs(np.sum(g_rho * rho)) <= 1e-12 * np.linalg.norm(g_rho) * np.linalg.norm(rho)
