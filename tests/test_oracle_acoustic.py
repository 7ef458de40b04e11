"""Pins of the FP64 acoustic oracle against facts fixed outside it.

Each test checks the oracle against something other than itself: a closed
form of the continuous or discrete wave equation, an exact invariant of the
scheme, brute force on a tiny grid, the continuous dispersion relation of the
absorbing model, or values the paper prints.
"""
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.special

import phantoms
from oracle import acoustic

HERE = os.path.dirname(os.path.abspath(__file__))


def homogeneous_setup(n=64, dx=1e-4, c=1500.0, rho=1000.0, nt=40, pml=0, cfl=0.3,
                      sensors=None, lossless=True, alpha_db=0.0, y=1.5):
    shape = (n, n)
    cc = np.full(shape, c)
    rr = np.full(shape, rho)
    dt = cfl * dx / c
    if sensors is None:
        sensors = np.zeros((1, 2))
    al = None if lossless else np.full(shape, alpha_db)
    return acoustic.make_setup(cc, rr, al, y, dx, dt, nt, pml, sensors, lossless=lossless)


def node_xy(S):
    n = S.shape[0]
    x = (np.arange(n) - (n - 1) / 2.0) * S.dx
    Y, X = np.meshgrid(x, x, indexing="ij")
    return X, Y


def test_fmax_matches_paper_section6():
    rows = np.loadtxt(os.path.join(HERE, "golden", "fmax_section6.txt"))
    for c_min, dx, f in rows:
        assert acoustic.max_supported_frequency(c_min, dx) == pytest.approx(f, rel=1e-3)


def test_wavenumbers_fft_order():
    # the DFT of exp(i k x_j) peaks at bin m with k = wavenumbers()[m]
    n, dx = 12, 0.3
    k = acoustic.wavenumbers(n, dx)
    x = np.arange(n) * dx
    for m in range(n):
        spec = np.fft.fft(np.exp(1j * k[m] * x))
        assert np.argmax(np.abs(spec)) == m
    assert k[n // 2] == pytest.approx(-math.pi / dx)


def test_gradient_transpose_identity_brute_force():
    """(d/dr_i^+)^T = -(d/dr_i^-) as explicit matrices, Nyquist bins included
    (the staggered symbol is real there, so both operators stay real)."""
    for shape in [(6, 8), (8, 8)]:
        cc = np.full(shape, 1500.0)
        S = acoustic.make_setup(cc, np.full(shape, 1000.0), None, 1.5, 1e-4, 2e-8, 2, 0,
                                np.zeros((1, 2)), lossless=True)
        G = int(np.prod(shape))
        for i in range(2):
            Dp = np.zeros((G, G))
            Dm = np.zeros((G, G))
            for j in range(G):
                e = np.zeros(G)
                e[j] = 1.0
                Dp[:, j] = acoustic.spectral(e.reshape(shape), S.D_plus[i]).ravel()
                Dm[:, j] = acoustic.spectral(e.reshape(shape), S.D_minus[i]).ravel()
            # imaginary parts are dropped by ``spectral``; verify they were round-off
            e = np.random.default_rng(1).standard_normal(shape)
            assert np.abs(np.fft.ifftn(S.D_plus[i] * np.fft.fftn(e)).imag).max() < 1e-9 * np.abs(Dp).max()
            np.testing.assert_allclose(Dp.T, -Dm, atol=1e-12 * np.abs(Dp).max())


def test_staggered_gradient_of_plane_wave():
    """d/dx^+ of cos(k x) on the grid is -k sin(k (x + dx/2)) times the k-space
    correction sinc(c_ref k dt / 2)."""
    S = homogeneous_setup(n=32, lossless=True)
    X, Y = node_xy(S)
    k = 2 * math.pi * 5 / (32 * S.dx)
    f = np.cos(k * X)
    g = acoustic.spectral(f, S.D_plus[0])
    x = S.c_ref * k * S.dt / 2
    expect = -k * np.sin(k * (X + S.dx / 2)) * math.sin(x) / x
    np.testing.assert_allclose(g, expect, atol=1e-9 * k)
    g = acoustic.spectral(np.cos(k * Y), S.D_minus[1])
    expect = -k * np.sin(k * (Y - S.dx / 2)) * math.sin(x) / x
    np.testing.assert_allclose(g, expect, atol=1e-9 * k)


def test_homogeneous_discrete_closed_form():
    """Homogeneous, lossless, periodic, c_ref = c: the scheme gives exactly
    p_n = F^-1{ P0(k) cos(n c |k| dt) } for n >= 1 and p_0 = P0 / 2."""
    S = homogeneous_setup(n=32, nt=30, lossless=True)
    P0 = np.random.default_rng(3).standard_normal(S.shape)
    fields = {}
    acoustic.forward_full(S, P0, callback=lambda n, v, r, p: fields.__setitem__(n + 1, p.copy()))
    kx = acoustic.wavenumbers(32, S.dx)
    K = np.sqrt(kx[None, :] ** 2 + kx[:, None] ** 2)
    F0 = np.fft.fftn(P0)
    c = math.sqrt(S.C[0, 0])
    np.testing.assert_allclose(fields[0], P0 / 2, atol=1e-13)
    for n in range(1, 30):
        expect = np.real(np.fft.ifftn(F0 * np.cos(n * c * K * S.dt)))
        np.testing.assert_allclose(fields[n], expect, atol=1e-11)


def test_gaussian_matches_continuous_2d_solution():
    """Continuous 2D wave equation with p(0) = Gaussian, dp/dt(0) = 0:
    p(r, t) = s^2 int_0^inf exp(-s^2 k^2 / 2) cos(c k t) J0(k r) k dk
    (Hankel transform).  With c_ref = c the k-space scheme is exact in time, so
    sensor samples n >= 1 equal this integral; sample 0 is half of p0
    (additive source split)."""
    n, dx, c = 128, 1e-4, 1500.0
    sig = 3.0 * dx
    x = (np.arange(n) - (n - 1) / 2.0) * dx
    xc = x[64]
    yc = x[60]
    sensors = np.array([[x[64 + 12], x[60]], [x[64], x[60 + 25]], [x[64 - 20], x[60 - 20]]])
    S = homogeneous_setup(n=n, dx=dx, c=c, nt=150, sensors=sensors, lossless=True)
    Y, X = np.meshgrid(x, x, indexing="ij")
    P0 = np.exp(-((X - xc) ** 2 + (Y - yc) ** 2) / (2 * sig * sig))
    data = acoustic.forward_full(S, P0)
    r = np.hypot(sensors[:, 0] - xc, sensors[:, 1] - yc)
    k = np.linspace(0, 12 / sig, 40001)
    for m in [1, 20, 60, 100, 149]:
        t = m * S.dt
        integrand = np.exp(-sig ** 2 * k[:, None] ** 2 / 2) * np.cos(c * k[:, None] * t) \
            * scipy.special.j0(k[:, None] * r[None, :]) * k[:, None]
        ref = sig ** 2 * scipy.integrate.simpson(integrand, x=k, axis=0)
        np.testing.assert_allclose(data[m], ref, atol=2e-9)
    np.testing.assert_allclose(data[0], 0.5 * np.exp(-r ** 2 / (2 * sig * sig)), atol=1e-12)


def test_energy_invariant_heterogeneous_lossless():
    """Lossless, periodic (no PML), heterogeneous c and rho:
    E_m = 1/2 <p_m, p_m / (rho c^2)> + 1/2 sum_i <rho_i v_i^(m-1/2), v_i^(m+1/2)>
    is exactly conserved after the source steps, because
    (d/dr^+)^T = -(d/dr^-)."""
    w = phantoms.small(n=28, pml=0, nt=80, lossless=True, sensors="circle")
    S = acoustic.setup_from_workload(w)
    P0 = acoustic.embed(S, phantoms.smooth_p0(w))
    ps, vs = {}, {}

    def cb(n, v, r, p):
        ps[n + 1] = p.copy()
        vs[n + 1] = [vi.copy() for vi in v]     # v^(n+1/2) is stored under m = n + 1

    acoustic.forward_full(S, P0, callback=cb)
    W = 1.0 / (S.rho0 * S.C)
    E = []
    for m in range(1, 78):
        e = 0.5 * np.sum(ps[m] * ps[m] * W)
        e += 0.5 * sum(np.sum(S.rho0_stag[i] * vs[m][i] * vs[m + 1][i]) for i in range(2))
        E.append(e)
    E = np.array(E)
    assert np.ptp(E) / abs(E.mean()) < 1e-12
    # the same quantity with the node density in place of the staggered one drifts
    E2 = [0.5 * np.sum(ps[m] ** 2 * W) + 0.5 * sum(np.sum(S.rho0 * vs[m][i] * vs[m + 1][i])
                                                   for i in range(2)) for m in range(1, 78)]
    assert np.ptp(E2) / abs(np.mean(E2)) > 1e-6


def _prony2(series):
    """Least-squares p_(n+1) = a p_n + b p_(n-1); returns roots and residual."""
    A = np.stack([series[1:-1], series[:-2]], 1)
    rhs = series[2:]
    (a, b), *_ = np.linalg.lstsq(A, rhs, rcond=None)
    resid = np.linalg.norm(A @ [a, b] - rhs) / np.linalg.norm(rhs)
    return np.roots([1.0, -a, -b]), resid


@pytest.mark.parametrize("y", [1.1, 1.5])
def test_plane_wave_attenuation_and_dispersion(y):
    """A single Fourier mode in a homogeneous absorbing medium decays at the
    temporal rate of the continuous model, omega^2 = c^2 k^2 (1 - eta k^(y-1)
    + i omega tau k^(y-2)), i.e. alpha0 c (c k)^y, which at 1 cm of travel is
    alpha0[dB MHz^-y cm^-1] * f^y dB: a check of the unit conversion, the
    sign of the absorption term and the fractional powers."""
    n, dx, c = 64, 1e-4, 1500.0
    alpha_db = 0.75
    S = homogeneous_setup(n=n, dx=dx, c=c, nt=400, lossless=False, alpha_db=alpha_db, y=y,
                          sensors=np.array([[-(n - 1) / 2 * dx, -(n - 1) / 2 * dx]]))
    X, Y = node_xy(S)
    m = 6
    k = 2 * math.pi * m / (n * dx)
    data = acoustic.forward_full(S, np.cos(k * (X - X[0, 0])))[:, 0]
    roots, resid = _prony2(data[3:])
    assert resid < 1e-10
    lam = roots[0]
    gamma_disc = -math.log(abs(lam)) / S.dt
    omega_disc = abs(np.angle(lam)) / S.dt
    # continuous model, solved exactly for complex omega at real k
    an = float(acoustic.db_to_neper(alpha_db, y))
    tau, eta = -2 * an * c ** (y - 1), 2 * an * c ** y * math.tan(math.pi * y / 2)
    b = 1j * tau * c * c * k ** y
    disc = np.sqrt(b * b + 4 * c * c * k * k * (1 - eta * k ** (y - 1)))
    omega = (b + disc) / 2
    assert gamma_disc == pytest.approx(-omega.imag, rel=0.02)
    assert omega_disc == pytest.approx(omega.real, rel=2e-3)
    # dB over 1 cm of travel at the mode's frequency
    f_mhz = omega_disc / (2 * math.pi) / 1e6
    db_per_cm = 20 * math.log10(math.e) * gamma_disc * (0.01 / c)
    assert db_per_cm == pytest.approx(alpha_db * f_mhz ** y, rel=0.03)
    assert gamma_disc > 0


def test_adjoint_brute_force_tiny():
    """H_a^* equals the transpose of the explicitly assembled H_a (PML,
    absorption, heterogeneity and both source steps included)."""
    w = phantoms.small(n=6, pml=3, nt=7, n_sensors=3, seed=5)
    S = acoustic.setup_from_workload(w)
    N = w.n * w.n
    H = np.zeros((w.nt * 3, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        H[:, j] = acoustic.forward(S, e.reshape(w.n, w.n)).ravel()
    Wd = np.random.default_rng(2).standard_normal((w.nt, 3))
    np.testing.assert_allclose(acoustic.adjoint(S, Wd).ravel(), H.T @ Wd.ravel(),
                               rtol=1e-11, atol=1e-13 * np.abs(H).max())


@pytest.mark.parametrize("lossless", [False, True])
def test_adjoint_dot_product(lossless):
    w = phantoms.small(n=20, pml=6, nt=60, lossless=lossless, seed=9)
    S = acoustic.setup_from_workload(w)
    p0 = phantoms.random_field(w.interior_shape, 1)
    Wd = phantoms.random_field((w.nt, w.n_sensors), 2)
    lhs = np.sum(acoustic.forward(S, p0) * Wd)
    rhs = np.sum(p0 * acoustic.adjoint(S, Wd))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs)) + 1e-300


def test_sensor_interpolation_exact_for_affine_fields():
    w = phantoms.small(n=16, pml=3)
    shape = w.shape
    pos = np.random.default_rng(4).uniform(-0.7e-3, 0.7e-3, size=(20, 2))
    M = acoustic.sensor_matrix(pos, shape, w.dx)
    x = phantoms.node_coords(w)
    Y, X = np.meshgrid(x, x, indexing="ij")
    f = 2.0 + 3e3 * X - 7e3 * Y + 1e7 * X * Y   # bilinear is exact on xy too
    np.testing.assert_allclose(M @ f.ravel(), 2.0 + 3e3 * pos[:, 0] - 7e3 * pos[:, 1]
                               + 1e7 * pos[:, 0] * pos[:, 1], rtol=1e-12)


def test_pml_profile_and_absorption():
    """The layer leaves the interior untouched, reaches alpha_max nepers per grid
    point at the outer node, and absorbs an outgoing pulse."""
    n, P, dx, c, dt = 40, 10, 1e-4, 1500.0, 2e-8
    A = acoustic.pml_profile(n, P, dx, c, dt, 2.0, False)
    assert np.all(A[P:n - P] == 1.0)
    assert A[0] == pytest.approx(math.exp(-2.0 * c / dx * dt / 2))
    assert A[n - 1] == pytest.approx(A[0])
    As = acoustic.pml_profile(n, P, dx, c, dt, 2.0, True)
    assert np.all(As[P:n - P - 1] == 1.0) and As[P - 1] < 1.0 and As[n - P - 1] < 1.0
    # energy left in the interior after the pulse has crossed the layer
    w = phantoms.small(n=40, pml=12, nt=300, lossless=True, seed=3)
    S = acoustic.setup_from_workload(w)
    P0 = acoustic.embed(S, phantoms.smooth_p0(w))
    last = {}
    acoustic.forward_full(S, P0, callback=lambda nn, v, r, p: last.__setitem__("p", p.copy()))
    e0 = np.sum(P0 ** 2)
    assert np.sum(last["p"] ** 2) < 1e-3 * e0


def test_homogeneous_discrete_closed_form_3d():
    """The 3D scheme, homogeneous lossless periodic: p_n = F^-1{P0 cos(n c |k| dt)}."""
    n, dx, c = 12, 1e-4, 1500.0
    shape = (n, n, n)
    S = acoustic.make_setup(np.full(shape, c), np.full(shape, 1000.0), None, 1.5, dx, 0.3 * dx / c, 20, 0,
                            np.zeros((1, 3)), lossless=True)
    P0 = np.random.default_rng(4).standard_normal(shape)
    fields = {}
    acoustic.forward_full(S, P0, callback=lambda nn, v, r, p: fields.__setitem__(nn + 1, p.copy()))
    k = acoustic.wavenumbers(n, dx)
    K = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    F0 = np.fft.fftn(P0)
    np.testing.assert_allclose(fields[0], P0 / 2, atol=1e-13)
    for m in range(1, 20):
        np.testing.assert_allclose(fields[m], np.real(np.fft.ifftn(F0 * np.cos(m * c * K * S.dt))), atol=1e-11)


def test_adjoint_brute_force_tiny_3d():
    """3D H_a^* equals the transpose of the assembled 3D H_a (PML, absorption,
    heterogeneity, trilinear sensors)."""
    w = phantoms.small(n=4, pml=2, nt=5, n_sensors=3, seed=6, dim=3)
    S = acoustic.setup_from_workload(w)
    N = w.n ** 3
    H = np.zeros((w.nt * 3, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        H[:, j] = acoustic.forward(S, e.reshape(w.interior_shape)).ravel()
    Wd = np.random.default_rng(3).standard_normal((w.nt, 3))
    np.testing.assert_allclose(acoustic.adjoint(S, Wd).ravel(), H.T @ Wd.ravel(), rtol=1e-11,
                               atol=1e-13 * np.abs(H).max())
