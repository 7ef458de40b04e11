"""GPU parity of the kappa derivatives of the composite map (Lemma 1,
delta-kappa rows) and of qpat_set_kappa, through the C ABI, against the FP64
oracle.  A heterogeneous kappa (seeded log-normal about the workload's
value) is installed with qpat_set_kappa and handed to the oracle as is.

The diffusion solves are iterative (PCG to a relative residual of 1e-13), so
FP64 comparisons use 1e-9, as for the mu derivatives."""
import numpy as np
import pytest

import phantoms
from oracle import optics, qpat
from gpu_helpers import make_pair, rel_l2, to_gpu, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _kappa(w, seed=3):
    rng = np.random.default_rng(seed)
    return phantoms.optical_diffusion(w) * np.exp(0.3 * rng.standard_normal(w.interior_shape))


@pytest.mark.parametrize("dim,prec,tol", [(2, "fp64", 1e-9), (2, "fp32", 2e-4), (3, "fp64", 1e-9)])
def test_kappa_jvp_vjp_match_oracle(dim, prec, tol):
    if dim == 2:
        w = phantoms.small(n=36, pml=6, nt=56, n_sensors=14, seed=4)
        illum = 0b0101
    else:
        w = phantoms.small(n=16, pml=4, nt=24, dim=3, n_sensors=12, seed=4)
        illum = 0b010001
    ctx, S = make_pair(w, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    mu = phantoms.optical_absorption(w)
    kappa = _kappa(w)
    ctx.set_kappa(to_gpu(kappa, torch.float64))
    v = phantoms.random_field(w.interior_shape, 5) * kappa
    W = phantoms.random_field((w.nt, w.n_sensors), 6)
    mu_g = to_gpu(mu, torch.float64)
    ref_f = qpat.forward(S, mu, kappa, illum)
    data, phi = ctx.forward(mu_g, illum, return_phi=True)
    assert rel_l2(to_np(data)[0], ref_f) <= tol
    ref_j = qpat.jvp_kappa(S, mu, kappa, illum, v)
    jv = ctx.jvp_kappa(mu_g, to_gpu(v, torch.float64), illum, phi0=phi)
    assert rel_l2(to_np(jv)[0], ref_j) <= tol
    jv2 = ctx.jvp_kappa(mu_g, to_gpu(v, torch.float64), illum)       # fluence solved inside
    assert rel_l2(to_np(jv2)[0], ref_j) <= tol
    ref_v = qpat.vjp_kappa(S, mu, kappa, illum, W)
    g = ctx.vjp_kappa(mu_g, to_gpu(W, dt), illum, phi0=phi)
    assert rel_l2(to_np(g)[0], ref_v) <= tol


def test_kappa_dot_product_fp64():
    w = phantoms.small(n=28, pml=6, nt=40, n_sensors=14, seed=8)
    ctx, _ = make_pair(w, "fp64")
    kappa = _kappa(w, seed=9)
    ctx.set_kappa(to_gpu(kappa, torch.float64))
    mu = to_gpu(phantoms.optical_absorption(w), torch.float64)
    v = to_gpu(phantoms.random_field(w.interior_shape, 1) * kappa, torch.float64)
    W = to_gpu(phantoms.random_field((w.nt, w.n_sensors), 2), torch.float64)
    jv = ctx.jvp_kappa(mu, v, 0b0010)
    g = ctx.vjp_kappa(mu, W, 0b0010)
    lhs = float(torch.sum(jv[0] * W))
    rhs = float(torch.sum(v * g[0]))
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs)


@pytest.mark.parametrize("da_precond", ["multigrid", "jacobi"])
def test_set_kappa_equals_a_fresh_context(da_precond):
    """After qpat_set_kappa the diffusion solve (fine operator and every
    multigrid level) is that of a context created with the new kappa."""
    from paper_1810_11685_gb300.binding import Context
    w = phantoms.small(n=32, pml=4, nt=30, n_sensors=10, seed=12)
    c, rho, alpha = phantoms.acoustic_medium(w)
    kappa = _kappa(w, seed=4)
    common = dict(dx=w.dx, dt=phantoms.time_step(w, c), nt=w.nt, pml=w.pml, y=w.y, precision="fp64",
                  da_precond=da_precond)
    a = Context(c, rho, alpha, phantoms.optical_diffusion(w), phantoms.sensor_positions(w), **common)
    b = Context(c, rho, alpha, kappa, phantoms.sensor_positions(w), **common)
    a.set_kappa(to_gpu(kappa, torch.float64))
    mu = to_gpu(phantoms.optical_absorption(w), torch.float64)
    for illum in (0b0001, 0b1010):
        pa = to_np(a.da_solve(mu, illum))[0]
        pb = to_np(b.da_solve(mu, illum))[0]
        assert rel_l2(pa, pb) <= 1e-11
        assert rel_l2(pb, optics.fluence(to_np(mu), kappa, w.dx, illum)) <= 1e-9
