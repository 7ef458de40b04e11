"""GPU parity of the diffusion solve and of the composite maps (eqs. DA,
com_des, J_des, Lemma 1) against the FP64 oracle, through the C ABI.

The diffusion solve is iterative (PCG to a relative residual of 1e-13), so
its FP64 comparisons use 1e-9; composite FP64 results inherit that bound."""
import numpy as np
import pytest

import phantoms
from oracle import acoustic, optics, qpat
from gpu_helpers import make_pair, rel_l2, to_gpu, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def problem(n=32, pml=4, nt=48, seed=21, **kw):
    """FFT extent n + 2 pml must factor into 2, 3, 5, 7."""
    return phantoms.small(n=n, pml=pml, nt=nt, n_sensors=14, seed=seed, **kw)


@pytest.mark.parametrize("illum", [0b0001, 0b0010, 0b0100, 0b1000, 0b0101])
def test_da_solve_matches_oracle(illum):
    w = problem()
    ctx, _ = make_pair(w, "fp64")
    mu = phantoms.optical_absorption(w)
    kappa = phantoms.optical_diffusion(w)
    ref = optics.fluence(mu, kappa, w.dx, illum)
    got = to_np(ctx.da_solve(to_gpu(mu, torch.float64), illum))[0]
    assert rel_l2(got, ref) <= 1e-9


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 2e-4)])
def test_forward_jvp_vjp_match_oracle(prec, tol):
    w = problem(n=36, pml=6, nt=56, seed=4)
    ctx, S = make_pair(w, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    mu = phantoms.optical_absorption(w)
    kappa = phantoms.optical_diffusion(w)
    v = phantoms.random_field(w.interior_shape, 5) * 3.0
    W = phantoms.random_field((w.nt, w.n_sensors), 6)
    illum = 0b0001
    ref_f = qpat.forward(S, mu, kappa, illum)
    ref_j = qpat.jvp(S, mu, kappa, illum, v)
    ref_v = qpat.vjp(S, mu, kappa, illum, W)
    mu_g = to_gpu(mu, torch.float64)
    data, phi = ctx.forward(mu_g, illum, return_phi=True)
    assert rel_l2(to_np(data)[0], ref_f) <= tol
    jv = ctx.jvp(mu_g, to_gpu(v, torch.float64), illum, phi0=phi)
    assert rel_l2(to_np(jv)[0], ref_j) <= tol
    jv2 = ctx.jvp(mu_g, to_gpu(v, torch.float64), illum)       # fluence solved inside
    assert rel_l2(to_np(jv2)[0], ref_j) <= tol
    g = ctx.vjp(mu_g, to_gpu(W, dt), illum, phi0=phi)
    assert rel_l2(to_np(g)[0], ref_v) <= tol


def test_composite_dot_product_fp64():
    w = problem(n=28, pml=6, nt=40, seed=8)
    ctx, _ = make_pair(w, "fp64")
    mu = to_gpu(phantoms.optical_absorption(w), torch.float64)
    v = to_gpu(phantoms.random_field(w.interior_shape, 1), torch.float64)
    W = to_gpu(phantoms.random_field((w.nt, w.n_sensors), 2), torch.float64)
    jv = ctx.jvp(mu, v, 0b0010)
    g = ctx.vjp(mu, W, 0b0010)
    lhs = float(torch.sum(jv[0] * W))
    rhs = float(torch.sum(v * g[0]))
    # both sides carry the PCG residual bound of the two diffusion solves
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs)


def test_jvp_central_differences_on_gpu():
    """J v against central differences of the GPU forward itself (FP64)."""
    w = problem(n=16, pml=4, nt=30, seed=13)
    ctx, _ = make_pair(w, "fp64")
    mu = phantoms.optical_absorption(w)
    rng = np.random.default_rng(0)
    for k in range(4):
        v = rng.standard_normal(w.interior_shape)
        eps = 1e-4 * np.linalg.norm(mu) / np.linalg.norm(v)
        fp = to_np(ctx.forward(to_gpu(mu + eps * v, torch.float64), 1))[0]
        fm = to_np(ctx.forward(to_gpu(mu - eps * v, torch.float64), 1))[0]
        jv = to_np(ctx.jvp(to_gpu(mu, torch.float64), to_gpu(v, torch.float64), 1))[0]
        assert rel_l2((fp - fm) / (2 * eps), jv) <= 1e-4
