"""GPU parity of the 3D path (x row pass, y and z passes) against the FP64
oracle on the same seeded inputs: H_a and H_a^* in FP64 (<= 1e-10) and FP32
(<= 2e-4), lossless and lossy, the 3D diffusion solve and the composite
jvp/vjp."""
import numpy as np
import pytest

import phantoms
from oracle import acoustic, optics, qpat
from gpu_helpers import make_pair, rel_l2, to_gpu, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "lossy-24": dict(n=16, pml=4, nt=30, dim=3),            # 24^3 FFT grid
    "lossless-24": dict(n=16, pml=4, nt=30, dim=3, lossless=True),
    "lossy-20x": dict(n=12, pml=4, nt=24, dim=3, y=1.1, seed=4),   # 20^3 (radix 4, 5)
}


def workload(name):
    kw = dict(CASES[name])
    kw.setdefault("n_sensors", 10)
    return phantoms.small(**kw)


@pytest.mark.parametrize("name", list(CASES))
def test_forward_adjoint_fp64_3d(name):
    w = workload(name)
    ctx, S = make_pair(w, "fp64")
    p0 = phantoms.smooth_p0(w) + 0.1 * phantoms.random_field(w.interior_shape, 3)
    got = to_np(ctx.acoustic_forward(to_gpu(p0, torch.float64)))[0]
    assert rel_l2(got, acoustic.forward(S, p0)) <= 1e-10
    W = phantoms.random_field((w.nt, w.n_sensors), 4)
    got = to_np(ctx.acoustic_adjoint(to_gpu(W, torch.float64)))[0]
    assert rel_l2(got, acoustic.adjoint(S, W)) <= 1e-10
    ctx.sync()


@pytest.mark.parametrize("name", ["lossy-24", "lossless-24"])
def test_forward_adjoint_fp32_3d(name):
    w = workload(name)
    ctx, S = make_pair(w, "fp32", max_batch=2)
    p0 = np.stack([phantoms.smooth_p0(w, 0), phantoms.smooth_p0(w, 1)])
    got = to_np(ctx.acoustic_forward(to_gpu(p0, torch.float32)))
    for b in range(2):
        assert rel_l2(got[b], acoustic.forward(S, p0[b])) <= 2e-4
    W = phantoms.random_field((w.nt, w.n_sensors), 4)
    got = to_np(ctx.acoustic_adjoint(to_gpu(W, torch.float32)))[0]
    assert rel_l2(got, acoustic.adjoint(S, W)) <= 2e-4


def test_dot_product_3d_fp64():
    w = workload("lossy-24")
    ctx, _ = make_pair(w, "fp64")
    p0 = to_gpu(phantoms.random_field(w.interior_shape, 11), torch.float64)
    W = to_gpu(phantoms.random_field((w.nt, w.n_sensors), 12), torch.float64)
    lhs = ctx.dot(ctx.acoustic_forward(p0), W.unsqueeze(0))[0]
    rhs = ctx.dot(p0.reshape(1, -1), ctx.acoustic_adjoint(W).reshape(1, -1))[0]
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("illum", [0b000001, 0b010000, 0b100100])
def test_da_solve_3d(illum):
    w = phantoms.small(n=16, pml=4, nt=10, n_sensors=6, seed=2, dim=3)
    ctx, _ = make_pair(w, "fp64")
    mu = phantoms.optical_absorption(w)
    ref = optics.fluence(mu, phantoms.optical_diffusion(w), w.dx, illum)
    got = to_np(ctx.da_solve(to_gpu(mu, torch.float64), illum))[0]
    assert rel_l2(got, ref) <= 1e-9


def test_jvp_vjp_3d():
    w = phantoms.small(n=14, pml=5, nt=20, n_sensors=8, seed=6, dim=3)   # 24^3
    ctx, S = make_pair(w, "fp64")
    mu = phantoms.optical_absorption(w)
    kappa = phantoms.optical_diffusion(w)
    v = phantoms.random_field(w.interior_shape, 5)
    W = phantoms.random_field((w.nt, w.n_sensors), 6)
    mu_g = to_gpu(mu, torch.float64)
    assert rel_l2(to_np(ctx.jvp(mu_g, to_gpu(v, torch.float64), 0b100000))[0],
                  qpat.jvp(S, mu, kappa, 0b100000, v)) <= 1e-9
    assert rel_l2(to_np(ctx.vjp(mu_g, to_gpu(W, torch.float64), 0b100000))[0],
                  qpat.vjp(S, mu, kappa, 0b100000, W)) <= 1e-9


@pytest.mark.parametrize("generic", [False, True])
def test_fp32_3d_48_specialised_and_generic(generic):
    # 48^3: the compile-time Stockham 3D passes (and, with generic_fft, the
    # runtime-radix ones) against the oracle, two problems in one batch
    w = phantoms.small(n=40, pml=4, nt=24, n_sensors=12, seed=8, dim=3)
    ctx, S = make_pair(w, "fp32", max_batch=2, generic_fft=generic)
    p0 = np.stack([phantoms.smooth_p0(w, 2), phantoms.random_field(w.interior_shape, 9)])
    got = to_np(ctx.acoustic_forward(to_gpu(p0, torch.float32)))
    for b in range(2):
        assert rel_l2(got[b], acoustic.forward(S, p0[b])) <= 2e-4
    W = np.stack([phantoms.random_field((w.nt, w.n_sensors), 13), phantoms.random_field((w.nt, w.n_sensors), 14)])
    got = to_np(ctx.acoustic_adjoint(to_gpu(W, torch.float32)))
    for b in range(2):
        assert rel_l2(got[b], acoustic.adjoint(S, W[b])) <= 2e-4


def test_fp32_3d_full_size_against_fp64_and_dot():
    # the 256^3-interior workload on its 288^3 FFT grid, in the launch
    # configuration the bench uses (FP32, specialised passes), for a shortened
    # loop: against the FP64 GPU path (itself pinned to the oracle above), and
    # the adjoint dot test <H p0, w> = <p0, H^* w> with w = H p0 + noise, so
    # that the inner product has no cancellation to amplify FP32 rounding
    import dataclasses
    w = dataclasses.replace(phantoms.C5, nt=16)
    ctx32, _ = make_pair(w, "fp32", nt=16)
    # white noise: in 16 steps only sources near the sensor plane reach it, so
    # a smooth central p0 would leave the sensors with rounding-level tails
    p0 = phantoms.random_field(w.interior_shape, 7)
    p0g = to_gpu(p0, torch.float32)
    d32 = ctx32.acoustic_forward(p0g)
    noise = to_gpu(phantoms.random_field((w.nt, w.n_sensors), 21), torch.float32)
    W = (d32[0] + 0.1 * d32.abs().max() * noise).contiguous()
    a32 = ctx32.acoustic_adjoint(W)
    lhs = ctx32.dot(d32, W.unsqueeze(0))[0]
    rhs = ctx32.dot(p0g.reshape(1, -1), a32.reshape(1, -1))[0]
    d32, a32 = to_np(d32)[0], to_np(a32)[0]
    del ctx32
    torch.cuda.empty_cache()
    ctx64, _ = make_pair(w, "fp64", nt=16)
    d64 = to_np(ctx64.acoustic_forward(to_gpu(p0, torch.float64)))[0]
    a64 = to_np(ctx64.acoustic_adjoint(W.double()))[0]
    errs = (abs(lhs - rhs) / abs(lhs), rel_l2(d32, d64), rel_l2(a32, a64))
    assert errs[0] <= 1e-5 and errs[1] <= 2e-4 and errs[2] <= 2e-4, errs
