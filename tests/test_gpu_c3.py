"""Full-size checks of the differentiable 2D workload: 1024^2 interior
(1080^2 FFT grid), Nt = 4000, FP32 propagation with FP64 reductions, four
illuminated sides, a smooth random mu (Gaussian-filtered noise, sigma = 8
cells).  The oracle cannot run this size, so the checks are properties that
hold at any size:

* the gradient of 1/2 sum_q ||P_q(mu) - d_q||^2 through the
  torch.autograd.Function (qpat_vjp after the forward's fluence) along 32
  random directions: in FP64 on a cropped grid of the same configuration
  against central differences, every direction within 1e-4; at full size in
  FP32 against the FP64 GPU gradient and against central differences of the
  FP32 objective;
* forward-state checkpoints every 64 steps: resuming from a checkpoint
  reproduces the rest of the series bit for bit."""
import dataclasses

import numpy as np
import pytest

import phantoms
from gpu_helpers import to_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ILLUMS = (0b0001, 0b0010, 0b0100, 0b1000)


@pytest.fixture(scope="module")
def c3():
    from paper_1810_11685_gb300.binding import context_from_workload
    w = phantoms.C3
    ctx = context_from_workload(w, precision="fp32", max_batch=2)
    return w, ctx


def _objective(ctx, data):
    from paper_1810_11685_gb300.autograd import qpat_data

    def f(m):
        """per problem of the batch m ([B][n1][n0]), FP64 accumulation"""
        tot = 0.0
        for q, d in zip(ILLUMS, data):
            r = qpat_data(ctx, m, q).double() - d
            tot = tot + 0.5 * (r * r).sum(dim=(1, 2))
        return tot
    return f


def _gradient(f, mu):
    m = mu.clone().unsqueeze(0).requires_grad_(True)
    f(m).sum().backward()
    return m.grad[0].clone()


def _directions(w, k=32):
    rng = np.random.default_rng(5)
    return [to_gpu(rng.standard_normal(w.interior_shape), torch.float64) for _ in range(k)]


def test_c3_fp64_gradient_against_central_differences_cropped():
    """The differentiable workload's configuration (dx 0.05 mm, 28-cell PML,
    six inclusions, smooth random mu, four illuminated sides) on a cropped
    264^2 interior (320^2 FFT grid) with Nt = 1000, in FP64: the gradient of
    1/2 sum_q ||P_q(mu) - d_q||^2 against central differences (relative step
    1e-3) along 32 random directions, each within 1e-4 (measured max 2.4e-5)."""
    from paper_1810_11685_gb300.binding import context_from_workload
    w = dataclasses.replace(phantoms.C3, n=264, nt=1000)
    ctx = context_from_workload(w, precision="fp64", max_batch=2)
    mu = to_gpu(phantoms.optical_absorption(w), torch.float64)
    f = _objective(ctx, [ctx.forward(mu * 1.05, q)[0].double() for q in ILLUMS])
    g = _gradient(f, mu)
    errs = []
    with torch.no_grad():
        for v in _directions(w):
            eps = 1e-3 * float(torch.linalg.norm(mu) / torch.linalg.norm(v))
            fv = f(torch.stack([mu + eps * v, mu - eps * v]))
            an = float((g * v).sum())
            errs.append(abs(float(fv[0] - fv[1]) / (2 * eps) - an) / abs(an))
    assert max(errs) <= 1e-4, errs


def test_c3_gradient_fp32_against_fp64_and_central_differences(c3):
    """Full size, FP32 propagation.  (1) The FP32 gradient against the FP64
    GPU gradient (whose finite-difference check is the cropped test above),
    along the 32 directions: each directional derivative within 1e-4 of the
    RMS directional derivative, and the median within 1e-4 relative (measured:
    relative L2 1.3e-5 over the whole gradient; median 1.3e-5; the largest
    relative error, 5.5e-4, falls on a direction whose derivative is small).
    (2) Central differences of the FP32 objective at the relative step 1e-2
    (the measured crossover of truncation and FP32 rounding), each within
    5e-4 of the RMS derivative (measured below 1.1e-4 on six directions):
    the FP32 objective's rounding, divided by the step, keeps central
    differences from the 1e-4 bar in every direction."""
    from paper_1810_11685_gb300.binding import context_from_workload
    w, ctx = c3
    mu = to_gpu(phantoms.optical_absorption(w), torch.float64)
    dirs = _directions(w)
    c64 = context_from_workload(w, precision="fp64", max_batch=1)
    g64 = _gradient(_objective(c64, [c64.forward(mu * 1.05, q)[0].double() for q in ILLUMS]), mu)
    del c64
    torch.cuda.empty_cache()
    f = _objective(ctx, [ctx.forward(mu * 1.05, q)[0].double() for q in ILLUMS])
    g32 = _gradient(f, mu)
    an64 = np.array([float((g64 * v).sum()) for v in dirs])
    an32 = np.array([float((g32 * v).sum()) for v in dirs])
    rms = np.sqrt(np.mean(an64 ** 2))
    assert np.max(np.abs(an32 - an64)) <= 1e-4 * rms, (an32 - an64) / rms
    assert np.median(np.abs(an32 - an64) / np.abs(an64)) <= 1e-4
    fds = []
    with torch.no_grad():
        for v in dirs:
            eps = 1e-2 * float(torch.linalg.norm(mu) / torch.linalg.norm(v))
            fv = f(torch.stack([mu + eps * v, mu - eps * v]))
            fds.append(float(fv[0] - fv[1]) / (2 * eps))
    fds = np.array(fds)
    assert np.max(np.abs(fds - an32)) <= 5e-4 * rms, (fds - an32) / rms


def test_c3_checkpoints_every_64_steps(c3):
    w, ctx = c3
    p0 = to_gpu(phantoms.smooth_p0(w), torch.float32)
    K = 64
    data, ck = ctx.acoustic_forward_ckpt(p0, K)
    assert torch.equal(data, ctx.acoustic_forward(p0))
    n_ck = (w.nt - 1) // K
    assert n_ck == 62
    for m in (0, 31, n_ck - 1):
        out = ctx.acoustic_resume(ck, K, m, batch=1)
        first = (m + 1) * K
        assert torch.equal(out[:, first:], data[:, first:]), m
