"""Full-size checks of the differentiable 2D workload: 1024^2 interior
(1080^2 FFT grid), Nt = 4000, FP32 propagation with FP64 reductions, four
illuminated sides, a smooth random mu (Gaussian-filtered noise, sigma = 8
cells).  The oracle cannot run this size, so the checks are properties that
hold at any size:

* the gradient of 1/2 sum_q ||P_q(mu) - d_q||^2 through the
  torch.autograd.Function (qpat_vjp after the forward's fluence) against
  central differences of the GPU objective along 32 random directions;
* forward-state checkpoints every 64 steps: resuming from a checkpoint
  reproduces the rest of the series bit for bit."""
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


def test_c3_gradient_against_central_differences(c3):
    from paper_1810_11685_gb300.autograd import qpat_data
    w, ctx = c3
    mu = to_gpu(phantoms.optical_absorption(w), torch.float64)
    data = [ctx.forward(mu * 1.05, q)[0].double() for q in ILLUMS]

    def objective(m):
        """per problem of the batch m ([B][n1][n0]), FP64 accumulation"""
        tot = 0.0
        for q, d in zip(ILLUMS, data):
            r = qpat_data(ctx, m, q).double() - d
            tot = tot + 0.5 * (r * r).sum(dim=(1, 2))
        return tot

    m = mu.clone().unsqueeze(0).requires_grad_(True)
    objective(m).sum().backward()
    g = m.grad[0].clone()
    rng = np.random.default_rng(5)
    fds, ans = [], []
    with torch.no_grad():
        for _ in range(32):
            v = to_gpu(rng.standard_normal(w.interior_shape), torch.float64)
            eps = 1e-3 * float(torch.linalg.norm(mu) / torch.linalg.norm(v))
            f = objective(torch.stack([mu + eps * v, mu - eps * v]))
            fds.append(float(f[0] - f[1]) / (2 * eps))
            ans.append(float((g * v).sum()))
    fds, ans = np.array(fds), np.array(ans)
    # FP32 series, FP64 objective: each central difference carries the FP32
    # rounding of two forward runs (measured: 5e-5 to 2e-3 of the directional
    # derivative), so the median relative error is bounded, and every
    # direction's error against the typical derivative size
    rel = np.abs(fds - ans) / np.abs(ans)
    assert np.median(rel) <= 1e-3, rel
    assert np.max(np.abs(fds - ans)) <= 1e-2 * np.sqrt(np.mean(ans ** 2)), rel


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
