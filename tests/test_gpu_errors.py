"""Error returns and degenerate sizes through the C ABI (GPU): invalid
configurations and arguments come back as status codes before any kernel
runs, and the smallest valid problem (8-point FFT extent, two samples)
matches the oracle."""
import numpy as np
import pytest

import phantoms
from oracle import acoustic
from gpu_helpers import make_pair, rel_l2, to_gpu, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EINVAL, EUNSTABLE = 1, 2


def _ctx_args(w, **over):
    c, rho, alpha = phantoms.acoustic_medium(w)
    kw = dict(dx=w.dx, dt=phantoms.time_step(w, c), nt=w.nt, pml=w.pml, y=w.y, precision="fp64")
    kw.update(over)
    return (c, rho, alpha, phantoms.optical_diffusion(w), phantoms.sensor_positions(w)), kw


def _status(fn):
    from paper_1810_11685_gb300.binding import QpatError
    with pytest.raises(QpatError) as e:
        fn()
    return e.value.status


def test_create_rejects_invalid_configurations():
    from paper_1810_11685_gb300.binding import Context
    w = phantoms.small(n=14, pml=4, nt=10, n_sensors=6, seed=1)          # FFT extent 22 = 2 x 11
    a, kw = _ctx_args(w)
    assert _status(lambda: Context(*a, **kw)) == EINVAL
    w = phantoms.small(n=16, pml=4, nt=10, n_sensors=6, seed=1)
    a, kw = _ctx_args(w, nt=1)
    assert _status(lambda: Context(*a, **kw)) == EINVAL
    a, kw = _ctx_args(w)
    kw["dt"] *= 10.0                                                    # c dt / dx far above the limit
    assert _status(lambda: Context(*a, **kw)) == EUNSTABLE
    a, kw = _ctx_args(w)
    far = np.array([[1.0, 1.0]])                                        # 1 m away: outside the grid
    assert _status(lambda: Context(a[0], a[1], a[2], a[3], far, **kw)) == EINVAL
    a, kw = _ctx_args(w, y=2.0)                                         # tan(pi y / 2) singular
    assert _status(lambda: Context(*a, **kw)) == EINVAL


def test_calls_reject_invalid_arguments():
    w = phantoms.small(n=16, pml=4, nt=10, n_sensors=6, seed=1)
    ctx, _ = make_pair(w, "fp64", max_batch=2)
    p0 = to_gpu(np.zeros((3,) + w.interior_shape), torch.float64)     # batch 3 > max_batch 2
    assert _status(lambda: ctx.acoustic_forward(p0)) == EINVAL
    mu = to_gpu(phantoms.optical_absorption(w), torch.float64)
    assert _status(lambda: ctx.da_solve(mu, 0)) == EINVAL              # no illuminated side
    assert _status(lambda: ctx.da_solve(mu, 1 << 4)) == EINVAL         # side 4 does not exist in 2D
    data = torch.zeros(0, w.nt, w.n_sensors, dtype=torch.float64, device="cuda")
    assert _status(lambda: ctx.ld_solve(data, (), mu, k_max=1)) == EINVAL


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-4)])
def test_smallest_problem_matches_oracle(prec, tol):
    """8-point FFT extent (4 interior nodes, PML 2), two samples: the first
    sample sees half the source (eq. s1), the second one step."""
    w = phantoms.small(n=4, pml=2, nt=2, n_sensors=3, seed=2)
    ctx, S = make_pair(w, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    p0 = phantoms.smooth_p0(w)
    got = to_np(ctx.acoustic_forward(to_gpu(p0, dt)))[0]
    assert rel_l2(got, acoustic.forward(S, p0)) <= tol
    W = phantoms.random_field((w.nt, w.n_sensors), 3)
    got = to_np(ctx.acoustic_adjoint(to_gpu(W, dt)))[0]
    assert rel_l2(got, acoustic.adjoint(S, W)) <= tol


def test_grid_barrier_wait_gives_up_and_device_stays_usable():
    """The bounded grid barrier of the cooperative kernels: with one CTA that
    never arrives, the others' waits give up after the limit and the call
    reports QPAT_ETIMEOUT; the device then runs the full check and a
    propagation normally."""
    from paper_1810_11685_gb300.binding import qpat_barrier_check
    assert qpat_barrier_check(blocks=152, rounds=8, absent=0, limit_s=1.0) == 0
    assert qpat_barrier_check(blocks=152, rounds=8, absent=1, limit_s=0.05) == 5
    assert qpat_barrier_check(blocks=152, rounds=8, absent=0, limit_s=1.0) == 0
    w = phantoms.small(n=24, pml=4, nt=20, n_sensors=8, seed=3)
    ctx, S = make_pair(w, "fp64")
    p0 = phantoms.random_field(w.interior_shape, 2)
    got = to_np(ctx.acoustic_forward(to_gpu(p0, torch.float64)))[0]
    assert rel_l2(got, acoustic.forward(S, p0)) <= 1e-10
    ctx.sync()
