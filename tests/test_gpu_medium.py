"""GPU parity of the derivatives of H_a in the sound speed and the density
(qpat_jvp_medium, qpat_vjp_medium) through the C ABI, against the FP64
oracle (``oracle/medium.py``), element by element, 2D, lossy and lossless,
with FP64 sweeps and with FP32 sweeps (FP64 gradient sums).  At the
128^2-interior, 600-step size of the paper's 2D grids the tests check the
transpose identity and the density-scale invariance, which hold at any size,
and compare the first 60 steps with the oracle.

FP32 bounds: each FP32 sweep rounds every field once per operation (unit
roundoff 6e-8) through about ten FFT stages and pointwise updates per step.
Measured on GB300: relative l2 errors of 3e-7 to 1e-6 for the tangent and the
gradients on the small grids over 24-30 steps; at 168^2 over 600 steps
0.8e-5 to 1.9e-5 against the FP64 sweeps and 5e-6 to 1.3e-5 for the
transpose identity, whose two sides come from independent FP32 sweeps.  The bound is
1e-4 (the FP32 sensor-series bound of the propagation tests, halved) for
all of them."""
import numpy as np
import pytest

import phantoms
from oracle import acoustic, medium
from gpu_helpers import make_pair, rel_l2, to_gpu, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs(w, S, seed):
    rng = np.random.default_rng(seed)
    c = np.sqrt(S.C)
    p0 = phantoms.smooth_p0(w, seed)
    dc = c * rng.standard_normal(S.shape) * 0.05
    drho = S.rho0 * rng.standard_normal(S.shape) * 0.05
    W = rng.standard_normal((w.nt, w.n_sensors))
    return p0, dc, drho, W


@pytest.mark.parametrize("n,pml,nt,lossless", [(16, 4, 30, False), (16, 4, 30, True), (20, 4, 24, False)])
def test_medium_derivatives_match_oracle(n, pml, nt, lossless):
    w = phantoms.small(n=n, pml=pml, nt=nt, lossless=lossless, seed=n + nt, n_sensors=10)
    ctx, S = make_pair(w, "fp64")
    p0, dc, drho, W = _inputs(w, S, 7)
    P0 = acoustic.embed(S, p0)
    ref = medium.jvp_medium(S, w.y, P0, dc, drho)
    got = ctx.jvp_medium(to_gpu(p0, torch.float64), to_gpu(dc, torch.float64), to_gpu(drho, torch.float64))
    assert rel_l2(to_np(got), ref) <= 1e-10
    only_c = ctx.jvp_medium(to_gpu(p0, torch.float64), to_gpu(dc, torch.float64))
    assert rel_l2(to_np(only_c), medium.jvp_medium(S, w.y, P0, dc, 0 * drho)) <= 1e-10
    rc, rr = medium.vjp_medium(S, w.y, P0, W)
    gc, gr = ctx.vjp_medium(to_gpu(p0, torch.float64), to_gpu(W, torch.float64))
    assert rel_l2(to_np(gc), rc) <= 1e-10
    assert rel_l2(to_np(gr), rr) <= 1e-10


def test_medium_derivatives_full_size_properties():
    """128^2 interior with a 20-node PML (168^2 FFT grid), 600 steps: the
    transpose identity to 1e-12, the density-scale invariance, and the first
    60 steps against the oracle."""
    w = phantoms.C1
    ctx, S = make_pair(w, "fp64")
    p0, dc, drho, W = _inputs(w, S, 11)
    g = lambda a: to_gpu(a, torch.float64)
    jv = to_np(ctx.jvp_medium(g(p0), g(dc), g(drho)))
    gc, gr = ctx.vjp_medium(g(p0), g(W))
    gc, gr = to_np(gc), to_np(gr)
    lhs = float(np.sum(jv * W))
    rhs_c, rhs_r = float(np.sum(gc * dc)), float(np.sum(gr * drho))
    assert abs(lhs - rhs_c - rhs_r) <= 1e-12 * (abs(rhs_c) + abs(rhs_r))
    assert abs(float(np.sum(gr * S.rho0))) <= 1e-11 * np.linalg.norm(gr) * np.linalg.norm(S.rho0)
    ctx60, S60 = make_pair(w, "fp64", nt=60)
    ref = medium.jvp_medium(S60, w.y, acoustic.embed(S60, p0), dc, drho)
    got = to_np(ctx60.jvp_medium(g(p0), g(dc), g(drho)))
    assert rel_l2(got, ref) <= 1e-10
    np.testing.assert_allclose(got, jv[:60], rtol=0, atol=1e-12 * np.abs(jv[:60]).max())


FP32_TOL = 1e-4


@pytest.mark.parametrize("n,pml,nt,lossless", [(16, 4, 30, False), (16, 4, 30, True), (20, 4, 24, False)])
def test_medium_derivatives_fp32_sweeps_match_oracle(n, pml, nt, lossless):
    """FP32 sweeps with FP64 gradient sums against the FP64 oracle."""
    w = phantoms.small(n=n, pml=pml, nt=nt, lossless=lossless, seed=n + nt, n_sensors=10)
    ctx, S = make_pair(w, "fp32")
    p0, dc, drho, W = _inputs(w, S, 7)
    P0 = acoustic.embed(S, p0)
    g = lambda a: to_gpu(a, torch.float64)
    ref = medium.jvp_medium(S, w.y, P0, dc, drho)
    got = ctx.jvp_medium(g(p0), g(dc), g(drho))
    assert got.dtype == torch.float64
    e = rel_l2(to_np(got), ref)
    assert e <= FP32_TOL, e
    rc, rr = medium.vjp_medium(S, w.y, P0, W)
    gc, gr = ctx.vjp_medium(g(p0), g(W))
    ec, er = rel_l2(to_np(gc), rc), rel_l2(to_np(gr), rr)
    assert ec <= FP32_TOL and er <= FP32_TOL, (ec, er)


def test_medium_derivatives_fp32_full_size():
    """128^2 interior (168^2 FFT grid), 600 steps, FP32 sweeps: the transpose
    identity, the first 60 steps of the tangent against the oracle, and the
    FP32-sweep tangent and gradient against the FP64-sweep ones."""
    w = phantoms.C1
    ctx, S = make_pair(w, "fp32")
    p0, dc, drho, W = _inputs(w, S, 11)
    g = lambda a: to_gpu(a, torch.float64)
    jv = to_np(ctx.jvp_medium(g(p0), g(dc), g(drho)))
    gc, gr = ctx.vjp_medium(g(p0), g(W))
    gc, gr = to_np(gc), to_np(gr)
    lhs = float(np.sum(jv * W))
    rhs_c, rhs_r = float(np.sum(gc * dc)), float(np.sum(gr * drho))
    ident = abs(lhs - rhs_c - rhs_r) / (abs(rhs_c) + abs(rhs_r))
    assert ident <= FP32_TOL, ident
    ctx64, _ = make_pair(w, "fp64")
    jv64 = to_np(ctx64.jvp_medium(g(p0), g(dc), g(drho)))
    gc64, gr64 = (to_np(t) for t in ctx64.vjp_medium(g(p0), g(W)))
    errs = rel_l2(jv, jv64), rel_l2(gc, gc64), rel_l2(gr, gr64)
    assert max(errs) <= FP32_TOL, errs
    ctx60, S60 = make_pair(w, "fp32", nt=60)
    ref = medium.jvp_medium(S60, w.y, acoustic.embed(S60, p0), dc, drho)
    e = rel_l2(to_np(ctx60.jvp_medium(g(p0), g(dc), g(drho))), ref)
    assert e <= FP32_TOL, e


def test_medium_errors():
    from paper_1810_11685_gb300.binding import QpatError
    w = phantoms.small(n=16, pml=4, nt=12, seed=3, n_sensors=6)
    w3 = phantoms.small(n=8, pml=4, nt=6, dim=3, seed=3, n_sensors=6)
    ctx3, _ = make_pair(w3, "fp64")
    with pytest.raises(QpatError) as e:
        ctx3.jvp_medium(to_gpu(phantoms.smooth_p0(w3, 1), torch.float64))
    assert e.value.status == 1
    p0 = to_gpu(phantoms.smooth_p0(w, 1), torch.float64)
    ctx64, _ = make_pair(w, "fp64")
    assert ctx64._lib.qpat_jvp_medium(ctx64._ptr, None, None, None, None) == 1
    assert ctx64._lib.qpat_vjp_medium(ctx64._ptr, p0.data_ptr(), None, None, None) == 1
    zero = to_np(ctx64.jvp_medium(p0))                   # no direction: zero derivative
    assert np.all(zero == 0.0)


@pytest.mark.parametrize("lossless,prec", [(False, "fp64"), (True, "fp64"), (False, "fp32")])
def test_medium_gradient_checkpoints_give_the_same_gradient(lossless, prec):
    """The gradient from forward-state checkpoints (the tape recomputed segment
    by segment) equals the whole-history gradient bit for bit, for segment
    lengths that divide Nt and that leave a short last segment, and matches
    the oracle."""
    w = phantoms.small(n=20, pml=4, nt=30, lossless=lossless, seed=5, n_sensors=10)
    ctx, S = make_pair(w, prec)
    p0, _, _, W = _inputs(w, S, 13)
    g = lambda a: to_gpu(a, torch.float64)
    ctx.set_medium_checkpoints(w.nt)
    full = [t.clone() for t in ctx.vjp_medium(g(p0), g(W))]
    for K in (1, 5, 7, 29):
        ctx.set_medium_checkpoints(K)
        got = ctx.vjp_medium(g(p0), g(W))
        assert torch.equal(got[0], full[0]) and torch.equal(got[1], full[1]), K
    ctx.set_medium_checkpoints(0)
    rc, rr = medium.vjp_medium(S, w.y, acoustic.embed(S, p0), W)
    tol = 1e-10 if prec == "fp64" else FP32_TOL
    assert rel_l2(to_np(full[0]), rc) <= tol
    assert rel_l2(to_np(full[1]), rr) <= tol
