"""GPU parity of H_a and H_a^* (Section 3.2.3 and Lemma 2) against the FP64
oracle, element by element on the same seeded inputs, through the C ABI.

Tolerances: FP64 path vs oracle relative L2 <= 1e-10; FP32 path vs oracle
relative L2 <= 2e-4 over the whole sensor series; dot-product test
<= 1e-12 (FP64) and <= 1e-5 (FP32)."""
import numpy as np
import pytest

import phantoms
from oracle import acoustic
from gpu_helpers import make_pair, rel_l2, to_gpu, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    # interior n, pml -> FFT extents 56 (8 7), 40 (8 5), 54 (2 27)
    "lossy-56": dict(n=40, pml=8, nt=70),
    "lossless-56": dict(n=40, pml=8, nt=70, lossless=True),
    "lossy-40-y11": dict(n=30, pml=5, nt=50, y=1.1),
    "lossy-54": dict(n=44, pml=5, nt=64, seed=3),
}


def workload(name):
    kw = dict(CASES[name])
    kw.setdefault("n_sensors", 16)
    return phantoms.small(**kw)


@pytest.mark.parametrize("name", list(CASES))
def test_forward_fp64_matches_oracle(name):
    w = workload(name)
    ctx, S = make_pair(w, "fp64")
    p0 = phantoms.smooth_p0(w) + 0.1 * phantoms.random_field(w.interior_shape, 3)
    ref = acoustic.forward(S, p0)
    got = to_np(ctx.acoustic_forward(to_gpu(p0, torch.float64)))[0]
    ctx.sync()
    assert rel_l2(got, ref) <= 1e-10


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_fp64_matches_oracle(name):
    w = workload(name)
    ctx, S = make_pair(w, "fp64")
    W = phantoms.random_field((w.nt, w.n_sensors), 4)
    ref = acoustic.adjoint(S, W)
    got = to_np(ctx.acoustic_adjoint(to_gpu(W, torch.float64)))[0]
    ctx.sync()
    assert rel_l2(got, ref) <= 1e-10


@pytest.mark.parametrize("name", ["lossy-56", "lossless-56"])
def test_forward_fp32_matches_oracle(name):
    w = workload(name)
    ctx, S = make_pair(w, "fp32")
    p0 = phantoms.smooth_p0(w)
    ref = acoustic.forward(S, p0)
    got = to_np(ctx.acoustic_forward(to_gpu(p0, torch.float32)))[0]
    assert rel_l2(got, ref) <= 2e-4
    W = phantoms.random_field((w.nt, w.n_sensors), 4)
    ref = acoustic.adjoint(S, W)
    got = to_np(ctx.acoustic_adjoint(to_gpu(W, torch.float32)))[0]
    assert rel_l2(got, ref) <= 2e-4


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_dot_product_on_gpu(prec, tol):
    w = workload("lossy-54")
    ctx, _ = make_pair(w, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    p0 = to_gpu(phantoms.random_field(w.interior_shape, 11), dt)
    W = to_gpu(phantoms.random_field((w.nt, w.n_sensors), 12), dt)
    Hp = ctx.acoustic_forward(p0)
    HtW = ctx.acoustic_adjoint(W)
    lhs = ctx.dot(Hp, W.unsqueeze(0))[0]
    rhs = ctx.dot(p0.unsqueeze(0), HtW)[0]
    assert abs(lhs - rhs) <= tol * max(abs(lhs), abs(rhs))


def test_batch_equals_single():
    w = workload("lossy-40-y11")
    ctx, _ = make_pair(w, "fp32", max_batch=3)
    p0 = torch.stack([to_gpu(phantoms.random_field(w.interior_shape, 20 + b), torch.float32) for b in range(3)])
    batched = ctx.acoustic_forward(p0)
    for b in range(3):
        single = ctx.acoustic_forward(p0[b])
        assert torch.equal(batched[b], single[0])
    W = to_gpu(np.stack([phantoms.random_field((w.nt, w.n_sensors), 30 + b) for b in range(3)]), torch.float32)
    batched = ctx.acoustic_adjoint(W)
    for b in range(3):
        assert torch.equal(batched[b], ctx.acoustic_adjoint(W[b])[0])


def test_c1_fp64_full_size():
    """128^2 interior + 20-cell PML (168^2 FFT grid), Nt = 600, 128 sensors on
    a 5.5 mm circle: the FP64 path against the oracle over the full series,
    and the FP32 path against the same oracle."""
    w = phantoms.C1
    ctx, S = make_pair(w, "fp64")
    p0 = phantoms.smooth_p0(w)
    ref = acoustic.forward(S, p0)
    got = to_np(ctx.acoustic_forward(to_gpu(p0, torch.float64)))[0]
    assert rel_l2(got, ref) <= 1e-10
    ctx32, _ = make_pair(w, "fp32")
    got32 = to_np(ctx32.acoustic_forward(to_gpu(p0, torch.float32)))[0]
    assert rel_l2(got32, ref) <= 2e-4


def test_nonfinite_detection():
    """A NaN in the input surfaces as QPAT_ENONFINITE at the next sync."""
    from paper_1810_11685_gb300 import QpatError
    w = workload("lossy-56")
    ctx, _ = make_pair(w, "fp32")
    p0 = np.zeros(w.interior_shape)
    p0[5, 7] = np.nan
    ctx.acoustic_forward(to_gpu(p0, torch.float32))
    with pytest.raises(QpatError) as e:
        ctx.sync()
    assert e.value.status == 3
    ctx.acoustic_forward(to_gpu(np.ones(w.interior_shape), torch.float32))
    ctx.sync()   # flag cleared, healthy call passes
