"""Element-by-element parity of the length-specialised passes that only the
large workloads use, against the FP64 oracle on the same seeded inputs, in
the launch configuration of those workloads:

* 2D extents 1080 (the 1024^2 differentiable workload, pml 28) and 1024
  (960^2 interior, pml 32): FP32 (specialised passes, 4-column CTAs) and FP64
  over the first 40 steps, batch of two white-noise initial pressures (so that
  the perimeter sensors see signal from the first step), forward and adjoint;
* 3D extent 288 (the 256^3 workload): FP32 (specialised x, y and z passes)
  and FP64 over its first three steps, batch of one, the sensor series and the
  whole adjoint field (256^3 values).

The oracle runs in spawned worker processes, one evaluation each."""
import dataclasses

import numpy as np
import pytest

import phantoms
from gpu_helpers import make_pair, oracle_many, rel_l2, to_gpu, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NT2 = 40
W2 = {
    "1080": dataclasses.replace(phantoms.C3, nt=NT2),
    "1024": dataclasses.replace(phantoms.C3, n=960, pml=32, nt=NT2, name="2d-960"),
}


@pytest.fixture(scope="module")
def oracle2d():
    inputs, jobs = {}, []
    for name, w in W2.items():
        p0 = np.stack([phantoms.random_field(w.interior_shape, 40), phantoms.random_field(w.interior_shape, 41)])
        W = phantoms.random_field((NT2, w.n_sensors), 9)
        inputs[name] = (p0, W)
        jobs += [("forward", w, NT2, p0[0]), ("forward", w, NT2, p0[1]), ("adjoint", w, NT2, W)]
    res = oracle_many(jobs)
    return {name: (inputs[name], res[3 * k:3 * k + 3]) for k, name in enumerate(W2)}


@pytest.mark.parametrize("name", list(W2))
@pytest.mark.parametrize("prec,tol", [("fp32", 2e-4), ("fp64", 1e-10)])
def test_large_2d_extent_against_oracle(oracle2d, name, prec, tol):
    w = W2[name]
    assert w.grid == int(name)
    (p0, W), (f0, f1, adj) = oracle2d[name]
    ctx, _ = make_pair(w, prec, max_batch=2, nt=NT2)
    dt = torch.float32 if prec == "fp32" else torch.float64
    got = to_np(ctx.acoustic_forward(to_gpu(p0, dt)))
    assert rel_l2(got[0], f0) <= tol
    assert rel_l2(got[1], f1) <= tol
    a = to_np(ctx.acoustic_adjoint(to_gpu(np.stack([W, W]), dt)))
    assert rel_l2(a[0], adj) <= tol
    assert np.array_equal(a[0], a[1])
    ctx.sync()


NT3 = 3
W3 = dataclasses.replace(phantoms.C5, nt=NT3)


@pytest.fixture(scope="module")
def oracle3d():
    p0 = phantoms.random_field(W3.interior_shape, 7)
    W = phantoms.random_field((NT3, W3.n_sensors), 8)
    f, a = oracle_many([("forward", W3, NT3, p0), ("adjoint", W3, NT3, W)])
    return p0, W, f, a


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-4), ("fp64", 1e-10)])
def test_3d_288_against_oracle(oracle3d, prec, tol):
    p0, W, f, a = oracle3d
    assert W3.grid == 288
    ctx, _ = make_pair(W3, prec, nt=NT3)
    dt = torch.float32 if prec == "fp32" else torch.float64
    got = to_np(ctx.acoustic_forward(to_gpu(p0, dt)))[0]
    assert rel_l2(got, f) <= tol
    got = to_np(ctx.acoustic_adjoint(to_gpu(W, dt)))[0]
    assert got.shape == W3.interior_shape
    assert rel_l2(got, a) <= tol
    ctx.sync()
    del ctx
    torch.cuda.empty_cache()
