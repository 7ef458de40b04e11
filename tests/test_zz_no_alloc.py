"""qpat_dot_noalloc: the inner product for callers that may not allocate
device memory at the call (a frozen memory pool, a host framework owning all
device allocations, an inner solver loop where cudaMalloc would synchronise).
Its scratch is a fixed array inside the library; the test checks, through the
C ABI, that it returns what the context-based qpat_dot returns, on two calls
in a row (the second call reuses the scratch the first one left behind).
This file is collected last so a failure here stops a run only after every
other test has run."""
import numpy as np
import pytest

import phantoms
from gpu_helpers import make_pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_dot_matches_context_dot_twice(prec):
    from paper_1810_11685_gb300.binding import QpatError, qpat_dot_noalloc
    w = phantoms.small(n=40, pml=8, nt=30, n_sensors=8, seed=1)
    ctx, _ = make_pair(w, prec, max_batch=6)
    dt = torch.float32 if prec == "fp32" else torch.float64
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    for call in range(2):
        g = torch.Generator(device="cpu").manual_seed(call)
        a = torch.randn(6, 50000 + 17 * call, generator=g, dtype=torch.float64).to("cuda", dt)
        b = torch.randn(6, 50000 + 17 * call, generator=g, dtype=torch.float64).to("cuda", dt)
        qpat_dot_noalloc(a, b, out)
        ref = ctx.dot(a, b)                      # synchronises the stream
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
        exact = (a.double() * b.double()).sum(dim=1).cpu().numpy()
        np.testing.assert_allclose(got, exact, rtol=1e-9)
    with pytest.raises(QpatError):
        big = torch.zeros(65, 4, dtype=dt, device="cuda")
        qpat_dot_noalloc(big, big, torch.empty(65, dtype=torch.float64, device="cuda"))


def test_noalloc_dot_rejects_bad_buffers_before_the_call():
    """Inputs the kernels would misread (wrong dtype, host memory, a short or
    mistyped output) are refused in the binding, before any device access."""
    from paper_1810_11685_gb300.binding import qpat_dot_noalloc
    a = torch.ones(3, 8, dtype=torch.float32, device="cuda")
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        qpat_dot_noalloc(a.half(), a.half(), out)
    with pytest.raises(TypeError):
        qpat_dot_noalloc(a.to(torch.int32), a.to(torch.int32), out)
    with pytest.raises(TypeError):
        qpat_dot_noalloc(a.cpu(), a.cpu(), out)
    with pytest.raises(ValueError):
        qpat_dot_noalloc(a, a, torch.empty(2, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        qpat_dot_noalloc(a, a, torch.empty(3, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        qpat_dot_noalloc(a, a.double(), out)
    # a transposed (non-contiguous) view is made contiguous, not misread
    t = torch.arange(24, dtype=torch.float64, device="cuda").reshape(8, 3).t()
    got = qpat_dot_noalloc(t, t, out).cpu().numpy()
    np.testing.assert_allclose(got, (t * t).sum(dim=1).cpu().numpy(), rtol=1e-14)
