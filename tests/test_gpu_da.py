"""GPU parity of the diffusion solve (eq. DA, finite-volume form) under both
preconditioners of its conjugate gradients, against the FP64 oracle's sparse
direct solve, through the C ABI.

The multigrid V-cycle and the diagonal preconditioner must reach the same
solution (relative residual 1e-13, compared at 1e-9); the V-cycle must do it
in a few tens of iterations where the grid halves down to a small one."""
import dataclasses

import numpy as np
import pytest

import phantoms
from oracle import optics
from gpu_helpers import make_pair, rel_l2, to_gpu, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def batch_mu(w, B):
    return np.stack([phantoms.optical_absorption(w, seed_offset=b) for b in range(B)])


@pytest.mark.parametrize("precond", ["multigrid", "jacobi"])
@pytest.mark.parametrize("n,pml", [(32, 4), (36, 6), (30, 5), (42, 3)])
def test_da_solve_batch_matches_oracle(precond, n, pml):
    # 32: halves down to 2 x 2; 36: to 9 x 9; 30: one coarse level (15 x 15);
    # 42: to 21 x 21
    w = phantoms.small(n=n, pml=pml, nt=8, n_sensors=6, seed=5)
    B, illum = 3, 0b1011
    ctx, _ = make_pair(w, "fp64", max_batch=B, da_precond=precond)
    mu = batch_mu(w, B)
    kappa = phantoms.optical_diffusion(w)
    got = to_np(ctx.da_solve(to_gpu(mu, torch.float64), illum))
    iters = ctx.stats()["pcg_iterations"]
    for b in range(B):
        ref = optics.fluence(mu[b], kappa, w.dx, illum)
        assert rel_l2(got[b], ref) <= 1e-9, (b, rel_l2(got[b], ref))
    assert iters > 0
    if precond == "multigrid" and n in (32, 36):
        assert iters <= 40, iters


def test_da_solve_graph_and_direct_launches_agree():
    w = phantoms.small(n=32, pml=4, nt=8, n_sensors=6, seed=9)
    mu = to_gpu(batch_mu(w, 2), torch.float64)
    out = []
    for no_graphs in (False, True):
        ctx, _ = make_pair(w, "fp64", max_batch=2, no_graphs=no_graphs)
        out.append(to_np(ctx.da_solve(mu, 0b0110)))
        # a second call replays the cached chunk (or relaunches directly)
        out.append(to_np(ctx.da_solve(mu, 0b0110)))
    for o in out[1:]:
        assert np.array_equal(o, out[0])


def test_da_solve_512_multigrid_sampled_parity():
    # the 512 x 512 optical grid of the 2D workloads (dx = 0.05 mm)
    w = dataclasses.replace(phantoms.C2, nt=8)
    ctx, _ = make_pair(w, "fp64", max_batch=1, nt=8)
    mu = phantoms.optical_absorption(w)
    kappa = phantoms.optical_diffusion(w)
    got = to_np(ctx.da_solve(to_gpu(mu[None], torch.float64), 0b1111))[0]
    iters = ctx.stats()["pcg_iterations"]
    ref = optics.fluence(mu, kappa, w.dx, 0b1111)
    assert rel_l2(got, ref) <= 1e-9
    assert iters <= 40, iters
