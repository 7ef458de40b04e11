"""Multi-rank host logic on CPU with two gloo ranks: unit assignment,
max-over-ranks timing, and the gradient sum over illuminations (eq. fre)
computed with the FP64 oracle, compared with the single-process sum."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import phantoms
    from oracle import acoustic, qpat
    from paper_1810_11685_gb300 import replicas
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = phantoms.small(n=12, pml=4, nt=20, n_sensors=8, seed=3)
    S = acoustic.setup_from_workload(w)
    mu = phantoms.optical_absorption(w)
    kappa = phantoms.optical_diffusion(w)
    g = np.zeros(w.interior_shape)
    for q in replicas.assign(4, rank, world):                  # 4 illuminations, one side each
        d = qpat.forward(S, mu * 1.1, kappa, 1 << q)          # synthetic measured data
        r = qpat.forward(S, mu, kappa, 1 << q) - d
        g += qpat.vjp(S, mu, kappa, 1 << q, r)
    gt = torch.from_numpy(g)
    replicas.sum_over_ranks(gt)
    tmax = replicas.max_over_ranks(1.0 + rank)
    out[rank] = (gt.numpy().copy(), tmax, replicas.assign(4, rank, world))
    dist.destroy_process_group()


def test_two_rank_gradient_sum_and_timing():
    import phantoms
    from oracle import acoustic, qpat
    from paper_1810_11685_gb300 import replicas
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    w = phantoms.small(n=12, pml=4, nt=20, n_sensors=8, seed=3)
    S = acoustic.setup_from_workload(w)
    mu = phantoms.optical_absorption(w)
    kappa = phantoms.optical_diffusion(w)
    ref = np.zeros(w.interior_shape)
    for q in range(4):
        d = qpat.forward(S, mu * 1.1, kappa, 1 << q)
        ref += qpat.vjp(S, mu, kappa, 1 << q, qpat.forward(S, mu, kappa, 1 << q) - d)
    for rank in range(2):
        g, tmax, units = out[rank]
        np.testing.assert_allclose(g, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        assert tmax == 2.0
    assert sorted(out[0][2] + out[1][2]) == [0, 1, 2, 3]
    assert replicas.throughput(10.0, 2, 4.0) == 5.0


def test_assign_balanced():
    from paper_1810_11685_gb300 import replicas
    for n in range(0, 13):
        for W in (1, 2, 3, 4, 8):
            parts = [replicas.assign(n, r, W) for r in range(W)]
            flat = [u for p in parts for u in p]
            assert flat == list(range(n))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
