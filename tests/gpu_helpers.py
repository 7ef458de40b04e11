"""Shared set-up for the GPU parity tests: one seeded workload feeds both the
CUDA context and the FP64 oracle (inputs from ``phantoms`` only)."""
import numpy as np

import phantoms
from oracle import acoustic


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make_pair(w, precision="fp64", max_batch=1, nt=None, **kw):
    """(GPU context, oracle setup) for workload ``w``."""
    from paper_1810_11685_gb300.binding import context_from_workload
    ctx = context_from_workload(w, precision=precision, max_batch=max_batch, nt=nt, **kw)
    S = acoustic.setup_from_workload(w, nt=nt)
    return ctx, S


def to_gpu(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def to_np(t):
    return t.detach().double().cpu().numpy()


def _oracle_job(job):
    """One oracle evaluation in a worker process: ("forward" | "adjoint",
    workload, nt, input array)."""
    kind, w, nt, x = job
    S = acoustic.setup_from_workload(w, nt=nt)
    return acoustic.forward(S, x) if kind == "forward" else acoustic.adjoint(S, x)


def oracle_many(jobs, procs=None):
    """Run independent oracle evaluations in spawned processes (safe after
    CUDA is up); results in job order."""
    import concurrent.futures
    import multiprocessing as mp
    import os
    n = procs or min(len(jobs), max(1, (os.cpu_count() or 1)))
    with concurrent.futures.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_oracle_job, jobs))
