"""Host side of the benchmark's CPU legs: the all-core oracle run spawns one
single-threaded process per problem, starts them together and times them
from the common start to the last finish."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import phantoms  # noqa: E402


def test_oracle_rate_parallel_two_workers():
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    before = {k: os.environ.get(k) for k in keys}
    w = phantoms.small(n=12, pml=4, nt=6, n_sensors=8, seed=3)
    rate, t = bench.oracle_rate_parallel(w, 6, 2, seed=5)
    assert t > 0
    assert rate == 2 * w.grid * w.grid * 6 * 2 / t
    assert {k: os.environ.get(k) for k in keys} == before      # thread caps are for the workers only


def test_host_cores_positive():
    assert bench.host_cores() >= 1



def test_host_cpu_record():
    h = bench.host_cpu()
    assert set(h) == {"machine", "cpu", "nproc"}
    assert h["nproc"] >= 1 and h["machine"]
