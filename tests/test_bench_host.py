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


def test_algorithmic_bytes_per_cell_step():
    """State z_n read and written ((2 d + 1) fields), one read of c, rho-bar,
    the d staggered rho-bar_i and alpha0 where it varies: 60 B in 2D FP32
    with alpha0(r), 76 B in 3D FP32 with a uniform alpha0."""
    assert bench.b_alg(2) == 60
    assert bench.b_alg(3, alpha_varies=False) == 76
    assert bench.b_alg(2, "f64") == 120


def test_step_roofline_fraction_is_recomputable():
    r = bench.roofline_step(2.0e10, 2, 12 * 576 * 576, traffic=123.0, what="step")
    assert r["achieved"] == 2.0e10 * 60 / 1e9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15
    assert r["alg_bytes_per_launch"] == 60 * 12 * 576 * 576 and r["traffic"] == 123.0


def test_parse_medium_precision(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "medium", "--medium-precision", "fp32"])
    a = bench.parse()
    assert a.workload == "medium" and a.medium_precision == "fp32"
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    assert bench.parse().medium_precision == "fp64"
