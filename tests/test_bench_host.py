"""Host-side pieces of bench.py (no GPU): the oracle legs over several spawned
processes count the same units as one process, and the reference arm prints one
JSON line of the contract's shape."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench(ora):
    import bench as b

    return b


def test_split_rows_cover_the_same_work(bench):
    w = dict(model=2, N=4096, eps=1e-4, dt=0.01, seed=4)
    u1, e1, d1 = bench.oracle_steps(w, 12, 1)
    u2, e2, d2 = bench.oracle_steps(w, 12, 1, 0, 3)
    assert u1 == u2 == 3 * 12 * 4096
    assert e1 > 0 and e2 > 0
    assert "split over 3 processes" in d2 and "split" not in d1


def test_hmf_replicas_count_every_process(bench):
    w = dict(model=0, N=10**6, eps=0.0, dt=0.1, seed=2)
    u, el, d = bench.oracle_steps(w, 5000, 2, 1, 2)
    assert u == 2 * 5000 * 2 and el > 0 and d.startswith("2 processes")


def test_sample_size_scales_rows_with_processes(bench):
    w = dict(model=1, N=8192, eps=0.01, dt=0.05, seed=3)
    n = bench.oracle_sample_size(w, 0.2, 1, 4)
    assert 4 <= n <= 8192 and n % 4 == 0 or n == 8192
    w0 = dict(model=0, N=5 * 10**7, eps=0.0, dt=0.1, seed=2)
    assert bench.oracle_sample_size(w0, 60.0, 1, 8) <= 2_000_000


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "ring", "--steps", "1",
                        "--warmup", "0", "--cpu-cores", "2", "--n", "2048"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "pair-interactions/s" and d["value"] > 0
    assert d["cpu_baseline"]["cores"] == 2 and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_oracle_gradient_leg_counts_both_passes(bench):
    w = dict(model=2, N=262144, eps=1e-4, dt=0.01, seed=4)
    u, el, d = bench.oracle_grad(w, 0.3, 1, nsteps=4, cores=2)
    n = int(d.split(" particles")[0].split()[-1])
    assert u == 2 * float(n) * n * (6 * 4 + 1) and el > 0 and d.startswith("2 processes")


def test_reference_arm_under_torchrun_prints_once():
    """Two ranks launched as the multi-GPU bench is: rank 0 alone times the oracle and
    prints the line; the other rank exits 0 without work."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", "29613", "bench.py", "--impl", "reference",
                        "--gpus", "2", "--workload", "ring", "--steps", "1", "--warmup", "0", "--cpu-cores", "2",
                        "--particles", "2048"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0


def test_fp64_hmf_roofline_counts_three_stages_of_fp64_operations(bench):
    """The FP64 HMF path's roofline: 3 stages x 12 FP64 operations per particle-step
    against SMs x FP64 FMA per SM per clock x the sampled SM clock; without a clock
    record, the rate's own clock."""
    import numpy as np

    rates = np.zeros(19)
    rates[0], rates[13], rates[14] = 152, 2.0, 1900.0
    r = bench.hmf_fp64_roofline(1.45e10, rates, {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0})
    assert r["bound"] == "alu" and r["pipe"] == "fp64" and r["unit"] == "FP64 op/s"
    assert r["achieved"] == pytest.approx(1.45e10 * 3 * 12)
    assert r["peak"] == pytest.approx(152 * 2.0 * 2070e6)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"]) and 0.8 < r["frac"] < 0.85
    assert r["frac_at_max_clock"] == pytest.approx(r["frac"])
    r2 = bench.hmf_fp64_roofline(1.45e10, rates, {})
    assert r2["peak"] == pytest.approx(152 * 2.0 * 1900e6)
    json.dumps(r)
