"""Host side of the benchmark: the product count behind GFLOP/s, the
algorithmic bytes behind the roofline fraction, and the reference arm's JSON
line (the oracle on the host cores), all without a GPU."""
import json
import os
import subprocess
import sys

import numpy as np

import gen
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_products_count_matches_oracle_and_brute_force():
    import bench
    A = gen.er_variable(300, 200, 12, 3, np.float64, "uniform", p_empty=0.2)
    B = gen.er_variable(200, 250, 9, 4, np.float64, "uniform", p_empty=0.2)
    brute = sum(int(B.rowptr[k + 1] - B.rowptr[k]) for i in range(A.nrows)
                for k in A.col[A.rowptr[i]:A.rowptr[i + 1]])
    assert bench.products(A, B) == brute == int(oracle.row_products(A, B).sum())


def test_algorithmic_bytes_by_hand():
    import bench
    # A: 2 x 3 with 3 entries, B: 3 x 2 with 4 entries, C with 3 entries
    A = gen.CSR(2, 3, np.array([0, 2, 3]), np.array([0, 2, 1], dtype=np.int32), np.ones(3))
    B = gen.CSR(3, 2, np.array([0, 2, 3, 4]), np.array([0, 1, 0, 1], dtype=np.int32), np.ones(4))
    num, sym = bench.algorithmic_bytes(A, B, 3, val_bytes=8)
    # numeric: A (row_ptr 12 + 3 x 12) + B (row_ptr 16 + 4 x 12) + C row_ptr 12 + C 3 x 12
    assert num == (12 + 36) + (16 + 48) + 12 + 36
    # symbolic: A (12 + 3 x 4) + B (16 + 4 x 4) + C row_ptr 12
    assert sym == (12 + 12) + (16 + 16) + 12
    num4, _ = bench.algorithmic_bytes(A, B, 3, val_bytes=4)
    assert num - num4 == 4 * (3 + 4 + 3)


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n-log2", "11",
                          "--d", "8", "--steps", "2", "--warmup", "1"], capture_output=True, text=True, env=env,
                         timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert d["config"]["workload"].startswith("ER A*B n=2^11 d=8")
    assert set(d["config"]) == {"workload", "parallelism"}
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_other_ranks_of_the_reference_arm_exit_quietly():
    env = dict(os.environ, RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n-log2", "10",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300,
                         cwd=ROOT)
    assert out.returncode == 0 and not [x for x in out.stdout.splitlines() if x.startswith("{")]


def test_cpu_baseline_reports_trials_threads_and_model():
    import bench
    A = gen.er(2048, 2048, 8, 0)
    cb = bench.cpu_baseline(A, A, 512, trials=2)
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1
    assert cb["all_cores"]["threads"] == cb["cores"] and cb["single_thread"]["threads"] == 1
    assert cb["all_cores"]["best"] >= cb["all_cores"]["mean"] > 0
    assert isinstance(cb["cpu_model"], str) and cb["cpu_model"]
    assert oracle.get_threads() == cb["cores"]  # the thread count is restored


def test_workload_roofline_arithmetic():
    import bench
    r = bench.workload_roofline(6_000_000_000, 2.0, "k")
    assert r["achieved"] == 3000.0 and r["unit"] == "GB/s" and r["bound"] == "hbm"
    assert abs(r["frac"] - 3000.0 / r["peak"]) < 1e-4
    assert bench.csr_bytes(3, 5, 8) == 16 + 60 and bench.csr_bytes(3, 5, 4) == 16 + 40
