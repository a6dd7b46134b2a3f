"""Host-side pieces of bench.py that need no GPU: the algorithmic-byte count, the ncu
record lookup (counters are used only while the kernel source is unchanged), the
issue-rate roofline, the CPU baseline's DAG sample and its threaded oracle runs."""
import hashlib
import json
import os

import numpy as np

import bench
import inputs
import oracle


def test_algorithmic_bytes_follow_the_stated_formula():
    b = inputs.layered(6, cfg=2, n_max=300)
    n, m, nd = b.n_total, b.m_total, b.ndag
    a = bench.algorithmic_bytes(b)
    csr = 4 * (n + nd) + 4 * m
    assert a["k_ia"] == csr + 4 * n
    assert a["k_ie_pull"] == csr + n + 4 * n
    assert a["k_sim"] == csr + n + 4 * n + 8 * n + 20 * n + 8 * nd


def test_path_bytes_count_each_input_and_output_once():
    """Per task 4 + 4 x out-degree + 1 + 8 + 20 bytes, per DAG 4 + 8 + the cost table; on the
    headline workload's shape that is about 109 bytes per task."""
    b = inputs.layered(6, cfg=2, n_max=300)
    n, m, nd = b.n_total, b.m_total, b.ndag
    assert bench.path_bytes(b) == 33 * n + 4 * m + 12 * nd + 16 * nd * b.n_types
    t = inputs.tiled(inputs.KIND_CHOLESKY, 8, 2)
    assert bench.path_bytes(t) == 33 * t.n_total + 4 * t.m_total + 12 * t.ndag + 16 * t.n_total
    big = inputs.layered4096(256)
    per_task = bench.path_bytes(big) / big.n_total
    assert 100 < per_task < 120


def _fake_root(tmp_path, src_text, sha):
    (tmp_path / "profiles").mkdir()
    d = tmp_path / "paper_2404_03226_b300" / "csrc"
    d.mkdir(parents=True)
    (d / "k_x.cu").write_text(src_text)
    rec = {"k_x": {"source": "k_x.cu", "source_sha": sha, "workload": "layered:4096", "bytes_per_step_small": 100,
                   "bytes_per_step_full": 4000, "inst_per_step_small": 10, "inst_per_step_full": 2_000_000_000}}
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(rec))


def test_profile_counters_only_for_the_unchanged_source_and_their_workload(tmp_path, monkeypatch):
    src = "__global__ void k_x() {}\n"
    sha = hashlib.sha256(src.encode()).hexdigest()[:16]
    _fake_root(tmp_path, src, sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    w = "layered:4096"
    assert bench.traffic_from_profile("k_x", 2.0, w) == 2000.0  # per launch: two launches per step
    assert bench.traffic_from_profile("k_missing", 1.0, w) is None
    # counters of another workload (or the same kernel on a prefix of it) do not apply
    assert bench.traffic_from_profile("k_x", 1.0, "tiled") is None
    assert bench.profile_record("k_x", "layered:2048") is None
    (tmp_path / "paper_2404_03226_b300" / "csrc" / "k_x.cu").write_text(src + "// edited\n")
    assert bench.traffic_from_profile("k_x", 1.0, w) is None
    assert bench.profile_record("k_x", w) is None


def test_issue_roofline_arithmetic(tmp_path, monkeypatch):
    src = "__global__ void k_x() {}\n"
    _fake_root(tmp_path, src, hashlib.sha256(src.encode()).hexdigest()[:16])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # 2 G warp instructions per step, 10 steps in 20 ms of kernel time: 1000 G/s; peak 148 x 4 x 2 GHz
    r = bench.issue_roofline(["k_x", "k_y"], np.array([20.0, 5.0]), 10, 148, 2000.0, "k_x", "layered:4096")
    assert r["peak"] == 1184.0
    assert r["achieved"] == 1000.0 and abs(r["frac"] - 1000.0 / 1184.0) < 1e-4
    assert r["per_kernel"]["k_y"] is None
    assert bench.issue_roofline(["k_x"], np.array([20.0]), 10, 148, 2000.0, "k_x", "mixed")["achieved"] is None


def test_cpu_sample_and_threaded_oracle():
    b = inputs.layered(12, cfg=2, n_max=200)
    idx, tasks = bench.first_dags(b, 500)
    assert tasks >= 500 and tasks - int(b.task_base[idx[-1] + 1] - b.task_base[idx[-1]]) < 500
    assert idx == list(range(len(idx)))
    dags = [b.dag(d) for d in idx]
    bench.run_oracle(dags, inputs.MACHINE_LAYERED, 1)
    bench.run_oracle(dags, inputs.MACHINE_LAYERED, 3)
    one = [oracle.simulate(g, inputs.MACHINE_LAYERED)["makespan"] for g in dags]
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(3) as ex:
        many = list(ex.map(lambda g: oracle.simulate(g, inputs.MACHINE_LAYERED)["makespan"], dags))
    assert one == many
    assert bench.host_cores() >= 1 and os.cpu_count() >= 1
