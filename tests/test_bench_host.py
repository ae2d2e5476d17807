"""Host-side pieces of bench.py (no GPU): the CPU oracle baselines report the
cores they used and the host's, and the code hash that keys committed traffic
figures ignores comments but not code."""
import os
import shutil

import numpy as np

import bench
import workloads


def test_batched_oracle_baseline_uses_every_host_core():
    d = workloads.batched_uniform(batch=24, n_min=64, n_max=400, seed=workloads.SEED_BASE + 4)
    rate, done, writes, threads, dt = bench.batched_oracle_rate(d, "set", budget_s=1.0)
    assert threads == (os.cpu_count() or 1)
    assert 0 < done <= 24 and writes > 0 and rate > 0 and dt > 0
    assert writes == sum(int(d["trip_ptr"][i + 1] - d["trip_ptr"][i])
                         for i in np.random.default_rng(7).permutation(24)[:done])


def test_differentiable_oracle_baseline_runs():
    f = workloads.fem_q1(n_el=16, dtype=np.float32, seed=3)
    rate, dt = bench.diff_oracle_rate(f, "sum")
    assert rate > 0 and dt > 0


def test_code_hash_ignores_comments(tmp_path, monkeypatch):
    root = tmp_path / "r"
    shutil.copytree(os.path.join(bench.ROOT, "paper_1805_03380_gb300", "csrc"),
                    root / "paper_1805_03380_gb300" / "csrc")
    shutil.copytree(os.path.join(bench.ROOT, "include"), root / "include")
    monkeypatch.setattr(bench, "ROOT", str(root))
    h0 = bench.source_hash()
    f = root / "paper_1805_03380_gb300" / "csrc" / "resolve.cu"
    text = f.read_text()
    f.write_text("// a new comment\n" + text.replace("namespace spm {", "namespace spm {  /* here too */", 1))
    assert bench.source_hash() == h0
    f.write_text(text.replace("constexpr uint32_t kDense = 3072;", "constexpr uint32_t kDense = 2048;"))
    assert bench.source_hash() != h0
