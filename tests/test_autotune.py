"""The autotuner: its cache on the CPU, and one small search on the GPU."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_cache_roundtrip_and_candidates(tmp_path, monkeypatch):
    from paper_1805_03380_gb300 import autotune as at
    p = str(tmp_path / "tune.json")
    key = at.cache_key((10, 20), 300, torch.float64, "sum")
    assert "10x20" in key and "m=300" in key and "f64" in key and key.endswith("flags=0")
    assert at.load_cache(p) == {}
    at.store_cache(key, {"tuning": {"bucket_target": 4096}, "ms": 1.0}, p)
    at.store_cache("other", {"tuning": {}, "ms": 2.0}, p)
    assert json.load(open(p))[key]["ms"] == 1.0
    monkeypatch.setenv("SPM_TUNE_CACHE", p)
    assert at.load_cache()[key]["tuning"] == {"bucket_target": 4096}
    cands = at.default_candidates()
    assert len(cands) == np.prod([len(v) for v in at.SEARCH_SPACE.values()])
    assert all(set(c) == set(at.SEARCH_SPACE) for c in cands)


@pytest.mark.gpu
def test_small_search_on_the_gpu(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1805_03380_gb300 as spm
    import workloads
    from paper_1805_03380_gb300 import autotune as at
    from tests.gpu_helpers import to_dev
    spm.spm_set_tuning(reset=True)
    t0 = spm.spm_get_tuning()
    d = workloads.zipf_batch(m=400_003, n=20_000, seed=workloads.SEED_BASE + 70)
    p = str(tmp_path / "tune.json")
    cands = [dict(bucket_target=2048, sub_bits=10), dict(bucket_target=3584, partition_threads=512)]
    best = at.autotune(to_dev(d["rows"]), to_dev(d["cols"]), to_dev(d["vals"]), d["shape"], "sum",
                       candidates=cands, reps=3, warmup=2, path=p, apply=False)
    assert best["tried"] == 2 and best["rejected"] == []
    assert spm.spm_get_tuning() == t0  # apply=False leaves the tuning alone
    entry = json.load(open(p))[at.cache_key(d["shape"], len(d["rows"]), torch.float64, "sum")]
    assert entry["tuning"] == best["tuning"] and entry["ms"] > 0
    assert at.apply_cached(d["shape"], len(d["rows"]), torch.float64, "sum", path=p) == best["tuning"]
    spm.spm_set_tuning(reset=True)


def test_every_candidate_is_a_valid_tuning():
    # the library accepts every candidate of the search space (host check, no GPU)
    import paper_1805_03380_gb300 as spm
    from paper_1805_03380_gb300 import autotune as at
    t0 = spm.spm_get_tuning()
    try:
        for cand in at.default_candidates():
            spm.spm_set_tuning(reset=True)
            t = spm.spm_set_tuning(**cand)
            assert all(t[k] == v for k, v in cand.items())
    finally:
        spm.spm_set_tuning(reset=True)
        spm.spm_set_tuning(**t0)


def test_batch_cache_key_follows_the_layout():
    from paper_1805_03380_gb300 import autotune as at
    n = np.array([64, 100, 300])
    tp = np.array([0, 40, 90, 200])
    k1 = at.batch_cache_key(n, n, tp, torch.float32, "set")
    assert k1 == at.batch_cache_key(list(n), list(n), list(tp), torch.float32, "set")
    assert "batch=3" in k1 and "m=200" in k1 and k1.endswith("f32|set|flags=0")
    # another shape, another split of the same writes, another mode: other keys
    assert at.batch_cache_key(n + 1, n, tp, torch.float32, "set") != k1
    assert at.batch_cache_key(n, n, np.array([0, 41, 90, 200]), torch.float32, "set") != k1
    assert at.batch_cache_key(n, n, tp, torch.float32, "sum") != k1
