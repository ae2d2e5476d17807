"""bench.py's workload table (no GPU): every workload the command line offers
has a specification, and the small ones generate inputs of the stated sizes."""
import os
import re
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _choices():
    text = open(os.path.join(ROOT, "bench.py")).read()
    block = text[text.index('ap.add_argument("--workload"'):]
    block = block[block.index("choices=[") + len("choices=["):block.index("])")]
    return re.findall(r'"([^"]+)"', block)


def test_every_offered_workload_has_a_spec():
    sys.path.insert(0, ROOT)
    import bench
    names = _choices()
    assert "n8" in names and len(names) >= 20
    for name in names:
        spec = bench.workload_spec(name)
        assert spec["desc"] and spec["kind"] in ("zipf", "fem", "ordered", "update", "lookup", "coo", "trace",
                                                 "lastwrite", "density", "batched", "diff")


def test_small_workloads_generate_the_stated_sizes():
    sys.path.insert(0, ROOT)
    import bench
    d, spec = bench.make_workload("c1")
    assert len(d["rows"]) == 10_000 and d["shape"] == (1000, 1000) and spec["mode"] == "set"
    d, spec = bench.make_workload("n4_0.01")
    assert len(d["rows"]) == 10_000 and d["shape"] == (10_000, 10_000)
    assert d["vals"].dtype == np.float64
