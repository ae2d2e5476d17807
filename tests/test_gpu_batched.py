"""Batched assembly (many independent matrices in one call) against the oracle
run matrix by matrix."""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_helpers import abs_contrib_per_entry, assert_bit_exact, assert_sum_within_tol, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _run_batched(rows, cols, vals, n_rows, n_cols, trip_ptr, mode, seq=None, keep_map=False):
    import paper_1805_03380_gb300 as spm
    s = None if seq is None else to_dev(np.asarray(seq, np.uint64).view(np.int64))
    cp, ri, v, nnz, mp = spm.assemble_csc_batched(to_dev(rows), to_dev(cols), to_dev(vals), n_rows, n_cols, trip_ptr,
                                                  mode=mode, seq=s, keep_map=keep_map)
    return cp.cpu().numpy(), ri.cpu().numpy(), v.cpu().numpy(), nnz.cpu().numpy(), \
        (mp.cpu().numpy() if mp is not None else None)


def _compare(rows, cols, vals, n_rows, n_cols, trip_ptr, mode, seq=None, keep_map=False):
    cp, ri, v, nnz, mp = _run_batched(rows, cols, vals, n_rows, n_cols, trip_ptr, mode, seq, keep_map)
    cbase = 0
    for i in range(len(n_rows)):
        a, b = int(trip_ptr[i]), int(trip_ptr[i + 1])
        wc, wr, wv, *wm = oracle.assemble_csc(rows[a:b], cols[a:b], vals[a:b], (int(n_rows[i]), int(n_cols[i])),
                                              mode=mode, seq=None if seq is None else seq[a:b], with_map=keep_map)
        k = int(nnz[i])
        assert k == len(wr), f"matrix {i}"
        np.testing.assert_array_equal(cp[cbase:cbase + int(n_cols[i]) + 1], wc)
        np.testing.assert_array_equal(ri[a:a + k], wr)
        if mode == "set":
            assert_bit_exact(v[a:a + k], wv.astype(vals.dtype))
        else:
            shape = (int(n_rows[i]), int(n_cols[i]))
            scale = abs_contrib_per_entry(rows[a:b], cols[a:b], vals[a:b], shape, wc, wr)
            assert_sum_within_tol(v[a:a + k], wv, scale, vals.dtype)
        if keep_map:
            np.testing.assert_array_equal(mp[a:b], wm[0])
        cbase += int(n_cols[i]) + 1


@pytest.mark.parametrize("mode", ["set", "sum"])
def test_batched_uneven_matrices(mode):
    d = workloads.batched_uniform(batch=96, n_min=64, n_max=1500, seed=workloads.SEED_BASE + 40)
    n = d["n"]
    _compare(d["rows"], d["cols"], d["vals"], n, n, d["trip_ptr"], mode)


def test_batched_with_seq_and_map():
    d = workloads.batched_uniform(batch=40, n_min=64, n_max=600, seed=workloads.SEED_BASE + 41)
    rng = np.random.Generator(np.random.PCG64(5))
    seq = rng.integers(0, 50, d["trip_ptr"][-1]).astype(np.uint64)
    n = d["n"]
    _compare(d["rows"], d["cols"], d["vals"], n, n, d["trip_ptr"], "set", seq=seq, keep_map=True)


def test_batched_edge_matrices():
    # empty matrices, a 1 x 1, a zero-row matrix, a matrix larger than the others,
    # rectangular shapes
    rng = np.random.Generator(np.random.PCG64(9))
    shapes = [(5, 7), (1, 1), (0, 4), (300, 2), (3000, 4000), (9, 9), (64, 64), (2, 1)]
    counts = [0, 5, 0, 600, 40_000, 0, 2000, 3]
    rows, cols, vals = [], [], []
    for (nr, nc), m in zip(shapes, counts):
        rows.append(rng.integers(0, max(nr, 1), m))
        cols.append(rng.integers(0, max(nc, 1), m))
        vals.append(rng.standard_normal(m).astype(np.float32))
    trip_ptr = np.concatenate([[0], np.cumsum(counts)])
    rows = np.concatenate(rows).astype(np.int32)
    cols = np.concatenate(cols).astype(np.int32)
    vals = np.concatenate(vals)
    n_rows = np.array([s[0] for s in shapes])
    n_cols = np.array([s[1] for s in shapes])
    for mode in ("set", "sum"):
        _compare(rows, cols, vals, n_rows, n_cols, trip_ptr, mode)


def test_batched_equals_single_calls():
    import paper_1805_03380_gb300 as spm
    d = workloads.batched_uniform(batch=12, n_min=100, n_max=3000, seed=workloads.SEED_BASE + 42)
    cp, ri, v, nnz, _ = _run_batched(d["rows"], d["cols"], d["vals"], d["n"], d["n"], d["trip_ptr"], "set")
    cbase = 0
    for i in range(12):
        a, b = int(d["trip_ptr"][i]), int(d["trip_ptr"][i + 1])
        n = int(d["n"][i])
        A = spm.assemble_csc(to_dev(d["rows"][a:b]), to_dev(d["cols"][a:b]), to_dev(d["vals"][a:b]), (n, n), "set")
        np.testing.assert_array_equal(cp[cbase:cbase + n + 1], A.col_ptr.cpu().numpy())
        np.testing.assert_array_equal(ri[a:a + A.nnz], A.row_idx.cpu().numpy())
        assert_bit_exact(v[a:a + A.nnz], A.vals.cpu().numpy())
        cbase += n + 1


def test_batched_mismatched_device_sizes_reported():
    import paper_1805_03380_gb300 as spm
    rows = np.zeros(4, np.int32)
    cols = np.zeros(4, np.int32)
    vals = np.ones(4, np.float32)
    hr = torch.tensor([3, 3], dtype=torch.int64)
    hc = torch.tensor([3, 3], dtype=torch.int64)
    ht = torch.tensor([0, 2, 4], dtype=torch.int64)
    ws = spm.spm_assemble_csc_batched_workspace(hr, hc, ht, torch.float32, "set")
    dev = torch.device("cuda")
    bad_rows = torch.tensor([3, 300], dtype=torch.int64, device=dev)  # differs from the host copy
    out = dict(col_ptr=torch.empty(8, dtype=torch.int64, device=dev), row_idx=torch.empty(4, dtype=torch.int32,
               device=dev), out_vals=torch.empty(4, device=dev), d_nnz=torch.empty(2, dtype=torch.int64, device=dev),
               d_status=torch.zeros(1, dtype=torch.int32, device=dev))
    spm.spm_assemble_csc_batched(hr, hc, ht, bad_rows, hc.to(dev), ht.to(dev), to_dev(rows), to_dev(cols),
                                 to_dev(vals), None, "set", 0, out["col_ptr"], out["row_idx"], out["out_vals"],
                                 out["d_nnz"], None, out["d_status"], torch.empty(ws, dtype=torch.uint8, device=dev))
    torch.cuda.synchronize()
    assert int(out["d_status"].item()) == 1


def _redraw(d, seed, dtype):
    """New writes for the same batch layout: the same sizes and write counts,
    new coordinates, values and rewrites."""
    rng = np.random.default_rng(seed)
    n, tp = np.asarray(d["n"], np.int64), np.asarray(d["trip_ptr"], np.int64)
    cnt = np.diff(tp)
    lim = np.repeat(n, cnt)
    rows = (rng.random(int(tp[-1])) * lim).astype(np.int32)
    cols = (rng.random(int(tp[-1])) * lim).astype(np.int32)
    # about 10 % rewrites of an earlier coordinate of the same matrix
    rep = np.nonzero(rng.random(int(tp[-1])) < 0.1)[0]
    start = np.repeat(tp[:-1], cnt)[rep]
    src = start + (rng.random(len(rep)) * (rep - start + 1)).astype(np.int64)
    rows[rep], cols[rep] = rows[src], cols[src]
    vals = rng.standard_normal(int(tp[-1])).astype(dtype)
    return rows, cols, vals


@pytest.mark.parametrize("mode", ["set", "sum"])
def test_batched_cuda_graph_capture_and_replay(mode):
    # capture one batched call in a CUDA graph, replay it on new writes of the
    # same layout, and compare every matrix with the oracle after each replay
    import paper_1805_03380_gb300 as spm
    d = workloads.batched_uniform(batch=48, n_min=64, n_max=900, seed=workloads.SEED_BASE + 44)
    n, tp = np.asarray(d["n"], np.int64), np.asarray(d["trip_ptr"], np.int64)
    dtype = np.float64 if mode == "sum" else np.float32
    first = _redraw(d, 1, dtype)
    rows, cols, vals = (to_dev(a) for a in first)
    asm = spm.BatchedAssembler(n, n, tp, dtype=vals.dtype, mode=mode)
    asm.run(rows, cols, vals)  # first call on the device (sets kernel attributes)
    asm.result()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            asm.run(rows, cols, vals, stream=s)
    for seed in (2, 3):
        r, c, v = _redraw(d, seed, dtype)
        rows.copy_(to_dev(r))
        cols.copy_(to_dev(c))
        vals.copy_(to_dev(v))
        g.replay()
        torch.cuda.synchronize()
        cp, ri, ov, nnz, _ = asm.result()
        cp, ri, ov, nnz = cp.cpu().numpy(), ri.cpu().numpy(), ov.cpu().numpy(), nnz.cpu().numpy()
        cbase = 0
        for i in range(len(n)):
            a, b = int(tp[i]), int(tp[i + 1])
            shape = (int(n[i]), int(n[i]))
            wc, wr, wv = oracle.assemble_csc(r[a:b], c[a:b], v[a:b], shape, mode=mode)
            k = int(nnz[i])
            assert k == len(wr), f"replay {seed}, matrix {i}"
            np.testing.assert_array_equal(cp[cbase:cbase + shape[1] + 1], wc)
            np.testing.assert_array_equal(ri[a:a + k], wr)
            if mode == "set":
                assert_bit_exact(ov[a:a + k], wv.astype(dtype))
            else:
                scale = abs_contrib_per_entry(r[a:b], c[a:b], v[a:b], shape, wc, wr)
                assert_sum_within_tol(ov[a:a + k], wv, scale, dtype)
            cbase += shape[1] + 1


def test_batched_autotune_cache_and_identical_results(tmp_path):
    import json

    import paper_1805_03380_gb300 as spm
    from paper_1805_03380_gb300 import autotune as at
    spm.spm_set_tuning(reset=True)
    t0 = spm.spm_get_tuning()
    d = workloads.batched_uniform(batch=64, n_min=64, n_max=2000, seed=workloads.SEED_BASE + 45)
    n, tp = np.asarray(d["n"], np.int64), np.asarray(d["trip_ptr"], np.int64)
    p = str(tmp_path / "tune.json")
    cands = [dict(bucket_target=4096, sub_bits=11), dict(bucket_target=7168, partition_threads=512)]
    best = at.autotune_batched(to_dev(d["rows"]), to_dev(d["cols"]), to_dev(d["vals"]), n, n, tp, "set",
                               candidates=cands, reps=3, warmup=2, path=p, apply=False)
    # every candidate gives the default tuning's bytes
    assert best["tried"] == 2 and best["rejected"] == []
    assert spm.spm_get_tuning() == t0
    key = at.batch_cache_key(n, n, tp, torch.float32, "set")
    assert json.load(open(p))[key]["tuning"] == best["tuning"]
    assert at.apply_cached_batched(n, n, tp, torch.float32, "set", path=p) == best["tuning"]
    spm.spm_set_tuning(reset=True)
