"""The workloads at their full sizes, in the launch configuration bench.py
times (one spm_assemble_csc call through spm.Assembler).

Where the oracle cannot run on everything in seconds, it runs on sampled
columns: the writes of a set of columns form a stream of their own whose CSC
is exactly those columns' part of the full CSC.  Properties that hold at any
size (CSC invariants, nnz = distinct coordinates with a non-zero value, the
FEM pattern) are checked on the whole output on the device.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_helpers import (abs_contrib_per_entry, assert_bit_exact, assert_correctly_rounded,
                               assert_sum_within_tol, to_dev)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1805_03380_gb300 as spm
    spm.spm_set_tuning(reset=True)


def _assemble(d, mode):
    import paper_1805_03380_gb300 as spm
    rows, cols, vals = to_dev(d["rows"]), to_dev(d["cols"]), to_dev(d["vals"])
    a = spm.Assembler(d["shape"], len(d["rows"]), vals.dtype, mode)
    a.run(rows, cols, vals)
    A = a.result()
    return A, rows, cols


def _device_invariants(A, shape):
    cp, ri, v = A.col_ptr, A.row_idx, A.vals
    assert int(cp[0]) == 0 and int(cp[-1]) == A.nnz
    assert bool((cp[1:] >= cp[:-1]).all())
    assert bool((ri >= 0).all()) and bool((ri < shape[0]).all())
    assert not bool((v == 0).any())
    col_of = torch.repeat_interleave(torch.arange(shape[1], device=cp.device), cp[1:] - cp[:-1])
    same = col_of[1:] == col_of[:-1]
    assert bool((ri[1:][same] > ri[:-1][same]).all())
    return col_of


def _sampled_columns(d, A, mode, sel, rounded):
    mask = np.isin(d["cols"], sel)
    sub = dict(rows=d["rows"][mask], cols=d["cols"][mask], vals=d["vals"][mask], shape=d["shape"])
    wc, wr, wv = oracle.assemble_csc(sub["rows"], sub["cols"], sub["vals"], sub["shape"], mode=mode)
    cp = A.col_ptr.cpu().numpy()
    scale = abs_contrib_per_entry(sub["rows"], sub["cols"], sub["vals"], sub["shape"], wc, wr)
    for c in sel:
        g0, g1 = int(cp[c]), int(cp[c + 1])
        w0, w1 = int(wc[c]), int(wc[c + 1])
        assert g1 - g0 == w1 - w0, f"column {c}"
        np.testing.assert_array_equal(A.row_idx[g0:g1].cpu().numpy(), wr[w0:w1])
        got = A.vals[g0:g1].cpu().numpy()
        if mode == "set":
            assert_bit_exact(got, wv[w0:w1].astype(got.dtype))
        else:
            assert_sum_within_tol(got, wv[w0:w1], scale[w0:w1], got.dtype)
    if rounded and mode == "sum":
        # the sub-stream's CSC holds exactly the selected columns, in increasing order
        got_all = np.concatenate([A.vals[int(cp[c]):int(cp[c + 1])].cpu().numpy() for c in sorted(sel)])
        assert_correctly_rounded(got_all, sub, wc, wr)


def test_n8_hundred_million_writes_sampled_columns():
    d = workloads.zipf_batch(m=100_000_000, n=100_000, dtype=np.float64)
    A, rows, cols = _assemble(d, "sum")
    _device_invariants(A, d["shape"])
    # every distinct coordinate is stored (a continuous sum is never exactly zero)
    key = cols.long() * d["shape"][0] + rows.long()
    assert torch.unique(key).numel() == A.nnz
    del key
    _sampled_columns(d, A, "sum", [0, 2, 17, 1000, 54321, 99999], rounded=False)
    _sampled_columns(d, A, "sum", [1, 3, 500, 77777], rounded=True)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_batch_insertion_1e7_full_oracle(dtype):
    d = workloads.zipf_batch(m=10_000_000, n=100_000, dtype=dtype)
    A, _, _ = _assemble(d, "sum")
    wc, wr, wv = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="sum")
    np.testing.assert_array_equal(A.col_ptr.cpu().numpy(), wc)
    np.testing.assert_array_equal(A.row_idx.cpu().numpy(), wr)
    got = A.vals.cpu().numpy()
    scale = abs_contrib_per_entry(d["rows"], d["cols"], d["vals"], d["shape"], wc, wr)
    assert_sum_within_tol(got, wv, scale, dtype)


def test_fem_2048_full_size():
    d = workloads.fem_q1(n_el=2048, dtype=np.float64)
    A, _, _ = _assemble(d, "sum")
    nn = 2049
    assert A.nnz == (3 * nn - 2) ** 2 == 37_761_025
    _device_invariants(A, d["shape"])
    cnt = (A.col_ptr[1:] - A.col_ptr[:-1])
    assert set(torch.unique(cnt).cpu().tolist()) == {4, 6, 9}
    rng = np.random.Generator(np.random.PCG64(1))
    sel = sorted(set([0, nn - 1, nn * nn - 1, nn * 1024 + 1024] + rng.integers(0, nn * nn, 12).tolist()))
    _sampled_columns(d, A, "sum", sel, rounded=True)


def test_batched_4096_full_size_sampled_matrices():
    import paper_1805_03380_gb300 as spm
    d = workloads.batched_uniform()
    tp = d["trip_ptr"]
    n = d["n"]
    cp, ri, v, nnz, _ = spm.assemble_csc_batched(to_dev(d["rows"]), to_dev(d["cols"]), to_dev(d["vals"]), n, n, tp,
                                                 mode="set")
    nnz = nnz.cpu().numpy()
    cbase = np.concatenate([[0], np.cumsum(n + 1)])
    rng = np.random.Generator(np.random.PCG64(2))
    picks = sorted(set([0, len(n) - 1, int(np.argmax(np.diff(tp)))] + rng.integers(0, len(n), 13).tolist()))
    for i in picks:
        a, b = int(tp[i]), int(tp[i + 1])
        wc, wr, wv = oracle.assemble_csc(d["rows"][a:b], d["cols"][a:b], d["vals"][a:b], (int(n[i]), int(n[i])),
                                         mode="set")
        assert int(nnz[i]) == len(wr)
        np.testing.assert_array_equal(cp[cbase[i]:cbase[i + 1]].cpu().numpy(), wc)
        np.testing.assert_array_equal(ri[a:a + len(wr)].cpu().numpy(), wr)
        assert_bit_exact(v[a:a + len(wr)].cpu().numpy(), wv.astype(np.float32))
    # every matrix: offsets start at 0 and end at its nnz
    cpn = cp.cpu().numpy()
    assert np.all(cpn[cbase[:-1]] == 0)
    assert np.all(cpn[cbase[1:] - 1] == nnz)
    assert np.all(nnz <= np.diff(tp))
