"""The two-pass partition (writes go first to groups of buckets, then to their
buckets) against the oracle.

By default only calls with many writes whose one-pass scatter would keep
many write fronts open take it; here both thresholds are set to zero so
that it runs on sizes the oracle finishes in seconds: several groups,
buckets with a ragged tail, batched matrices whose groups straddle matrix
boundaries, last-write and sum modes, both value types and the map.  Without
seq the result must not depend on which partition path ran: it is compared
bit for bit with the one-pass path as well.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests._refimpl import check_csc_invariants
from tests.gpu_helpers import (abs_contrib_per_entry, assert_bit_exact, assert_correctly_rounded,
                               assert_same_structure, assert_sum_within_tol, gpu_assemble, to_dev)

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
    yield
    spm.spm_set_tuning(reset=True)


def _both_paths(d, mode, keep_map=False, offset=0):
    import paper_1805_03380_gb300 as spm
    spm.spm_set_tuning(two_pass_min_writes=0, two_pass_min_fronts=0)
    try:
        two = gpu_assemble(d, mode, keep_map=keep_map, offset=offset)
    finally:
        spm.spm_set_tuning(reset=True)
    spm.spm_set_tuning(two_pass_min_writes=2**31 - 1)
    try:
        one = gpu_assemble(d, mode, keep_map=keep_map, offset=offset)
    finally:
        spm.spm_set_tuning(reset=True)
    for a, b in zip(two, one):
        np.testing.assert_array_equal(np.asarray(a).view(np.uint8), np.asarray(b).view(np.uint8))
    return two


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("mode", ["set", "sum"])
def test_zipf_two_pass_against_oracle(dtype, mode):
    d = workloads.zipf_batch(m=1_500_007, n=60_000, dtype=dtype, seed=workloads.SEED_BASE + 60)
    got = _both_paths(d, mode)
    want = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode=mode)
    assert_same_structure(got, want)
    check_csc_invariants(got[0], got[1], got[2], d["shape"])
    if mode == "set":
        assert_bit_exact(got[2], want[2].astype(dtype))
    else:
        scale = abs_contrib_per_entry(d["rows"], d["cols"], d["vals"], d["shape"], want[0], want[1])
        assert_sum_within_tol(got[2], want[2], scale, dtype)
        assert_correctly_rounded(got[2], d, got[0], got[1])


def test_fem_two_pass_against_oracle():
    d = workloads.fem_q1(n_el=256, dtype=np.float64)
    got = _both_paths(d, "sum", offset=1)
    want = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="sum")
    assert_same_structure(got, want)
    scale = abs_contrib_per_entry(d["rows"], d["cols"], d["vals"], d["shape"], want[0], want[1])
    assert_sum_within_tol(got[2], want[2], scale, np.float64)


def test_two_pass_keep_map():
    d = workloads.zipf_batch(m=300_001, n=20_000, seed=workloads.SEED_BASE + 61)
    for mode in ("set", "sum"):
        got = _both_paths(d, mode, keep_map=True)
        want = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode=mode, with_map=True)
        assert_same_structure(got, want)
        np.testing.assert_array_equal(got[3], want[3])


@pytest.mark.parametrize("mode", ["set", "sum"])
def test_two_pass_batched(mode):
    import paper_1805_03380_gb300 as spm
    d = workloads.batched_uniform(batch=300, n_min=64, n_max=2500, seed=workloads.SEED_BASE + 62)
    n, tp = d["n"], d["trip_ptr"]
    outs = []
    for thr in (0, 2**31 - 1):
        spm.spm_set_tuning(two_pass_min_writes=thr, two_pass_min_fronts=0)
        try:
            cp, ri, v, nnz, _ = spm.assemble_csc_batched(to_dev(d["rows"]), to_dev(d["cols"]), to_dev(d["vals"]), n, n,
                                                         tp, mode=mode)
        finally:
            spm.spm_set_tuning(reset=True)
        outs.append((cp.cpu().numpy(), ri.cpu().numpy(), v.cpu().numpy(), nnz.cpu().numpy()))
    (cp, ri, v, nnz), (cp1, ri1, v1, nnz1) = outs
    np.testing.assert_array_equal(cp, cp1)
    np.testing.assert_array_equal(nnz, nnz1)
    for i in range(len(n)):  # each matrix's stored elements (the rest of its slice is unused)
        a, k = int(tp[i]), int(nnz[i])
        np.testing.assert_array_equal(ri[a:a + k], ri1[a:a + k])
        np.testing.assert_array_equal(v[a:a + k].view(np.uint8), v1[a:a + k].view(np.uint8))
    cbase = np.concatenate([[0], np.cumsum(n + 1)])
    for i in [0, 1, 57, 150, 299]:
        a, b = int(tp[i]), int(tp[i + 1])
        wc, wr, wv = oracle.assemble_csc(d["rows"][a:b], d["cols"][a:b], d["vals"][a:b], (int(n[i]), int(n[i])),
                                         mode=mode)
        k = int(nnz[i])
        assert k == len(wr)
        np.testing.assert_array_equal(cp[cbase[i]:cbase[i + 1]], wc)
        np.testing.assert_array_equal(ri[a:a + k], wr)
        if mode == "set":
            assert_bit_exact(v[a:a + k], wv.astype(v.dtype))
        else:
            scale = abs_contrib_per_entry(d["rows"][a:b], d["cols"][a:b], d["vals"][a:b], (int(n[i]), int(n[i])),
                                          wc, wr)
            assert_sum_within_tol(v[a:a + k], wv, scale, v.dtype)


def test_two_pass_is_not_used_with_seq():
    # seq is carried by the one-pass path only; the threshold must not change the result
    d = workloads.last_write_1000(shuffled_seq=True)
    import paper_1805_03380_gb300 as spm
    spm.spm_set_tuning(two_pass_min_writes=0, two_pass_min_fronts=0)
    try:
        got = gpu_assemble(d, "set", seq=d["seq"])
    finally:
        spm.spm_set_tuning(reset=True)
    ordered = workloads.last_write_1000()
    want = oracle.assemble_csc(ordered["rows"], ordered["cols"], ordered["vals"], ordered["shape"], mode="set")
    assert_same_structure(got, want)
    assert_bit_exact(got[2], want[2])
