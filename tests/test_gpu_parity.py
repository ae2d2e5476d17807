"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Structure (col_ptr, row_idx) and last-write values must match bit for bit;
summed values within |d| <= 1e-12 * sum|contributions| (float64) or 1e-5 *
sum|contributions| (float32) of the oracle's write-order sum.  The library
rounds the exact sum once, so its sums are also checked against math.fsum
(correct rounding), and bit for bit against the oracle on dyadic inputs, where
every summation order is exact.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests import _golden
from tests._refimpl import assert_sums_match_exact, brute_force_csc, check_csc_invariants, exact_sums
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
    spm.spm_debug_withhold_publication(-1)


def _oracle(d, mode, seq=None, with_map=False):
    return oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode=mode, seq=seq, with_map=with_map)


def _check(d, mode, seq=None, rounded=False, offset=0):
    """Set mode: bit-exact against the oracle.  Sum mode: within tolerance of
    the oracle; with `rounded`, also correctly rounded (math.fsum)."""
    got = gpu_assemble(d, mode, seq=seq, offset=offset)
    want = _oracle(d, mode, seq)
    assert_same_structure(got, want)
    check_csc_invariants(got[0], got[1], got[2], d["shape"])
    if mode == "set":
        assert_bit_exact(got[2], want[2])
    else:
        scale = abs_contrib_per_entry(d["rows"], d["cols"], d["vals"], d["shape"], want[0], want[1])
        assert_sum_within_tol(got[2], want[2], scale, np.asarray(d["vals"]).dtype)
        if rounded:
            assert_correctly_rounded(got[2], d, got[0], got[1])
    return got


# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("case", _golden.all_cases(), ids=lambda c: c["path"].rsplit("/", 1)[-1])
def test_golden_fixtures(case):
    cp, ri, v = gpu_assemble(case, case["mode"])
    np.testing.assert_array_equal(cp, case["col_ptr"])
    np.testing.assert_array_equal(ri, case["row_idx"])
    np.testing.assert_array_equal(v, case["vals_expected"])


@pytest.mark.parametrize("mode", ["set", "sum"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("use_seq", [False, True])
def test_tiny_against_brute_force(mode, dtype, use_seq):
    rng = np.random.Generator(np.random.PCG64(100 + (mode == "sum") + 2 * (dtype == np.float32) + 4 * use_seq))
    # specials include values far apart in magnitude (1e300 next to 3.25e-300)
    specials = np.array([0.0, -0.0, np.nan, np.inf, -np.inf, 1.0, -1.0, 0.5, 3.25e-300, 1e300, -1e300])
    if dtype == np.float32:
        specials = np.array([0.0, -0.0, np.nan, np.inf, -np.inf, 1.0, -1.0, 0.5, 1e-40, 3e38, -3e38])
    for trial in range(25):
        n_rows, n_cols = int(rng.integers(1, 50)), int(rng.integers(1, 50))
        m = int(rng.integers(0, 600))
        n_coord = int(rng.integers(1, 80))
        cr, cc = rng.integers(0, n_rows, n_coord), rng.integers(0, n_cols, n_coord)
        pick = rng.integers(0, n_coord, m)
        vals = rng.standard_normal(m)
        sel = rng.random(m) < 0.15
        vals[sel] = specials[rng.integers(0, len(specials), int(sel.sum()))]
        d = dict(rows=cr[pick].astype(np.int32), cols=cc[pick].astype(np.int32), vals=vals.astype(dtype),
                 shape=(n_rows, n_cols))
        seq = rng.integers(0, 6, m).astype(np.uint64) if use_seq else None
        got = gpu_assemble(d, mode, seq=seq)
        if mode == "sum":
            # against the exact sums: within tol * sum|contributions| per element,
            # cancellation-ambiguous elements (|exact| <= that bound) may vanish
            check_csc_invariants(got[0], got[1], got[2], d["shape"])
            ref = exact_sums(d["rows"], d["cols"], d["vals"], d["shape"])
            assert_sums_match_exact(got, ref, d["shape"], 1e-12 if dtype == np.float64 else 1e-5,
                                    out_f32=dtype == np.float32)
            continue
        want = brute_force_csc(d["rows"], d["cols"], d["vals"].astype(np.float64), d["shape"], mode, seq=seq,
                               out_f32=dtype == np.float32)
        assert_same_structure(got, want)
        assert_bit_exact(got[2], want[2].astype(dtype))


def test_last_write_1000():
    d = workloads.last_write_1000()
    _check(d, "set")


def test_last_write_1000_shuffled_with_seq():
    d = workloads.last_write_1000(shuffled_seq=True)
    got = _check(d, "set", seq=d["seq"])
    ordered = workloads.last_write_1000()
    want = _oracle(ordered, "set")
    assert_same_structure(got, want)
    assert_bit_exact(got[2], want[2])


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_zipf_batch_insertion(dtype):
    # 100,000 x 100,000 with Zipf columns, 2,000,003 writes (a ragged tail)
    d = workloads.zipf_batch(m=2_000_003, n=100_000, dtype=dtype, seed=workloads.SEED_BASE + 20)
    _check(d, "sum", rounded=True)


def test_dyadic_sums_bit_exact_against_the_oracle():
    # multiples of 2^-24: every summation order is exact, so GPU == oracle bit for bit
    d = workloads.zipf_batch(m=1_000_001, n=5000, seed=workloads.SEED_BASE + 27)
    d["vals"] = workloads.dyadic_values(len(d["rows"]), seed=5)
    # force some exact cancellations: append the negated sum of a few coordinates
    got = gpu_assemble(d, "sum")
    want = _oracle(d, "sum")
    assert_same_structure(got, want)
    assert_bit_exact(got[2], want[2])


def test_zipf_last_write_unaligned_pointers():
    d = workloads.zipf_batch(m=500_001, n=30_000, dtype=np.float64, seed=workloads.SEED_BASE + 21)
    _check(d, "set", offset=1)
    _check(d, "sum", offset=3, rounded=True)


def test_fem_q1_sum():
    d = workloads.fem_q1(n_el=256, dtype=np.float64)
    got = _check(d, "sum")
    nn = 257
    assert got[0][-1] == (3 * nn - 2) ** 2
    assert set(np.unique(np.diff(got[0])).tolist()) == {4, 6, 9}


def test_fem_q1_unperturbed_closed_form():
    d = workloads.fem_q1(n_el=64, dtype=np.float64, unperturbed=True)
    cp, ri, v = gpu_assemble(d, "sum")
    nn = 65
    assert cp[-1] == (3 * nn - 2) ** 2
    col_of = np.repeat(np.arange(nn * nn), np.diff(cp))
    diag = v[ri == col_of]
    node = np.arange(nn * nn)
    ix, iy = node % nn, node // nn
    bx = (ix == 0) | (ix == nn - 1)
    by = (iy == 0) | (iy == nn - 1)
    expect = np.where(bx & by, 2 / 3, np.where(bx ^ by, 4 / 3, 8 / 3))
    np.testing.assert_allclose(diag, expect, rtol=0, atol=1e-14)
    # every row sums to zero
    row_sum = np.zeros(nn * nn)
    np.add.at(row_sum, ri, v)
    assert np.max(np.abs(row_sum)) < 1e-13


def test_density_sweep_shapes():
    for dens in (1e-4, 1e-3, 1e-2):
        d = workloads.density_sweep(dens)
        _check(d, "set")


def test_empty_and_degenerate():
    # m = 0
    d = dict(rows=np.zeros(0, np.int32), cols=np.zeros(0, np.int32), vals=np.zeros(0), shape=(7, 5))
    cp, ri, v = gpu_assemble(d, "set")
    np.testing.assert_array_equal(cp, np.zeros(6))
    assert ri.size == 0
    # single row / column, 1 x 1
    rng = np.random.Generator(np.random.PCG64(3))
    for shape in [(1, 900), (900, 1), (1, 1)]:
        m = 3000
        d = dict(rows=rng.integers(0, shape[0], m).astype(np.int32), cols=rng.integers(0, shape[1], m).astype(np.int32),
                 vals=rng.standard_normal(m), shape=shape)
        _check(d, "set")
        _check(d, "sum", rounded=True)
    # all writes to one coordinate, the last one decides / zero removal
    vals = np.array([1.0, 0.0] * 50 + [0.0])
    d = dict(rows=np.full(101, 2, np.int32), cols=np.full(101, 3, np.int32), vals=vals, shape=(4, 4))
    cp, ri, v = gpu_assemble(d, "set")
    assert cp[-1] == 0
    d["vals"] = np.concatenate([vals[:-1], [-0.0]])
    cp, ri, v = gpu_assemble(d, "set")
    assert cp[-1] == 0
    d["vals"] = np.concatenate([vals[:-1], [np.nan]])
    cp, ri, v = gpu_assemble(d, "set")
    assert cp[-1] == 1 and np.isnan(v[0])
    # +inf + -inf = nan in sum mode is kept; x + (-x) = 0 is removed
    d = dict(rows=np.array([0, 0, 1, 1], np.int32), cols=np.array([0, 0, 0, 0], np.int32),
             vals=np.array([np.inf, -np.inf, 2.5, -2.5]), shape=(2, 1))
    cp, ri, v = gpu_assemble(d, "sum")
    assert list(cp) == [0, 1] and list(ri) == [0] and np.isnan(v[0])


def test_keep_map_matches_oracle():
    d = workloads.last_write_1000()
    for mode in ("set", "sum"):
        got = gpu_assemble(d, mode, keep_map=True)
        want = _oracle(d, mode, with_map=True)
        assert_same_structure(got, want)
        np.testing.assert_array_equal(got[3], want[3])


def test_out_of_range_index_is_reported():
    import paper_1805_03380_gb300 as spm
    d = dict(rows=np.array([0, 1, 5], np.int32), cols=np.array([0, 1, 1], np.int32), vals=np.ones(3), shape=(5, 5))
    with pytest.raises(spm.SpmError) as e:
        gpu_assemble(d, "set")
    assert e.value.code == 2
    d["rows"] = np.array([0, -1, 2], np.int32)
    with pytest.raises(spm.SpmError) as e:
        gpu_assemble(d, "sum")
    assert e.value.code == 2
    # the next call is unaffected
    d["rows"] = np.array([0, 1, 2], np.int32)
    cp, ri, v = gpu_assemble(d, "sum")
    assert cp[-1] == 3


def test_workspace_too_small_is_rejected_on_the_host():
    import paper_1805_03380_gb300 as spm
    d = workloads.last_write_1000()
    a = spm.Assembler(d["shape"], len(d["rows"]), torch.float64, "set")
    a.workspace = a.workspace[:100]
    with pytest.raises(spm.SpmError) as e:
        a.run(to_dev(d["rows"]), to_dev(d["cols"]), to_dev(d["vals"]))
    assert e.value.code == 3


def test_deterministic_output():
    d = workloads.zipf_batch(m=1_000_000, n=20_000, seed=workloads.SEED_BASE + 22)
    a = gpu_assemble(d, "sum")
    b = gpu_assemble(d, "sum")
    for x, y in zip(a, b):
        assert x.tobytes() == y.tobytes()


def test_cuda_graph_capture_and_replay():
    import paper_1805_03380_gb300 as spm
    d1 = workloads.zipf_batch(m=300_000, n=5000, seed=workloads.SEED_BASE + 23)
    d2 = workloads.zipf_batch(m=300_000, n=5000, seed=workloads.SEED_BASE + 24)
    rows, cols, vals = to_dev(d1["rows"]), to_dev(d1["cols"]), to_dev(d1["vals"])
    a = spm.Assembler(d1["shape"], 300_000, torch.float64, "sum")
    a.run(rows, cols, vals)  # first call on the device (sets kernel attributes)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            a.run(rows, cols, vals, stream=s)
    for d in (d2, d1):
        rows.copy_(to_dev(d["rows"]))
        cols.copy_(to_dev(d["cols"]))
        vals.copy_(to_dev(d["vals"]))
        g.replay()
        torch.cuda.synchronize()
        A = a.result()
        want = _oracle(d, "sum")
        np.testing.assert_array_equal(A.col_ptr.cpu().numpy(), want[0])
        np.testing.assert_array_equal(A.row_idx.cpu().numpy(), want[1])
        assert_correctly_rounded(A.vals.cpu().numpy(), d, want[0], want[1])


def test_oversize_buckets_window_path():
    # a bucket target above the shared-memory capacity makes many buckets
    # overflow it, which exercises the windowed path
    import paper_1805_03380_gb300 as spm
    spm.spm_set_tuning(bucket_target=65536)
    try:
        d = workloads.density_sweep(3e-3, n=10_000)
        d["vals"][::7] = 0.0
        a = spm.Assembler(d["shape"], len(d["rows"]), torch.float64, "set")
        a.run(to_dev(d["rows"]), to_dev(d["cols"]), to_dev(d["vals"]))
        a.result()
        st = spm.spm_debug_plan_stats(a)
        assert st["over_capacity"] > 0 and st["largest"] > st["capacity"]
        _check(d, "set")
        d2 = workloads.zipf_batch(m=400_000, n=2000, seed=workloads.SEED_BASE + 25)
        _check(d2, "sum", rounded=True)
        got = gpu_assemble(d2, "set", keep_map=True)
        want = _oracle(d2, "set", with_map=True)
        np.testing.assert_array_equal(got[3], want[3])
    finally:
        spm.spm_set_tuning(reset=True)


def test_single_key_with_more_writes_than_fit():
    rng = np.random.Generator(np.random.PCG64(77))
    m = 50_000
    rows = np.where(rng.random(m) < 0.6, 3, rng.integers(0, 50, m)).astype(np.int32)
    cols = np.where(rows == 3, 7, rng.integers(0, 50, m)).astype(np.int32)
    d = dict(rows=rows, cols=cols, vals=rng.standard_normal(m), shape=(50, 50))
    _check(d, "set")
    seq = rng.integers(0, 1000, m).astype(np.uint64)
    _check(d, "set", seq=seq)
    _check(d, "sum", rounded=True)
    got = gpu_assemble(d, "set", keep_map=True)
    want = _oracle(d, "set", with_map=True)
    np.testing.assert_array_equal(got[3], want[3])


def test_bounded_wait_reports_timeout_and_recovers():
    # with the map, each bucket's elements are placed at once, after a bounded
    # wait for the counts of the buckets before it; a bucket that never
    # publishes its count makes that wait expire.  Without the map no block
    # waits for another (the offsets come from a scan between two kernels).
    import paper_1805_03380_gb300 as spm
    d = workloads.density_sweep(2e-3, n=10_000)  # uniform: every bucket takes the in-shared-memory path
    spm.spm_debug_withhold_publication(1)
    try:
        with pytest.raises(spm.SpmError) as e:
            gpu_assemble(d, "sum", keep_map=True)
        assert e.value.code == 6
        _check(d, "sum")  # nothing waits without the map
    finally:
        spm.spm_debug_withhold_publication(-1)
    got = gpu_assemble(d, "set", keep_map=True)
    want = _oracle(d, "set", with_map=True)
    assert_same_structure(got, want)
    np.testing.assert_array_equal(got[3], want[3])
    _check(d, "sum", rounded=True)
    _check(d, "set")
