"""GPU parity of the single pass for write streams already in column-major
order (incremental construction; the paper's quasi-ordered insertion) against
the CPU oracle, through the C ABI; the general path must take over whenever
the stream is not in order."""
import numpy as np
import pytest

import oracle
import workloads
from tests._refimpl import check_csc_invariants
from tests.gpu_helpers import assert_bit_exact, assert_same_structure, to_dev

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


def _run(d, mode, dtype=None):
    """Assemble on the GPU; returns the CSC (numpy) and whether the single pass finished the call."""
    import paper_1805_03380_gb300 as spm
    vals = d["vals"] if dtype is None else d["vals"].astype(dtype)
    a = spm.Assembler(d["shape"], len(d["rows"]), torch.from_numpy(vals).dtype, mode)
    a.run(to_dev(d["rows"], np.int32), to_dev(d["cols"], np.int32), to_dev(vals))
    A = a.result()
    st = spm.spm_debug_plan_stats(a)
    return (A.col_ptr.cpu().numpy(), A.row_idx.cpu().numpy().astype(np.int64), A.vals.cpu().numpy()), st["ordered_pass"]


def _dyadic(d, seed):
    d = dict(d)
    d["vals"] = workloads.dyadic_values(len(d["rows"]), seed, bits=20)
    return d


@pytest.mark.parametrize("mode", ["set", "sum"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("dup", [0.05, 0.6])
def test_ordered_stream_parity(mode, dtype, dup):
    d = _dyadic(workloads.quasi_ordered(m=300_000, n=3000, dup_frac=dup, swap_frac=0.0), 5)
    d["vals"][::11] = 0.0
    got, taken = _run(d, mode, dtype)
    assert taken == 1
    want = oracle.assemble_csc(d["rows"], d["cols"], d["vals"].astype(dtype), d["shape"], mode=mode)
    check_csc_invariants(*got, d["shape"])
    assert_same_structure(got, want)
    assert_bit_exact(got[2], want[2].astype(dtype))


def test_same_result_with_and_without_the_single_pass():
    import paper_1805_03380_gb300 as spm
    d = workloads.quasi_ordered(m=500_000, n=5000, dup_frac=0.3, swap_frac=0.0, seed=workloads.SEED_BASE + 61)
    for mode in ("set", "sum"):
        got1, taken = _run(d, mode)
        assert taken == 1
        spm.spm_set_tuning(ordered_path=0)
        try:
            got0, taken0 = _run(d, mode)
        finally:
            spm.spm_set_tuning(reset=True)
        assert taken0 == 0
        assert_same_structure(got1, got0)
        # both paths sum each run exactly at the run's own binary point and
        # round once: the same bits in both modes
        assert_bit_exact(got1[2], got0[2])


def test_streams_out_of_order_take_the_general_path():
    for swap in (0.01, 1e-5):
        d = workloads.quasi_ordered(m=300_000, n=3000, swap_frac=swap, seed=workloads.SEED_BASE + 62)
        got, taken = _run(d, "sum")
        assert taken == 0
        want = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="sum")
        assert_same_structure(got, want)
        np.testing.assert_allclose(got[2], want[2], rtol=1e-12, atol=1e-12)


def test_long_runs_and_edges():
    # one write; all writes to one element (a run longer than a tile reads); long runs inside tiles
    one = dict(rows=np.array([4], dtype=np.int32), cols=np.array([2], dtype=np.int32), vals=np.array([1.5]),
               shape=(7, 5))
    got, taken = _run(one, "set")
    assert taken == 1 and got[0].tolist() == [0, 0, 0, 1, 1, 1] and got[1].tolist() == [4]
    same = dict(rows=np.full(20_000, 3, dtype=np.int32), cols=np.full(20_000, 1, dtype=np.int32),
                vals=workloads.dyadic_values(20_000, 3), shape=(9, 4))
    got, taken = _run(same, "sum")
    assert taken == 0
    want = oracle.assemble_csc(same["rows"], same["cols"], same["vals"], same["shape"], mode="sum")
    assert_same_structure(got, want)
    assert_bit_exact(got[2], want[2])
    rng = np.random.default_rng(9)
    keys = np.repeat(np.arange(0, 40_000, 3), rng.integers(1, 60, len(np.arange(0, 40_000, 3))))
    d = dict(rows=(keys % 200).astype(np.int32), cols=(keys // 200).astype(np.int32),
             vals=workloads.dyadic_values(len(keys), 4), shape=(200, 200))
    for mode in ("set", "sum"):
        got, _ = _run(d, mode)
        want = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode=mode)
        assert_same_structure(got, want)
        assert_bit_exact(got[2], want[2])


def test_ordered_stream_with_a_bad_index_is_reported():
    import paper_1805_03380_gb300 as spm
    d = workloads.quasi_ordered(m=100_000, n=1000, swap_frac=0.0, seed=workloads.SEED_BASE + 63)
    d["rows"][50_000] = 1000
    with pytest.raises(spm.SpmError, match=spm.STATUS_NAMES[2]):
        _run(d, "sum")
    got, taken = _run(workloads.quasi_ordered(m=1000, n=100, swap_frac=0.0), "sum")
    assert taken == 1


def test_update_with_ordered_writes():
    """The update's own assembly of ordered writes (zeros kept in last-write mode) takes the single pass."""
    import paper_1805_03380_gb300 as spm
    da = workloads.update_batch(n_rows=800, n_cols=500, m_a=40_000, m=0, seed=64)
    A = oracle.assemble_csc(da["a_rows"], da["a_cols"], da["a_vals"], da["shape"], mode="sum")
    w = workloads.quasi_ordered(m=20_000, n=500, dup_frac=0.2, swap_frac=0.0, seed=workloads.SEED_BASE + 65)
    w["rows"] = (w["rows"].astype(np.int64) * 800 // 500).astype(np.int32)  # stretch rows to the 800-row matrix
    w["vals"][::5] = 0.0
    for mode in ("set", "sum"):
        want = oracle.csc_update(*A, da["shape"], w["rows"], w["cols"], w["vals"], mode=mode)
        out = spm.csc_update((to_dev(A[0], np.int64), to_dev(A[1], np.int32), to_dev(A[2]), da["shape"]),
                             to_dev(w["rows"], np.int32), to_dev(w["cols"], np.int32), to_dev(w["vals"]), mode=mode)
        got = (out.col_ptr.cpu().numpy(), out.row_idx.cpu().numpy().astype(np.int64), out.vals.cpu().numpy())
        assert_same_structure(got, want)
        if mode == "set":
            assert_bit_exact(got[2], want[2])
        else:
            np.testing.assert_allclose(got[2], want[2], rtol=1e-12, atol=1e-12)


def test_ordered_at_scale():
    """4*10^6 ordered writes on a 100,000 x 100,000 matrix (many tiles and look-back rounds)."""
    d = workloads.quasi_ordered(m=4_000_000, n=100_000, swap_frac=0.0, seed=workloads.SEED_BASE + 66)
    got, taken = _run(d, "sum")
    assert taken == 1
    want = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="sum")
    assert_same_structure(got, want)
    np.testing.assert_allclose(got[2], want[2], rtol=1e-12, atol=1e-12)


def test_graph_replay_switches_between_the_two_paths():
    """One captured call replayed on an ordered stream (single pass) and on an unordered one
    (general path): both results match the oracle."""
    import paper_1805_03380_gb300 as spm
    m, n = 200_000, 2000
    d_ord = workloads.quasi_ordered(m=m, n=n, swap_frac=0.0, seed=workloads.SEED_BASE + 67)
    d_rnd = workloads.zipf_batch(m=m, n=n, seed=workloads.SEED_BASE + 68)
    rows, cols, vals = to_dev(d_ord["rows"], np.int32), to_dev(d_ord["cols"], np.int32), to_dev(d_ord["vals"])
    a = spm.Assembler((n, n), m, torch.float64, "sum")
    a.run(rows, cols, vals)  # first call on the device (sets kernel attributes)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            a.run(rows, cols, vals, stream=s)
    for d, ordered in ((d_rnd, 0), (d_ord, 1), (d_rnd, 0)):
        rows.copy_(to_dev(d["rows"], np.int32))
        cols.copy_(to_dev(d["cols"], np.int32))
        vals.copy_(to_dev(d["vals"]))
        g.replay()
        torch.cuda.synchronize()
        A = a.result()
        assert spm.spm_debug_plan_stats(a)["ordered_pass"] == ordered
        want = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], (n, n), mode="sum")
        got = (A.col_ptr.cpu().numpy(), A.row_idx.cpu().numpy().astype(np.int64), A.vals.cpu().numpy())
        assert_same_structure(got, want)
        np.testing.assert_allclose(got[2], want[2], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_pairs_across_the_exponent_window_match_the_general_path(dtype):
    # runs of two writes whose exponents differ by 0..60 binades, with ties
    # to even and values just above and below them: the single pass (one IEEE
    # addition inside the window, the accumulator outside it) and the general
    # path give the same bits
    import paper_1805_03380_gb300 as spm
    rng = np.random.default_rng(71)
    n = 4000
    big = (1.0 + rng.integers(0, 2**20, n) / 2**20) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    shift = rng.integers(0, 61, n)
    ulp_frac = rng.choice([0.5, 0.5 + 2.0**-30, 0.5 - 2.0**-30, 0.25, 1.0], n)
    mant_bits = 53 if dtype == np.float64 else 24
    small = np.ldexp(np.ones(n), -(mant_bits - 1)) * ulp_frac * np.where(shift < 40, 1.0, 0.0)
    small = np.where(shift < 40, small, np.ldexp(rng.standard_normal(n), -shift.astype(np.int64)))
    small = small * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    rows = np.repeat(np.arange(n, dtype=np.int32), 2)
    cols = np.zeros(2 * n, dtype=np.int32)
    vals = np.empty(2 * n)
    vals[0::2], vals[1::2] = big, small
    d = dict(rows=rows, cols=cols, vals=vals.astype(dtype), shape=(n, 1))
    got1, taken = _run(d, "sum")
    assert taken == 1
    spm.spm_set_tuning(ordered_path=0)
    try:
        got0, taken0 = _run(d, "sum")
    finally:
        spm.spm_set_tuning(reset=True)
    assert taken0 == 0
    assert_same_structure(got1, got0)
    assert_bit_exact(got1[2], got0[2])
