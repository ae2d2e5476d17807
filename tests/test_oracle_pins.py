"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: hand-written CSC
fixtures derived from the paper's examples, the dense brute-force definition
on tiny inputs, CSC invariants, scipy's COO->CSC conversion, numpy.lexsort,
exact dyadic sums and the closed-form FEM matrices.  Each family is chosen so
that a plausible slip in the oracle (wrong key order, a lost zero test, a sum
that restarts, a swapped row/column, a wrong seq tie-break) fails one of them.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from tests import _golden
from tests._refimpl import (assert_sums_match_exact, brute_force_csc, check_csc_invariants, contribution_abs_sums, densify,
                            distinct_nonzero_count)


def _assert_csc_equal(got, want):
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])
    np.testing.assert_array_equal(got[2], want[2])


# --------------------------------------------------------------------------------------------
# Hand-written fixtures (Table 1, Fig. 2, Section 3.1)
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("case", _golden.all_cases(), ids=lambda c: c["path"].rsplit("/", 1)[-1])
def test_golden_fixtures(case):
    cp, ri, v = oracle.assemble_csc(case["rows"], case["cols"], case["vals"], case["shape"], mode=case["mode"])
    np.testing.assert_array_equal(cp, case["col_ptr"])
    np.testing.assert_array_equal(ri, case["row_idx"])
    np.testing.assert_array_equal(v, case["vals_expected"])


# --------------------------------------------------------------------------------------------
# Brute force on tiny inputs
# --------------------------------------------------------------------------------------------
SPECIALS = np.array([0.0, -0.0, np.nan, np.inf, -np.inf, 1.0, -1.0, 0.5, 3.25e-300, 1e300])


def _tiny_case(rng, with_specials):
    n_rows = int(rng.integers(1, 40))
    n_cols = int(rng.integers(1, 40))
    m = int(rng.integers(0, 400))
    # few distinct coordinates so that duplicates are frequent
    n_coord = int(rng.integers(1, max(2, min(n_rows * n_cols, 60))))
    coord_r = rng.integers(0, n_rows, n_coord)
    coord_c = rng.integers(0, n_cols, n_coord)
    pick = rng.integers(0, n_coord, m)
    rows, cols = coord_r[pick], coord_c[pick]
    vals = rng.standard_normal(m)
    if with_specials and m:
        sel = rng.random(m) < 0.15
        vals[sel] = SPECIALS[rng.integers(0, len(SPECIALS), int(sel.sum()))]
    return rows, cols, vals, (n_rows, n_cols)


@pytest.mark.parametrize("mode", ["set", "sum"])
@pytest.mark.parametrize("use_seq", [False, True])
@pytest.mark.parametrize("out_f32", [False, True])
def test_brute_force_seeded(mode, use_seq, out_f32):
    rng = np.random.Generator(np.random.PCG64(7 + use_seq * 2 + out_f32 * 4 + (mode == "sum") * 8))
    for trial in range(40):
        rows, cols, vals, shape = _tiny_case(rng, with_specials=(trial % 2 == 0))
        seq = rng.integers(0, 5, len(rows)).astype(np.uint64) if use_seq else None  # many ties
        if out_f32:
            vals = vals.astype(np.float32)
        got = oracle.assemble_csc(rows, cols, vals, shape, mode=mode, seq=seq, out_f32=out_f32)
        want = brute_force_csc(rows, cols, np.asarray(vals, np.float64), shape, mode, seq=seq, out_f32=out_f32)
        _assert_csc_equal(got, want)
        check_csc_invariants(*got, shape)
        assert len(got[1]) == distinct_nonzero_count(rows, cols, np.asarray(vals, np.float64), shape, mode, seq)


def test_brute_force_hypothesis():
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=150, deadline=None)
    @hyp.given(st.data())
    def run(data):
        n_rows = data.draw(st.integers(1, 64))
        n_cols = data.draw(st.integers(1, 64))
        m = data.draw(st.integers(0, 500))
        rows = np.array(data.draw(st.lists(st.integers(0, n_rows - 1), min_size=m, max_size=m)), dtype=np.int64)
        cols = np.array(data.draw(st.lists(st.integers(0, n_cols - 1), min_size=m, max_size=m)), dtype=np.int64)
        vals = np.array(data.draw(st.lists(st.one_of(st.sampled_from([0.0, -0.0, 1.0, -1.0, 2.5]),
                                                     st.floats(allow_nan=True, allow_infinity=True)),
                                           min_size=m, max_size=m)), dtype=np.float64)
        mode = data.draw(st.sampled_from(["set", "sum"]))
        seq = None
        if data.draw(st.booleans()):
            seq = np.array(data.draw(st.lists(st.integers(0, 3), min_size=m, max_size=m)), dtype=np.uint64)
        got = oracle.assemble_csc(rows, cols, vals, (n_rows, n_cols), mode=mode, seq=seq, out_f32=False)
        want = brute_force_csc(rows, cols, vals, (n_rows, n_cols), mode, seq=seq)
        _assert_csc_equal(got, want)

    run()


def test_degenerate_shapes():
    # m = 0: all-zero col_ptr
    cp, ri, v = oracle.assemble_csc(np.zeros(0), np.zeros(0), np.zeros(0), (7, 5))
    np.testing.assert_array_equal(cp, np.zeros(6, dtype=np.int64))
    assert ri.size == 0 and v.size == 0
    # single row / single column
    for shape in [(1, 9), (9, 1)]:
        rng = np.random.Generator(np.random.PCG64(3))
        rows = rng.integers(0, shape[0], 50)
        cols = rng.integers(0, shape[1], 50)
        vals = rng.standard_normal(50)
        for mode in ("set", "sum"):
            _assert_csc_equal(oracle.assemble_csc(rows, cols, vals, shape, mode=mode),
                              brute_force_csc(rows, cols, vals, shape, mode))
    # every write to one coordinate, alternating value / 0.0: the last write decides
    rows = np.full(11, 2)
    cols = np.full(11, 3)
    vals = np.array([1.0, 0.0] * 5 + [0.0])
    cp, ri, v = oracle.assemble_csc(rows, cols, vals, (4, 4), mode="set")
    assert cp[-1] == 0
    vals[-1] = 5.0
    cp, ri, v = oracle.assemble_csc(rows, cols, vals, (4, 4), mode="set")
    assert list(ri) == [2] and list(v) == [5.0] and list(cp) == [0, 0, 0, 0, 1]


def test_out_of_range_is_an_error():
    with pytest.raises(oracle.OracleError):
        oracle.assemble_csc(np.array([0, 5]), np.array([0, 0]), np.ones(2), (5, 5))
    with pytest.raises(oracle.OracleError):
        oracle.assemble_csc(np.array([0, -1]), np.array([0, 0]), np.ones(2), (5, 5))


def test_seq_orders_writes():
    # presented in reverse, seq restores the write order: the original last write wins
    rows = np.array([1, 1, 1])
    cols = np.array([0, 0, 0])
    vals = np.array([3.0, 2.0, 1.0])
    seq = np.array([2, 1, 0], dtype=np.uint64)
    _, _, v = oracle.assemble_csc(rows, cols, vals, (2, 1), mode="set", seq=seq)
    assert list(v) == [3.0]
    # equal seq keeps stream order: the later write wins
    seq = np.array([0, 0, 0], dtype=np.uint64)
    _, _, v = oracle.assemble_csc(rows, cols, vals, (2, 1), mode="set", seq=seq)
    assert list(v) == [1.0]


def test_shuffled_stream_with_seq_equals_ordered_stream():
    ordered = workloads.last_write_1000()
    shuffled = workloads.last_write_1000(shuffled_seq=True)
    a = oracle.assemble_csc(ordered["rows"], ordered["cols"], ordered["vals"], ordered["shape"], mode="set")
    b = oracle.assemble_csc(shuffled["rows"], shuffled["cols"], shuffled["vals"], shuffled["shape"], mode="set",
                            seq=shuffled["seq"])
    _assert_csc_equal(a, b)


def test_last_write_1000_invariants():
    d = workloads.last_write_1000()
    cp, ri, v = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="set")
    check_csc_invariants(cp, ri, v, d["shape"])
    assert len(ri) == distinct_nonzero_count(d["rows"], d["cols"], d["vals"], d["shape"], "set")
    # 8,000 distinct coordinates were written; about 5 % of them end on 0.0
    assert 7400 < len(ri) < 7900


# --------------------------------------------------------------------------------------------
# Library special cases
# --------------------------------------------------------------------------------------------
def test_sum_mode_is_within_tolerance_of_exact_sums():
    """Add mode against the exact (rational) sum of each element's writes:
    within 1e-12 * sum|contributions| (float64) or 1e-5 (float32 values,
    float64 accumulation), special values by IEEE rules, across values far
    apart in magnitude (1e300 next to 3.25e-300, subnormals); elements whose
    exact sum is within that bound of zero may vanish either way."""
    from tests._refimpl import exact_sums
    rng = np.random.default_rng(808)
    for out_f32 in (False, True):
        specials = ([0.0, -0.0, np.nan, np.inf, -np.inf, 1e300, -1e300, 3.25e-300, 5e-324 * 3] if not out_f32 else
                    [0.0, -0.0, np.nan, np.inf, -np.inf, 3e38, -3e38, 1e-40, 1.4e-45 * 3])
        for trial in range(40):
            n_rows, n_cols = int(rng.integers(1, 30)), int(rng.integers(1, 30))
            m = int(rng.integers(0, 400))
            n_coord = int(rng.integers(1, 50))
            cr, cc = rng.integers(0, n_rows, n_coord), rng.integers(0, n_cols, n_coord)
            pick = rng.integers(0, n_coord, m)
            vals = rng.standard_normal(m) * np.exp(rng.uniform(-20, 20, m))
            sel = rng.random(m) < 0.2
            vals[sel] = np.array(specials)[rng.integers(0, len(specials), int(sel.sum()))]
            dt = np.float32 if out_f32 else np.float64
            rows, cols, v = cr[pick].astype(np.int32), cc[pick].astype(np.int32), vals.astype(dt)
            got = oracle.assemble_csc(rows, cols, v, (n_rows, n_cols), mode="sum")
            check_csc_invariants(*got, (n_rows, n_cols))
            assert_sums_match_exact(got, exact_sums(rows, cols, v, (n_rows, n_cols)), (n_rows, n_cols),
                                    1e-5 if out_f32 else 1e-12, out_f32=out_f32)


def test_sum_mode_matches_scipy():
    sp = pytest.importorskip("scipy.sparse")
    d = workloads.zipf_batch(m=200_000, n=3000)
    cp, ri, v = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="sum")
    A = sp.coo_matrix((d["vals"], (d["rows"].astype(np.int64), d["cols"].astype(np.int64))), shape=d["shape"]).tocsc()
    A.sum_duplicates()
    A.eliminate_zeros()
    A.sort_indices()
    np.testing.assert_array_equal(cp, A.indptr)
    np.testing.assert_array_equal(ri, A.indices)
    scale = contribution_abs_sums(d["rows"], d["cols"], d["vals"], d["shape"], cp, ri)
    assert np.all(np.abs(v - A.data) <= 1e-12 * scale)


def test_distinct_nonzero_stream_is_a_lexsort():
    rng = np.random.Generator(np.random.PCG64(11))
    n_rows, n_cols, m = 5000, 3000, 100_000
    lin = rng.choice(n_rows * n_cols, size=m, replace=False)
    rows, cols = lin % n_rows, lin // n_rows
    rows, cols = rows[rng.permutation(m)], cols[rng.permutation(m)]  # decorrelate and shuffle
    keep = np.unique(cols.astype(np.int64) * n_rows + rows, return_index=True)[1]
    rows, cols = rows[keep], cols[keep]
    perm = rng.permutation(len(rows))
    rows, cols = rows[perm], cols[perm]
    vals = rng.uniform(0.5, 1.5, len(rows)) * rng.choice([-1.0, 1.0], len(rows))
    for mode in ("set", "sum"):
        cp, ri, v = oracle.assemble_csc(rows, cols, vals, (n_rows, n_cols), mode=mode)
        order = np.lexsort((rows, cols))
        np.testing.assert_array_equal(ri, rows[order])
        np.testing.assert_array_equal(v, vals[order])
        np.testing.assert_array_equal(cp, np.concatenate([[0], np.cumsum(np.bincount(cols, minlength=n_cols))]))


def test_dyadic_sums_are_exact():
    # Multiples of 2^-24 with at most 2^20 terms per coordinate sum exactly in
    # float64 in any order, so the oracle must equal the exact integer sum, and
    # coordinates whose integer sum is 0 must be absent.
    rng = np.random.Generator(np.random.PCG64(5))
    n_rows, n_cols, n_coord, m = 300, 200, 500, 60_000
    cr = rng.integers(0, n_rows, n_coord)
    cc = rng.integers(0, n_cols, n_coord)
    pick = rng.integers(0, n_coord, m)
    rows, cols = cr[pick], cc[pick]
    k = rng.integers(-(1 << 24) + 1, 1 << 24, m)
    # force exact cancellation on a few coordinates: append the negated sum
    first = np.unique(pick)[:25]
    extra_r, extra_c, extra_k = [], [], []
    for q in first:
        tot = int(k[pick == q].sum())
        extra_r.append(cr[q])
        extra_c.append(cc[q])
        extra_k.append(-tot)
    rows = np.concatenate([rows, extra_r])
    cols = np.concatenate([cols, extra_c])
    k = np.concatenate([k, extra_k])
    vals = k.astype(np.float64) * 2.0 ** -24
    cp, ri, v = oracle.assemble_csc(rows, cols, vals, (n_rows, n_cols), mode="sum")
    exact = {}
    for r, c, kk in zip(rows.tolist(), cols.tolist(), k.tolist()):
        exact[(r, c)] = exact.get((r, c), 0) + kk
    want = sorted(((c, r), s) for (r, c), s in exact.items() if s != 0)
    assert len(ri) == len(want)
    col_of = np.repeat(np.arange(n_cols), np.diff(cp))
    for q, ((c, r), s) in enumerate(want):
        assert (col_of[q], ri[q]) == (c, r)
        assert v[q] == s * 2.0 ** -24


# --------------------------------------------------------------------------------------------
# Closed forms: the unperturbed Q1 Laplacian
# --------------------------------------------------------------------------------------------
def test_fem_closed_form():
    n_el = 32
    nn = n_el + 1
    d = workloads.fem_q1(n_el=n_el, unperturbed=True)
    cp, ri, v = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="sum")
    check_csc_invariants(cp, ri, v, d["shape"])
    assert cp[-1] == (3 * nn - 2) ** 2 == 9409
    assert set(np.unique(np.diff(cp)).tolist()) == {4, 6, 9}
    A = densify(cp, ri, v, d["shape"])
    ix, iy = np.meshgrid(np.arange(nn), np.arange(nn))
    on_x = (ix == 0) | (ix == nn - 1)
    on_y = (iy == 0) | (iy == nn - 1)
    diag = np.diag(A).reshape(nn, nn)
    np.testing.assert_allclose(diag[~on_x & ~on_y], 8 / 3, rtol=0, atol=1e-14)
    np.testing.assert_allclose(diag[on_x ^ on_y], 4 / 3, rtol=0, atol=1e-14)
    np.testing.assert_allclose(diag[on_x & on_y], 2 / 3, rtol=0, atol=1e-14)
    # an interior node couples to its 8 neighbours with -1/3 each
    node = 5 * nn + 7
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dx or dy:
                assert abs(A[node, node + dy * nn + dx] + 1 / 3) < 1e-15
    # along the boundary edge only one element is shared: -1/6
    assert abs(A[3, 4] + 1 / 6) < 1e-15
    # rows sum to zero (constants are in the Laplacian's null space)
    Y = oracle.csc_mm(d["shape"], cp, ri, v, np.ones((nn * nn, 1)))
    assert np.max(np.abs(Y)) < 1e-13
    # symmetric
    np.testing.assert_allclose(A, A.T, rtol=0, atol=0)


# --------------------------------------------------------------------------------------------
# csc_mm and dvals
# --------------------------------------------------------------------------------------------
def test_csc_mm_matches_dense_matmul():
    rng = np.random.Generator(np.random.PCG64(9))
    shape = (70, 45)
    rows = rng.integers(0, shape[0], 900)
    cols = rng.integers(0, shape[1], 900)
    vals = rng.standard_normal(900)
    cp, ri, v = oracle.assemble_csc(rows, cols, vals, shape, mode="sum")
    A = densify(cp, ri, v, shape)
    X = rng.standard_normal((shape[1], 16))
    np.testing.assert_allclose(oracle.csc_mm(shape, cp, ri, v, X), A @ X, rtol=1e-13, atol=1e-13)
    X2 = rng.standard_normal((shape[0], 5))
    np.testing.assert_allclose(oracle.csc_mm(shape, cp, ri, v, X2, transpose=True), A.T @ X2, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("mode", ["set", "sum"])
def test_dvals_matches_finite_differences_and_dense_gradient(mode):
    rng = np.random.Generator(np.random.PCG64(13 + (mode == "sum")))
    shape = (20, 15)
    m = 300
    rows = rng.integers(0, shape[0], m)
    cols = rng.integers(0, shape[1], m)
    vals = rng.standard_normal(m)
    vals[:10] = 0.0  # some writes of 0.0 (removed coordinates keep their gradient)
    X = rng.standard_normal((shape[1], 4))
    dY = rng.standard_normal((shape[0], 4))
    _, _, _, mp = oracle.assemble_csc(rows, cols, vals, shape, mode=mode, with_map=True)
    g = oracle.dvals(rows, cols, dY, X, map=mp if mode == "set" else None)
    # dense gradient: d<dY, A X>/dA = dY X^T, and A[r,c] depends on the winner (set)
    # or on every contribution (sum)
    G = dY @ X.T
    winner = {}
    for t in range(m):
        winner[(rows[t], cols[t])] = t
    for t in range(m):
        expect = G[rows[t], cols[t]] if (mode == "sum" or winner[(rows[t], cols[t])] == t) else 0.0
        assert abs(g[t] - expect) < 1e-12
    # central finite differences through the oracle itself
    def f(vv):
        cp, ri, v = oracle.assemble_csc(rows, cols, vv, shape, mode=mode)
        return float(np.sum(dY * oracle.csc_mm(shape, cp, ri, v, X)))
    h = 1e-6
    for t in rng.choice(m, 25, replace=False).tolist() + [0, 1, 2]:
        e = np.zeros(m)
        e[t] = h
        fd = (f(vals + e) - f(vals - e)) / (2 * h)
        assert abs(fd - g[t]) < 1e-6 * max(1.0, abs(g[t]))
    # map: -1 exactly for overwritten writes in set mode, never in sum mode
    if mode == "sum":
        assert np.all(mp != -1)
    else:
        for t in range(m):
            assert (mp[t] == -1) == (winner[(rows[t], cols[t])] != t)


# --------------------------------------------------------------------------------------------
# Batch insertion into an existing CSC matrix (Section 3.1 sort-then-merge, Section 3.4 sync)
# --------------------------------------------------------------------------------------------
def _dyadic(rng, k, bits=12):
    return rng.integers(-(1 << bits) + 1, 1 << bits, size=k).astype(np.float64) * 2.0 ** -bits


def _tiny_update_case(rng, zero_frac=0.2, hit_frac=0.5):
    """A canonical CSC matrix built by scipy from a dense array, and writes,
    part of them to A's elements; dyadic values (all sums exact)."""
    sp = pytest.importorskip("scipy.sparse")
    n_rows = int(rng.integers(1, 25))
    n_cols = int(rng.integers(1, 25))
    dense = np.where(rng.random((n_rows, n_cols)) < 0.3, _dyadic(rng, n_rows * n_cols).reshape(n_rows, n_cols), 0.0)
    A = sp.csc_matrix(dense)
    A.sort_indices()
    m = int(rng.integers(0, 80))
    rows = rng.integers(0, n_rows, m)
    cols = rng.integers(0, n_cols, m)
    nz_r, nz_c = np.nonzero(dense)
    if len(nz_r) and m:
        hit = rng.random(m) < hit_frac
        pick = rng.integers(0, len(nz_r), m)
        rows[hit], cols[hit] = nz_r[pick[hit]], nz_c[pick[hit]]
    vals = _dyadic(rng, m)
    vals[rng.random(m) < zero_frac] = 0.0
    if m and len(nz_r):  # writes that cancel an element exactly (sum mode removes it)
        k = int(rng.integers(0, m))
        rows[k], cols[k] = nz_r[0], nz_c[0]
        vals[k] = -dense[nz_r[0], nz_c[0]]
    return (A.indptr.astype(np.int64), A.indices.astype(np.int64), A.data.astype(np.float64), (n_rows, n_cols),
            rows, cols, vals)


@pytest.mark.parametrize("mode", ["set", "sum"])
@pytest.mark.parametrize("use_seq", [False, True])
@pytest.mark.parametrize("out_f32", [False, True])
def test_update_matches_dense_sequential_writes(mode, use_seq, out_f32):
    rng = np.random.default_rng(1805_2 + 7 * use_seq + 3 * out_f32 + (mode == "sum"))
    from tests._refimpl import brute_force_update
    for _ in range(40):
        cp, ri, v, shape, rows, cols, vals = _tiny_update_case(rng)
        seq = rng.integers(0, 4, len(rows)).astype(np.uint64) if use_seq else None
        wv = vals.astype(np.float32) if out_f32 else vals
        av = v.astype(np.float32) if out_f32 else v
        got = oracle.csc_update(cp, ri, av, shape, rows, cols, wv, mode=mode, seq=seq)
        want = brute_force_update(cp, ri, v, shape, rows, cols, vals, mode, seq=seq, out_f32=out_f32)
        _assert_csc_equal(got, want)
        check_csc_invariants(*got, shape)


def test_update_sum_is_scipy_addition():
    """Sum mode: A + (the new writes assembled with duplicates summed), by scipy."""
    sp = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(18053)
    for _ in range(40):
        cp, ri, v, shape, rows, cols, vals = _tiny_update_case(rng)
        A = sp.csc_matrix((v, ri, cp), shape=shape)
        Bm = sp.coo_matrix((vals, (rows, cols)), shape=shape).tocsc()
        C = (A + Bm).tocsc()
        C.eliminate_zeros()
        C.sort_indices()
        got = oracle.csc_update(cp, ri, v, shape, rows, cols, vals, mode="sum")
        np.testing.assert_array_equal(got[0], C.indptr)
        np.testing.assert_array_equal(got[1], C.indices)
        np.testing.assert_array_equal(got[2], C.data)


def test_update_special_cases():
    rng = np.random.default_rng(18054)
    for _ in range(20):
        cp, ri, v, shape, rows, cols, vals = _tiny_update_case(rng, zero_frac=0.0)
        # no writes: A itself (A holds no zeros)
        _assert_csc_equal(oracle.csc_update(cp, ri, v, shape, rows[:0], cols[:0], vals[:0]), (cp, ri, v))
        # an empty A: the plain assembly of the writes
        empty = (np.zeros(shape[1] + 1, dtype=np.int64), np.zeros(0, dtype=np.int64), np.zeros(0))
        for mode in ("set", "sum"):
            _assert_csc_equal(oracle.csc_update(*empty, shape, rows, cols, vals, mode=mode),
                              oracle.assemble_csc(rows, cols, vals, shape, mode=mode))
        # last-write mode composes: two batches in turn equal their concatenation
        h = len(rows) // 2
        once = oracle.csc_update(cp, ri, v, shape, rows, cols, vals, mode="set")
        first = oracle.csc_update(cp, ri, v, shape, rows[:h], cols[:h], vals[:h], mode="set")
        twice = oracle.csc_update(*first, shape, rows[h:], cols[h:], vals[h:], mode="set")
        _assert_csc_equal(twice, once)
        # zeros written over every element of A (set) or its negation added (sum) empty the matrix
        colj = np.repeat(np.arange(shape[1]), np.diff(cp))
        for mode, w in (("set", np.zeros(len(ri))), ("sum", -v)):
            cp2, ri2, v2 = oracle.csc_update(cp, ri, v, shape, ri, colj, w, mode=mode)
            assert cp2[-1] == 0 and len(ri2) == 0


def test_update_rejects_malformed_matrices():
    cp, ri, v = np.array([0, 2, 3]), np.array([0, 2, 1]), np.array([1.0, 2.0, 3.0])
    shape = (3, 2)
    none = (np.zeros(0, dtype=np.int64),) * 2 + (np.zeros(0),)
    oracle.csc_update(cp, ri, v, shape, *none)
    bad = {
        "invalid argument": [(np.array([1, 2, 3]), ri), (np.array([0, 3, 2]), ri), (np.array([0, 2, 2]), ri),
                             (cp, np.array([2, 0, 1])), (cp, np.array([1, 1, 1]))],
        "index out of range": [(cp, np.array([0, 3, 1])), (cp, np.array([-1, 2, 1]))],
    }
    for msg, cases in bad.items():
        for c, r in cases:
            with pytest.raises(oracle.OracleError, match=msg):
                oracle.csc_update(c, r, v, shape, *none)
    with pytest.raises(oracle.OracleError, match="index out of range"):
        oracle.csc_update(cp, ri, v, shape, np.array([3]), np.array([0]), np.array([1.0]))


# --------------------------------------------------------------------------------------------
# Element lookup (Section 3.1) and coordinate-list export (Section 3.2)
# --------------------------------------------------------------------------------------------
def test_lookup_matches_dense_indexing():
    rng = np.random.default_rng(18055)
    for _ in range(30):
        cp, ri, v, shape, rows, cols, vals = _tiny_update_case(rng)
        X = densify(cp, ri, v, shape)
        qr = rng.integers(0, shape[0], 60)
        qc = rng.integers(0, shape[1], 60)
        got, pos = oracle.csc_lookup(cp, ri, v, shape, qr, qc)
        np.testing.assert_array_equal(got, X[qr, qc])
        stored = pos >= 0
        np.testing.assert_array_equal(stored, X[qr, qc] != 0)
        np.testing.assert_array_equal(ri[pos[stored]], qr[stored])
        assert np.all((cp[qc[stored]] <= pos[stored]) & (pos[stored] < cp[qc[stored] + 1]))
    with pytest.raises(oracle.OracleError, match="index out of range"):
        oracle.csc_lookup(cp, ri, v, shape, [shape[0]], [0])


def test_coo_export_matches_scipy_and_round_trips():
    sp = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(18056)
    for _ in range(30):
        cp, ri, v, shape, *_ = _tiny_update_case(rng)
        r, c, x = oracle.csc_to_coo(cp, ri, v)
        coo = sp.csc_matrix((v, ri, cp), shape=shape).tocoo()
        order = np.lexsort((coo.row, coo.col))
        np.testing.assert_array_equal(r, coo.row[order])
        np.testing.assert_array_equal(c, coo.col[order])
        np.testing.assert_array_equal(x, coo.data[order])
        # the coordinate list assembles back to the same matrix
        _assert_csc_equal(oracle.assemble_csc(r, c, x, shape, mode="set"), (cp, ri, v))


# --------------------------------------------------------------------------------------------
# trace(A^T B) without the transpose or the product (Section 2, Fig. 1b)
# --------------------------------------------------------------------------------------------
def test_trace_matches_dense_and_scipy():
    sp = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(18057)
    for _ in range(40):
        cp, ri, v, shape, *_ = _tiny_update_case(rng)
        dense_b = np.where(rng.random(shape) < 0.4, _dyadic(rng, shape[0] * shape[1]).reshape(shape), 0.0)
        B = sp.csc_matrix(dense_b)
        B.sort_indices()
        got = oracle.csc_trace_atb(cp, ri, v, B.indptr, B.indices, B.data)
        A = densify(cp, ri, v, shape)
        assert got == np.trace(A.T @ dense_b)           # dyadic values: exact in any order
        assert got == float(sp.csc_matrix((v, ri, cp), shape=shape).multiply(B).sum())
        assert got == oracle.csc_trace_atb(B.indptr, B.indices, B.data, cp, ri, v)  # trace(A^T B) = trace(B^T A)


def _hyp_csc(data, st, n_rows, n_cols, values):
    """A canonical CSC matrix drawn by hypothesis: a dense pattern with values from `values`
    (zero excluded), converted column by column."""
    cp, ri, v = [0], [], []
    for _ in range(n_cols):
        rows = sorted(set(data.draw(st.lists(st.integers(0, n_rows - 1), max_size=min(n_rows, 6)))))
        for r in rows:
            ri.append(r)
            v.append(data.draw(st.sampled_from(values)))
        cp.append(len(ri))
    return np.array(cp, dtype=np.int64), np.array(ri, dtype=np.int64), np.array(v, dtype=np.float64)


def test_update_hypothesis():
    """Writes to an existing matrix, drawn by hypothesis (repeats, zeros, -0.0, NaN and
    infinities, seq ties): the oracle equals sequential writes on a dense array."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")
    from tests._refimpl import brute_force_update
    a_values = [1.0, -1.0, 2.5, 0.25, np.inf, -np.inf, np.nan]
    w_values = a_values + [0.0, -0.0]

    @hyp.settings(max_examples=150, deadline=None)
    @hyp.given(st.data())
    def run(data):
        n_rows = data.draw(st.integers(1, 12))
        n_cols = data.draw(st.integers(1, 12))
        cp, ri, v = _hyp_csc(data, st, n_rows, n_cols, a_values)
        m = data.draw(st.integers(0, 60))
        rows = np.array(data.draw(st.lists(st.integers(0, n_rows - 1), min_size=m, max_size=m)), dtype=np.int64)
        cols = np.array(data.draw(st.lists(st.integers(0, n_cols - 1), min_size=m, max_size=m)), dtype=np.int64)
        vals = np.array(data.draw(st.lists(st.sampled_from(w_values), min_size=m, max_size=m)), dtype=np.float64)
        mode = data.draw(st.sampled_from(["set", "sum"]))
        seq = None
        if data.draw(st.booleans()):
            seq = np.array(data.draw(st.lists(st.integers(0, 3), min_size=m, max_size=m)), dtype=np.uint64)
        got = oracle.csc_update(cp, ri, v, (n_rows, n_cols), rows, cols, vals, mode=mode, seq=seq, out_f32=False)
        want = brute_force_update(cp, ri, v, (n_rows, n_cols), rows, cols, vals, mode, seq=seq)
        _assert_csc_equal(got, want)

    run()


def test_trace_hypothesis():
    """trace(A^T B) of matrices drawn by hypothesis (small dyadic values, so every order
    of summation is exact) equals the dense trace of A^T B."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")
    values = [1.0, -1.0, 2.5, 0.25, -0.125, 3.0]

    @hyp.settings(max_examples=150, deadline=None)
    @hyp.given(st.data())
    def run(data):
        n_rows = data.draw(st.integers(1, 12))
        n_cols = data.draw(st.integers(1, 12))
        A = _hyp_csc(data, st, n_rows, n_cols, values)
        B = _hyp_csc(data, st, n_rows, n_cols, values)
        got = oracle.csc_trace_atb(*A, *B)
        DA = densify(*A, (n_rows, n_cols))
        DB = densify(*B, (n_rows, n_cols))
        assert got == float(np.trace(DA.T @ DB))

    run()
