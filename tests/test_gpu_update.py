"""GPU parity of spm_csc_update (batch insertion into an existing CSC matrix,
Section 3.1; the sync of Section 3.4) against the CPU oracle, through the C ABI.

Structure must match bit for bit; last-write values bit for bit; summed
values bit for bit on dyadic inputs (every order exact) and within
1e-12 (float64) / 1e-5 (float32) of the magnitudes involved otherwise.
The existing matrices A come from the oracle's assembly of seeded writes.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests._refimpl import check_csc_invariants
from tests.gpu_helpers import assert_bit_exact, to_dev

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


def _matrix_a(d, dtype):
    cp, ri, v = oracle.assemble_csc(d["a_rows"], d["a_cols"], d["a_vals"], d["shape"], mode="sum")
    return cp, ri, v.astype(dtype)


def _gpu_update(A, shape, rows, cols, vals, mode, seq=None):
    import paper_1805_03380_gb300 as spm
    cp, ri, v = A
    s = None if seq is None else torch.from_numpy(np.asarray(seq, dtype=np.uint64).view(np.int64)).cuda()
    out = spm.csc_update((to_dev(cp, np.int64), to_dev(ri, np.int32), to_dev(v), shape), to_dev(rows, np.int32),
                         to_dev(cols, np.int32), to_dev(vals), mode=mode, seq=s)
    return out.col_ptr.cpu().numpy(), out.row_idx.cpu().numpy().astype(np.int64), out.vals.cpu().numpy()


def _check(got, want, mode, exact, dtype, scale=None):
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])
    if mode == "set" or exact:
        assert_bit_exact(got[2], want[2])
    else:
        assert scale is not None, "sums are checked against the sum of |contributions| of each element"
        tol = 1e-12 if dtype == np.float64 else 1e-5
        w = np.asarray(want[2], dtype=np.float64)
        g = got[2].astype(np.float64)
        assert np.all(np.abs(g - w) <= tol * scale)


def _scale(A, d, want, shape):
    """|A's element| + sum of |writes| per output element (the sum's magnitude)."""
    n_rows = shape[0]
    acc = {}
    cp, ri, v = A
    for j in range(shape[1]):
        for e in range(int(cp[j]), int(cp[j + 1])):
            acc[int(ri[e]) + j * n_rows] = abs(float(v[e]))
    for r, c, x in zip(d["rows"].tolist(), d["cols"].tolist(), np.asarray(d["vals"], dtype=np.float64).tolist()):
        k = r + c * n_rows
        acc[k] = acc.get(k, 0.0) + abs(x)
    out = np.empty(len(want[1]))
    p = 0
    for j in range(shape[1]):
        for q in range(int(want[0][j]), int(want[0][j + 1])):
            out[p] = max(acc[int(want[1][q]) + j * n_rows], 1e-300)
            p += 1
    return out


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("mode", ["set", "sum"])
@pytest.mark.parametrize("dyadic", [True, False])
@pytest.mark.parametrize("zipf", [None, 1.1])
def test_update_parity(dtype, mode, dyadic, zipf):
    d = workloads.update_batch(n_rows=3000, n_cols=2000 if zipf is None else 300, m_a=60_000, m=20_000,
                               zipf_s=zipf, dtype=dtype, dyadic=dyadic)
    A = _matrix_a(d, dtype)
    want = oracle.csc_update(*A, d["shape"], d["rows"], d["cols"], d["vals"], mode=mode)
    got = _gpu_update(A, d["shape"], d["rows"], d["cols"], d["vals"], mode)
    check_csc_invariants(*got, d["shape"])
    scale = None if (mode == "set" or dyadic) else _scale(A, d, want, d["shape"])
    _check(got, want, mode, dyadic, dtype, scale)


def test_update_with_seq():
    d = workloads.update_batch(n_rows=500, n_cols=400, m_a=20_000, m=30_000, hit_frac=0.5, seed=11)
    A = _matrix_a(d, np.float64)
    seq = np.random.default_rng(5).integers(0, 50, len(d["rows"])).astype(np.uint64)
    want = oracle.csc_update(*A, d["shape"], d["rows"], d["cols"], d["vals"], mode="set", seq=seq)
    got = _gpu_update(A, d["shape"], d["rows"], d["cols"], d["vals"], "set", seq=seq)
    _check(got, want, "set", True, np.float64)


def test_pairs_across_tile_cuts():
    """One column: A holds every even row, the writes hit every one of them,
    so the merged sequence alternates A, B and tile cuts fall between pairs."""
    n = 20_000
    rows_a = np.arange(0, n, 2)
    A = (np.array([0, len(rows_a)], dtype=np.int64), rows_a.astype(np.int64), np.ones(len(rows_a)))
    wr = rows_a[::-1].copy()
    wc = np.zeros(len(wr), dtype=np.int64)
    wv = np.full(len(wr), 0.5)
    wv[::7] = 0.0
    for mode in ("set", "sum"):
        want = oracle.csc_update(*A, (n, 1), wr, wc, wv, mode=mode)
        got = _gpu_update(A, (n, 1), wr, wc, wv, mode)
        _check(got, want, mode, True, np.float64)


@pytest.mark.parametrize("mode", ["set", "sum"])
def test_degenerate_updates(mode):
    d = workloads.update_batch(n_rows=700, n_cols=90, m_a=5000, m=3000, seed=21)
    A = _matrix_a(d, np.float64)
    shape = d["shape"]
    e = np.zeros(0, dtype=np.int64)
    # no writes: A itself
    got = _gpu_update(A, shape, e, e, np.zeros(0), mode)
    _check(got, A, mode, True, np.float64)
    # empty A: the plain assembly of the writes
    empty = (np.zeros(shape[1] + 1, dtype=np.int64), e, np.zeros(0))
    want = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], shape, mode=mode)
    got = _gpu_update(empty, shape, d["rows"], d["cols"], d["vals"], mode)
    _check(got, want, mode, mode == "set", np.float64, None if mode == "set" else _scale(empty, d, want, shape))
    # both empty
    got = _gpu_update(empty, shape, e, e, np.zeros(0), mode)
    assert got[0].tolist() == [0] * (shape[1] + 1) and len(got[1]) == 0
    # every element of A removed: zeros written (set) or its negation added (sum)
    colj = np.repeat(np.arange(shape[1]), np.diff(A[0]))
    w = np.zeros(len(A[1])) if mode == "set" else -A[2]
    got = _gpu_update(A, shape, A[1], colj, w, mode)
    assert got[0][-1] == 0 and len(got[1]) == 0
    # single row and single column matrices
    for shp in ((1, 57), (57, 1)):
        dd = workloads.update_batch(n_rows=shp[0], n_cols=shp[1], m_a=40, m=70, seed=31)
        AA = _matrix_a(dd, np.float64)
        want = oracle.csc_update(*AA, shp, dd["rows"], dd["cols"], dd["vals"], mode=mode)
        got = _gpu_update(AA, shp, dd["rows"], dd["cols"], dd["vals"], mode)
        _check(got, want, mode, False, np.float64, None if mode == "set" else _scale(AA, dd, want, shp))


def test_stored_zeros_in_a_are_removed():
    A = (np.array([0, 3, 4], dtype=np.int64), np.array([0, 1, 4, 2], dtype=np.int64), np.array([1.0, 0.0, -0.0, 2.0]))
    got = _gpu_update(A, (5, 2), np.array([3]), np.array([1]), np.array([7.0]), "set")
    want = oracle.csc_update(*A, (5, 2), np.array([3]), np.array([1]), np.array([7.0]), mode="set")
    _check(got, want, "set", True, np.float64)
    assert got[1].tolist() == [0, 2, 3]


def test_malformed_inputs_are_reported():
    import paper_1805_03380_gb300 as spm
    shape = (3, 2)
    v = np.array([1.0, 2.0, 3.0])
    one = (np.array([1]), np.array([0]), np.array([5.0]))
    cases = [
        ((np.array([1, 2, 3]), np.array([0, 2, 1])), spm.STATUS_NAMES[1]),   # col_ptr does not start at 0
        ((np.array([0, 3, 2]), np.array([0, 2, 1])), spm.STATUS_NAMES[1]),   # decreasing
        ((np.array([0, 2, 2]), np.array([0, 2, 1])), spm.STATUS_NAMES[1]),   # last entry != nnz
        ((np.array([0, 2, 3]), np.array([2, 0, 1])), spm.STATUS_NAMES[1]),   # rows not increasing
        ((np.array([0, 2, 3]), np.array([1, 1, 1])), spm.STATUS_NAMES[1]),   # repeated row
        ((np.array([0, 2, 3]), np.array([0, 3, 1])), spm.STATUS_NAMES[2]),   # row outside the matrix
    ]
    for (cp, ri), name in cases:
        with pytest.raises(spm.SpmError, match=name):
            _gpu_update((cp, ri, v), shape, *one, "set")
    # a write outside the matrix
    with pytest.raises(spm.SpmError, match=spm.STATUS_NAMES[2]):
        _gpu_update((np.array([0, 2, 3]), np.array([0, 2, 1]), v), shape, np.array([3]), np.array([0]),
                    np.array([1.0]), "sum")
    # the map is not offered by the update: rejected before anything runs
    with pytest.raises(spm.SpmError, match=spm.STATUS_NAMES[1]):
        spm.spm_csc_update_workspace(3, 2, 3, 1, torch.float64, "set", spm.KEEP_MAP)
    # and the library still works afterwards
    got = _gpu_update((np.array([0, 2, 3]), np.array([0, 2, 1]), v), shape, *one, "set")
    assert got[1].tolist() == [0, 1, 2, 1]


def test_update_at_scale_sampled():
    """10^6 existing elements from a Zipf stream, 3*10^5 writes: full parity."""
    d = workloads.zipf_batch(m=1_000_000, n=100_000, seed=workloads.SEED_BASE + 71)
    w = workloads.zipf_batch(m=300_000, n=100_000, seed=workloads.SEED_BASE + 72)
    A = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="sum")
    rng = np.random.default_rng(73)
    rows, cols, vals = w["rows"].copy(), w["cols"].copy(), w["vals"].copy()
    # a third of the writes hit existing elements
    hit = rng.random(len(rows)) < 1 / 3
    pick = rng.integers(0, len(A[1]), len(rows))
    colj = np.repeat(np.arange(d["shape"][1]), np.diff(A[0]))
    rows[hit], cols[hit] = A[1][pick[hit]], colj[pick[hit]]
    for mode in ("set", "sum"):
        want = oracle.csc_update(*A, d["shape"], rows, cols, vals, mode=mode)
        got = _gpu_update(A, d["shape"], rows, cols, vals, mode)
        w = dict(rows=rows, cols=cols, vals=vals)
        _check(got, want, mode, False, np.float64, None if mode == "set" else _scale(A, w, want, d["shape"]))
