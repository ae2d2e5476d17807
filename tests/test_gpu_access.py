"""GPU parity of element lookup (Section 3.1) and coordinate-list export
(Section 3.2) against the CPU oracle, through the C ABI.  Values, positions
and indices must match exactly."""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_helpers import assert_bit_exact, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    yield


def _matrix(d, dtype):
    cp, ri, v = oracle.assemble_csc(d["a_rows"], d["a_cols"], d["a_vals"], d["shape"], mode="sum")
    return cp, ri, v.astype(dtype)


def _dev_csc(A, shape):
    cp, ri, v = A
    return (to_dev(cp, np.int64), to_dev(ri, np.int32), to_dev(v), shape)


def _queries(A, shape, q, rng):
    """Half of the queries ask for stored elements, half for random ones."""
    cp, ri, _ = A
    colj = np.repeat(np.arange(shape[1]), np.diff(cp))
    qr = rng.integers(0, shape[0], q)
    qc = rng.integers(0, shape[1], q)
    if len(ri):
        hit = rng.random(q) < 0.5
        pick = rng.integers(0, len(ri), q)
        qr[hit], qc[hit] = ri[pick[hit]], colj[pick[hit]]
    return qr, qc


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("zipf", [None, 1.1])
def test_lookup_parity(dtype, zipf):
    import paper_1805_03380_gb300 as spm
    d = workloads.update_batch(n_rows=3000, n_cols=2000 if zipf is None else 300, m_a=60_000, m=0, zipf_s=zipf,
                               dtype=dtype)
    A = _matrix(d, dtype)
    qr, qc = _queries(A, d["shape"], 20_000, np.random.default_rng(3))
    want_v, want_p = oracle.csc_lookup(*A, d["shape"], qr, qc)
    got_v, got_p = spm.csc_lookup(_dev_csc(A, d["shape"]), to_dev(qr, np.int32), to_dev(qc, np.int32))
    np.testing.assert_array_equal(got_p.cpu().numpy(), want_p)
    assert_bit_exact(got_v.cpu().numpy(), want_v.astype(dtype))


def test_lookup_at_scale_properties():
    """A 10^6-write Zipf matrix, 2*10^5 queries: every hit points at the
    queried row inside the queried column; every miss has no such row
    (checked with a sorted search per column)."""
    import paper_1805_03380_gb300 as spm
    d = workloads.zipf_batch(m=1_000_000, n=100_000, seed=workloads.SEED_BASE + 81)
    A = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="sum")
    qr, qc = _queries(A, d["shape"], 200_000, np.random.default_rng(4))
    got_v, got_p = spm.csc_lookup(_dev_csc(A, d["shape"]), to_dev(qr, np.int32), to_dev(qc, np.int32))
    v, p = got_v.cpu().numpy(), got_p.cpu().numpy()
    cp, ri, x = A
    lo, hi = cp[qc], cp[qc + 1]
    hit = p >= 0
    assert np.all((p[hit] >= lo[hit]) & (p[hit] < hi[hit]))
    np.testing.assert_array_equal(ri[p[hit]], qr[hit])
    np.testing.assert_array_equal(v[hit], x[p[hit]])
    assert np.all(v[~hit] == 0)
    for k in np.flatnonzero(~hit)[:2000]:
        col = ri[lo[k]:hi[k]]
        s = np.searchsorted(col, qr[k])
        assert s == len(col) or col[s] != qr[k]
    assert hit.mean() > 0.45


def test_lookup_errors():
    import paper_1805_03380_gb300 as spm
    A = (np.array([0, 2, 3]), np.array([0, 2, 1]), np.array([1.0, 2.0, 3.0]))
    with pytest.raises(spm.SpmError, match=spm.STATUS_NAMES[2]):
        spm.csc_lookup(_dev_csc(A, (3, 2)), to_dev([3], np.int32), to_dev([0], np.int32))
    bad = (np.array([0, 4, 3]), A[1], A[2])
    with pytest.raises(spm.SpmError, match=spm.STATUS_NAMES[1]):
        spm.csc_lookup(_dev_csc(bad, (3, 2)), to_dev([1], np.int32), to_dev([0], np.int32))
    v, p = spm.csc_lookup(_dev_csc(A, (3, 2)), to_dev([2, 1, 0], np.int32), to_dev([0, 0, 1], np.int32))
    assert v.cpu().tolist() == [2.0, 0.0, 0.0] and p.cpu().tolist() == [1, -1, -1]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("shape,m_a,zipf", [((3000, 2000), 60_000, None), ((3000, 300), 60_000, 1.1),
                                            ((5, 1_000_000), 3000, None), ((40_000, 1), 9000, None),
                                            ((7, 7), 0, None)])
def test_coo_export_parity(dtype, shape, m_a, zipf):
    import paper_1805_03380_gb300 as spm
    d = workloads.update_batch(n_rows=shape[0], n_cols=shape[1], m_a=m_a, m=0, zipf_s=zipf, dtype=dtype)
    A = _matrix(d, dtype)
    want = oracle.csc_to_coo(*A)
    r, c, v = spm.csc_to_coo(_dev_csc(A, shape))
    np.testing.assert_array_equal(r.cpu().numpy(), want[0])
    np.testing.assert_array_equal(c.cpu().numpy(), want[1])
    assert_bit_exact(v.cpu().numpy(), want[2].astype(dtype))


def test_coo_round_trip_on_the_gpu():
    """COO export followed by the assembly gives back the matrix."""
    import paper_1805_03380_gb300 as spm
    d = workloads.zipf_batch(m=500_000, n=50_000, seed=workloads.SEED_BASE + 82)
    A = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="sum")
    r, c, v = spm.csc_to_coo(_dev_csc(A, d["shape"]))
    B = spm.assemble_csc(r, c, v, d["shape"], mode="set")
    np.testing.assert_array_equal(B.col_ptr.cpu().numpy(), A[0])
    np.testing.assert_array_equal(B.row_idx.cpu().numpy(), A[1])
    assert_bit_exact(B.vals.cpu().numpy(), A[2])


def test_coo_export_malformed_offsets():
    import paper_1805_03380_gb300 as spm
    bad = (np.array([0, 2, 1, 3]), np.array([0, 2, 1]), np.array([1.0, 2.0, 3.0]))
    with pytest.raises(spm.SpmError, match=spm.STATUS_NAMES[1]):
        spm.csc_to_coo(_dev_csc(bad, (3, 3)))
