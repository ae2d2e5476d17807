"""GPU parity of trace(A^T B) evaluated without the transpose or the product
(Section 2; Fig. 1b's workload: 10,000 x 10,000 random matrices at densities
0.01 % .. 10 %) against the CPU oracle, through the C ABI.

The library sums the products in double precision in its own fixed order, so
it is compared with the oracle within 1e-12 of the sum of |A(i,j) B(i,j)|,
and bit for bit on dyadic values, where every order is exact."""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    yield


def _random_csc(density, seed, n=10_000, dtype=np.float64, dyadic=False):
    d = workloads.density_sweep(density, n=n, dtype=dtype, seed=seed)
    vals = workloads.dyadic_values(len(d["rows"]), seed + 1, bits=10).astype(dtype) if dyadic else d["vals"]
    cp, ri, v = oracle.assemble_csc(d["rows"], d["cols"], vals, d["shape"], mode="set")
    return cp, ri, v.astype(dtype), d["shape"]


def _dev(A):
    cp, ri, v, shape = A
    return (to_dev(cp, np.int64), to_dev(ri, np.int32), to_dev(v), shape)


def _abs_products(A, B):
    return oracle.csc_trace_atb(A[0], A[1], np.abs(A[2]), B[0], B[1], np.abs(B[2]))


@pytest.mark.parametrize("density", [0.0001, 0.001, 0.01])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_trace_parity(density, dtype):
    import paper_1805_03380_gb300 as spm
    A = _random_csc(density, workloads.SEED_BASE + 91, dtype=dtype)
    B = _random_csc(density, workloads.SEED_BASE + 92, dtype=dtype)
    want = oracle.csc_trace_atb(A[0], A[1], A[2], B[0], B[1], B[2])
    got = spm.csc_trace_atb(_dev(A), _dev(B))
    assert abs(got - want) <= 1e-12 * _abs_products(A, B) + 1e-300
    # the same bits on a second call
    assert spm.csc_trace_atb(_dev(A), _dev(B)) == got


def test_trace_dyadic_is_exact():
    import paper_1805_03380_gb300 as spm
    A = _random_csc(0.01, workloads.SEED_BASE + 93, dyadic=True)
    B = _random_csc(0.01, workloads.SEED_BASE + 94, dyadic=True)
    want = oracle.csc_trace_atb(A[0], A[1], A[2], B[0], B[1], B[2])
    assert spm.csc_trace_atb(_dev(A), _dev(B)) == want
    assert spm.csc_trace_atb(_dev(A), _dev(A)) == oracle.csc_trace_atb(A[0], A[1], A[2], A[0], A[1], A[2])


def test_trace_at_ten_percent_density_properties():
    """10 % density (10^7 elements each): against scipy's elementwise product,
    and trace(A^T A) against the sum of squares of the values."""
    sp = pytest.importorskip("scipy.sparse")
    import paper_1805_03380_gb300 as spm
    A = _random_csc(0.1, workloads.SEED_BASE + 95)
    B = _random_csc(0.1, workloads.SEED_BASE + 96)
    sa = sp.csc_matrix((A[2], A[1], A[0]), shape=A[3])
    sb = sp.csc_matrix((B[2], B[1], B[0]), shape=B[3])
    prod = sa.multiply(sb)
    want = float(prod.sum())
    scale = float(abs(prod).sum())
    got = spm.csc_trace_atb(_dev(A), _dev(B))
    assert abs(got - want) <= 1e-12 * scale
    ss = float(np.sum(A[2] * A[2]))
    assert abs(spm.csc_trace_atb(_dev(A), _dev(A)) - ss) <= 1e-12 * ss


def test_trace_degenerate_and_errors():
    import paper_1805_03380_gb300 as spm
    z = np.zeros(0, dtype=np.int64)
    empty = (np.zeros(4, dtype=np.int64), z, np.zeros(0), (5, 3))
    A = (np.array([0, 2, 2, 3]), np.array([0, 4, 1]), np.array([1.5, 2.0, -3.0]), (5, 3))
    B = (np.array([0, 1, 1, 2]), np.array([4, 1]), np.array([2.0, 0.5]), (5, 3))
    assert spm.csc_trace_atb(_dev(empty), _dev(A)) == 0.0
    assert spm.csc_trace_atb(_dev(A), _dev(empty)) == 0.0
    assert spm.csc_trace_atb(_dev(A), _dev(B)) == 2.5  # (4, 0) and (1, 2) are in both: 2 * 2 - 3 * 0.5
    for shape in ((1, 4000), (4000, 1)):
        d = workloads.update_batch(n_rows=shape[0], n_cols=shape[1], m_a=3000, m=3000, hit_frac=0.5, seed=97)
        AA = oracle.assemble_csc(d["a_rows"], d["a_cols"], d["a_vals"], shape, mode="set") + (shape,)
        BB = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], shape, mode="set") + (shape,)
        want = oracle.csc_trace_atb(*AA[:3], *BB[:3])
        got = spm.csc_trace_atb(_dev(AA), _dev(BB))
        assert abs(got - want) <= 1e-12 * _abs_products(AA, BB) + 1e-300
    unsorted = (np.array([0, 2, 2, 2]), np.array([3, 1]), np.array([1.0, 1.0]), (5, 3))
    with pytest.raises(spm.SpmError, match=spm.STATUS_NAMES[1]):
        spm.csc_trace_atb(_dev(A), _dev(unsorted))
    with pytest.raises(spm.SpmError, match=spm.STATUS_NAMES[1]):
        spm.csc_trace_atb(_dev((np.array([0, 3, 2, 3]), A[1], A[2], (5, 3))), _dev(B))
    with pytest.raises(spm.SpmError, match=spm.STATUS_NAMES[2]):
        spm.csc_trace_atb(_dev(A), _dev((B[0], np.array([5, 1]), B[2], (5, 3))))
    # and the library still answers afterwards
    assert spm.csc_trace_atb(_dev(B), _dev(A)) == 2.5
