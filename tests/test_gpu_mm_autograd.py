"""spm_csc_mm, spm_triplet_dvals and the AssembleMM autograd function against
the oracle, float64 central differences and a dense reference gradient."""
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


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("transpose", [False, True])
def test_csc_mm_matches_oracle(dtype, transpose):
    import paper_1805_03380_gb300 as spm
    d = workloads.fem_q1(n_el=64, dtype=dtype)
    cp, ri, v = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="sum")
    n = d["shape"][0]
    X = workloads.dense_rhs(n, 16, dtype=dtype)
    Y = spm.csc_mm(to_dev(cp), to_dev(ri.astype(np.int32)), to_dev(v.astype(dtype)), d["shape"], to_dev(X),
                   transpose=transpose).cpu().numpy()
    W = oracle.csc_mm(d["shape"], cp, ri, v.astype(dtype).astype(np.float64), X.astype(np.float64),
                      transpose=transpose)
    # |error| <= k eps sum |a x| per output entry
    A_abs = oracle.csc_mm(d["shape"], cp, ri, np.abs(v.astype(dtype).astype(np.float64)),
                          np.abs(X.astype(np.float64)), transpose=transpose)
    eps = 1e-12 if dtype == np.float64 else 1e-5
    assert np.all(np.abs(Y - W) <= eps * A_abs + 1e-300)


def test_csc_mm_constant_null_space():
    import paper_1805_03380_gb300 as spm
    d = workloads.fem_q1(n_el=128, dtype=np.float64, unperturbed=True)
    A = spm.assemble_csc(to_dev(d["rows"]), to_dev(d["cols"]), to_dev(d["vals"]), d["shape"], "sum")
    ones = torch.ones(d["shape"][0], 3, dtype=torch.float64, device="cuda")
    for tr in (False, True):
        Y = spm.csc_mm(A.col_ptr, A.row_idx, A.vals, d["shape"], ones, transpose=tr)
        assert float(Y.abs().max()) < 1e-12


@pytest.mark.parametrize("mode", ["sum", "set"])
def test_dvals_matches_oracle(mode):
    import paper_1805_03380_gb300 as spm
    d = workloads.fem_q1(n_el=32, dtype=np.float64)
    n = d["shape"][0]
    rng = np.random.Generator(np.random.PCG64(3))
    X, dY = rng.standard_normal((n, 16)), rng.standard_normal((n, 16))
    A = spm.assemble_csc(to_dev(d["rows"]), to_dev(d["cols"]), to_dev(d["vals"]), d["shape"], mode,
                         keep_map=(mode == "set"))
    g = spm.triplet_dvals(to_dev(d["rows"]), to_dev(d["cols"]), A.map, to_dev(dY), to_dev(X)).cpu().numpy()
    _, _, _, mp = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode=mode, with_map=True)
    w = oracle.dvals(d["rows"], d["cols"], dY, X, map=mp if mode == "set" else None)
    np.testing.assert_allclose(g, w, rtol=1e-12, atol=1e-12)
    # float32 k = 16 fast path
    g32 = spm.triplet_dvals(to_dev(d["rows"]), to_dev(d["cols"]), A.map, to_dev(dY.astype(np.float32)),
                            to_dev(X.astype(np.float32))).cpu().numpy()
    np.testing.assert_allclose(g32, w, rtol=0, atol=1e-4 * np.max(np.abs(w)))


@pytest.mark.parametrize("mode,keep_map", [("sum", True), ("set", True), ("set", False)])
def test_assemble_mm_gradients_fd_and_dense(mode, keep_map):
    import paper_1805_03380_gb300 as spm
    d = workloads.fem_q1(n_el=32, dtype=np.float64)  # 1,089 nodes, 16,384 writes
    n = d["shape"][0]
    rows, cols = to_dev(d["rows"]), to_dev(d["cols"])
    vals = to_dev(d["vals"]).requires_grad_(True)
    rng = np.random.Generator(np.random.PCG64(11))
    X = to_dev(rng.standard_normal((n, 16))).requires_grad_(True)
    W = to_dev(rng.standard_normal((n, 16)))
    Y = spm.AssembleMM.apply(rows, cols, vals, d["shape"], X, mode, keep_map)
    loss = (Y * W).sum()
    loss.backward()
    gv, gX = vals.grad.detach().clone(), X.grad.detach().clone()

    # dense reference: A[r, c] = sum (or last) of writes, Y = A X
    def dense_forward(v, Xd):
        if mode == "sum":
            A = torch.zeros(n, n, dtype=torch.float64, device="cuda")
            A = A.index_put((rows.long(), cols.long()), v, accumulate=True)
        else:
            key = cols.long() * n + rows.long()
            last = torch.zeros(n * n, dtype=torch.long, device="cuda")
            last.scatter_reduce_(0, key, torch.arange(len(key), device="cuda"), reduce="amax", include_self=False)
            win = last[key] == torch.arange(len(key), device="cuda")
            A = torch.zeros(n, n, dtype=torch.float64, device="cuda")
            A = A.index_put((rows.long()[win], cols.long()[win]), v[win], accumulate=True)
        return A @ Xd

    v2 = vals.detach().clone().requires_grad_(True)
    X2 = X.detach().clone().requires_grad_(True)
    (dense_forward(v2, X2) * W).sum().backward()
    torch.testing.assert_close(gv, v2.grad, rtol=1e-6, atol=1e-9)
    torch.testing.assert_close(gX, X2.grad, rtol=1e-6, atol=1e-9)
    torch.testing.assert_close(Y.detach(), dense_forward(vals.detach(), X.detach()), rtol=1e-12, atol=1e-12)

    # float64 central differences on sampled write values and X entries
    h = 1e-6

    def f(v, Xd):
        with torch.no_grad():
            return float((spm.AssembleMM.apply(rows, cols, v, d["shape"], Xd, mode, keep_map) * W).sum())

    for t in rng.choice(len(d["rows"]), 12, replace=False):
        e = torch.zeros_like(vals)
        e[t] = h
        fd = (f(vals.detach() + e, X.detach()) - f(vals.detach() - e, X.detach())) / (2 * h)
        assert abs(fd - float(gv[t])) <= 1e-6 * max(1.0, abs(fd))
    for _ in range(6):
        i, j = int(rng.integers(0, n)), int(rng.integers(0, 16))
        e = torch.zeros_like(X)
        e[i, j] = h
        fd = (f(vals.detach(), X.detach() + e) - f(vals.detach(), X.detach() - e)) / (2 * h)
        assert abs(fd - float(gX[i, j])) <= 1e-6 * max(1.0, abs(fd))


def test_assemble_mm_float32_512_mesh():
    import paper_1805_03380_gb300 as spm
    d = workloads.fem_q1(n_el=512, dtype=np.float32)
    n = d["shape"][0]
    rows, cols = to_dev(d["rows"]), to_dev(d["cols"])
    vals = to_dev(d["vals"]).requires_grad_(True)
    X = to_dev(workloads.dense_rhs(n, 16)).requires_grad_(True)
    Y = spm.AssembleMM.apply(rows, cols, vals, d["shape"], X, "sum", True)
    dY = torch.ones_like(Y)
    Y.backward(dY)
    # Y against the oracle product of the oracle CSC
    cp, ri, v = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="sum")
    Xn = X.detach().cpu().numpy().astype(np.float64)
    W = oracle.csc_mm(d["shape"], cp, ri, v, Xn)
    Wabs = oracle.csc_mm(d["shape"], cp, ri, np.abs(v), np.abs(Xn))
    assert np.all(np.abs(Y.detach().cpu().numpy() - W) <= 1e-5 * Wabs + 1e-30)
    # dvals = <1, X[c]> = row sums of X
    want = Xn.sum(axis=1)[d["cols"]]
    np.testing.assert_allclose(vals.grad.cpu().numpy(), want, rtol=1e-5, atol=1e-4)


def _random_csc(n_rows, n_cols, m, seed, dtype=np.float64):
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.integers(0, n_rows, m).astype(np.int32)
    c = rng.integers(0, n_cols, m).astype(np.int32)
    v = rng.standard_normal(m).astype(dtype)
    cp, ri, vv = oracle.assemble_csc(r, c, v, (n_rows, n_cols), mode="set")
    return cp, ri.astype(np.int32), vv.astype(dtype)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_csc_transpose_matches_oracle(dtype):
    # the transpose is the CSC of the swapped coordinates: structure and values
    # bit for bit (every coordinate occurs once), including empty rows and
    # columns; transposing twice gives A back
    import paper_1805_03380_gb300 as spm
    shape = (700, 1300)
    cp, ri, v = _random_csc(*shape, 20_000, 5, dtype)
    cols = np.repeat(np.arange(shape[1], dtype=np.int32), np.diff(cp))
    want = oracle.assemble_csc(cols, ri, v, (shape[1], shape[0]), mode="set")
    At = spm.csc_transpose(to_dev(cp), to_dev(ri), to_dev(v), shape)
    assert At.shape == (shape[1], shape[0])
    np.testing.assert_array_equal(At.col_ptr.cpu().numpy(), want[0])
    np.testing.assert_array_equal(At.row_idx.cpu().numpy(), want[1])
    assert At.vals.cpu().numpy().tobytes() == want[2].astype(dtype).tobytes()
    Att = spm.csc_transpose(At.col_ptr, At.row_idx, At.vals, At.shape)
    np.testing.assert_array_equal(Att.col_ptr.cpu().numpy(), cp)
    np.testing.assert_array_equal(Att.row_idx.cpu().numpy(), ri)
    assert Att.vals.cpu().numpy().tobytes() == v.tobytes()


def test_csc_transpose_keeps_explicit_zeros_and_empty_matrices():
    import paper_1805_03380_gb300 as spm
    cp = np.array([0, 2, 2, 3], dtype=np.int64)
    ri = np.array([0, 4, 2], dtype=np.int32)
    v = np.array([0.0, -0.0, 2.5])
    At = spm.csc_transpose(to_dev(cp), to_dev(ri), to_dev(v), (5, 3))
    np.testing.assert_array_equal(At.col_ptr.cpu().numpy(), [0, 1, 1, 2, 2, 3])
    np.testing.assert_array_equal(At.row_idx.cpu().numpy(), [0, 2, 0])
    assert At.vals.cpu().numpy().tobytes() == np.array([0.0, 2.5, -0.0]).tobytes()
    E = spm.csc_transpose(to_dev(np.zeros(4, np.int64)), to_dev(np.zeros(0, np.int32)), to_dev(np.zeros(0)), (6, 3))
    assert E.nnz == 0 and E.col_ptr.cpu().numpy().tolist() == [0] * 7


def test_csc_transpose_reports_bad_rows():
    import paper_1805_03380_gb300 as spm
    cp = np.array([0, 1, 2], dtype=np.int64)
    ri = np.array([1, 9], dtype=np.int32)  # 9 is outside the 5 rows
    with pytest.raises(spm.SpmError, match="INDEX_OUT_OF_RANGE"):
        spm.csc_transpose(to_dev(cp), to_dev(ri), to_dev(np.ones(2)), (5, 2))
    with pytest.raises(spm.SpmError, match="INDEX_OUT_OF_RANGE"):
        spm.csc_mm(to_dev(cp), to_dev(ri), to_dev(np.ones(2)), (5, 2), torch.ones(2, 3, dtype=torch.float64,
                                                                                       device="cuda"))
    with pytest.raises(spm.SpmError, match="INDEX_OUT_OF_RANGE"):
        spm.csc_mm(to_dev(cp), to_dev(ri), to_dev(np.ones(2)), (5, 2), torch.ones(5, 3, dtype=torch.float64,
                                                                                       device="cuda"), transpose=True)


def _fma_chain(terms):
    """fl(...fl(fl(0 + a0 x0) + a1 x1)...) with each step a fused multiply-add
    rounded once (exact rationals, then the correctly rounded double)."""
    from fractions import Fraction
    acc = 0.0
    for a, x in terms:
        acc = float(Fraction(acc) + Fraction(float(a)) * Fraction(float(x)))
    return acc


@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("k,strided", [(1, False), (3, False), (4, True), (16, False)])
def test_csc_mm_sums_in_storage_order_bit_for_bit(transpose, k, strided):
    # float64: every output entry equals the chain of fused multiply-adds over
    # its row (A X: increasing column) or column (A^T X: increasing row) of A,
    # bit for bit, for every vector width; and repeated calls give the same bits
    import paper_1805_03380_gb300 as spm
    shape = (90, 70)
    cp, ri, v = _random_csc(*shape, 900, 6)
    v[::13] = 0.0
    rng = np.random.Generator(np.random.PCG64(7))
    n_in = shape[0] if transpose else shape[1]
    Xfull = rng.standard_normal((n_in, k + 3 if strided else k))
    Xd = to_dev(Xfull)[:, :k] if strided else to_dev(Xfull)
    X = Xfull[:, :k]
    Y1 = spm.csc_mm(to_dev(cp), to_dev(ri), to_dev(v), shape, Xd, transpose=transpose).cpu().numpy()
    Y2 = spm.csc_mm(to_dev(cp), to_dev(ri), to_dev(v), shape, Xd, transpose=transpose).cpu().numpy()
    assert Y1.tobytes() == Y2.tobytes()
    cols = np.repeat(np.arange(shape[1]), np.diff(cp))
    if transpose:  # output row c: column c of A, increasing row
        groups = {c: [(v[p], X[ri[p]]) for p in range(cp[c], cp[c + 1])] for c in range(shape[1])}
    else:  # output row r: row r of A, increasing column
        order = np.lexsort((cols, ri))
        groups = {r: [] for r in range(shape[0])}
        for p in order:
            groups[int(ri[p])].append((v[p], X[cols[p]]))
    for out, terms in groups.items():
        for j in range(k):
            assert Y1[out, j] == _fma_chain([(a, x[j]) for a, x in terms]), (out, j)


def test_assemble_mm_is_deterministic():
    import paper_1805_03380_gb300 as spm
    d = workloads.fem_q1(n_el=48, dtype=np.float32)
    rows, cols, vals = to_dev(d["rows"]), to_dev(d["cols"]), to_dev(d["vals"])
    X = torch.randn(d["shape"][0], 16, device="cuda", dtype=torch.float32, requires_grad=True)
    G = torch.randn(d["shape"][0], 16, device="cuda", dtype=torch.float32)
    outs = []
    for _ in range(2):
        v = vals.clone().requires_grad_(True)
        X.grad = None
        Y = spm.AssembleMM.apply(rows, cols, v, d["shape"], X, "sum", True)
        (Y * G).sum().backward()
        outs.append((Y.detach().cpu().numpy().tobytes(), v.grad.cpu().numpy().tobytes(),
                     X.grad.cpu().numpy().tobytes()))
    assert outs[0] == outs[1]
