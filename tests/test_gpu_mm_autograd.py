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
