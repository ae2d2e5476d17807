"""The update, lookup, COO export and ordered-stream workloads at the full
sizes bench.py times them at, on one GB300.

The oracle runs on sampled columns: the writes of a set of columns (for the
update: A's writes and the new writes of those columns) form streams of their
own whose results are exactly those columns' part of the full result.
Properties that hold at any size (CSC invariants, element counts, every read
and every exported column) are checked on the whole output on the device,
against torch's own sort-based primitives.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_helpers import abs_contrib_per_entry, assert_bit_exact, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N = 100_000


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1805_03380_gb300 as spm
    spm.spm_set_tuning(reset=True)


@pytest.fixture(scope="module")
def n8():
    """The 10^8-write Zipf stream (bench.py's n8) and its matrix, assembled on the device."""
    import paper_1805_03380_gb300 as spm
    d = workloads.zipf_batch(m=100_000_000, n=N, dtype=np.float64, seed=workloads.SEED_BASE + 2)
    rows, cols, vals = to_dev(d["rows"]), to_dev(d["cols"]), to_dev(d["vals"])
    A = spm.assemble_csc(rows, cols, vals, d["shape"], mode="sum")
    keys = cols.long() * N + rows.long()
    del rows, cols, vals
    torch.cuda.empty_cache()
    return d, (A.col_ptr, A.row_idx.clone(), A.vals.clone()), keys


def _invariants(cp, ri, v, shape, nnz):
    assert int(cp[0]) == 0 and int(cp[-1]) == nnz
    assert bool((cp[1:] >= cp[:-1]).all())
    assert bool((ri >= 0).all()) and bool((ri < shape[0]).all())
    assert not bool((v == 0).any())
    col_of = torch.repeat_interleave(torch.arange(shape[1], device=cp.device), cp[1:] - cp[:-1])
    same = col_of[1:] == col_of[:-1]
    assert bool((ri[1:][same] > ri[:-1][same]).all())
    return col_of


def _sel(rng, extra=12):
    return sorted(set([0, 97, N // 2, N - 1] + rng.integers(0, N, extra).tolist()))


def test_update_n8_full_size_sampled_columns(n8):
    import paper_1805_03380_gb300 as spm
    d, (a_cp, a_ri, a_v), a_keys = n8
    w = workloads.zipf_batch(m=10_000_000, n=N, dtype=np.float64, seed=workloads.SEED_BASE + 8)
    wr, wc, wv = to_dev(w["rows"]), to_dev(w["cols"]), to_dev(w["vals"])
    out = spm.csc_update((a_cp, a_ri, a_v, d["shape"]), wr, wc, wv, mode="sum")
    _invariants(out.col_ptr, out.row_idx, out.vals, d["shape"], out.nnz)
    # every coordinate written for A or by the new writes is stored (continuous sums are never 0)
    union = torch.unique(torch.cat([a_keys, wc.long() * N + wr.long()]))
    assert out.nnz == union.numel()
    del union
    sel = _sel(np.random.default_rng(101))
    ma, mw = np.isin(d["cols"], sel), np.isin(w["cols"], sel)
    sub_a = oracle.assemble_csc(d["rows"][ma], d["cols"][ma], d["vals"][ma], d["shape"], mode="sum")
    want = oracle.csc_update(*sub_a, d["shape"], w["rows"][mw], w["cols"][mw], w["vals"][mw], mode="sum")
    # sum of |contributions| per element: A's element and the new writes
    a_cols = np.repeat(np.arange(d["shape"][1]), np.diff(sub_a[0]))
    scale_all = abs_contrib_per_entry(np.concatenate([sub_a[1], w["rows"][mw]]), np.concatenate([a_cols, w["cols"][mw]]),
                                      np.concatenate([sub_a[2], w["vals"][mw]]), d["shape"], want[0], want[1])
    cp = out.col_ptr.cpu().numpy()
    for c in sel:
        g0, g1, w0, w1 = int(cp[c]), int(cp[c + 1]), int(want[0][c]), int(want[0][c + 1])
        assert g1 - g0 == w1 - w0, f"column {c}"
        np.testing.assert_array_equal(out.row_idx[g0:g1].cpu().numpy(), want[1][w0:w1])
        got = out.vals[g0:g1].cpu().numpy()
        assert np.all(np.abs(got - want[2][w0:w1]) <= 1e-12 * scale_all[w0:w1]), f"column {c}"


def test_lookup_and_coo_n8_full_size(n8):
    import paper_1805_03380_gb300 as spm
    d, (cp, ri, v), _ = n8
    nnz = ri.numel()
    # COO export: the column of every element, rows and values copied
    r, c, x = spm.csc_to_coo((cp, ri, v, d["shape"]))
    col_of = torch.repeat_interleave(torch.arange(N, device=cp.device, dtype=torch.int32), cp[1:] - cp[:-1])
    assert torch.equal(c, col_of) and torch.equal(r, ri) and torch.equal(x.view(torch.int64), v.view(torch.int64))
    # 10^7 reads, half of them stored elements (bench.py's lookup_n8)
    g = torch.Generator(device=cp.device)
    g.manual_seed(7)
    q = 10_000_000
    pick = torch.randint(0, nnz, (q,), device=cp.device, generator=g)
    hit = torch.rand(q, device=cp.device, generator=g) < 0.5
    qr = torch.where(hit, ri[pick], torch.randint(0, N, (q,), device=cp.device, generator=g, dtype=torch.int32))
    qc = torch.where(hit, col_of[pick], torch.randint(0, N, (q,), device=cp.device, generator=g, dtype=torch.int32))
    vals, pos = spm.csc_lookup((cp, ri, v, d["shape"]), qr, qc)
    # expected positions from a sorted search over the stored elements' linear indices
    keys = col_of.long() * N + ri.long()
    qk = qc.long() * N + qr.long()
    s = torch.searchsorted(keys, qk)
    found = (s < nnz) & (keys[s.clamp(max=nnz - 1)] == qk)
    want_pos = torch.where(found, s, torch.full_like(s, -1))
    assert torch.equal(pos, want_pos)
    want_v = torch.where(found, v[s.clamp(max=nnz - 1)], torch.zeros_like(vals))
    assert torch.equal(vals.view(torch.int64), want_v.view(torch.int64))
    assert 0.45 < float(found.double().mean()) < 0.6


def test_ordered_n8_full_size_sampled_columns():
    """10^8 writes in column-major order (bench.py's ordered_n8): the single pass finishes it."""
    import paper_1805_03380_gb300 as spm
    d = workloads.quasi_ordered(m=100_000_000, n=N, swap_frac=0.0, dtype=np.float64,
                                seed=workloads.SEED_BASE + 10)
    rows, cols, vals = to_dev(d["rows"]), to_dev(d["cols"]), to_dev(d["vals"])
    a = spm.Assembler(d["shape"], len(d["rows"]), vals.dtype, "sum")
    a.run(rows, cols, vals)
    A = a.result()
    assert spm.spm_debug_plan_stats(a)["ordered_pass"] == 1
    _invariants(A.col_ptr, A.row_idx, A.vals, d["shape"], A.nnz)
    keys = cols.long() * N + rows.long()
    assert A.nnz == torch.unique_consecutive(keys).numel()
    del rows, cols, vals, keys
    sel = _sel(np.random.default_rng(102))
    mask = np.isin(d["cols"], sel)
    want = oracle.assemble_csc(d["rows"][mask], d["cols"][mask], d["vals"][mask], d["shape"], mode="sum")
    scale_all = abs_contrib_per_entry(d["rows"][mask], d["cols"][mask], d["vals"][mask], d["shape"], want[0], want[1])
    cp = A.col_ptr.cpu().numpy()
    for c in sel:
        g0, g1, w0, w1 = int(cp[c]), int(cp[c + 1]), int(want[0][c]), int(want[0][c + 1])
        assert g1 - g0 == w1 - w0, f"column {c}"
        np.testing.assert_array_equal(A.row_idx[g0:g1].cpu().numpy(), want[1][w0:w1])
        got = A.vals[g0:g1].cpu().numpy()
        assert np.all(np.abs(got - want[2][w0:w1]) <= 1e-12 * scale_all[w0:w1])
    # the same matrix written in last-write mode keeps the last value of every run, bit for bit
    a2 = spm.Assembler(d["shape"], len(d["rows"]), torch.float64, "set")
    a2.run(to_dev(d["rows"]), to_dev(d["cols"]), to_dev(d["vals"]))
    B = a2.result()
    wset = oracle.assemble_csc(d["rows"][mask], d["cols"][mask], d["vals"][mask], d["shape"], mode="set")
    cpb = B.col_ptr.cpu().numpy()
    for c in sel:
        g0, g1, w0, w1 = int(cpb[c]), int(cpb[c + 1]), int(wset[0][c]), int(wset[0][c + 1])
        np.testing.assert_array_equal(B.row_idx[g0:g1].cpu().numpy(), wset[1][w0:w1])
        assert_bit_exact(B.vals[g0:g1].cpu().numpy(), wset[2][w0:w1])
