"""Helpers for the GPU parity tests: move numpy workloads to the device, run
the library, bring the CSC back, and compare it with the oracle's."""
from __future__ import annotations

import numpy as np

TOL = {np.float64: 1e-12, np.float32: 1e-5}


def to_dev(a, dtype=None):
    import torch
    a = np.ascontiguousarray(a if dtype is None else np.asarray(a, dtype=dtype))
    return torch.from_numpy(a).cuda()


def gpu_assemble(d, mode, seq=None, keep_map=False, offset=0):
    """Run spm.assemble_csc on the workload dict d; `offset` > 0 passes views
    that start `offset` elements into padded buffers (unaligned pointers)."""
    import torch

    import paper_1805_03380_gb300 as spm
    rows = np.ascontiguousarray(d["rows"], dtype=np.int32)
    cols = np.ascontiguousarray(d["cols"], dtype=np.int32)
    vals = np.ascontiguousarray(d["vals"])
    if offset:
        pad = lambda a: np.concatenate([np.zeros(offset, dtype=a.dtype), a])  # noqa: E731
        r, c, v = to_dev(pad(rows))[offset:], to_dev(pad(cols))[offset:], to_dev(pad(vals))[offset:]
    else:
        r, c, v = to_dev(rows), to_dev(cols), to_dev(vals)
    s = None if seq is None else torch.from_numpy(np.asarray(seq, dtype=np.uint64).view(np.int64)).cuda()
    A = spm.assemble_csc(r, c, v, d["shape"], mode=mode, seq=s, keep_map=keep_map)
    out = (A.col_ptr.cpu().numpy(), A.row_idx.cpu().numpy().astype(np.int64), A.vals.cpu().numpy())
    if keep_map:
        out = out + (A.map.cpu().numpy().astype(np.int64),)
    return out


def assert_same_structure(got, want):
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])


def assert_bit_exact(got_vals, want_vals):
    got = np.asarray(got_vals)
    want = np.asarray(want_vals, dtype=got.dtype)
    nan_g, nan_w = np.isnan(got), np.isnan(want)
    np.testing.assert_array_equal(nan_g, nan_w)
    ui = np.uint64 if got.dtype.itemsize == 8 else np.uint32
    np.testing.assert_array_equal(got[~nan_g].view(ui), want[~nan_w].view(ui))


def assert_sum_within_tol(got_vals, want_vals, scale, dtype):
    tol = TOL[np.float64 if dtype == np.float64 else np.float32]
    got = np.asarray(got_vals, dtype=np.float64)
    want = np.asarray(want_vals, dtype=np.float64)
    fin = np.isfinite(want)
    assert np.all(np.abs(got[fin] - want[fin]) <= tol * scale[fin] + 0.0), \
        f"max |d|/scale = {np.max(np.abs(got[fin] - want[fin]) / np.maximum(scale[fin], 1e-300))}"
    np.testing.assert_array_equal(np.isnan(got), np.isnan(want))


def abs_contrib_per_entry(rows, cols, vals, shape, col_ptr, row_idx):
    """Sum of |contribution| of each stored CSC entry (vectorised, numpy)."""
    n_rows = shape[0]
    key = cols.astype(np.int64) * n_rows + rows.astype(np.int64)
    uk, inv = np.unique(key, return_inverse=True)
    s = np.zeros(uk.shape[0])
    np.add.at(s, inv, np.abs(np.asarray(vals, dtype=np.float64)))
    col_of = np.repeat(np.arange(shape[1], dtype=np.int64), np.diff(col_ptr))
    ek = col_of * n_rows + row_idx
    return s[np.searchsorted(uk, ek)]


def correctly_rounded_sums(d, col_ptr, row_idx):
    """Per stored element: math.fsum of its writes (the exact sum rounded once
    to float64), then float32 when the values are float32."""
    import math
    n_rows = d["shape"][0]
    rows = np.asarray(d["rows"], dtype=np.int64)
    cols = np.asarray(d["cols"], dtype=np.int64)
    vals = np.asarray(d["vals"], dtype=np.float64)
    key = cols * n_rows + rows
    order = np.argsort(key, kind="stable")
    sk, sv = key[order], vals[order]
    cut = np.flatnonzero(np.diff(sk)) + 1
    starts = np.concatenate([[0], cut])
    ends = np.concatenate([cut, [len(sk)]])
    ukeys = sk[starts]
    col_of = np.repeat(np.arange(d["shape"][1], dtype=np.int64), np.diff(np.asarray(col_ptr)))
    ek = col_of * n_rows + np.asarray(row_idx, dtype=np.int64)
    gi = np.searchsorted(ukeys, ek)
    out = np.array([math.fsum(sv[starts[g]:ends[g]]) for g in gi.tolist()])
    return out


def assert_correctly_rounded(got_vals, d, col_ptr, row_idx):
    """float64: bit-equal to fsum; float32: within one float32 ulp of fsum
    rounded to float32 (fsum then float32 may round twice)."""
    want = correctly_rounded_sums(d, col_ptr, row_idx)
    got = np.asarray(got_vals)
    if got.dtype == np.float64:
        assert_bit_exact(got, want)
    else:
        w32 = want.astype(np.float32)
        diff = np.abs(got.view(np.int32).astype(np.int64) - w32.view(np.int32).astype(np.int64))
        assert np.all(diff <= 1), f"{np.count_nonzero(diff > 1)} values more than 1 ulp from the rounded exact sum"
