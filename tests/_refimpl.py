"""Independent checkers used to pin the oracle (and, on the GPU, the library).

Nothing here is shared with either implementation: these are the textbook
definitions written out on dense arrays or through library routines.
"""
from __future__ import annotations

import numpy as np


def brute_force_csc(rows, cols, vals, shape, mode, seq=None, out_f32=False):
    """Dense definition: apply the writes in (seq, position) order to a dense
    zero matrix with X[r,c] = v (set) or X[r,c] += v (sum), then read the
    non-zero entries column by column (Section 3.1)."""
    n_rows, n_cols = shape
    A = np.zeros((n_rows, n_cols), dtype=np.float64)
    m = len(rows)
    order = list(range(m))
    if seq is not None:
        order.sort(key=lambda t: (int(seq[t]), t))
    for t in order:
        r, c, v = int(rows[t]), int(cols[t]), float(vals[t])
        if mode == "set":
            A[r, c] = v
        else:
            A[r, c] += v
    if out_f32:
        A = A.astype(np.float32).astype(np.float64)
    col_ptr = [0]
    row_idx = []
    out = []
    for c in range(n_cols):
        for r in range(n_rows):
            if A[r, c] != 0:
                row_idx.append(r)
                out.append(A[r, c])
        col_ptr.append(len(row_idx))
    return (np.array(col_ptr, dtype=np.int64), np.array(row_idx, dtype=np.int64),
            np.array(out, dtype=np.float64))


def check_csc_invariants(col_ptr, row_idx, vals, shape):
    """c[0] = 0, c non-decreasing, c[n_cols] = N (Section 3.1); rows strictly
    increasing inside each column and in range; no stored zeros."""
    n_rows, n_cols = shape
    col_ptr = np.asarray(col_ptr)
    row_idx = np.asarray(row_idx)
    vals = np.asarray(vals)
    assert col_ptr.shape == (n_cols + 1,)
    assert col_ptr[0] == 0
    assert np.all(np.diff(col_ptr) >= 0)
    nnz = int(col_ptr[-1])
    assert row_idx.shape[0] == nnz and vals.shape[0] == nnz
    if nnz:
        assert row_idx.min() >= 0 and row_idx.max() < n_rows
        assert not np.any(vals == 0)
        col_of = np.repeat(np.arange(n_cols), np.diff(col_ptr))
        same_col = col_of[1:] == col_of[:-1]
        assert np.all(row_idx[1:][same_col] > row_idx[:-1][same_col])


def distinct_nonzero_count(rows, cols, vals, shape, mode, seq=None):
    """Number of distinct coordinates whose final value is non-zero, counted
    with a hash map (dict) instead of an ordered structure."""
    final = {}
    m = len(rows)
    order = list(range(m))
    if seq is not None:
        order.sort(key=lambda t: (int(seq[t]), t))
    for t in order:
        key = (int(rows[t]), int(cols[t]))
        v = float(vals[t])
        if mode == "set" or key not in final:
            final[key] = v
        else:
            final[key] += v
    return sum(1 for v in final.values() if v != 0)


def densify(col_ptr, row_idx, vals, shape):
    A = np.zeros(shape, dtype=np.float64)
    for c in range(shape[1]):
        for p in range(int(col_ptr[c]), int(col_ptr[c + 1])):
            A[int(row_idx[p]), c] = vals[p]
    return A


def contribution_abs_sums(rows, cols, vals, shape, col_ptr, row_idx):
    """Sum of |contribution| per stored CSC entry (the scale of the summation
    tolerance), computed with a dict keyed by coordinate."""
    acc = {}
    for r, c, v in zip(np.asarray(rows).tolist(), np.asarray(cols).tolist(), np.asarray(vals).tolist()):
        acc[(r, c)] = acc.get((r, c), 0.0) + abs(v)
    out = np.empty(len(row_idx))
    n_cols = shape[1]
    p = 0
    for c in range(n_cols):
        for q in range(int(col_ptr[c]), int(col_ptr[c + 1])):
            out[q] = acc[(int(row_idx[q]), c)]
    return out


def brute_force_update(col_ptr, row_idx, vals, shape, rows, cols, wvals, mode, seq=None, out_f32=False):
    """Dense definition of writes to an existing matrix: start from A as a
    dense array, apply each write in (seq, position) order as X[r,c] = v
    (set) or X[r,c] += v (sum), then read the non-zero entries column by
    column.  With dyadic values every summation order is exact, so this
    equals any correctly implemented update bit for bit."""
    X = densify(col_ptr, row_idx, vals, shape)
    m = len(rows)
    order = list(range(m))
    if seq is not None:
        order.sort(key=lambda t: (int(seq[t]), t))
    for t in order:
        r, c, v = int(rows[t]), int(cols[t]), float(wvals[t])
        if mode == "set":
            X[r, c] = v
        else:
            X[r, c] += v
    if out_f32:
        X = X.astype(np.float32).astype(np.float64)
    n_cols = shape[1]
    cp, ri, out = [0], [], []
    for c in range(n_cols):
        nz = np.nonzero(X[:, c])[0]
        ri.extend(nz.tolist())
        out.extend(X[nz, c].tolist())
        cp.append(len(ri))
    return np.array(cp, dtype=np.int64), np.array(ri, dtype=np.int64), np.array(out, dtype=np.float64)


def exact_sums(rows, cols, vals, shape):
    """The element-wise sums of the writes computed exactly (rational
    arithmetic on the binary values), with IEEE special-value rules: NaN when
    a NaN or both infinities occur, otherwise the infinity that occurs.
    Returns {linear index: (exact sum as Fraction or float special, sum of
    |finite contributions|)} (Fig. 2: X(r,c) += v)."""
    from fractions import Fraction
    n_rows = shape[0]
    acc = {}
    for r, c, v in zip(np.asarray(rows).tolist(), np.asarray(cols).tolist(),
                       np.asarray(vals, dtype=np.float64).tolist()):
        k = int(r) + int(c) * n_rows
        s, a, nan, pinf, ninf = acc.get(k, (Fraction(0), 0.0, False, False, False))
        if v != v:
            nan = True
        elif v == float("inf"):
            pinf = True
        elif v == float("-inf"):
            ninf = True
        else:
            s += Fraction(v)
            a += abs(v)
        acc[k] = (s, a, nan, pinf, ninf)
    out = {}
    for k, (s, a, nan, pinf, ninf) in acc.items():
        if nan or (pinf and ninf):
            out[k] = (float("nan"), a)
        elif pinf:
            out[k] = (float("inf"), a)
        elif ninf:
            out[k] = (float("-inf"), a)
        else:
            out[k] = (s, a)
    return out


def assert_sums_match_exact(got, ref, shape, tol, out_f32=False):
    """The CSC `got` (col_ptr, row_idx, vals) against exact_sums `ref`:
    elements whose exact sum is special, or larger than tol * sum|c| in
    magnitude (after rounding to the output type), must be stored with a value
    within tol * sum|c| (specials equal); elements whose exact sum lies within
    tol * sum|c| of zero are cancellation-ambiguous (the order of additions
    decides whether they vanish): they may be absent, and if stored their value
    lies within that bound too.  Nothing else may be stored."""
    col_ptr, row_idx, vals = (np.asarray(x) for x in got)
    n_rows = shape[0]
    col_of = np.repeat(np.arange(shape[1]), np.diff(col_ptr))
    stored = {}
    for j, r, v in zip(col_of.tolist(), row_idx.tolist(), vals.astype(np.float64).tolist()):
        stored[int(r) + int(j) * n_rows] = v
    for k, (s, a) in ref.items():
        if isinstance(s, float):  # a special value
            assert k in stored, f"element {k}: special sum {s} not stored"
            g = stored.pop(k)
            assert (g != g and s != s) or g == s, f"element {k}: {g} != {s}"
            continue
        try:
            sf = float(s)
        except OverflowError:
            sf = float("inf") if s > 0 else float("-inf")
        with np.errstate(over="ignore"):
            rounded = float(np.float32(sf)) if out_f32 else sf
        if rounded in (float("inf"), float("-inf")):  # the rounded sum overflows
            assert stored.pop(k, None) == rounded, f"element {k}: exact sum {sf} rounds to {rounded}"
            continue
        ambiguous = abs(sf) <= tol * a or rounded == 0.0
        if k in stored:
            g = stored.pop(k)
            assert abs(g - sf) <= tol * a, f"element {k}: {g} vs exact {sf} (sum|c| {a})"
        else:
            assert ambiguous, f"element {k}: exact sum {sf} (sum|c| {a}) not stored"
    assert not stored, f"{len(stored)} elements stored that were never written"
