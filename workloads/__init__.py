"""Seeded synthetic element-write streams shaped like the paper's workloads.

This module only draws inputs: (rows, cols, vals[, seq]) arrays and, for the
differentiable case, dense right-hand sides.  It contains none of the sync
step's arithmetic (no keys, no sorting, no duplicate resolution, no CSC), so
both the CPU oracle and the CUDA library can be fed from it without sharing
any part of the method.

Every generator takes a seed; the defaults are 1805033800 + workload number.
All arrays are numpy (host) arrays.

Workloads
---------
* ``last_write_1000``  1000 x 1000, 10,000 writes, 20 % of them rewrite an
  already-written coordinate, 5 % of values exactly 0.0, the rest N(0,1);
  element-set semantics (Table 1 ``X(1,2) = 3``).
* ``zipf_batch``       n x n (default 100,000 x 100,000) batch insertion with
  add semantics: column index bounded Zipf(s=1.1) (column 0 hottest), row
  uniform, values U(-1,1) in float64 or float32.  m = 10^7 is the paper-shaped
  batch insertion; m = 10^8 is the large assembly.
* ``fem_q1``           bilinear (Q1) quad mesh with n_el x n_el elements; each
  element emits its 4 x 4 local stiffness block (unit-square Laplacian stencil)
  with every entry scaled by an independent N(1, 0.1) factor; int32 indices.
* ``batched_uniform``  many independent square matrices of uneven size for the
  batched path (set semantics, float32 N(0,1) values, 10 % rewrites).
* ``density_sweep``    the shape of the paper's unordered-insertion experiment:
  10,000 x 10,000, uniform coordinates, m = density * 10^8.
* ``quasi_ordered``    incremental construction: writes in column-major order
  with random gaps, 5 % repeated, 1 % of adjacent pairs swapped (the paper's
  quasi-ordered insertion experiment).
* ``update_batch``     writes that build an existing matrix plus a batch of
  new writes to it, part of them hitting existing elements, part of them
  zero (insertion into a matrix already in CSC, Section 3.1).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1805033800

# Q1 element stiffness of the Laplacian on the unit square, nodes counter-
# clockwise from (0,0): (0,0), (1,0), (1,1), (0,1).  This is the input stencil
# of the FEM-shaped workload, not part of the assembly method.
Q1_STENCIL = np.array([[4.0, -1.0, -2.0, -1.0],
                       [-1.0, 4.0, -1.0, -2.0],
                       [-2.0, -1.0, 4.0, -1.0],
                       [-1.0, -2.0, -1.0, 4.0]]) / 6.0


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def last_write_1000(seed=SEED_BASE + 1, n=1000, m=10_000, rewrite_frac=0.2, zero_frac=0.05,
                    shuffled_seq=False):
    """Element writes with rewrites and explicit zeros (set semantics).

    Exactly ``round(rewrite_frac*m)`` write slots (chosen by the seed among
    positions 1..m-1) rewrite a coordinate drawn uniformly from those already
    written; the other writes take fresh uniform coordinates (rejecting
    already-written ones).  With ``shuffled_seq`` the stream is presented in a
    random order together with ``seq`` = the original position.
    Returns dict(rows, cols, vals, seq, shape).
    """
    rng = _rng(seed)
    n_rewrite = int(round(rewrite_frac * m))
    is_rewrite = np.zeros(m, dtype=bool)
    if m > 1 and n_rewrite > 0:
        is_rewrite[rng.choice(np.arange(1, m), size=min(n_rewrite, m - 1), replace=False)] = True
    rows = np.empty(m, dtype=np.int32)
    cols = np.empty(m, dtype=np.int32)
    written = []
    seen = set()
    for t in range(m):
        if is_rewrite[t] and written:
            r, c = written[int(rng.integers(0, len(written)))]
        else:
            while True:
                r = int(rng.integers(0, n))
                c = int(rng.integers(0, n))
                if (r, c) not in seen:
                    break
            seen.add((r, c))
            written.append((r, c))
        rows[t] = r
        cols[t] = c
    vals = rng.standard_normal(m)
    vals[rng.random(m) < zero_frac] = 0.0
    seq = None
    if shuffled_seq:
        perm = rng.permutation(m)
        seq = perm.astype(np.uint64)  # presented write i is original write perm[i]
        rows, cols, vals = rows[perm], cols[perm], vals[perm]
    return dict(rows=rows, cols=cols, vals=vals, seq=seq, shape=(n, n))


def zipf_cdf(n_cols, s=1.1):
    w = np.arange(1, n_cols + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    return cdf / cdf[-1]


def zipf_batch(m=10_000_000, n=100_000, s=1.1, dtype=np.float64, seed=SEED_BASE + 2, chunk=1 << 24):
    """Batch insertion stream: col ~ bounded Zipf(s) over ranks 1..n (col = rank-1),
    row ~ U{0..n-1}, value ~ U(-1,1).  Returns dict(rows, cols, vals, shape)."""
    rng = _rng(seed)
    cdf = zipf_cdf(n, s)
    rows = np.empty(m, dtype=np.int32)
    cols = np.empty(m, dtype=np.int32)
    vals = np.empty(m, dtype=dtype)
    for a in range(0, m, chunk):
        b = min(m, a + chunk)
        u = rng.random(b - a)
        cols[a:b] = np.minimum(np.searchsorted(cdf, u, side="right"), n - 1)
        rows[a:b] = rng.integers(0, n, size=b - a, dtype=np.int64)
        vals[a:b] = rng.uniform(-1.0, 1.0, size=b - a).astype(dtype)
    return dict(rows=rows, cols=cols, vals=vals, seq=None, shape=(n, n))


def fem_q1(n_el=2048, dtype=np.float64, sigma=0.1, seed=SEED_BASE + 3, unperturbed=False):
    """Q1 quad-mesh element-block stream.

    Nodes: (n_el+1)^2, id = iy*(n_el+1) + ix.  Element (ex, ey) has local nodes
    (counter-clockwise) n0 = ey*(n_el+1) + ex, n0+1, n0+n_el+2, n0+n_el+1.  The
    16 writes of an element are emitted element-major, then a-major:
    (row = g[a], col = g[b], value = Q1_STENCIL[a][b] * f), f ~ N(1, sigma)
    independently per entry (f = 1 with ``unperturbed``).
    """
    rng = _rng(seed)
    nn = n_el + 1
    ey, ex = np.divmod(np.arange(n_el * n_el, dtype=np.int64), n_el)
    n0 = ey * nn + ex
    g = np.stack([n0, n0 + 1, n0 + nn + 1, n0 + nn], axis=1)  # (E, 4)
    rows = np.repeat(g, 4, axis=1).astype(np.int32).reshape(-1)        # g[a] repeated over b
    cols = np.tile(g, (1, 4)).astype(np.int32).reshape(-1)             # g[b] cycling
    base = np.tile(Q1_STENCIL.reshape(-1), n_el * n_el)
    if unperturbed:
        vals = base.astype(dtype)
    else:
        f = rng.normal(1.0, sigma, size=base.shape[0])
        vals = (base * f).astype(dtype)
    n_nodes = nn * nn
    return dict(rows=rows, cols=cols, vals=vals, seq=None, shape=(n_nodes, n_nodes))


def update_batch(n_rows=3000, n_cols=2000, m_a=60_000, m=20_000, hit_frac=0.3, zero_frac=0.05, zipf_s=None,
                 dtype=np.float64, dyadic=False, seed=SEED_BASE + 7):
    """Writes to a matrix that is already held in CSC.

    ``a_rows, a_cols, a_vals`` (m_a writes) are the writes that built the
    existing matrix A (the caller assembles them); ``rows, cols, vals`` are
    the m new writes: a fraction ``hit_frac`` of them targets coordinates
    written for A (an update of an existing element), the rest uniform
    coordinates; a fraction ``zero_frac`` has value 0.0 (which removes an
    element in last-write mode).  Columns are uniform, or bounded Zipf(s)
    (column 0 hottest) with ``zipf_s``.  Values N(0,1), or dyadic multiples of
    2^-20 with ``dyadic`` (every sum of a few of them is exact in float32).
    """
    rng = _rng(seed)

    def draw_cols(k):
        if zipf_s is None:
            return rng.integers(0, n_cols, size=k)
        return np.minimum(np.searchsorted(zipf_cdf(n_cols, zipf_s), rng.random(k), side="right"), n_cols - 1)

    def draw_vals(k):
        if dyadic:
            return (rng.integers(-(1 << 20) + 1, 1 << 20, size=k).astype(np.float64) * 2.0 ** -20).astype(dtype)
        return rng.standard_normal(k).astype(dtype)

    a_rows = rng.integers(0, n_rows, size=m_a).astype(np.int32)
    a_cols = draw_cols(m_a).astype(np.int32)
    a_vals = draw_vals(m_a)
    rows = rng.integers(0, n_rows, size=m).astype(np.int32)
    cols = draw_cols(m).astype(np.int32)
    if m_a > 0:
        hit = rng.random(m) < hit_frac
        src = rng.integers(0, m_a, size=m)
        rows[hit] = a_rows[src[hit]]
        cols[hit] = a_cols[src[hit]]
    vals = draw_vals(m)
    vals[rng.random(m) < zero_frac] = 0.0
    return dict(a_rows=a_rows, a_cols=a_cols, a_vals=a_vals, rows=rows, cols=cols, vals=vals, seq=None,
                shape=(n_rows, n_cols))


def quasi_ordered(m=100_000_000, n=100_000, dup_frac=0.05, swap_frac=0.01, dtype=np.float64,
                  seed=SEED_BASE + 10, chunk=1 << 24):
    """Incremental construction (the paper's quasi-ordered insertion): writes
    walk the n x n matrix in column-major order.  The gap between the linear
    positions of consecutive writes is 0 with probability ``dup_frac`` (a
    repeated write) and otherwise uniform in 1 .. 2*(n*n/m) - 1, so the walk
    spans the matrix; then a fraction ``swap_frac`` of adjacent pairs is
    swapped (quasi-ordered).  Values U(-1,1).  Returns dict(rows, cols, vals)."""
    rng = _rng(seed)
    span = max(1, (2 * n * n) // m - 1)
    pos = np.empty(m, dtype=np.int64)
    base = 0
    for a in range(0, m, chunk):
        b = min(m, a + chunk)
        gaps = rng.integers(1, span + 1, size=b - a)
        gaps[rng.random(b - a) < dup_frac] = 0
        pos[a:b] = base + np.cumsum(gaps)
        base = int(pos[b - 1])
    pos = np.minimum(pos, n * n - 1)
    sw = np.flatnonzero(rng.random(m - 1) < swap_frac) if m > 1 else np.zeros(0, dtype=np.int64)
    sw = sw[np.concatenate([[True], np.diff(sw) > 1])] if len(sw) else sw  # disjoint pairs
    pos[sw], pos[sw + 1] = pos[sw + 1].copy(), pos[sw].copy()
    cols = (pos // n).astype(np.int32)
    rows = (pos - cols.astype(np.int64) * n).astype(np.int32)
    vals = rng.uniform(-1.0, 1.0, size=m).astype(dtype)
    return dict(rows=rows, cols=cols, vals=vals, seq=None, shape=(n, n))


def dense_rhs(n, k=16, dtype=np.float32, seed=SEED_BASE + 5):
    """X ~ N(0,1) of shape (n, k)."""
    return _rng(seed).standard_normal((n, k)).astype(dtype)


def batched_uniform(batch=4096, n_min=64, n_max=8192, d_min=0.001, d_max=0.02, rewrite_frac=0.1,
                    dtype=np.float32, seed=SEED_BASE + 4, max_total=None):
    """Independent square matrices: n_i ~ U{n_min..n_max}, density d_i ~ U[d_min, d_max],
    m_i = round(d_i * n_i^2) writes, of which a fraction ``rewrite_frac`` rewrite an
    earlier coordinate of the same matrix; values N(0,1).  Set semantics.
    Returns dict(rows, cols, vals, n (per matrix), trip_ptr)."""
    rng = _rng(seed)
    ns = rng.integers(n_min, n_max + 1, size=batch)
    ds = rng.uniform(d_min, d_max, size=batch)
    ms = np.maximum(1, np.round(ds * ns.astype(np.float64) ** 2)).astype(np.int64)
    if max_total is not None and ms.sum() > max_total:
        ms = np.maximum(1, (ms * (max_total / ms.sum())).astype(np.int64))
    trip_ptr = np.zeros(batch + 1, dtype=np.int64)
    trip_ptr[1:] = np.cumsum(ms)
    total = int(trip_ptr[-1])
    rows = np.empty(total, dtype=np.int32)
    cols = np.empty(total, dtype=np.int32)
    for i in range(batch):
        a, b = int(trip_ptr[i]), int(trip_ptr[i + 1])
        mi, ni = b - a, int(ns[i])
        r = rng.integers(0, ni, size=mi)
        c = rng.integers(0, ni, size=mi)
        nrw = min(int(round(rewrite_frac * mi)), mi - 1)
        if nrw > 0:
            slots = np.sort(rng.choice(np.arange(1, mi), size=nrw, replace=False))
            fresh = np.ones(mi, dtype=bool)
            fresh[slots] = False
            fresh_pos = np.flatnonzero(fresh)
            # a rewrite copies the coordinate of a uniformly chosen earlier fresh write
            n_before = slots - np.arange(nrw)
            src = fresh_pos[(rng.random(nrw) * n_before).astype(np.int64)]
            r[slots] = r[src]
            c[slots] = c[src]
        rows[a:b] = r
        cols[a:b] = c
    vals = rng.standard_normal(total).astype(dtype)
    return dict(rows=rows, cols=cols, vals=vals, n=ns.astype(np.int64), trip_ptr=trip_ptr)


def density_sweep(density, n=10_000, dtype=np.float64, seed=SEED_BASE + 6):
    """Uniform random coordinates, m = density * n^2, values N(0,1) (set semantics)."""
    rng = _rng(seed)
    m = int(round(density * n * n))
    rows = rng.integers(0, n, size=m).astype(np.int32)
    cols = rng.integers(0, n, size=m).astype(np.int32)
    vals = rng.standard_normal(m).astype(dtype)
    return dict(rows=rows, cols=cols, vals=vals, seq=None, shape=(n, n))


def dyadic_values(m, seed, bits=24):
    """Values that are integer multiples of 2^-bits in (-1, 1): sums of up to
    2^(52-bits) of them are exact in float64 in any order."""
    rng = _rng(seed)
    k = rng.integers(-(1 << bits) + 1, 1 << bits, size=m)
    return k.astype(np.float64) * 2.0 ** (-bits)
