"""GPU parity of add mode (batch insertion, X(r,c) += v, Fig. 2) at any dynamic
range: every element's sum is compared with its exact (rational) value and with
the oracle, per element, within 1e-12 * sum|contributions| (float64) or 1e-5 *
sum|contributions| (float32), the structure bit for bit.

The cases put, in one bucket, elements whose writes are ~1 next to elements
whose writes are many binades smaller (1e-25, 1e-40, 1e-300, subnormals), so
an element's sum must not depend on the magnitudes of other elements; and one
element with more writes than a bucket holds in shared memory, of
near-maximum magnitude, so the exact accumulator must not overflow.
"""
import numpy as np
import pytest

import oracle
from tests._refimpl import assert_sums_match_exact, check_csc_invariants, exact_sums
from tests.gpu_helpers import abs_contrib_per_entry, assert_same_structure, gpu_assemble

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
    spm.spm_set_tuning(reset=True)


def _compare(d, dtype):
    tol = 1e-12 if dtype == np.float64 else 1e-5
    got = gpu_assemble(d, "sum")
    check_csc_invariants(got[0], got[1], got[2], d["shape"])
    # exact sums: per element within tol * sum|c|; nothing vanishes here
    ref = exact_sums(d["rows"], d["cols"], d["vals"], d["shape"])
    assert_sums_match_exact(got, ref, d["shape"], tol, out_f32=dtype == np.float32)
    # the oracle: the same structure, values within tol * sum|c|
    want = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="sum")
    assert_same_structure(got, want)
    scale = abs_contrib_per_entry(d["rows"], d["cols"], d["vals"], d["shape"], want[0], want[1])
    g, w = got[2].astype(np.float64), want[2].astype(np.float64)
    assert np.all(np.abs(g - w) <= tol * scale), f"max |d|/scale {np.max(np.abs(g - w) / scale)}"
    return got


def _wide_range_stream(dtype, seed):
    """64 x 64 matrix: a background of ~1 values (single writes and runs of
    up to 40), and elements whose 3, 5 or 40 writes are ~1e-25, ~1e-40,
    ~1e-300 or subnormal, in random order; all in the key range of one bucket."""
    rng = np.random.default_rng(seed)
    n = 64
    tiny = [1e-25, 1e-40, 1e-300, 5e-324 * 7] if dtype == np.float64 else [1e-25, 1e-38, 1e-40, 1.4e-45 * 3]
    rows, cols, vals = [], [], []
    k = 0
    for mag in tiny:
        for count in (3, 5, 40):
            for sign in (1.0, -1.0):
                r, c = k % n, (k * 7) % n
                k += 1
                if mag < 1e-300:  # subnormal multiples: exactly representable
                    v = np.full(count, mag) * rng.integers(1, 9, count)
                else:
                    v = mag * (1.0 + rng.random(count))
                rows += [r] * count
                cols += [c] * count
                vals += list(sign * v)
    used = {(r, c) for r, c in zip(rows, cols)}
    # background: ~1 values, including long runs, in the same columns
    for _ in range(400):
        r, c = int(rng.integers(0, n)), int(rng.integers(0, n))
        if (r, c) in used:
            continue
        count = int(rng.choice([1, 1, 2, 3, 40]))
        rows += [r] * count
        cols += [c] * count
        vals += list(rng.standard_normal(count))
    order = rng.permutation(len(rows))
    return dict(rows=np.array(rows, dtype=np.int32)[order], cols=np.array(cols, dtype=np.int32)[order],
                vals=np.array(vals, dtype=dtype)[order], shape=(n, n))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_small_elements_next_to_large_ones(dtype):
    d = _wide_range_stream(dtype, 11)
    got = _compare(d, dtype)
    # every tiny element is stored, with a value of its own magnitude
    assert got[0][-1] == len(exact_sums(d["rows"], d["cols"], d["vals"], d["shape"]))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_wide_range_inside_one_element(dtype):
    # one element holds 1.0-sized and much smaller writes; values more than
    # the accumulator's window below the largest may be truncated, which stays
    # far inside tol * sum|c|
    rng = np.random.default_rng(12)
    small = 1e-300 if dtype == np.float64 else 1e-40
    v = np.concatenate([rng.standard_normal(30), small * (1 + rng.random(30)), [0.5, -0.25, 1e-20]])
    m = len(v)
    d = dict(rows=np.full(m, 3, dtype=np.int32), cols=np.full(m, 5, dtype=np.int32),
             vals=rng.permutation(v).astype(dtype), shape=(10, 10))
    _compare(d, dtype)


def test_more_writes_than_a_bucket_holds_no_overflow():
    # 70,000 writes of the largest double below 2 to one element (more than the
    # 65,536 a 58-bit binary point would allow in 128 bits), next to a small
    # matrix of ordinary elements
    big = 1.9999999999999998
    m1 = 70_000
    rng = np.random.default_rng(13)
    r2 = rng.integers(0, 200, 5000)
    c2 = rng.integers(0, 200, 5000)
    d = dict(rows=np.concatenate([np.full(m1, 17), r2]).astype(np.int32),
             cols=np.concatenate([np.full(m1, 23), c2]).astype(np.int32),
             vals=np.concatenate([np.full(m1, big), rng.standard_normal(5000)]), shape=(200, 200))
    order = rng.permutation(len(d["rows"]))
    d = {k: (v[order] if isinstance(v, np.ndarray) else v) for k, v in d.items()}
    got = _compare(d, np.float64)
    # the long run is exact: every write has the same exponent, so the sum is
    # the correctly rounded value of 70000 * big
    from fractions import Fraction
    col_of = np.repeat(np.arange(200), np.diff(got[0]))
    pos = np.nonzero((col_of == 23) & (got[1] == 17))[0]
    assert len(pos) == 1
    assert got[2][pos[0]] == float(Fraction(big) * m1)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_long_runs_across_lanes_and_warps(dtype):
    # one element with thousands of writes inside one bucket (its run spans many
    # lanes and warps), and runs of every length up to 300 around it
    rng = np.random.default_rng(14)
    rows, cols, vals = [], [], []
    rows += [5] * 6000
    cols += [9] * 6000
    vals += list(rng.standard_normal(6000) * np.exp(rng.uniform(-30, 30, 6000)))
    for L in range(1, 301):
        rows += [L % 97] * L
        cols += [(L * 13) % 50] * L
        vals += list(rng.standard_normal(L))
    order = rng.permutation(len(rows))
    d = dict(rows=np.array(rows, dtype=np.int32)[order], cols=np.array(cols, dtype=np.int32)[order],
             vals=np.array(vals, dtype=dtype)[order], shape=(100, 50))
    _compare(d, dtype)


def _narrow_stream(dtype, seed, m=40_000, n_rows=2000):
    """m writes into an n_rows x 1 matrix: every bucket's key range is narrow
    (the direct-addressed table path); values of wide dynamic range."""
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, n_rows, m).astype(np.int32)
    vals = (rng.standard_normal(m) * np.exp(rng.uniform(-20, 20, m))).astype(dtype)
    vals[rng.random(m) < 0.02] = 0.0
    return dict(rows=rows, cols=np.zeros(m, np.int32), vals=vals, shape=(n_rows, 1))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_narrow_buckets_table_path_matches_exact_and_sorted_path(dtype):
    # the table path (narrow key ranges) against the exact sums and the oracle,
    # and bit for bit against the same elements spread over a key range wide
    # enough that the sort path resolves them
    d = _narrow_stream(dtype, 21)
    got = _compare(d, dtype)
    wide = dict(rows=d["rows"] * 997, cols=d["cols"], vals=d["vals"], shape=(2000 * 997, 1))
    g2 = gpu_assemble(wide, "sum")
    assert np.array_equal(got[0], g2[0])
    np.testing.assert_array_equal(got[1] * 997, g2[1])
    assert got[2].tobytes() == g2[2].tobytes()


def test_narrow_buckets_with_nan_and_infinity_fall_back():
    d = _narrow_stream(np.float64, 22, m=20_000)
    d["vals"][5] = np.nan
    d["vals"][17] = np.inf
    d["vals"][18] = -np.inf
    got = gpu_assemble(d, "sum")
    want = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="sum")
    assert_same_structure(got, want)
    both_nan = np.isnan(got[2]) & np.isnan(want[2])
    fin = ~both_nan
    assert np.array_equal(np.isnan(got[2]), np.isnan(want[2]))
    scale = abs_contrib_per_entry(d["rows"], d["cols"], np.nan_to_num(d["vals"], nan=0.0, posinf=0.0, neginf=0.0),
                                  d["shape"], want[0], want[1])
    g, w = got[2][fin], want[2][fin]
    ok = (g == w) | (np.abs(g - w) <= 1e-12 * scale[fin])
    assert np.all(ok)


def test_narrow_buckets_last_write_bit_exact():
    d = _narrow_stream(np.float64, 23)
    got = gpu_assemble(d, "set")
    want = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="set")
    assert_same_structure(got, want)
    assert got[2].tobytes() == want[2].tobytes()


@pytest.mark.parametrize("mode", ["sum", "set"])
def test_banded_matrix_structure_and_values(mode):
    # rows within a band around the diagonal (the band-transformed sort keys),
    # near the first and last columns too, rectangular: structure bit for bit,
    # sums within the bar, last writes bit for bit
    rng = np.random.default_rng(31)
    n_rows, n_cols, m = 300_000, 250_000, 600_000
    cols = rng.integers(0, n_cols, m)
    rows = np.clip(cols + rng.integers(-37, 38, m), 0, n_rows - 1)
    rep = rng.random(m) < 0.3
    src = rng.integers(0, m, m)
    rows[rep], cols[rep] = rows[src[rep]], cols[src[rep]]
    d = dict(rows=rows.astype(np.int32), cols=cols.astype(np.int32), vals=rng.standard_normal(m),
             shape=(n_rows, n_cols))
    if mode == "sum":
        _compare(d, np.float64)
    else:
        got = gpu_assemble(d, "set")
        want = oracle.assemble_csc(d["rows"], d["cols"], d["vals"], d["shape"], mode="set")
        assert_same_structure(got, want)
        assert got[2].tobytes() == want[2].tobytes()
