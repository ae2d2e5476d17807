"""The C-ABI library: builds for sm_103a, loads, exports every entry point that
include/spm.h declares, and rejects bad arguments on the host (no GPU needed:
nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(spm_[a-z0-9_]+)\s*\(", text, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def spm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1805_03380_gb300 as spm
    return spm


def test_library_exports_every_declared_symbol(spm):
    declared = _declared_functions()
    assert len(declared) >= 10
    lib = ctypes.CDLL(spm.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(declared) == set(spm.EXPORTED)


def test_status_strings_and_version(spm):
    L = spm.lib()
    assert L.spm_status_string(0) == b"SPM_OK"
    assert L.spm_status_string(6) == b"SPM_ERR_TIMEOUT"
    assert L.spm_version() >= 10000


def test_workspace_query_and_limits(spm):
    import torch
    m = 100_000_000
    ws = spm.spm_assemble_csc_workspace(100_000, 100_000, m, torch.float64, "sum")
    # records (16 bytes per write) and, above the two-pass threshold, the first
    # pass's records (16) and their buckets (4) dominate; planner tables and the
    # per-(block, bucket) counters are small next to them
    assert 36 * m < ws < 40 * m
    t0 = spm.spm_get_tuning()
    try:
        spm.spm_set_tuning(two_pass_min_writes=2**31 - 1)
        ws1 = spm.spm_assemble_csc_workspace(100_000, 100_000, m, torch.float64, "sum")
        assert 16 * m < ws1 < 20 * m
        assert ws - ws1 >= 19 * m
    finally:
        spm.spm_set_tuning(reset=True)
    assert spm.spm_get_tuning() == t0
    # seq is read from the caller's array: it needs no workspace of its own
    m = 1_000_000  # below the two-pass threshold
    ws_set = spm.spm_assemble_csc_workspace(100_000, 100_000, m, torch.float64, "set")
    ws_seq = spm.spm_assemble_csc_workspace(100_000, 100_000, m, torch.float64, "set", spm.SEQ_EXPLICIT)
    assert ws_seq == ws_set
    assert spm.spm_assemble_csc_workspace(1000, 1000, 0, torch.float32, "set") > 0
    with pytest.raises(spm.SpmError) as e:
        spm.spm_assemble_csc_workspace(1 << 30, 1 << 30, 10, torch.float64, "sum")  # 2^60 > 2^52 key space
    assert e.value.code == 4
    with pytest.raises(spm.SpmError) as e:
        spm.spm_assemble_csc_workspace(-1, 5, 10, torch.float64, "sum")
    assert e.value.code == 1
    with pytest.raises(spm.SpmError):
        spm.spm_assemble_csc_workspace(10, 10, 1 << 33, torch.float64, "sum")


def test_batched_workspace_query(spm):
    import torch
    ws = spm.spm_assemble_csc_batched_workspace([10, 20, 30], [10, 20, 30], [0, 5, 5, 40], torch.float32, "set")
    assert ws > 0
    with pytest.raises(spm.SpmError):  # trip_ptr must start at 0 and not decrease
        spm.spm_assemble_csc_batched_workspace([10, 20], [10, 20], [1, 5, 7], torch.float32, "set")
    with pytest.raises(spm.SpmError):
        spm.spm_assemble_csc_batched_workspace([10, 20], [10, 20], [0, 5, 3], torch.float32, "set")


def test_host_argument_validation_launches_nothing(spm):
    L = spm.lib()
    # invalid dtype / mode / flags / missing status pointer are rejected before any CUDA call
    args = dict(n_rows=10, n_cols=10, m=0)
    null = None
    assert L.spm_assemble_csc(10, 10, 0, null, null, null, null, 7, 0, 0, null, null, null, null, null, null, null, 0,
                              null) == 1
    assert L.spm_assemble_csc(10, 10, 0, null, null, null, null, 0, 9, 0, null, null, null, null, null, null, null, 0,
                              null) == 1
    assert L.spm_assemble_csc(10, 10, 0, null, null, null, null, 0, 0, 64, null, null, null, null, null, null, null,
                              0, null) == 1
    # SEQ_EXPLICIT without a seq pointer
    assert L.spm_assemble_csc(10, 10, 0, null, null, null, null, 0, 0, 4, null, null, null, null, null, null, null,
                              0, null) == 1
    # KEEP_MAP without a map pointer
    assert L.spm_assemble_csc(10, 10, 0, null, null, null, null, 0, 0, 1, null, null, null, null, null, null, null,
                              0, null) == 1
    # spm_csc_mm(n_rows, n_cols, nnz, col_ptr, row_idx, vals, dtype, transpose, k, X, ldx, Y, ldy, d_status,
    #            workspace, ws_bytes, stream)
    assert L.spm_csc_mm(-1, 5, 0, null, null, null, 0, 0, 4, null, 4, null, 4, null, null, 0, null) == 1
    assert L.spm_csc_mm(5, 5, 0, null, null, null, 0, 2, 4, null, 4, null, 4, null, null, 0, null) == 1
    # A X needs a status word and the workspace; k = 0 or an empty output launches nothing
    sz = ctypes.c_size_t(0)
    assert L.spm_csc_mm_workspace(5, 6, 7, 0, 1, ctypes.byref(sz)) == 0 and sz.value == 0
    assert L.spm_csc_mm_workspace(5, 6, 7, 0, 0, ctypes.byref(sz)) == 0 and sz.value > 7 * 4
    assert L.spm_csc_mm_workspace(5, 6, 7, 0, 3, ctypes.byref(sz)) == 1
    assert L.spm_csc_mm(5, 6, 7, 8, 8, 8, 0, 0, 4, 8, 4, 8, 4, null, 8, sz.value, null) == 1
    assert L.spm_csc_mm(5, 6, 7, 8, 8, 8, 0, 0, 4, 8, 4, 8, 4, 8, null, 0, null) == 3
    assert L.spm_csc_mm(5, 6, 7, 8, 8, 8, 0, 0, 4, 8, 4, 8, 4, 8, 8, sz.value - 1, null) == 3
    assert L.spm_csc_mm(5, 6, 7, null, null, null, 0, 1, 0, null, 0, null, 0, null, null, 0, null) == 0
    # spm_csc_transpose(n_rows, n_cols, nnz, col_ptr, row_idx, vals, dtype, t_col_ptr, t_row_idx, t_vals,
    #                   d_status, workspace, ws_bytes, stream)
    assert L.spm_csc_transpose_workspace(5, 6, -1, 0, ctypes.byref(sz)) == 1
    assert L.spm_csc_transpose_workspace(5, 6, 7, 2, ctypes.byref(sz)) == 1
    assert L.spm_csc_transpose_workspace(5, 6, 7, 1, ctypes.byref(sz)) == 0 and sz.value >= 7 * 4
    assert L.spm_csc_transpose(5, 6, 7, 8, 8, 8, 1, 8, 8, 8, null, 8, sz.value, null) == 1
    assert L.spm_csc_transpose(5, 6, 7, 8, null, 8, 1, 8, 8, 8, 8, 8, sz.value, null) == 1
    assert L.spm_csc_transpose(5, 6, 7, 8, 8, 8, 1, 8, 8, 8, 8, 8, sz.value - 1, null) == 3
    assert L.spm_triplet_dvals(-3, null, null, null, 0, 4, null, 4, null, 4, null, null) == 1
    assert L.spm_triplet_dvals(0, null, null, null, 0, 4, null, 4, null, 4, null, null) == 0
    del args


def test_tuning_roundtrip(spm):
    t0 = spm.spm_get_tuning()
    try:
        assert t0["ordered_path"] == 1
        t = spm.spm_set_tuning(bucket_target=2048, sub_bits=10, partition_threads=512, resolve_threads=512,
                               two_pass_min_writes=0, two_pass_min_fronts=7, ordered_path=0)
        assert t == {"bucket_target": 2048, "sub_bits": 10, "partition_threads": 512, "resolve_threads": 512,
                     "two_pass_min_writes": 0, "two_pass_min_fronts": 7, "ordered_path": 0}
        with pytest.raises(spm.SpmError):
            spm.spm_set_tuning(ordered_path=2)
        with pytest.raises(spm.SpmError):
            spm.spm_set_tuning(bucket_target=100)
        with pytest.raises(spm.SpmError):
            spm.spm_set_tuning(two_pass_min_writes=-1)
        with pytest.raises(spm.SpmError):
            spm.spm_set_tuning(resolve_threads=768)
    finally:
        spm.spm_set_tuning(reset=True)
    assert spm.spm_get_tuning() == t0


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1805_03380_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), fn
                assert "spm_oracle" not in text, fn
    for fn in os.listdir(os.path.join(ROOT, "oracle")):
        if fn.endswith((".py", ".cpp")):
            text = open(os.path.join(ROOT, "oracle", fn)).read()
            assert not re.search(r"^\s*(import|from)\s+paper_1805_03380_gb300\b", text, re.M), fn
            assert not re.search(r"#\s*include\s*[<\"]spm\.h", text), fn
            assert "libspm.so" not in text, fn


def test_update_trace_lookup_coo_host_checks(spm):
    """Workspace sizes and argument checks of the update, trace, lookup and
    COO entry points (all return before anything is launched)."""
    import torch
    m, nnz_a, n = 1_000_000, 5_000_000, 100_000
    asm = spm.spm_assemble_csc_workspace(n, n, m, torch.float64, "sum")
    upd = spm.spm_csc_update_workspace(n, n, nnz_a, m, torch.float64, "sum")
    # the resolved writes (col_ptr, rows, values), one cut and one state per 2047 merged elements,
    # then the assembly's own workspace
    assert asm + 12 * m + 8 * (n + 1) < upd < asm + 12 * m + 8 * (n + 1) + 41 * (nnz_a + m) // 2047 + 4096
    assert spm.spm_csc_update_workspace(n, n, 2 * nnz_a, m, torch.float64, "sum") > upd
    for bad in (dict(nnz_a=-1), dict(m=-1)):
        args = dict(n_rows=n, n_cols=n, nnz_a=nnz_a, m=m, dtype=torch.float64, mode="sum")
        args.update(bad)
        with pytest.raises(spm.SpmError):
            spm.spm_csc_update_workspace(**args)
    with pytest.raises(spm.SpmError, match="INVALID_ARG"):
        spm.spm_csc_update_workspace(n, n, nnz_a, m, torch.float64, "set", spm.KEEP_MAP)
    tr = spm.spm_csc_trace_atb_workspace(n, nnz_a, nnz_a)
    assert 40 * (2 * nnz_a) // 2047 <= tr < 40 * (2 * nnz_a) // 2047 + 4096
    with pytest.raises(spm.SpmError):
        spm.spm_csc_trace_atb_workspace(-1, 0, 0)
    L = spm.lib()
    null = None
    # NULL pointers and negative sizes are refused on the host
    assert L.spm_csc_update(n, n, null, null, null, 0, 0, null, null, null, null, 1, 1, 0, null, null, null, null,
                            null, null, 0, null) == 1
    assert L.spm_csc_trace_atb(n, n, null, null, null, 0, null, null, null, 0, 1, null, null, null, 0, null) == 1
    assert L.spm_csc_lookup(-1, n, 0, null, null, null, 1, 0, null, null, null, null, null, null) == 1
    assert L.spm_csc_lookup(n, n, 0, null, null, null, 1, 0, null, null, null, null, null, null) == 1
    assert L.spm_csc_to_coo(-1, 0, null, null, null, 1, null, null, null, null, null) == 1
    assert L.spm_csc_to_coo(n, 0, null, null, null, 1, null, null, null, null, null) == 1
