"""GB300-native sync step of the hybrid sparse matrix class (arXiv 1805.03380).

An unordered stream of element writes (row, col, value[, seq]) becomes a
canonical CSC matrix (Section 3.1 of the paper), resolving repeated writes as
element setting (last write wins, Table 1 ``X(1,2) = 3``) or as batch insertion
with accumulation (``X(3,4) += 4.56``, Fig. 2).

This module is the thin Python binding of ``libspm.so`` (C ABI declared in
``include/spm.h``): it only checks and marshals torch tensors (device memory
and streams) into the C calls; every step of the computation runs in the
library's CUDA kernels.  There is no CPU fallback: if the library is missing
or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from collections import namedtuple

import torch

__all__ = [
    "SpmError", "lib", "spm_assemble_csc", "spm_assemble_csc_workspace", "spm_assemble_csc_batched",
    "spm_assemble_csc_batched_workspace", "spm_csc_mm", "spm_triplet_dvals", "spm_set_tuning", "spm_get_tuning",
    "spm_csc_update", "spm_csc_update_workspace", "spm_csc_lookup", "spm_csc_to_coo", "csc_lookup", "csc_to_coo", "csc_transpose",
    "spm_csc_transpose", "spm_csc_transpose_workspace", "spm_csc_mm_workspace",
    "spm_csc_trace_atb", "spm_csc_trace_atb_workspace", "csc_trace_atb",
    "assemble_csc", "assemble_csc_batched", "csc_update", "csc_mm", "triplet_dvals", "AssembleMM", "Assembler",
    "BatchedAssembler", "CSC",
    "MODE_LAST_WRITE", "MODE_SUM", "KEEP_MAP", "SEQ_EXPLICIT", "LIB_PATH",
]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libspm.so")

SPM_OK = 0
STATUS_NAMES = {0: "SPM_OK", 1: "SPM_ERR_INVALID_ARG", 2: "SPM_ERR_INDEX_OUT_OF_RANGE",
                3: "SPM_ERR_WORKSPACE_TOO_SMALL", 4: "SPM_ERR_UNSUPPORTED", 5: "SPM_ERR_CUDA", 6: "SPM_ERR_TIMEOUT"}
MODE_LAST_WRITE, MODE_SUM = 0, 1
F32, F64 = 0, 1
KEEP_MAP, CHECK_BOUNDS, SEQ_EXPLICIT = 1, 2, 4

EXPORTED = ["spm_status_string", "spm_version", "spm_assemble_csc_workspace", "spm_assemble_csc",
            "spm_assemble_csc_batched_workspace", "spm_assemble_csc_batched", "spm_csc_mm", "spm_triplet_dvals",
            "spm_set_tuning", "spm_get_tuning", "spm_debug_withhold_publication", "spm_debug_stage_timing",
            "spm_debug_stage_times", "spm_debug_launch_count", "spm_debug_plan_stats", "spm_assemble_csc_static",
            "spm_csc_update_workspace", "spm_csc_update", "spm_csc_lookup", "spm_csc_to_coo",
            "spm_csc_trace_atb_workspace", "spm_csc_trace_atb", "spm_csc_transpose_workspace", "spm_csc_transpose",
            "spm_csc_mm_workspace"]


class SpmError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = int(code)
        super().__init__(f"{where}: {STATUS_NAMES.get(self.code, self.code)}")


class _Tuning(ctypes.Structure):
    _fields_ = [("bucket_target", ctypes.c_int32), ("sub_bits", ctypes.c_int32),
                ("partition_threads", ctypes.c_int32), ("resolve_threads", ctypes.c_int32),
                ("two_pass_min_writes", ctypes.c_int32), ("two_pass_min_fronts", ctypes.c_int32),
                ("ordered_path", ctypes.c_int32)]


_lib = None


def lib():
    """Load libspm.so (built in-tree by __graft_entry__.build()); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    p, i64, i32, u32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_size_t
    L.spm_status_string.argtypes = [ctypes.c_int]
    L.spm_status_string.restype = ctypes.c_char_p
    L.spm_version.restype = i32
    L.spm_assemble_csc_workspace.argtypes = [i64, i64, i64, ctypes.c_int, ctypes.c_int, u32, ctypes.POINTER(sz)]
    L.spm_assemble_csc.argtypes = [i64, i64, i64, p, p, p, p, ctypes.c_int, ctypes.c_int, u32, p, p, p, p, p, p, p,
                                   sz, p]
    L.spm_assemble_csc_batched_workspace.argtypes = [i64, p, p, p, ctypes.c_int, ctypes.c_int, u32,
                                                     ctypes.POINTER(sz)]
    L.spm_assemble_csc_batched.argtypes = [i64, p, p, p, p, p, p, p, p, p, p, ctypes.c_int, ctypes.c_int, u32, p, p,
                                           p, p, p, p, p, sz, p]
    L.spm_assemble_csc_static.argtypes = [i64, i64, i64, p, p, p, p, ctypes.c_int, ctypes.c_int, u32, p, p, p, p, p,
                                          p, p]
    L.spm_csc_update_workspace.argtypes = [i64, i64, i64, i64, ctypes.c_int, ctypes.c_int, u32, ctypes.POINTER(sz)]
    L.spm_csc_update.argtypes = [i64, i64, p, p, p, i64, i64, p, p, p, p, ctypes.c_int, ctypes.c_int, u32, p, p, p,
                                 p, p, p, sz, p]
    L.spm_csc_lookup.argtypes = [i64, i64, i64, p, p, p, ctypes.c_int, i64, p, p, p, p, p, p]
    L.spm_csc_to_coo.argtypes = [i64, i64, p, p, p, ctypes.c_int, p, p, p, p, p]
    L.spm_csc_trace_atb_workspace.argtypes = [i64, i64, i64, ctypes.POINTER(sz)]
    L.spm_csc_trace_atb.argtypes = [i64, i64, p, p, p, i64, p, p, p, i64, ctypes.c_int, p, p, p, sz, p]
    L.spm_csc_transpose_workspace.argtypes = [i64, i64, i64, ctypes.c_int, ctypes.POINTER(sz)]
    L.spm_csc_transpose.argtypes = [i64, i64, i64, p, p, p, ctypes.c_int, p, p, p, p, p, sz, p]
    L.spm_csc_mm_workspace.argtypes = [i64, i64, i64, ctypes.c_int, i32, ctypes.POINTER(sz)]
    L.spm_csc_mm.argtypes = [i64, i64, i64, p, p, p, ctypes.c_int, i32, i64, p, i64, p, i64, p, p, sz, p]
    L.spm_triplet_dvals.argtypes = [i64, p, p, p, ctypes.c_int, i64, p, i64, p, i64, p, p]
    L.spm_set_tuning.argtypes = [ctypes.POINTER(_Tuning)]
    L.spm_get_tuning.argtypes = [ctypes.POINTER(_Tuning)]
    L.spm_debug_withhold_publication.argtypes = [i64]
    L.spm_debug_stage_timing.argtypes = [i32]
    L.spm_debug_stage_times.argtypes = [i32, ctypes.POINTER(ctypes.c_float), i32]
    L.spm_debug_launch_count.argtypes = []
    L.spm_debug_plan_stats.argtypes = [p, sz, i64, i64, i64, ctypes.c_int, ctypes.c_int, u32,
                                       ctypes.POINTER(ctypes.c_int64), i32]
    for name in EXPORTED:
        if name not in ("spm_status_string", "spm_version", "spm_debug_launch_count"):
            getattr(L, name).restype = ctypes.c_int
    L.spm_debug_launch_count.restype = i64
    _lib = L
    return L


def _check(code, where):
    if code != SPM_OK:
        raise SpmError(code, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_code(dt):
    if dt == torch.float32:
        return F32
    if dt == torch.float64:
        return F64
    raise TypeError(f"values must be float32 or float64, got {dt}")


def _mode_code(mode):
    if mode in ("set", "last_write", MODE_LAST_WRITE):
        return MODE_LAST_WRITE
    if mode in ("sum", "add", MODE_SUM):
        return MODE_SUM
    raise ValueError(f"mode must be 'set' or 'sum', got {mode!r}")


# ------------------------------------------------------------------------------------------
# One-to-one wrappers of the C entry points (torch tensors in, status checked)
# ------------------------------------------------------------------------------------------
def spm_assemble_csc_workspace(n_rows, n_cols, m, dtype, mode, flags=0):
    out = ctypes.c_size_t(0)
    _check(lib().spm_assemble_csc_workspace(int(n_rows), int(n_cols), int(m), _dtype_code(dtype), _mode_code(mode),
                                            int(flags), ctypes.byref(out)), "spm_assemble_csc_workspace")
    return int(out.value)


def spm_assemble_csc(n_rows, n_cols, rows, cols, vals, seq, mode, flags, col_ptr, row_idx, out_vals, d_nnz, map,
                     d_status, workspace, stream=None):
    m = rows.numel()
    code = lib().spm_assemble_csc(int(n_rows), int(n_cols), int(m), _ptr(rows), _ptr(cols), _ptr(vals), _ptr(seq),
                                  _dtype_code(vals.dtype), _mode_code(mode), int(flags), _ptr(col_ptr),
                                  _ptr(row_idx), _ptr(out_vals), _ptr(d_nnz), _ptr(map), _ptr(d_status),
                                  _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream))
    _check(code, "spm_assemble_csc")


def spm_assemble_csc_static(n_rows, n_cols, rows, cols, vals, seq, mode, flags, col_ptr, row_idx, out_vals, d_nnz,
                            map, d_status, stream=None):
    """spm_assemble_csc without a workspace: the library's built-in 32 MiB
    device scratch array is used instead (for callers that cannot allocate)."""
    code = lib().spm_assemble_csc_static(int(n_rows), int(n_cols), rows.numel(), _ptr(rows), _ptr(cols), _ptr(vals),
                                         _ptr(seq), _dtype_code(vals.dtype), _mode_code(mode), int(flags),
                                         _ptr(col_ptr), _ptr(row_idx), _ptr(out_vals), _ptr(d_nnz), _ptr(map),
                                         _ptr(d_status), _stream(stream))
    _check(code, "spm_assemble_csc_static")


def spm_csc_update_workspace(n_rows, n_cols, nnz_a, m, dtype, mode, flags=0):
    out = ctypes.c_size_t(0)
    _check(lib().spm_csc_update_workspace(int(n_rows), int(n_cols), int(nnz_a), int(m), _dtype_code(dtype),
                                          _mode_code(mode), int(flags), ctypes.byref(out)), "spm_csc_update_workspace")
    return int(out.value)


def spm_csc_update(n_rows, n_cols, a_col_ptr, a_row_idx, a_vals, rows, cols, vals, seq, mode, flags, col_ptr, row_idx,
                   out_vals, d_nnz, d_status, workspace, stream=None):
    """Existing CSC A (a_col_ptr, a_row_idx, a_vals) updated by the writes
    (rows, cols, vals[, seq]); outputs as for spm_assemble_csc."""
    code = lib().spm_csc_update(int(n_rows), int(n_cols), _ptr(a_col_ptr), _ptr(a_row_idx), _ptr(a_vals),
                                a_row_idx.numel(), rows.numel(), _ptr(rows), _ptr(cols), _ptr(vals), _ptr(seq),
                                _dtype_code(vals.dtype), _mode_code(mode), int(flags), _ptr(col_ptr), _ptr(row_idx),
                                _ptr(out_vals), _ptr(d_nnz), _ptr(d_status), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream(stream))
    _check(code, "spm_csc_update")


def spm_csc_lookup(n_rows, n_cols, col_ptr, row_idx, vals, q_rows, q_cols, out_vals, out_pos, d_status,
                   stream=None):
    """Values of the elements (q_rows[i], q_cols[i]) of a CSC matrix (0 where not stored)."""
    code = lib().spm_csc_lookup(int(n_rows), int(n_cols), row_idx.numel(), _ptr(col_ptr), _ptr(row_idx), _ptr(vals),
                                _dtype_code(vals.dtype), q_rows.numel(), _ptr(q_rows), _ptr(q_cols), _ptr(out_vals),
                                _ptr(out_pos), _ptr(d_status), _stream(stream))
    _check(code, "spm_csc_lookup")


def spm_csc_to_coo(n_cols, col_ptr, row_idx, vals, out_rows, out_cols, out_vals, d_status, stream=None):
    """Column of every stored element (and copies of rows and values when given)."""
    code = lib().spm_csc_to_coo(int(n_cols), row_idx.numel(), _ptr(col_ptr), _ptr(row_idx), _ptr(vals),
                                _dtype_code(vals.dtype), _ptr(out_rows), _ptr(out_cols), _ptr(out_vals),
                                _ptr(d_status), _stream(stream))
    _check(code, "spm_csc_to_coo")


def spm_csc_trace_atb_workspace(n_cols, nnz_a, nnz_b):
    out = ctypes.c_size_t(0)
    _check(lib().spm_csc_trace_atb_workspace(int(n_cols), int(nnz_a), int(nnz_b), ctypes.byref(out)),
           "spm_csc_trace_atb_workspace")
    return int(out.value)


def spm_csc_trace_atb(n_rows, n_cols, a_col_ptr, a_row_idx, a_vals, b_col_ptr, b_row_idx, b_vals, d_result, d_status,
                      workspace, stream=None):
    """trace(A^T B) of two CSC matrices into the device double d_result."""
    if a_vals.dtype != b_vals.dtype:
        raise TypeError("A and B must have the same value type")
    code = lib().spm_csc_trace_atb(int(n_rows), int(n_cols), _ptr(a_col_ptr), _ptr(a_row_idx), _ptr(a_vals),
                                   a_row_idx.numel(), _ptr(b_col_ptr), _ptr(b_row_idx), _ptr(b_vals),
                                   b_row_idx.numel(), _dtype_code(a_vals.dtype), _ptr(d_result), _ptr(d_status),
                                   _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream))
    _check(code, "spm_csc_trace_atb")


def _host_i64(a):
    return torch.as_tensor(a, dtype=torch.int64).contiguous().cpu()


def spm_assemble_csc_batched_workspace(n_rows, n_cols, trip_ptr, dtype, mode, flags=0):
    hr, hc, ht = _host_i64(n_rows), _host_i64(n_cols), _host_i64(trip_ptr)
    out = ctypes.c_size_t(0)
    _check(lib().spm_assemble_csc_batched_workspace(hr.numel(), _ptr(hr), _ptr(hc), _ptr(ht), _dtype_code(dtype),
                                                    _mode_code(mode), int(flags), ctypes.byref(out)),
           "spm_assemble_csc_batched_workspace")
    return int(out.value)


def spm_assemble_csc_batched(h_n_rows, h_n_cols, h_trip_ptr, d_n_rows, d_n_cols, d_trip_ptr, rows, cols, vals, seq,
                             mode, flags, col_ptr, row_idx, out_vals, d_nnz, map, d_status, workspace, stream=None):
    code = lib().spm_assemble_csc_batched(
        h_n_rows.numel(), _ptr(h_n_rows), _ptr(h_n_cols), _ptr(h_trip_ptr), _ptr(d_n_rows), _ptr(d_n_cols),
        _ptr(d_trip_ptr), _ptr(rows), _ptr(cols), _ptr(vals), _ptr(seq), _dtype_code(vals.dtype), _mode_code(mode),
        int(flags), _ptr(col_ptr), _ptr(row_idx), _ptr(out_vals), _ptr(d_nnz), _ptr(map), _ptr(d_status),
        _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream))
    _check(code, "spm_assemble_csc_batched")


def spm_csc_transpose_workspace(n_rows, n_cols, nnz, dtype):
    out = ctypes.c_size_t(0)
    _check(lib().spm_csc_transpose_workspace(int(n_rows), int(n_cols), int(nnz), _dtype_code(dtype), ctypes.byref(out)),
           "spm_csc_transpose_workspace")
    return int(out.value)


def spm_csc_transpose(n_rows, n_cols, col_ptr, row_idx, vals, t_col_ptr, t_row_idx, t_vals, d_status, workspace,
                      stream=None):
    code = lib().spm_csc_transpose(int(n_rows), int(n_cols), row_idx.numel(), _ptr(col_ptr), _ptr(row_idx),
                                   _ptr(vals), _dtype_code(vals.dtype), _ptr(t_col_ptr), _ptr(t_row_idx),
                                   _ptr(t_vals), _ptr(d_status), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), _stream(stream))
    _check(code, "spm_csc_transpose")


def spm_csc_mm_workspace(n_rows, n_cols, nnz, dtype, transpose):
    out = ctypes.c_size_t(0)
    _check(lib().spm_csc_mm_workspace(int(n_rows), int(n_cols), int(nnz), _dtype_code(dtype), int(bool(transpose)),
                                      ctypes.byref(out)), "spm_csc_mm_workspace")
    return int(out.value)


def spm_csc_mm(n_rows, n_cols, col_ptr, row_idx, vals, transpose, X, Y, d_status=None, workspace=None, stream=None):
    k = X.shape[1]
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    code = lib().spm_csc_mm(int(n_rows), int(n_cols), row_idx.numel(), _ptr(col_ptr), _ptr(row_idx), _ptr(vals),
                            _dtype_code(vals.dtype), int(bool(transpose)), int(k), _ptr(X), X.stride(0), _ptr(Y),
                            Y.stride(0), _ptr(d_status), _ptr(workspace), ws_bytes, _stream(stream))
    _check(code, "spm_csc_mm")


def spm_triplet_dvals(rows, cols, map, dY, X, dvals, stream=None):
    code = lib().spm_triplet_dvals(rows.numel(), _ptr(rows), _ptr(cols), _ptr(map), _dtype_code(dY.dtype),
                                   int(X.shape[1]), _ptr(dY), dY.stride(0), _ptr(X), X.stride(0), _ptr(dvals),
                                   _stream(stream))
    _check(code, "spm_triplet_dvals")


def spm_set_tuning(bucket_target=None, sub_bits=None, partition_threads=None, resolve_threads=None,
                   two_pass_min_writes=None, two_pass_min_fronts=None, ordered_path=None, reset=False):
    """Set the process-wide tuning (fields left as None keep their value); returns the new tuning."""
    if reset:
        _check(lib().spm_set_tuning(None), "spm_set_tuning")
        return spm_get_tuning()
    cur = spm_get_tuning()
    new = dict(bucket_target=bucket_target, sub_bits=sub_bits, partition_threads=partition_threads,
               resolve_threads=resolve_threads, two_pass_min_writes=two_pass_min_writes,
               two_pass_min_fronts=two_pass_min_fronts, ordered_path=ordered_path)
    t = _Tuning(*[cur[f] if new[f] is None else int(new[f]) for f, _ in _Tuning._fields_])
    _check(lib().spm_set_tuning(ctypes.byref(t)), "spm_set_tuning")
    return spm_get_tuning()


def spm_debug_withhold_publication(bucket):
    """Test-only fault injection (see include/spm.h); -1 switches it off."""
    _check(lib().spm_debug_withhold_publication(int(bucket)), "spm_debug_withhold_publication")


STAGES = ("plan", "hist", "offsets", "partition", "resolve", "place")


def spm_debug_stage_timing(enable):
    """Record CUDA events at the stage boundaries of later assembly calls."""
    _check(lib().spm_debug_stage_timing(1 if enable else 0), "spm_debug_stage_timing")


def spm_debug_stage_times(back=0):
    """Stage durations (ms) of the assembly call made `back` calls ago (stream must be complete)."""
    arr = (ctypes.c_float * len(STAGES))()
    _check(lib().spm_debug_stage_times(int(back), arr, len(STAGES)), "spm_debug_stage_times")
    return dict(zip(STAGES, [float(x) for x in arr]))


def spm_debug_launch_count():
    """Kernels launched by the library so far in this process."""
    return int(lib().spm_debug_launch_count())


def spm_debug_plan_stats(asm):
    """Bucket-plan statistics of the last call of an Assembler (synchronous)."""
    out = (ctypes.c_int64 * 8)()
    _check(lib().spm_debug_plan_stats(_ptr(asm.workspace), asm.workspace.numel(), asm.n_rows, asm.n_cols, asm.m,
                                      _dtype_code(asm.dtype), _mode_code(asm.mode), asm.flags, out, 8),
           "spm_debug_plan_stats")
    keys = ("buckets", "largest", "over_capacity", "writes_over_capacity", "capacity", "l2_tables", "bucket_bound",
            "ordered_pass")
    return dict(zip(keys, [int(x) for x in out]))


def spm_get_tuning():
    t = _Tuning()
    _check(lib().spm_get_tuning(ctypes.byref(t)), "spm_get_tuning")
    return {f: getattr(t, f) for f, _ in _Tuning._fields_}


# ------------------------------------------------------------------------------------------
# Convenience layer
# ------------------------------------------------------------------------------------------
CSC = namedtuple("CSC", "col_ptr row_idx vals nnz map shape")


def _as_index(t, device):
    t = torch.as_tensor(t, device=device)
    if t.dtype != torch.int32:
        t = t.to(torch.int32)
    return t.contiguous()


def _raise_status(d_status, where):
    code = int(d_status.item())
    if code != SPM_OK:
        raise SpmError(code, where)


class Assembler:
    """Reusable single-matrix assembly with its own workspace and output buffers.

    ``run()`` only enqueues the kernels (no host synchronisation), so it can
    be timed with CUDA events or captured in a CUDA graph; ``result()``
    synchronises, checks the device status and returns the CSC.
    """

    def __init__(self, shape, m, dtype=torch.float64, mode="sum", seq=False, keep_map=False, device="cuda"):
        self.n_rows, self.n_cols = int(shape[0]), int(shape[1])
        self.m = int(m)
        self.dtype = dtype
        self.mode = mode
        self.flags = (SEQ_EXPLICIT if seq else 0) | (KEEP_MAP if keep_map else 0)
        dev = torch.device(device)
        self.device = dev
        ws = spm_assemble_csc_workspace(self.n_rows, self.n_cols, self.m, dtype, mode, self.flags)
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=dev)
        self.col_ptr = torch.empty(self.n_cols + 1, dtype=torch.int64, device=dev)
        self.row_idx = torch.empty(max(self.m, 1), dtype=torch.int32, device=dev)
        self.out_vals = torch.empty(max(self.m, 1), dtype=dtype, device=dev)
        self.d_nnz = torch.zeros(1, dtype=torch.int64, device=dev)
        self.d_status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.map = torch.empty(max(self.m, 1), dtype=torch.int32, device=dev) if keep_map else None

    def run(self, rows, cols, vals, seq=None, stream=None):
        if rows.numel() != self.m:
            raise ValueError("stream length differs from the one the Assembler was built for")
        spm_assemble_csc(self.n_rows, self.n_cols, rows, cols, vals, seq, self.mode, self.flags, self.col_ptr,
                         self.row_idx, self.out_vals, self.d_nnz, self.map, self.d_status, self.workspace, stream)

    def result(self):
        torch.cuda.current_stream().synchronize()
        _raise_status(self.d_status, "spm_assemble_csc")
        nnz = int(self.d_nnz.item())
        return CSC(self.col_ptr, self.row_idx[:nnz], self.out_vals[:nnz], nnz,
                   self.map[:self.m] if self.map is not None else None, (self.n_rows, self.n_cols))


class BatchedAssembler:
    """Reusable batched assembly (many independent matrices, one call) with its
    own size tables, workspace and output buffers, for a fixed batch layout:
    matrix i has shape (n_rows[i], n_cols[i]) and its writes at
    [trip_ptr[i], trip_ptr[i+1]) of the concatenated streams.

    ``run()`` only enqueues the kernels (capturable in a CUDA graph; replays
    may change the writes but not the layout); ``result()`` synchronises,
    checks the device status and returns (col_ptr, row_idx, vals, nnz, map)
    as assemble_csc_batched does.
    """

    def __init__(self, n_rows, n_cols, trip_ptr, dtype=torch.float64, mode="set", seq=False, keep_map=False,
                 device="cuda"):
        dev = torch.device(device)
        self.device = dev
        self.h_n_rows, self.h_n_cols, self.h_trip_ptr = _host_i64(n_rows), _host_i64(n_cols), _host_i64(trip_ptr)
        if self.h_trip_ptr.numel() != self.h_n_rows.numel() + 1 or self.h_n_cols.numel() != self.h_n_rows.numel():
            raise ValueError("n_rows and n_cols need one entry per matrix and trip_ptr one more")
        self.d_n_rows, self.d_n_cols, self.d_trip_ptr = (t.to(dev) for t in (self.h_n_rows, self.h_n_cols,
                                                                              self.h_trip_ptr))
        self.B = self.h_n_rows.numel()
        self.m = int(self.h_trip_ptr[-1]) if self.B else 0
        self.dtype, self.mode = dtype, mode
        self.flags = (SEQ_EXPLICIT if seq else 0) | (KEEP_MAP if keep_map else 0)
        ws = spm_assemble_csc_batched_workspace(self.h_n_rows, self.h_n_cols, self.h_trip_ptr, dtype, mode,
                                                self.flags)
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=dev)
        self.col_ptr = torch.empty(int((self.h_n_cols + 1).sum()), dtype=torch.int64, device=dev)
        self.row_idx = torch.empty(max(self.m, 1), dtype=torch.int32, device=dev)
        self.out_vals = torch.empty(max(self.m, 1), dtype=dtype, device=dev)
        self.d_nnz = torch.zeros(max(self.B, 1), dtype=torch.int64, device=dev)
        self.d_status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.map = torch.empty(max(self.m, 1), dtype=torch.int32, device=dev) if keep_map else None

    def run(self, rows, cols, vals, seq=None, stream=None):
        if rows.numel() != self.m:
            raise ValueError("stream length differs from the batch layout")
        spm_assemble_csc_batched(self.h_n_rows, self.h_n_cols, self.h_trip_ptr, self.d_n_rows, self.d_n_cols,
                                 self.d_trip_ptr, rows, cols, vals, seq, self.mode, self.flags, self.col_ptr,
                                 self.row_idx, self.out_vals, self.d_nnz, self.map, self.d_status, self.workspace,
                                 stream)

    def result(self):
        torch.cuda.current_stream().synchronize()
        _raise_status(self.d_status, "spm_assemble_csc_batched")
        return (self.col_ptr, self.row_idx[:self.m], self.out_vals[:self.m], self.d_nnz[:self.B],
                self.map[:self.m] if self.map is not None else None)


def assemble_csc(rows, cols, vals, shape, mode="set", seq=None, keep_map=False, stream=None):
    """Canonical CSC of the matrix the element writes produce (device tensors in and out)."""
    vals = torch.as_tensor(vals)
    if not vals.is_cuda:
        raise ValueError("vals must be a CUDA tensor")
    dev = vals.device
    rows = _as_index(rows, dev)
    cols = _as_index(cols, dev)
    vals = vals.contiguous()
    if seq is not None:
        seq = torch.as_tensor(seq, device=dev)
        if seq.dtype != torch.int64:
            seq = seq.to(torch.int64)
        seq = seq.contiguous()
    if not (rows.numel() == cols.numel() == vals.numel()) or (seq is not None and seq.numel() != rows.numel()):
        raise ValueError("rows, cols, vals (and seq) must have the same length")
    a = Assembler(shape, rows.numel(), vals.dtype, mode, seq is not None, keep_map, dev)
    a.run(rows, cols, vals, seq, stream)
    return a.result()


def csc_update(a, rows, cols, vals, mode="set", seq=None, stream=None):
    """The CSC ``a`` (a CSC tuple, or (col_ptr, row_idx, vals, shape)) after the
    element writes (rows, cols, vals[, seq]); a new CSC, ``a`` is not modified."""
    a_cp, a_ri, a_v, shape = _csc_parts(a)
    n_rows, n_cols = int(shape[0]), int(shape[1])
    vals = torch.as_tensor(vals)
    if not vals.is_cuda:
        raise ValueError("vals must be a CUDA tensor")
    dev = vals.device
    if a_v.dtype != vals.dtype:
        raise TypeError("the matrix and the writes must have the same value type")
    a_cp = torch.as_tensor(a_cp, device=dev).to(torch.int64).contiguous()
    a_ri = _as_index(a_ri, dev)
    a_v = a_v.contiguous()
    rows, cols, vals = _as_index(rows, dev), _as_index(cols, dev), vals.contiguous()
    if seq is not None:
        seq = torch.as_tensor(seq, device=dev).to(torch.int64).contiguous()
    if a_cp.numel() != n_cols + 1 or a_ri.numel() != a_v.numel():
        raise ValueError("col_ptr must have n_cols + 1 entries and row_idx/vals the same length")
    if not (rows.numel() == cols.numel() == vals.numel()) or (seq is not None and seq.numel() != rows.numel()):
        raise ValueError("rows, cols, vals (and seq) must have the same length")
    flags = SEQ_EXPLICIT if seq is not None else 0
    cap = max(a_ri.numel() + rows.numel(), 1)
    ws = spm_csc_update_workspace(n_rows, n_cols, a_ri.numel(), rows.numel(), vals.dtype, mode, flags)
    workspace = torch.empty(ws, dtype=torch.uint8, device=dev)
    col_ptr = torch.empty(n_cols + 1, dtype=torch.int64, device=dev)
    row_idx = torch.empty(cap, dtype=torch.int32, device=dev)
    out_vals = torch.empty(cap, dtype=vals.dtype, device=dev)
    d_nnz = torch.zeros(1, dtype=torch.int64, device=dev)
    d_status = torch.zeros(1, dtype=torch.int32, device=dev)
    spm_csc_update(n_rows, n_cols, a_cp, a_ri, a_v, rows, cols, vals, seq, mode, flags, col_ptr, row_idx, out_vals,
                   d_nnz, d_status, workspace, stream)
    (stream if stream is not None else torch.cuda.current_stream()).synchronize()
    _raise_status(d_status, "spm_csc_update")
    nnz = int(d_nnz.item())
    return CSC(col_ptr, row_idx[:nnz], out_vals[:nnz], nnz, None, (n_rows, n_cols))


def _csc_parts(a):
    if isinstance(a, CSC):
        return a.col_ptr, a.row_idx, a.vals, a.shape
    return a


def csc_lookup(a, rows, cols, stream=None):
    """Values (0 where not stored) and positions (-1 where not stored) of the
    elements (rows[i], cols[i]) of the CSC ``a`` (a CSC tuple, or
    (col_ptr, row_idx, vals, shape))."""
    cp, ri, v, shape = _csc_parts(a)
    dev = v.device
    rows, cols = _as_index(rows, dev), _as_index(cols, dev)
    if rows.numel() != cols.numel():
        raise ValueError("rows and cols must have the same length")
    cp = torch.as_tensor(cp, device=dev).to(torch.int64).contiguous()
    ri, v = _as_index(ri, dev), v.contiguous()
    out = torch.empty(rows.numel(), dtype=v.dtype, device=dev)
    pos = torch.empty(rows.numel(), dtype=torch.int64, device=dev)
    d_status = torch.zeros(1, dtype=torch.int32, device=dev)
    spm_csc_lookup(shape[0], shape[1], cp, ri, v, rows, cols, out, pos, d_status, stream)
    (stream if stream is not None else torch.cuda.current_stream()).synchronize()
    _raise_status(d_status, "spm_csc_lookup")
    return out, pos


def csc_trace_atb(a, b, stream=None):
    """trace(A^T B) (a Python float) of the CSC matrices ``a`` and ``b`` of one shape."""
    acp, ari, av, shape = _csc_parts(a)
    bcp, bri, bv, bshape = _csc_parts(b)
    if tuple(shape) != tuple(bshape):
        raise ValueError("A and B must have the same shape")
    dev = av.device
    acp = torch.as_tensor(acp, device=dev).to(torch.int64).contiguous()
    bcp = torch.as_tensor(bcp, device=dev).to(torch.int64).contiguous()
    ari, bri = _as_index(ari, dev), _as_index(bri, dev)
    av, bv = av.contiguous(), bv.contiguous()
    ws = torch.empty(spm_csc_trace_atb_workspace(shape[1], ari.numel(), bri.numel()), dtype=torch.uint8, device=dev)
    res = torch.zeros(1, dtype=torch.float64, device=dev)
    d_status = torch.zeros(1, dtype=torch.int32, device=dev)
    spm_csc_trace_atb(shape[0], shape[1], acp, ari, av, bcp, bri, bv, res, d_status, ws, stream)
    (stream if stream is not None else torch.cuda.current_stream()).synchronize()
    _raise_status(d_status, "spm_csc_trace_atb")
    return float(res.item())


def csc_to_coo(a, stream=None):
    """Coordinate list (rows, cols, vals) of the CSC ``a``, in column-major order."""
    cp, ri, v, shape = _csc_parts(a)
    dev = v.device
    cp = torch.as_tensor(cp, device=dev).to(torch.int64).contiguous()
    ri, v = _as_index(ri, dev), v.contiguous()
    rows = torch.empty_like(ri)
    cols = torch.empty_like(ri)
    vals = torch.empty_like(v)
    d_status = torch.zeros(1, dtype=torch.int32, device=dev)
    spm_csc_to_coo(shape[1], cp, ri, v, rows, cols, vals, d_status, stream)
    (stream if stream is not None else torch.cuda.current_stream()).synchronize()
    _raise_status(d_status, "spm_csc_to_coo")
    return rows, cols, vals


def assemble_csc_batched(rows, cols, vals, n_rows, n_cols, trip_ptr, mode="set", seq=None, keep_map=False):
    """Batch of independent matrices (concatenated write streams) in one call.

    Returns (col_ptr, row_idx, vals, nnz, map): col_ptr concatenated with
    n_cols_i + 1 entries per matrix; matrix i's elements start at trip_ptr[i].
    """
    vals = torch.as_tensor(vals).contiguous()
    dev = vals.device
    rows = _as_index(rows, dev)
    cols = _as_index(cols, dev)
    hr, hc, ht = _host_i64(n_rows), _host_i64(n_cols), _host_i64(trip_ptr)
    dr, dc, dt = hr.to(dev), hc.to(dev), ht.to(dev)
    if seq is not None:
        seq = torch.as_tensor(seq, device=dev).to(torch.int64).contiguous()
    flags = (SEQ_EXPLICIT if seq is not None else 0) | (KEEP_MAP if keep_map else 0)
    ws = spm_assemble_csc_batched_workspace(hr, hc, ht, vals.dtype, mode, flags)
    workspace = torch.empty(ws, dtype=torch.uint8, device=dev)
    total = int(ht[-1]) if ht.numel() else 0
    col_ptr = torch.empty(int((hc + 1).sum()), dtype=torch.int64, device=dev)
    row_idx = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
    out_vals = torch.empty(max(total, 1), dtype=vals.dtype, device=dev)
    d_nnz = torch.zeros(max(hr.numel(), 1), dtype=torch.int64, device=dev)
    d_status = torch.zeros(1, dtype=torch.int32, device=dev)
    mp = torch.empty(max(total, 1), dtype=torch.int32, device=dev) if keep_map else None
    spm_assemble_csc_batched(hr, hc, ht, dr, dc, dt, rows, cols, vals, seq, mode, flags, col_ptr, row_idx, out_vals,
                             d_nnz, mp, d_status, workspace)
    torch.cuda.current_stream().synchronize()
    _raise_status(d_status, "spm_assemble_csc_batched")
    return col_ptr, row_idx, out_vals, d_nnz[:hr.numel()], (mp[:total] if mp is not None else None)


def csc_mm(col_ptr, row_idx, vals, shape, X, transpose=False, stream=None, check=True):
    """Y = A X (or A^T X) for A in CSC; X row-major (inner stride 1).  Each
    output row is gathered in a fixed order (the same bits on every call).
    With ``check`` the call waits for the stream and raises on a malformed
    matrix; without it nothing synchronises (A must be well formed)."""
    if X.stride(1) != 1:
        X = X.contiguous()
    out_rows = shape[1] if transpose else shape[0]
    Y = torch.empty((out_rows, X.shape[1]), dtype=X.dtype, device=X.device)
    ws_bytes = spm_csc_mm_workspace(shape[0], shape[1], row_idx.numel(), vals.dtype, transpose)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=X.device) if ws_bytes else None
    d_status = torch.zeros(1, dtype=torch.int32, device=X.device) if (check or not transpose) else None
    spm_csc_mm(shape[0], shape[1], col_ptr, row_idx, vals, transpose, X, Y, d_status, ws, stream)
    if check:
        (stream or torch.cuda.current_stream()).synchronize()
        _raise_status(d_status, "spm_csc_mm")
    return Y


def csc_transpose(col_ptr, row_idx, vals, shape, stream=None):
    """The CSC of A^T (shape (n_cols, n_rows)) from the CSC of A: a CSC tuple
    whose row_idx holds A's column indices, increasing inside each column;
    values carried over bit for bit."""
    n_rows, n_cols = int(shape[0]), int(shape[1])
    dev = vals.device
    nnz = row_idx.numel()
    ws = torch.empty(spm_csc_transpose_workspace(n_rows, n_cols, nnz, vals.dtype), dtype=torch.uint8, device=dev)
    t_cp = torch.empty(n_rows + 1, dtype=torch.int64, device=dev)
    t_ri = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
    t_v = torch.empty(max(nnz, 1), dtype=vals.dtype, device=dev)
    d_status = torch.zeros(1, dtype=torch.int32, device=dev)
    spm_csc_transpose(n_rows, n_cols, col_ptr, _as_index(row_idx, dev), vals.contiguous(), t_cp, t_ri, t_v, d_status,
                      ws, stream)
    (stream or torch.cuda.current_stream()).synchronize()
    _raise_status(d_status, "spm_csc_transpose")
    return CSC(t_cp, t_ri[:nnz], t_v[:nnz], nnz, None, (n_cols, n_rows))


def triplet_dvals(rows, cols, map, dY, X, stream=None):
    """dL/dvals for Y = A X assembled from the writes (map: None in sum mode)."""
    if dY.stride(1) != 1:
        dY = dY.contiguous()
    if X.stride(1) != 1:
        X = X.contiguous()
    dvals = torch.empty(rows.numel(), dtype=dY.dtype, device=dY.device)
    spm_triplet_dvals(rows, cols, map, dY, X, dvals, stream)
    return dvals


class AssembleMM(torch.autograd.Function):
    """Y = A(vals) X where A is assembled from the writes (rows, cols, vals).

    backward: dvals[t] = <dY[rows[t]], X[cols[t]]> for every write that feeds
    its element (in set mode only the last write; overwritten writes get 0,
    read from the kept map, or from a re-assembly when ``keep_map`` is False),
    dX = A^T dY.  Both products are gathers in a fixed order: the forward
    walks the columns of A^T (built once by csc_transpose), the backward those
    of A, so every call gives the same bits.
    """

    @staticmethod
    def forward(ctx, rows, cols, vals, shape, X, mode="sum", keep_map=True):
        rows = _as_index(rows, vals.device)
        cols = _as_index(cols, vals.device)
        need_map = _mode_code(mode) == MODE_LAST_WRITE and keep_map
        A = assemble_csc(rows, cols, vals.detach(), shape, mode=mode, keep_map=need_map)
        At = csc_transpose(A.col_ptr, A.row_idx, A.vals, shape)
        Y = csc_mm(At.col_ptr, At.row_idx, At.vals, At.shape, X.detach(), transpose=True, check=False)
        ctx.save_for_backward(rows, cols, vals.detach(), X.detach(), A.col_ptr, A.row_idx, A.vals,
                              A.map if need_map else None)
        ctx.shape, ctx.mode = tuple(shape), mode
        return Y

    @staticmethod
    def backward(ctx, dY):
        rows, cols, vals, X, col_ptr, row_idx, avals, mp = ctx.saved_tensors
        dY = dY.contiguous()
        dvals = dX = None
        if ctx.needs_input_grad[2]:
            if _mode_code(ctx.mode) == MODE_LAST_WRITE and mp is None:
                # the map was not kept: recompute it by assembling again
                mp = assemble_csc(rows, cols, vals, ctx.shape, mode=ctx.mode, keep_map=True).map
            dvals = triplet_dvals(rows, cols, mp if _mode_code(ctx.mode) == MODE_LAST_WRITE else None, dY, X)
        if ctx.needs_input_grad[4]:
            dX = csc_mm(col_ptr, row_idx, avals, ctx.shape, dY, transpose=True, check=False)
        return None, None, dvals, None, dX, None, None
