"""Autotuner for the assembly kernels' tuning parameters (spm_tuning).

For one workload -- a device-resident write stream and its matrix shape,
value type and mode, or a batch of matrices with its layout -- it times
spm_assemble_csc (spm_assemble_csc_batched) under a list of candidate
tunings (CUDA events around each call, after warm-up), keeps only the
candidates whose CSC equals the one the default tuning produces bit for bit
(structure and values: the reduction of an element's writes does not depend
on how the work is split, so every tuning must give the same bytes), and
returns the fastest.  Results are cached in
a JSON file keyed by GPU, sizes, value type and mode: the path given, else
the environment variable SPM_TUNE_CACHE, else no cache.

    best = autotune(rows, cols, vals, shape, "sum")   # tunes, applies, caches
    apply_cached(shape, m, torch.float64, "sum")      # later: reuse the entry

    best = autotune_batched(rows, cols, vals, n_rows, n_cols, trip_ptr, "set")
    apply_cached_batched(n_rows, n_cols, trip_ptr, torch.float32, "set")

A batch is keyed by its matrix count, total writes and a digest of its
layout (n_rows, n_cols, trip_ptr): the same layout with other writes reuses
the entry.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

import numpy as np

import torch

from . import Assembler, BatchedAssembler, spm_get_tuning, spm_set_tuning

# the fields of spm_tuning the search varies, and the values it tries
SEARCH_SPACE = {
    "bucket_target": (4096, 5120, 6144, 7168),
    "partition_threads": (512, 1024),
    "sub_bits": (11, 12),
}


def default_candidates():
    keys = list(SEARCH_SPACE)
    return [dict(zip(keys, vals)) for vals in itertools.product(*(SEARCH_SPACE[k] for k in keys))]


def cache_key(shape, m, dtype, mode, flags=0, device=None):
    name = torch.cuda.get_device_name(device) if torch.cuda.is_available() else "cpu"
    dt = "f64" if dtype == torch.float64 else "f32"
    return f"{name}|{int(shape[0])}x{int(shape[1])}|m={int(m)}|{dt}|{mode}|flags={int(flags)}"


def batch_cache_key(n_rows, n_cols, trip_ptr, dtype, mode, flags=0, device=None):
    name = torch.cuda.get_device_name(device) if torch.cuda.is_available() else "cpu"
    dt = "f64" if dtype == torch.float64 else "f32"
    h = hashlib.sha256()
    for a in (n_rows, n_cols, trip_ptr):
        h.update(np.ascontiguousarray(np.asarray(a, dtype=np.int64)).tobytes())
        h.update(b"|")
    tp = np.asarray(trip_ptr, dtype=np.int64)
    return (f"{name}|batch={len(tp) - 1}|m={int(tp[-1]) if len(tp) else 0}|layout={h.hexdigest()[:16]}|{dt}|{mode}"
            f"|flags={int(flags)}")


def _cache_path(path):
    return path if path is not None else os.environ.get("SPM_TUNE_CACHE")


def load_cache(path=None):
    p = _cache_path(path)
    if not p or not os.path.exists(p):
        return {}
    with open(p) as f:
        return json.load(f)


def store_cache(key, entry, path=None):
    p = _cache_path(path)
    if not p:
        return
    data = load_cache(p)
    data[key] = entry
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def apply_cached(shape, m, dtype, mode, flags=0, path=None):
    """Set the cached tuning for this workload (if any); returns it or None."""
    entry = load_cache(path).get(cache_key(shape, m, dtype, mode, flags))
    if entry is None:
        return None
    spm_set_tuning(**entry["tuning"])
    return entry["tuning"]


def apply_cached_batched(n_rows, n_cols, trip_ptr, dtype, mode, flags=0, path=None):
    """Set the cached tuning for this batch layout (if any); returns it or None."""
    entry = load_cache(path).get(batch_cache_key(n_rows, n_cols, trip_ptr, dtype, mode, flags))
    if entry is None:
        return None
    spm_set_tuning(**entry["tuning"])
    return entry["tuning"]


def _same_result(a, b, mode):
    if a.nnz != b.nnz or not torch.equal(a.col_ptr, b.col_ptr) or not torch.equal(a.row_idx, b.row_idx):
        return False
    return a.nnz == 0 or torch.equal(a.vals.view(torch.uint8), b.vals.view(torch.uint8))


def _time_candidate(shape, rows, cols, vals, mode, reps, warmup):
    asm = Assembler(shape, rows.numel(), vals.dtype, mode, device=vals.device)
    for _ in range(warmup):
        asm.run(rows, cols, vals)
    res = asm.result()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in ev:
        e0.record()
        asm.run(rows, cols, vals)
        e1.record()
    torch.cuda.synchronize()
    ms = sorted(e0.elapsed_time(e1) for e0, e1 in ev)[reps // 2]
    out = asm.result()
    # copies: the next candidate reuses nothing of this Assembler
    return ms, type(out)(out.col_ptr.clone(), out.row_idx.clone(), out.vals.clone(), out.nnz, None, out.shape), res


def autotune(rows, cols, vals, shape, mode="sum", candidates=None, reps=5, warmup=3, path=None, apply=True):
    """Time the candidates on this workload; return the best entry
    {"tuning": {...}, "ms": median ms per call, "tried": n, "rejected": [...]}."""
    start = spm_get_tuning()
    rows, cols, vals = rows.contiguous(), cols.contiguous(), vals.contiguous()
    try:
        spm_set_tuning(reset=True)
        base_ms, ref, _ = _time_candidate(shape, rows, cols, vals, mode, reps, warmup)
        best = {"tuning": spm_get_tuning(), "ms": base_ms}
        rejected = []
        cands = candidates if candidates is not None else default_candidates()
        for cand in cands:
            spm_set_tuning(reset=True)
            spm_set_tuning(**cand)
            ms, out, _ = _time_candidate(shape, rows, cols, vals, mode, reps, warmup)
            if not _same_result(out, ref, mode):
                rejected.append(cand)
                continue
            if ms < best["ms"]:
                best = {"tuning": spm_get_tuning(), "ms": ms}
        best["tried"] = len(cands)
        best["rejected"] = rejected
        best["default_ms"] = base_ms
    finally:
        spm_set_tuning(reset=True)
        spm_set_tuning(**start)
    store_cache(cache_key(shape, rows.numel(), vals.dtype, mode), best, path)
    if apply:
        spm_set_tuning(**best["tuning"])
    return best


def _same_batch(a, b):
    return all(torch.equal(x.view(torch.uint8), y.view(torch.uint8)) for x, y in zip(a[:4], b[:4]))


def _time_batched(layout, rows, cols, vals, mode, reps, warmup):
    asm = BatchedAssembler(*layout, dtype=vals.dtype, mode=mode, device=vals.device)
    for _ in range(warmup):
        asm.run(rows, cols, vals)
    asm.result()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in ev:
        e0.record()
        asm.run(rows, cols, vals)
        e1.record()
    torch.cuda.synchronize()
    ms = sorted(e0.elapsed_time(e1) for e0, e1 in ev)[reps // 2]
    cp, ri, v, nnz, _ = asm.result()
    # the stored elements only (the tails of each matrix's slot are not written)
    tp, k = layout[2], nnz.cpu().numpy()
    idx = np.repeat(tp[:-1] - np.concatenate([[0], np.cumsum(k)[:-1]]), k) + np.arange(int(k.sum()))
    keep = torch.from_numpy(idx).to(ri.device)
    return ms, (cp.clone(), ri[keep].clone(), v[keep].clone(), nnz.clone())


def autotune_batched(rows, cols, vals, n_rows, n_cols, trip_ptr, mode="set", candidates=None, reps=5, warmup=3,
                     path=None, apply=True):
    """As autotune, for one batch layout and spm_assemble_csc_batched; the
    cache entry is keyed by the layout (batch_cache_key)."""
    start = spm_get_tuning()
    rows, cols, vals = rows.contiguous(), cols.contiguous(), vals.contiguous()
    layout = (np.asarray(n_rows, dtype=np.int64), np.asarray(n_cols, dtype=np.int64),
              np.asarray(trip_ptr, dtype=np.int64))
    try:
        spm_set_tuning(reset=True)
        base_ms, ref = _time_batched(layout, rows, cols, vals, mode, reps, warmup)
        best = {"tuning": spm_get_tuning(), "ms": base_ms}
        rejected = []
        cands = candidates if candidates is not None else default_candidates()
        for cand in cands:
            spm_set_tuning(reset=True)
            spm_set_tuning(**cand)
            ms, out = _time_batched(layout, rows, cols, vals, mode, reps, warmup)
            if not _same_batch(out, ref):
                rejected.append(cand)
                continue
            if ms < best["ms"]:
                best = {"tuning": spm_get_tuning(), "ms": ms}
        best["tried"] = len(cands)
        best["rejected"] = rejected
        best["default_ms"] = base_ms
    finally:
        spm_set_tuning(reset=True)
        spm_set_tuning(**start)
    store_cache(batch_cache_key(*layout, vals.dtype, mode), best, path)
    if apply:
        spm_set_tuning(**best["tuning"])
    return best
