"""Autotuner for the assembly kernels' tuning parameters (spm_tuning).

For one workload -- a device-resident write stream and its matrix shape,
value type and mode -- it times spm_assemble_csc under a list of candidate
tunings (CUDA events around each call, after warm-up), keeps only the
candidates whose CSC equals the one the default tuning produces bit for bit
(structure and values: the reduction of an element's writes does not depend
on how the work is split, so every tuning must give the same bytes), and
returns the fastest.  Results are cached in
a JSON file keyed by GPU, sizes, value type and mode: the path given, else
the environment variable SPM_TUNE_CACHE, else no cache.

    best = autotune(rows, cols, vals, shape, "sum")   # tunes, applies, caches
    apply_cached(shape, m, torch.float64, "sum")      # later: reuse the entry
"""
from __future__ import annotations

import itertools
import json
import os

import torch

from . import Assembler, spm_get_tuning, spm_set_tuning

# the fields of spm_tuning the search varies, and the values it tries
SEARCH_SPACE = {
    "bucket_target": (2048, 2560, 3072, 3584),
    "partition_threads": (512, 1024),
    "sub_bits": (10, 11),
}


def default_candidates():
    keys = list(SEARCH_SPACE)
    return [dict(zip(keys, vals)) for vals in itertools.product(*(SEARCH_SPACE[k] for k in keys))]


def cache_key(shape, m, dtype, mode, flags=0, device=None):
    name = torch.cuda.get_device_name(device) if torch.cuda.is_available() else "cpu"
    dt = "f64" if dtype == torch.float64 else "f32"
    return f"{name}|{int(shape[0])}x{int(shape[1])}|m={int(m)}|{dt}|{mode}|flags={int(flags)}"


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
