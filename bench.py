#!/usr/bin/env python
"""Benchmark of the sync step: unordered element writes -> canonical CSC.

Default workload (N=1): 100,000 x 100,000 matrix, 10^8 writes, column index
bounded Zipf(s=1.1), row uniform, values U(-1,1) in float64, add semantics
(duplicates summed) -- the 10^8-write assembly the headline metric is quoted
on.  One step = one spm_assemble_csc call (every kernel of the path) over the
whole stream, inputs resident in HBM (1.6 GB, larger than the 129 MB L2, so
no flush is needed between steps).

Prints ONE JSON line (rank 0).  Multi-GPU (torchrun, one rank per GPU): every
rank assembles its own replica of the workload (different seed), there is no
data-path collective; value = writes of all ranks / max over ranks of the
timed region (weak scaling).

--impl reference runs the CPU oracle (std::map build + in-order walk) on the
host cores instead, each step a bounded prefix of the same stream.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "assembled triplets/sec and achieved HBM GB/s (% of roofline) vs CPU oracle"
UNIT = "triplets/s"
FALLBACK_HBM_GBS = 6800.0


def workload_spec(name):
    import numpy as np
    specs = {
        "n8": dict(desc="100,000 x 100,000, 10^8 writes, Zipf(1.1) columns, uniform rows, U(-1,1) float64, sum mode",
                   m=100_000_000, n=100_000, dtype=np.float64, mode="sum", kind="zipf"),
        "zipf3e7": dict(desc="100,000 x 100,000, 3*10^7 writes, Zipf(1.1) columns, U(-1,1) float64, sum mode "
                             "(a smaller case of the same stream, for profiling)",
                        m=30_000_000, n=100_000, dtype=np.float64, mode="sum", kind="zipf"),
        "zipf1e7": dict(desc="100,000 x 100,000, 10^7 writes, Zipf(1.1) columns, U(-1,1) float64, sum mode",
                        m=10_000_000, n=100_000, dtype=np.float64, mode="sum", kind="zipf"),
        "zipf1e7_f32": dict(desc="100,000 x 100,000, 10^7 writes, Zipf(1.1) columns, U(-1,1) float32 values, "
                                 "float64 accumulation, sum mode",
                            m=10_000_000, n=100_000, dtype=np.float32, mode="sum", kind="zipf"),
        "fem2048": dict(desc="Q1 FEM 2048 x 2048 elements (4,198,401 nodes), 67,108,864 writes, float64, sum mode",
                        n_el=2048, dtype=np.float64, mode="sum", kind="fem"),
        "ordered_n8": dict(desc="100,000 x 100,000, 10^8 writes in column-major order with random gaps (5 % "
                                "repeated), U(-1,1) float64, sum mode",
                           m=100_000_000, n=100_000, dtype=np.float64, mode="sum", kind="ordered", swap=0.0),
        "ordered_2e7": dict(desc="as ordered_n8 with 2*10^7 writes (a smaller case, for profiling)",
                            m=20_000_000, n=100_000, dtype=np.float64, mode="sum", kind="ordered", swap=0.0),
        "quasi_n8": dict(desc="as ordered_n8 with 1 % of adjacent pairs swapped (quasi-ordered)",
                         m=100_000_000, n=100_000, dtype=np.float64, mode="sum", kind="ordered", swap=0.01),
        "c1": dict(desc="1000 x 1000, 10^4 writes (20 % rewrites, 5 % zeros), N(0,1) float64, set mode "
                        "(latency of one small call)", m=10_000, n=1000, dtype=np.float64, mode="set", kind="lastwrite"),
        "n4_0.01": dict(desc="10,000 x 10,000, uniform coordinates, density 0.01 % (10^4 writes), float64, set mode",
                        density=0.0001, n=10_000, dtype=np.float64, mode="set", kind="density"),
        "n4_0.1": dict(desc="10,000 x 10,000, uniform coordinates, density 0.1 % (10^5 writes), float64, set mode",
                       density=0.001, n=10_000, dtype=np.float64, mode="set", kind="density"),
        "n4_1": dict(desc="10,000 x 10,000, uniform coordinates, density 1 % (10^6 writes), float64, set mode",
                     density=0.01, n=10_000, dtype=np.float64, mode="set", kind="density"),
        "n4_10": dict(desc="10,000 x 10,000, uniform coordinates, density 10 % (10^7 writes), float64, set mode",
                      density=0.1, n=10_000, dtype=np.float64, mode="set", kind="density"),
        "batched4096": dict(desc="4096 independent square matrices, n ~ U{64..8192}, density ~ U[0.1 %, 2 %], 10 % "
                                 "rewrites, float32 N(0,1), set mode: one batched call vs single-matrix calls",
                            dtype=np.float32, mode="set", kind="batched"),
        "c5": dict(desc="Q1 FEM 512 x 512 elements (263,169 nodes, 4,194,304 writes), float32, sum mode; Y = A X "
                        "with X 263,169 x 16: forward + backward vs assembly + SpMM",
                   n_el=512, dtype=np.float32, mode="sum", kind="diff"),
        "update_n8": dict(desc="10^7 new writes (Zipf(1.1) columns, U(-1,1) float64) applied to the 100,000 x "
                               "100,000 CSC matrix that the 10^8-write Zipf stream assembles to, sum mode",
                          m=10_000_000, m_a=100_000_000, n=100_000, dtype=np.float64, mode="sum", kind="update"),
        "update_small": dict(desc="2*10^6 new writes applied to the 100,000 x 100,000 CSC matrix that 2*10^7 writes of "
                                  "the Zipf stream assemble to, sum mode (a smaller case, for profiling)",
                             m=2_000_000, m_a=20_000_000, n=100_000, dtype=np.float64, mode="sum", kind="update"),
        "lookup_n8": dict(desc="10^7 element reads (half of them stored elements) from the 100,000 x 100,000 CSC "
                               "matrix that the 10^8-write Zipf stream assembles to, float64",
                          q=10_000_000, m_a=100_000_000, n=100_000, dtype=np.float64, mode="sum", kind="lookup"),
        "coo_n8": dict(desc="coordinate-list export (column of every element, rows and values copied) of the "
                            "100,000 x 100,000 CSC matrix that the 10^8-write Zipf stream assembles to, float64",
                       m_a=100_000_000, n=100_000, dtype=np.float64, mode="sum", kind="coo"),
        "trace_10k": dict(desc="trace(A^T B) of two random 10,000 x 10,000 CSC matrices (uniform coordinates, "
                               "N(0,1) float64) at density 10 %; densities 0.01 %, 0.1 %, 1 % timed beside it",
                          n=10_000, density=0.1, dtype=np.float64, kind="trace"),
        "update_n8_set": dict(desc="as update_n8, last-write mode (the matrix assembled in sum mode)",
                              m=10_000_000, m_a=100_000_000, n=100_000, dtype=np.float64, mode="set",
                              kind="update"),
    }
    return specs[name]


def make_workload(name, rank=0):
    import workloads
    s = workload_spec(name)
    if s["kind"] == "zipf":
        d = workloads.zipf_batch(m=s["m"], n=s["n"], dtype=s["dtype"], seed=workloads.SEED_BASE + 2 + 1000 * rank)
    elif s["kind"] == "ordered":
        d = workloads.quasi_ordered(m=s["m"], n=s["n"], swap_frac=s["swap"], dtype=s["dtype"],
                                    seed=workloads.SEED_BASE + 10 + 1000 * rank)
    elif s["kind"] == "lastwrite":
        d = workloads.last_write_1000(seed=workloads.SEED_BASE + 1 + 1000 * rank)
    elif s["kind"] == "density":
        d = workloads.density_sweep(s["density"], n=s["n"], dtype=s["dtype"], seed=workloads.SEED_BASE + 6 + 1000 * rank)
    else:
        d = workloads.fem_q1(n_el=s["n_el"], dtype=s["dtype"], seed=workloads.SEED_BASE + 3 + 1000 * rank)
    return d, s


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _code_only(text):
    """The source without its comments and blank lines (edits to comments do
    not change the compiled kernels)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())


def source_hash():
    """Hash of the library's code (every kernel file and header, comments
    left out): a committed traffic figure is used only while it is unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1805_03380_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if not fn.endswith((".cu", ".cuh", ".h")):
            continue
        with open(os.path.join(csrc, fn), encoding="utf-8") as f:
            h.update(fn.encode() + _code_only(f.read()).encode())
    with open(os.path.join(ROOT, "include", "spm.h"), encoding="utf-8") as f:
        h.update(b"spm.h" + _code_only(f.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload, key="dram_bytes_per_call"):
    """DRAM bytes (read + written) per call, or per launch of one kernel, from
    the committed ncu summary of the workload, if it was taken on the current
    sources (otherwise None)."""
    p = os.path.join(ROOT, "profiles", f"traffic_{workload}.md")
    if not os.path.exists(p):
        return None
    vals = {}
    with open(p) as f:
        for line in f:
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("source_hash", "").split(" ")[0] != source_hash():
        return None
    try:
        return int(vals[key])
    except Exception:
        return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines += [ln for ln in out.splitlines() if ln.strip()]  # (several timed regions add up)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(elapsed_s, units, world, device):
    """Max of the timed region and sum of the units over ranks."""
    if world == 1:
        return elapsed_s, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def oracle_rate(d, mode, sample):
    """CPU oracle (single thread) on the first `sample` writes: writes/s."""
    import oracle
    r, c, v = d["rows"][:sample], d["cols"][:sample], d["vals"][:sample]
    t0 = time.perf_counter()
    oracle.assemble_csc(r, c, v, d["shape"], mode=mode)
    dt = time.perf_counter() - t0
    return sample / dt, dt


UPDATE_METRIC = "elements merged into an existing CSC matrix per second (existing elements + new writes)"
UPDATE_UNIT = "elements/s"


def update_oracle_rate(spec, sample):
    """CPU oracle of the update on a sample: the matrix assembled from the
    first `sample` writes of the matrix stream, then the first sample/10 new
    writes; (existing elements + writes) per second, and the seconds taken."""
    import oracle
    import workloads
    da = workloads.zipf_batch(m=sample, n=spec["n"], dtype=spec["dtype"], seed=workloads.SEED_BASE + 2)
    dw = workloads.zipf_batch(m=max(sample // 10, 1), n=spec["n"], dtype=spec["dtype"], seed=workloads.SEED_BASE + 8)
    A = oracle.assemble_csc(da["rows"], da["cols"], da["vals"], da["shape"], mode="sum")
    t0 = time.perf_counter()
    oracle.csc_update(*A, da["shape"], dw["rows"], dw["cols"], dw["vals"], mode=spec["mode"])
    dt = time.perf_counter() - t0
    return (len(A[1]) + len(dw["rows"])) / dt, dt, len(A[1]), len(dw["rows"])


def run_update(args, world, rank, local_rank):
    """spm_csc_update on the workload: CUDA events around each call, inputs
    resident in HBM.  The merge stage is the call minus the assembly of the
    new writes alone (timed the same way); the alternative without a merge,
    re-assembling the whole concatenated stream, is timed beside it."""
    import numpy as np
    import torch

    import paper_1805_03380_gb300 as spm
    import workloads
    spec = workload_spec(args.workload)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    sv = np.dtype(spec["dtype"]).itemsize
    da = workloads.zipf_batch(m=spec["m_a"], n=spec["n"], dtype=spec["dtype"],
                              seed=workloads.SEED_BASE + 2 + 1000 * rank)
    dw = workloads.zipf_batch(m=spec["m"], n=spec["n"], dtype=spec["dtype"],
                              seed=workloads.SEED_BASE + 8 + 1000 * rank)
    shape = da["shape"]
    n_rows, n_cols = shape
    ar, ac, av = (torch.from_numpy(da[k]).to(dev) for k in ("rows", "cols", "vals"))
    A = spm.assemble_csc(ar, ac, av, shape, mode="sum")
    a_cp, a_ri, a_v = A.col_ptr, A.row_idx.clone(), A.vals.clone()
    nnz_a = A.nnz
    wr, wc, wv = (torch.from_numpy(dw[k]).to(dev) for k in ("rows", "cols", "vals"))
    m = wr.numel()
    mode = spec["mode"]
    ws = torch.empty(spm.spm_csc_update_workspace(n_rows, n_cols, nnz_a, m, wv.dtype, mode), dtype=torch.uint8,
                     device=dev)
    o_cp = torch.empty(n_cols + 1, dtype=torch.int64, device=dev)
    o_ri = torch.empty(nnz_a + m, dtype=torch.int32, device=dev)
    o_v = torch.empty(nnz_a + m, dtype=wv.dtype, device=dev)
    d_nnz = torch.zeros(1, dtype=torch.int64, device=dev)
    d_status = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def update():
        spm.spm_csc_update(n_rows, n_cols, a_cp, a_ri, a_v, wr, wc, wv, None, mode, 0, o_cp, o_ri, o_v, d_nnz,
                           d_status, ws)

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for e0, e1 in ev:
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in ev]

    for _ in range(args.warmup):
        update()
    torch.cuda.synchronize()
    if int(d_status.item()) != 0:
        raise RuntimeError(f"spm_csc_update status {int(d_status.item())}")
    nnz_out = int(d_nnz.item())
    sampler = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    sampler.start()
    time.sleep(0.2)
    launches0 = spm.spm_debug_launch_count()
    if world > 1:
        torch.distributed.barrier()
    upd_ms = timed(update, args.steps)
    launches = spm.spm_debug_launch_count() - launches0
    sampler.stop()
    if int(d_status.item()) != 0 or int(d_nnz.item()) != nnz_out:
        raise RuntimeError("spm_csc_update changed its result between calls")
    # the assembly of the new writes alone (the update's first stage)
    asm_b = spm.Assembler(shape, m, wv.dtype, mode, device=dev)
    for _ in range(args.warmup):
        asm_b.run(wr, wc, wv)
    b_ms = timed(lambda: asm_b.run(wr, wc, wv), args.steps)
    nnz_b = asm_b.result().nnz
    del asm_b
    # re-assembling everything instead: A's elements as writes, then the new ones
    colj = torch.repeat_interleave(torch.arange(n_cols, device=dev, dtype=torch.int32), a_cp.diff())
    cr, cc, cv = torch.cat([a_ri, wr]), torch.cat([colj, wc]), torch.cat([a_v, wv])
    del colj
    asm_all = spm.Assembler(shape, cr.numel(), wv.dtype, mode, device=dev)
    for _ in range(args.warmup):
        asm_all.run(cr, cc, cv)
    all_ms = timed(lambda: asm_all.run(cr, cc, cv), args.steps)
    if asm_all.result().nnz != nnz_out:
        raise RuntimeError("re-assembly and update disagree on the number of elements")
    del asm_all, cr, cc, cv

    upd = statistics.mean(upd_ms)
    bms = statistics.mean(b_ms)
    merge_ms = max(upd - bms, 1e-6)
    tot_s, units = aggregate(sum(upd_ms) / 1000.0, (nnz_a + m) * args.steps, world, dev)
    peak, peak_kind = measured_peak()
    merge_bytes = (nnz_a + nnz_b + nnz_out) * (4 + sv) + 3 * (n_cols + 1) * 8
    achieved = merge_bytes / (merge_ms / 1000.0) / 1e9
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, dt, sa, sw = update_oracle_rate(spec, min(args.ref_sample, 1_000_000))
        cpu = {"value": rate, "unit": UPDATE_UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{sa} existing elements (first writes of the matrix stream) + {sw} new writes, "
                         f"dict + two-pointer merge in Python, 1 thread, {dt:.1f} s"}
    if rank == 0:
        line = {
            "metric": UPDATE_METRIC, "value": units / tot_s, "unit": UPDATE_UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64" if sv == 8 else "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "description": spec["desc"], "nnz_a": nnz_a, "m": m,
                       "nnz_b": nnz_b, "nnz_out": nnz_out, "mode": mode,
                       "l2": "inputs larger than the 129 MB L2 (no flush between steps)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_kind": peak_kind + " copy bandwidth",
                         "kernel": "merge stage (offset check, cuts, k_merge): call time minus the assembly of "
                                   "the new writes alone",
                         "algorithmic_bytes_per_launch": merge_bytes,
                         "bytes_formula": "(nnz_a + nnz_b + nnz_out)*(4+sv) + 3*(n_cols+1)*8",
                         "launch_ms_mean": merge_ms},
            "update_ms_mean": upd, "assemble_new_writes_ms_mean": bms, "reassemble_all_ms_mean": statistics.mean(all_ms),
            "cpu_baseline": cpu,
            "clocks": sampler.summary(),
            "gpu_launches": launches,
            "gpu": torch.cuda.get_device_name(dev),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_access(args, world, rank, local_rank):
    """Element lookup, coordinate-list export or trace(A^T B): CUDA events
    around each call, inputs resident in HBM."""
    import numpy as np
    import torch

    import paper_1805_03380_gb300 as spm
    import workloads
    spec = workload_spec(args.workload)
    kind = spec["kind"]
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    sv = np.dtype(spec["dtype"]).itemsize
    stream = torch.cuda.current_stream()

    sampler = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        sampler.start()  # clocks sampled during the timed calls only
        for e0, e1 in ev:
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        t_hold = time.perf_counter()  # the same load a moment longer, so that the sampler sees it
        while time.perf_counter() - t_hold < 0.5:
            fn()
            torch.cuda.synchronize()
        sampler.stop()
        return statistics.mean(e0.elapsed_time(e1) for e0, e1 in ev)

    def matrix_from(d):
        r, c, v = (torch.from_numpy(d[k]).to(dev) for k in ("rows", "cols", "vals"))
        A = spm.assemble_csc(r, c, v, d["shape"], mode="sum" if kind != "trace" else "set")
        return A.col_ptr, A.row_idx.clone(), A.vals.clone(), d["shape"]

    d_status = torch.zeros(1, dtype=torch.int32, device=dev)
    extra = {}
    launches0 = spm.spm_debug_launch_count()
    if kind in ("lookup", "coo"):
        cp, ri, v, shape = matrix_from(workloads.zipf_batch(m=spec["m_a"], n=spec["n"], dtype=spec["dtype"],
                                                            seed=workloads.SEED_BASE + 2 + 1000 * rank))
        nnz = ri.numel()
        n_cols = shape[1]
        if kind == "lookup":
            q = spec["q"]
            g = torch.Generator(device=dev)
            g.manual_seed(workloads.SEED_BASE + 9 + rank)
            colj = torch.repeat_interleave(torch.arange(n_cols, device=dev, dtype=torch.int32), cp.diff())
            pick = torch.randint(0, nnz, (q,), device=dev, generator=g)
            hit = torch.rand(q, device=dev, generator=g) < 0.5
            qr = torch.where(hit, ri[pick], torch.randint(0, shape[0], (q,), device=dev, generator=g,
                                                          dtype=torch.int32))
            qc = torch.where(hit, colj[pick], torch.randint(0, n_cols, (q,), device=dev, generator=g,
                                                            dtype=torch.int32))
            del colj, pick, hit
            out = torch.empty(q, dtype=v.dtype, device=dev)
            pos = torch.empty(q, dtype=torch.int64, device=dev)
            launches0 = spm.spm_debug_launch_count()
            ms = timed(lambda: spm.spm_csc_lookup(shape[0], n_cols, cp, ri, v, qr, qc, out, pos, d_status), args.steps)
            units = q
            unit = "reads/s"
            metric = "element reads from a CSC matrix per second (column start + binary search)"
            alg = q * (4 + 4 + sv + 8) + q * 16
            formula = "q*(4+4+sv+8) + q*16 (query in, value and position out, the column's two offsets)"
            kernel = "k_lookup (one thread per read)"
            extra = {"stored_fraction": float((pos >= 0).double().mean().item())}
        else:
            o_r, o_c, o_v = torch.empty_like(ri), torch.empty_like(ri), torch.empty_like(v)
            launches0 = spm.spm_debug_launch_count()
            ms = timed(lambda: spm.spm_csc_to_coo(n_cols, cp, ri, v, o_r, o_c, o_v, d_status), args.steps)
            units = nnz
            unit = "elements/s"
            metric = "elements exported from CSC to a coordinate list per second"
            alg = nnz * (4 + sv + 4 + 4 + sv) + (n_cols + 1) * 8
            formula = "nnz*(4+sv read + 4+4+sv written) + (n_cols+1)*8"
            kernel = "k_to_coo (tile of 2048 elements per block)"
        extra.update({"nnz": nnz, "n_rows": shape[0], "n_cols": n_cols})
    else:
        per = {}
        for dens in (0.0001, 0.001, 0.01, spec["density"]):
            A = matrix_from(workloads.density_sweep(dens, n=spec["n"], dtype=spec["dtype"],
                                                    seed=workloads.SEED_BASE + 6 + 1000 * rank))
            B = matrix_from(workloads.density_sweep(dens, n=spec["n"], dtype=spec["dtype"],
                                                    seed=workloads.SEED_BASE + 16 + 1000 * rank))
            ws = torch.empty(spm.spm_csc_trace_atb_workspace(spec["n"], A[1].numel(), B[1].numel()),
                             dtype=torch.uint8, device=dev)
            res = torch.zeros(1, dtype=torch.float64, device=dev)

            def call():
                spm.spm_csc_trace_atb(spec["n"], spec["n"], A[0], A[1], A[2], B[0], B[1], B[2], res, d_status, ws)
            launches0 = spm.spm_debug_launch_count()
            ms_d = timed(call, args.steps)
            per[f"{dens * 100:g}%"] = {"ms": ms_d, "nnz_a": A[1].numel(), "nnz_b": B[1].numel(),
                                       "trace": float(res.item())}
        ms = per[f"{spec['density'] * 100:g}%"]["ms"]
        nnz_a, nnz_b = per[f"{spec['density'] * 100:g}%"]["nnz_a"], per[f"{spec['density'] * 100:g}%"]["nnz_b"]
        units = nnz_a + nnz_b
        unit = "elements/s"
        metric = "elements of A and B reduced into trace(A^T B) per second"
        alg = (nnz_a + nnz_b) * (4 + sv) + 2 * (spec["n"] + 1) * 8
        formula = "(nnz_a + nnz_b)*(4+sv) + 2*(n_cols+1)*8"
        kernel = "whole call (offset checks, cuts, k_merge in dot form, final sum)"
        extra = {"densities": per}
    launches = spm.spm_debug_launch_count() - launches0
    torch.cuda.synchronize()
    if int(d_status.item()) != 0:
        raise RuntimeError(f"device status {int(d_status.item())}")
    tot_s, tot_units = aggregate(ms / 1000.0 * args.steps, units * args.steps, world, dev)
    peak, peak_kind = measured_peak()
    achieved = alg / (ms / 1000.0) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": metric, "value": tot_units / tot_s, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if sv == 8 else "f32", "data": "synthetic",
            "config": dict({"workload": args.workload, "description": spec["desc"]}, **extra),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind + " copy bandwidth",
                         "kernel": kernel, "algorithmic_bytes_per_launch": alg, "bytes_formula": formula,
                         "launch_ms_mean": ms},
            "gpu_launches": launches, "gpu": torch.cuda.get_device_name(dev), "clocks": sampler.summary()}),
              flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def batched_oracle_rate(d, mode, budget_s=20.0):
    """CPU oracle over the batch, one matrix per thread on every host core
    (ctypes releases the GIL during the oracle's C++ build): matrices in a
    seeded order until about budget_s of wall time; writes/s, the matrices
    and writes done, the threads used."""
    import concurrent.futures as cf

    import numpy as np

    import oracle
    tp = np.asarray(d["trip_ptr"], dtype=np.int64)
    ns = np.asarray(d["n"], dtype=np.int64)
    order = np.random.default_rng(7).permutation(len(ns))
    threads = os.cpu_count() or 1

    def one(i):
        a, b = int(tp[i]), int(tp[i + 1])
        oracle.assemble_csc(d["rows"][a:b], d["cols"][a:b], d["vals"][a:b], (int(ns[i]), int(ns[i])), mode=mode)
        return b - a

    done = writes = 0
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        while done < len(order) and time.perf_counter() - t0 < budget_s:
            chunk = order[done:done + 4 * threads]
            writes += sum(ex.map(one, chunk))
            done += len(chunk)
    dt = time.perf_counter() - t0
    return writes / dt, done, writes, threads, dt


def diff_oracle_rate(f, mode, k=16):
    """CPU oracle of the differentiable step (1 thread): assembly, Y = A X, and
    the backward (dvals and dX = A^T dY); writes/s and the seconds taken."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(5)
    n = f["shape"][0]
    X = rng.standard_normal((n, k))
    dY = rng.standard_normal((n, k))
    t0 = time.perf_counter()
    cp, ri, v = oracle.assemble_csc(f["rows"], f["cols"], f["vals"], f["shape"], mode=mode)
    oracle.csc_mm(f["shape"], cp, ri, v, X)
    oracle.dvals(f["rows"], f["cols"], dY, X)
    oracle.csc_mm(f["shape"], cp, ri, v, dY, transpose=True)
    dt = time.perf_counter() - t0
    return len(f["rows"]) / dt, dt


def run_batched_or_diff(args, world, rank, local_rank):
    """The batched workload (one spm_assemble_csc_batched call against the
    same matrices assembled one call each, the latter timed on every 16th
    matrix and scaled) or the differentiable one (AssembleMM forward +
    backward against assembly + SpMM).  CUDA events around each call."""
    import numpy as np
    import torch

    import paper_1805_03380_gb300 as spm
    import workloads
    spec = workload_spec(args.workload)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream()
    # the differentiable workload's operands (about 120 MB with the workspace)
    # fit in L2: a 512 MB write flushes it before every timed call
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev) if spec["kind"] == "diff" else None

    sampler = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        sampler.start()  # clocks sampled during the timed calls only
        for e0, e1 in ev:
            if flush is not None:
                flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        t_hold = time.perf_counter()  # the same load a moment longer, so that the sampler sees it
        while time.perf_counter() - t_hold < 0.5:
            fn()
            torch.cuda.synchronize()
        sampler.stop()
        return statistics.mean(e0.elapsed_time(e1) for e0, e1 in ev)

    if spec["kind"] == "batched":
        d = workloads.batched_uniform(seed=workloads.SEED_BASE + 4 + 1000 * rank)
        ns, tp = np.asarray(d["n"], dtype=np.int64), np.asarray(d["trip_ptr"], dtype=np.int64)
        rows, cols, vals = (torch.from_numpy(np.ascontiguousarray(d[k])).to(dev) for k in ("rows", "cols", "vals"))
        rows, cols = rows.to(torch.int32), cols.to(torch.int32)
        B, total = len(ns), int(tp[-1])
        # the project's autotuner picks the tuning (on the first 512 matrices of
        # the batch, whose layout stands for the rest) before anything is timed
        from paper_1805_03380_gb300 import autotune as at
        sub = 512
        tsub = int(tp[sub])
        best = at.autotune_batched(rows[:tsub], cols[:tsub], vals[:tsub], ns[:sub], ns[:sub], tp[:sub + 1],
                                   spec["mode"], candidates=[dict(bucket_target=t, partition_threads=p)
                                                             for t in (4096, 6144, 7168) for p in (512, 1024)],
                                   reps=3, warmup=1, apply=True)
        hr, hc, ht = torch.from_numpy(ns), torch.from_numpy(ns.copy()), torch.from_numpy(tp)
        dr, dc, dt = hr.to(dev), hc.to(dev), ht.to(dev)
        ws = torch.empty(spm.spm_assemble_csc_batched_workspace(hr, hc, ht, vals.dtype, spec["mode"]),
                         dtype=torch.uint8, device=dev)
        col_ptr = torch.empty(int((hc + 1).sum()), dtype=torch.int64, device=dev)
        row_idx = torch.empty(total, dtype=torch.int32, device=dev)
        out_vals = torch.empty(total, dtype=vals.dtype, device=dev)
        d_nnz = torch.zeros(B, dtype=torch.int64, device=dev)
        d_status = torch.zeros(1, dtype=torch.int32, device=dev)

        def batched():
            spm.spm_assemble_csc_batched(hr, hc, ht, dr, dc, dt, rows, cols, vals, None, spec["mode"], 0, col_ptr,
                                         row_idx, out_vals, d_nnz, None, d_status, ws)
        b_ms = timed(batched, args.steps)
        if int(d_status.item()) != 0:
            raise RuntimeError(f"batched status {int(d_status.item())}")
        sample = list(range(0, B, 16))
        asms = [spm.Assembler((int(ns[i]), int(ns[i])), int(tp[i + 1] - tp[i]), vals.dtype, spec["mode"], device=dev)
                for i in sample]
        views = [(rows[int(tp[i]):int(tp[i + 1])], cols[int(tp[i]):int(tp[i + 1])], vals[int(tp[i]):int(tp[i + 1])])
                 for i in sample]

        def singles():
            for a, (r, c, v) in zip(asms, views):
                a.run(r, c, v)
        s_ms = timed(singles, max(1, args.steps // 5)) * B / len(sample)
        units, ms = total, b_ms
        metric = "assembled triplets/sec, 4096 matrices in one batched call"
        extra = {"matrices": B, "writes": total, "nnz": int(d_nnz.sum().item()),
                 "single_calls_ms_scaled": s_ms, "single_calls_sample": f"every 16th matrix ({len(sample)}), scaled",
                 "batched_vs_single_speedup": s_ms / b_ms,
                 "tuning": {k: best["tuning"][k] for k in ("bucket_target", "partition_threads", "sub_bits")},
                 "autotune": f"{best['tried']} candidates timed on the first {sub} matrices, "
                             f"{len(best['rejected'])} rejected for different bits; default {best['default_ms']:.2f} ms, "
                             f"chosen {best['ms']:.2f} ms",
                 "l2": "inputs (about 12 GB) larger than the 129 MB L2 (no flush between steps)"}
        sv = 4
        alg = total * (4 + 4 + sv) + int(d_nnz.sum().item()) * (4 + sv) + int((hc + 1).sum()) * 8
    else:
        f = workloads.fem_q1(n_el=spec["n_el"], dtype=spec["dtype"], seed=workloads.SEED_BASE + 5 + 1000 * rank)
        shape = f["shape"]
        rows, cols = (torch.from_numpy(f[k]).to(dev).to(torch.int32) for k in ("rows", "cols"))
        vals = torch.from_numpy(f["vals"]).to(dev)
        g = torch.Generator(device=dev)
        g.manual_seed(workloads.SEED_BASE + 5)
        X = torch.randn(shape[0], 16, device=dev, dtype=vals.dtype, generator=g, requires_grad=True)
        G = torch.randn(shape[0], 16, device=dev, dtype=vals.dtype, generator=g)
        v = vals.clone().requires_grad_(True)

        def fwd_bwd():
            Y = spm.AssembleMM.apply(rows, cols, v, shape, X, spec["mode"], True)
            (Y * G).sum().backward()

        def asm_mm():
            A = spm.assemble_csc(rows, cols, vals, shape, mode=spec["mode"])
            spm.csc_mm(A.col_ptr, A.row_idx, A.vals, shape, X.detach())
        fb_ms = timed(fwd_bwd, args.steps)
        am_ms = timed(asm_mm, args.steps)
        # the product kernel alone: Y = A X gathered over the columns of A^T
        A = spm.assemble_csc(rows, cols, vals, shape, mode=spec["mode"])
        At = spm.csc_transpose(A.col_ptr, A.row_idx, A.vals, shape)
        Xd = X.detach()

        def gather():
            spm.csc_mm(At.col_ptr, At.row_idx, At.vals, At.shape, Xd, transpose=True, check=False)
        # the operands fit in L2: flush it (write 512 MB) before every timed launch
        for _ in range(args.warmup):
            gather()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(max(args.steps, 20))]
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            gather()
            e1.record(stream)
        torch.cuda.synchronize()
        mm_ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in evs)
        nnz_a = A.nnz
        mm_bytes = nnz_a * (4 + 4) + 2 * shape[0] * 16 * 4 + (shape[0] + 1) * 8
        mm_ach = mm_bytes / (mm_ms / 1000.0) / 1e9
        units, ms = len(f["rows"]), fb_ms
        metric = "assembled triplets/sec through assemble + SpMM forward and backward"
        extra = {"writes": len(f["rows"]), "nodes": shape[0], "nnz": nnz_a, "k": 16, "assembly_plus_spmm_ms": am_ms,
                 "forward_backward_over_assembly_spmm": fb_ms / am_ms,
                 "l2": "a 512 MB write flushes the 129 MB L2 before every timed call"}
        sv = 4
        alg = None
        peak0, peak_kind0 = measured_peak()
        spmm_roofline = {"bound": "hbm", "achieved": mm_ach, "peak": peak0, "unit": "GB/s", "frac": mm_ach / peak0,
                         "traffic": None, "peak_kind": peak_kind0 + " copy bandwidth",
                         "kernel": "k_mm_gather: Y = A X (263,169 x 16 float32) over the columns of A^T, "
                                   "CUDA events around each launch",
                         "algorithmic_bytes_per_launch": mm_bytes,
                         "bytes_formula": "nnz*(4+sv) + 2*n*k*sv + (n+1)*8", "launch_ms_mean": mm_ms,
                         "l2": "operands (about 55 MB) fit in the 129 MB L2: a 512 MB write flushes it before "
                               "every timed launch"}
    tot_s, tot_units = aggregate(ms / 1000.0 * args.steps, units * args.steps, world, dev)
    peak, peak_kind = measured_peak()
    line = {
        "metric": metric, "value": tot_units / tot_s, "unit": "triplets/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if sv == 4 else "f64", "data": "synthetic",
        "config": dict({"workload": args.workload, "description": spec["desc"]}, **extra),
        "gpu": torch.cuda.get_device_name(dev), "clocks": sampler.summary(),
    }
    if spec["kind"] == "diff":
        line["roofline"] = spmm_roofline
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if spec["kind"] == "batched":
            rate, done, wr, thr, dt = batched_oracle_rate(d, spec["mode"])
            line["cpu_baseline"] = {"value": rate, "unit": "triplets/s", "cores": thr, "host_cores": os.cpu_count(),
                                    "kind": "oracle",
                                    "sample": f"{done} of the {B} matrices ({wr} writes) in a seeded order, one "
                                              f"matrix per thread, std::map build + walk, {dt:.1f} s"}
        else:
            rate, dt = diff_oracle_rate(f, spec["mode"])
            line["cpu_baseline"] = {"value": rate, "unit": "triplets/s", "cores": 1, "host_cores": os.cpu_count(),
                                    "kind": "oracle",
                                    "sample": f"the whole workload: std::map assembly, Y = A X, dvals and A^T dY "
                                              f"(float64), 1 thread, {dt:.1f} s"}
    if alg is not None:
        achieved = alg / (ms / 1000.0) / 1e9
        line["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind + " copy bandwidth",
                            "kernel": "whole batched call", "algorithmic_bytes_per_launch": alg,
                            "bytes_formula": "m*(4+4+sv) + nnz*(4+sv) + sum(n_cols_i+1)*8", "launch_ms_mean": ms}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_reference(args, world, rank):
    import numpy as np  # noqa: F401
    import workloads
    if rank != 0:
        return
    spec = workload_spec(args.workload)
    sample = args.ref_sample
    if spec["kind"] in ("lookup", "coo", "trace", "batched", "diff"):
        print(json.dumps({"impl": "reference", "unavailable": "the CPU reference leg times the single-matrix "
                                                              "assembly and update workloads only"}), flush=True)
        return
    if spec["kind"] == "update":
        sample = min(sample, 200_000)
        times = []
        for k in range(args.warmup + args.steps):
            rate, dt, sa, sw = update_oracle_rate(spec, sample)
            if k >= args.warmup:
                times.append(dt)
        value = (sa + sw) * args.steps / sum(times)
        print(json.dumps({
            "metric": UPDATE_METRIC, "value": value, "unit": UPDATE_UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": spec["desc"],
                       "sample": f"{sa} existing elements + {sw} new writes per step"},
            "cpu_baseline": {"value": value, "unit": UPDATE_UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{sa} existing elements + {sw} new writes, Python dict + merge, 1 thread"},
            "e2e": {"value": value, "unit": UPDATE_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
            flush=True)
        return
    # the prefix of the same stream (the generator draws in fixed chunks of 2^24)
    if spec["kind"] == "zipf":
        d = workloads.zipf_batch(m=max(sample, min(spec["m"], 1 << 24)), n=spec["n"], dtype=spec["dtype"],
                                 seed=workloads.SEED_BASE + 2)
    elif spec["kind"] == "ordered":  # the gaps depend on m: draw the whole stream, use its prefix
        d = workloads.quasi_ordered(m=spec["m"], n=spec["n"], swap_frac=spec["swap"], dtype=spec["dtype"],
                                    seed=workloads.SEED_BASE + 10)
    elif spec["kind"] in ("lastwrite", "density"):
        d, _ = make_workload(args.workload)
        sample = min(sample, len(d["rows"]))
    else:
        d = workloads.fem_q1(n_el=spec["n_el"], dtype=spec["dtype"], seed=workloads.SEED_BASE + 3)
    for _ in range(args.warmup):
        oracle_rate(d, spec["mode"], sample)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_rate(d, spec["mode"], sample)
        times.append(dt)
    tot = sum(times)
    value = sample * args.steps / tot
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if spec["dtype"].__name__ == "float64" else "f32", "data": "synthetic",
        "config": {"workload": args.workload, "description": spec["desc"],
                   "sample": f"first {sample} writes of the same stream per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"first {sample} writes of the workload's stream, std::map build + walk, 1 thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_e2e(spm, asm0, d, rows, cols, vals, nnz, steps, args, world, dev):
    """End-to-end rate of the single-matrix call through the public API:
    every step copies its writes from pinned host memory to the device, runs
    spm_assemble_csc and copies the CSC (col_ptr and the stored elements)
    back to pinned host memory.  Two slots (device inputs, an Assembler,
    host outputs) alternate between steps so that the copies of neighbouring
    steps overlap the call.  Returns (writes/s, D2H bytes per step, H2D bytes
    per step)."""
    import torch
    m = len(d["rows"])
    n_cols = d["shape"][1]
    sv = vals.element_size()
    if args.profile or steps == 0:
        return None, 0, m * (8 + sv)
    h_in = [torch.from_numpy(d[k]).pin_memory() for k in ("rows", "cols", "vals")]
    slots = []
    for j in range(2):
        a = asm0 if j == 0 else spm.Assembler(d["shape"], m, vals.dtype, asm0.mode, device=dev)
        slots.append({
            "asm": a, "d_in": [torch.empty_like(t) for t in (rows, cols, vals)],
            "h_cp": torch.empty(n_cols + 1, dtype=torch.int64).pin_memory(),
            "h_ri": torch.empty(m, dtype=torch.int32).pin_memory(),
            "h_v": torch.empty(m, dtype=vals.dtype).pin_memory(),
            "h_nnz": torch.zeros(1, dtype=torch.int64).pin_memory(),
            "h2d": torch.cuda.Event(), "done": torch.cuda.Event(), "d2h": torch.cuda.Event(), "used": False})
    s_in = [torch.cuda.Stream(device=dev) for _ in range(3)]
    s_cmp = torch.cuda.Stream(device=dev)
    s_out = torch.cuda.Stream(device=dev)
    d2h_bytes = []

    def enqueue(k):
        sl = slots[k % 2]
        for st, dst, src in zip(s_in, sl["d_in"], h_in):
            if sl["used"]:
                st.wait_event(sl["done"])  # the call two steps back has read this slot's inputs
            with torch.cuda.stream(st):
                dst.copy_(src, non_blocking=True)
        ev_in = []
        for st in s_in:
            e = torch.cuda.Event()
            e.record(st)
            ev_in.append(e)
        for e in ev_in:
            s_cmp.wait_event(e)
        if sl["used"]:
            s_cmp.wait_event(sl["d2h"])  # this slot's outputs have been copied out
        sl["asm"].run(*sl["d_in"], stream=s_cmp)
        with torch.cuda.stream(s_cmp):
            sl["h_nnz"].copy_(sl["asm"].d_nnz, non_blocking=True)
        sl["done"].record(s_cmp)
        sl["used"] = True

    def drain(k):
        sl = slots[k % 2]
        sl["done"].synchronize()  # step k has ended (step k+1 is queued behind it)
        k_nnz = int(sl["h_nnz"][0])
        s_out.wait_event(sl["done"])
        a = sl["asm"]
        with torch.cuda.stream(s_out):
            sl["h_cp"].copy_(a.col_ptr, non_blocking=True)
            sl["h_ri"][:k_nnz].copy_(a.row_idx[:k_nnz], non_blocking=True)
            sl["h_v"][:k_nnz].copy_(a.out_vals[:k_nnz], non_blocking=True)
        sl["d2h"].record(s_out)
        d2h_bytes.append(8 + (n_cols + 1) * 8 + k_nnz * (4 + sv))

    def run(n):
        for k in range(n):
            enqueue(k)
            if k >= 1:
                drain(k - 1)
        drain(n - 1)
        s_out.synchronize()

    run(3)  # warm-up
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    d2h_bytes.clear()
    t0 = time.perf_counter()
    run(steps)
    e2e_s = time.perf_counter() - t0
    for sl in slots:
        spm._raise_status(sl["asm"].d_status, "spm_assemble_csc")
    k_nnz = int(slots[(steps - 1) % 2]["h_nnz"][0])
    if k_nnz != nnz or int(slots[(steps - 1) % 2]["h_cp"][-1]) != nnz:
        raise RuntimeError("end-to-end result differs from the device-timed one")
    e2e_tot_s, e2e_units = aggregate(max(e2e_s, 1e-9), m * steps, world, dev)
    return e2e_units / e2e_tot_s, statistics.mean(d2h_bytes), m * (8 + sv)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n8",
                    choices=["n8", "zipf3e7", "zipf1e7", "zipf1e7_f32", "fem2048", "update_n8", "update_n8_set",
                             "update_small", "lookup_n8", "coo_n8", "trace_10k", "ordered_n8",
                             "quasi_n8", "ordered_2e7", "c1", "n4_0.01", "n4_0.1", "n4_1", "n4_10", "batched4096",
                             "c5"])
    ap.add_argument("--cpu-sample", type=int, default=10_000_000, help="writes the CPU oracle baseline times")
    ap.add_argument("--ref-sample", type=int, default=1_000_000, help="writes per step of --impl reference")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="only the warm-up and timed steps (for ncu): no e2e, clock hold or CPU baseline")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if workload_spec(args.workload)["kind"] == "update":
        run_update(args, world, rank, local_rank)
        return
    if workload_spec(args.workload)["kind"] in ("lookup", "coo", "trace"):
        run_access(args, world, rank, local_rank)
        return
    if workload_spec(args.workload)["kind"] in ("batched", "diff"):
        run_batched_or_diff(args, world, rank, local_rank)
        return

    import numpy as np
    import torch

    import paper_1805_03380_gb300 as spm
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    d, spec = make_workload(args.workload, rank)
    m = len(d["rows"])
    n_rows, n_cols = d["shape"]
    sv = np.dtype(spec["dtype"]).itemsize
    rows = torch.from_numpy(d["rows"]).to(dev)
    cols = torch.from_numpy(d["cols"]).to(dev)
    vals = torch.from_numpy(d["vals"]).to(dev)
    asm = spm.Assembler(d["shape"], m, vals.dtype, spec["mode"], device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        asm.run(rows, cols, vals)
    A = asm.result()  # synchronises and checks the device status
    nnz = A.nnz

    # ---- timed region: K steps, inputs resident in HBM ----
    spm.spm_debug_stage_timing(True)
    sampler = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    sampler.start()
    time.sleep(0.2)
    launches0 = spm.spm_debug_launch_count()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    # inputs smaller than L2 (129 MB, with room for the workspace): a 512 MB
    # write flushes it before every step, outside the step's events, and the
    # rate is taken over the steps' own times
    flush_l2 = m * (8 + sv) < (256 << 20)
    flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device=dev) if flush_l2 else None
    t_start.record(stream)
    for k in range(args.steps):
        if flush_l2:
            flush_buf.zero_()
        starts[k].record(stream)
        asm.run(rows, cols, vals)
        ends[k].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = spm.spm_debug_launch_count() - launches0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    elapsed_s = (sum(step_ms) if flush_l2 else t_start.elapsed_time(t_end)) / 1000.0
    del flush_buf
    stages = {}
    nback = min(args.steps, 64)
    for back in range(nback):
        for kname, v in spm.spm_debug_stage_times(back).items():
            stages.setdefault(kname, []).append(v)
    # keep the GPU under the same load for a moment so the clock sampler sees it
    t_extra = time.perf_counter()
    while not args.profile and time.perf_counter() - t_extra < 1.0:
        asm.run(rows, cols, vals)
        torch.cuda.synchronize()
    sampler.stop()
    spm.spm_debug_stage_timing(False)
    A = asm.result()
    assert A.nnz == nnz

    tot_s, tot_units = aggregate(elapsed_s, m * args.steps, world, dev)
    value = tot_units / tot_s
    ms_per_step = 1000.0 * tot_s / args.steps

    # ---- roofline of the whole call (the sync step: one read of the writes,
    # one write of the CSC), CUDA events around each call on its stream; and
    # of its two largest kernels, CUDA events at their launch boundaries ----
    peak, peak_kind = measured_peak()
    stage_ms = {k: statistics.mean(v) for k, v in stages.items()}
    alg_bytes = m * (4 + 4 + sv) + nnz * (4 + sv) + (n_cols + 1) * 8
    mean_call_s = statistics.mean(step_ms) / 1000.0
    achieved = alg_bytes / mean_call_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profiled_traffic(args.workload), "peak_kind": peak_kind + " copy bandwidth",
                "kernel": f"spm_assemble_csc: the whole sync step ({launches // max(args.steps, 1)} kernel "
                          "launches), CUDA events around each call",
                "algorithmic_bytes_per_launch": alg_bytes,
                "bytes_formula": "m*(4+4+sv) + nnz*(4+sv) + (n_cols+1)*8", "launch_ms_mean": 1000 * mean_call_s,
                "stage_ms_mean": stage_ms}
    # k_resolve reads the 16-byte bucketed records and writes each bucket's
    # stored elements (row, value); k_place (with its offset scan) reads those
    # and writes the CSC
    res_bytes = m * 16 + nnz * (4 + sv)
    place_bytes = 2 * nnz * (4 + sv) + (n_cols + 1) * 8
    kernel_rooflines = []
    for name, stage, nbytes, formula in (("k_resolve", "resolve", res_bytes, "m*16 + nnz*(4+sv)"),
                                         ("k_place (+ offset scan)", "place", place_bytes,
                                          "2*nnz*(4+sv) + (n_cols+1)*8")):
        if stage in stage_ms and stage_ms[stage] > 0:
            a = nbytes / (stage_ms[stage] / 1000.0) / 1e9
            kernel_rooflines.append({"kernel": name, "bound": "hbm", "achieved": a, "peak": peak, "unit": "GB/s",
                                     "frac": a / peak, "algorithmic_bytes_per_launch": nbytes,
                                     "bytes_formula": formula, "launch_ms_mean": stage_ms[stage],
                                     "traffic": profiled_traffic(args.workload, f"{stage}_dram_bytes_per_launch")})

    # ---- end to end through the public API: pinned host buffers, copies
    # inside the timed region.  Consecutive steps overlap as a user streaming
    # batches would run them: the inputs of step k+1 travel to the device
    # while step k assembles and the CSC of step k-1 travels back; step k-1's
    # stored-element count is read once its call has ended, with step k
    # already queued behind it. ----
    e2e_steps = args.e2e_steps or min(args.steps, 20)
    e2e_value, d2h, h2d = run_e2e(spm, asm, d, rows, cols, vals, nnz, e2e_steps, args, world, dev)

    # ---- CPU oracle baseline (rank 0, N = 1 only) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.profile:
        sample = min(args.cpu_sample, m)
        rate, dt = oracle_rate(d, spec["mode"], sample)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
               "sample": f"first {sample} of the {m} writes of this stream, std::map build + in-order walk, "
                         f"1 thread, {dt:.1f} s"}

    clocks = sampler.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if sv == 8 else "f32", "data": "synthetic",
            "config": {"workload": args.workload, "description": spec["desc"], "m": m, "n_rows": n_rows,
                       "n_cols": n_cols, "nnz": nnz, "mode": spec["mode"],
                       "l2": ("a 512 MB write flushes the 129 MB L2 before every step (outside the step's "
                              "events); rate over the steps' event times") if flush_l2 else
                             "inputs larger than the 129 MB L2 (no flush between steps)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "kernel_rooflines": kernel_rooflines,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps, "overlap": "H2D of step k+1, call k and D2H of step k-1 on three streams"},
            "clocks": clocks,
            "gpu_launches": launches,
            "gpu": torch.cuda.get_device_name(dev),
            "source_hash": source_hash(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
