#!/usr/bin/env python3
"""Benchmark of the trident SpGEMM hot path on GB300.

Default workload (N=1): C = A B with A, B independent Erdos-Renyi CSR
matrices, n = 2^20, 16 nonzeros per row at distinct uniform columns, float64
values U(-1, 1), seeds 0 / 1 (268,435,456 intermediate products).  One step =
the whole product: analysis + symbolic + scan (+ nnz read back) + numeric.
Metric: SpGEMM GFLOP/s = 2 x intermediate products / second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                  [--n-log2 L] [--d D] [--no-cpu-baseline] [--no-e2e] [--no-extras]

The JSON line carries the roofline of the numeric kernel (achieved
algorithmic bytes per launch over its CUDA-event time, the measured peak,
the DRAM traffic of the committed ncu capture while the kernel sources match
it, and the per-product streaming model), the library's phase times, the
oracle on the host cores (cpu_baseline), the same product end to end from
pinned host memory (e2e), and, unless --no-extras, a "workloads" object with
one entry per further workload: the small ER case, the single-pass product,
the trident grid, 256 independent products, autograd, the restriction
operator, the permuted banded matrix with its trident loads and volumes, and
Markov clustering.  Rank 0 prints exactly one JSON line.

Under torchrun (N > 1) every rank runs its own replica of the workload
(independent problems, no collective on the data path); the time is the max
over ranks and the value counts all ranks' products.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpGEMM GFLOP/s (2x intermediate products/s)"
UNIT = "GFLOP/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["native", "reference"], default="native")
    p.add_argument("--n-log2", type=int, default=20)
    p.add_argument("--d", type=int, default=16)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--extras", dest="extras", action="store_true", default=True,
                   help="also time the trident grid, 256 products and the autograd workload")
    p.add_argument("--no-extras", dest="extras", action="store_false")
    p.add_argument("--only", default=None,
                   help="run one further workload alone (e.g. many_products, trident_grid) and print its entry")
    p.add_argument("--trident-n-log2", type=int, default=21,
                   help="n = 2^L of the trident-grid workload (smaller for profiling)")
    p.add_argument("--many-count", type=int, default=256,
                   help="products of the many_products workload (the first N of the 256; smaller for profiling)")
    return p.parse_args()


def workload(args):
    import gen
    n = 1 << args.n_log2
    A = gen.er(n, n, args.d, 0, np.float64)
    B = gen.er(n, n, args.d, 1, np.float64)
    return n, A, B


def workload_name(args) -> str:
    return f"ER A*B n=2^{args.n_log2} d={args.d} f64 (seeds 0/1), plain product"


def products(A, B) -> int:
    return int(np.diff(B.rowptr)[A.col].sum())


def algorithmic_bytes(A, B, nnz_c: int, val_bytes: int = 8):
    """Compulsory bytes of the numeric pass (read A and B once, read C's
    row_ptr, write C's columns and values) and of the symbolic pass (read the
    index arrays of A and B, write C's row_ptr)."""
    m, k = A.nrows, B.nrows
    numeric = (4 * (m + 1) + A.nnz * (4 + val_bytes) + 4 * (k + 1) + B.nnz * (4 + val_bytes)
               + 4 * (m + 1) + nnz_c * (4 + val_bytes))
    symbolic = 4 * (m + 1) + 4 * A.nnz + 4 * (k + 1) + 4 * B.nnz + 4 * (m + 1)
    return numeric, symbolic


def csr_bytes(nrows: int, nnz: int, val_bytes: int = 8) -> int:
    """Bytes of one CSR matrix: row_ptr (int32) + column indices + values."""
    return 4 * (nrows + 1) + nnz * (4 + val_bytes)


def workload_roofline(alg_bytes: int, ms: float, kernel: str, traffic=None) -> dict:
    """Roofline of one workload's timed launch set: algorithmic (compulsory)
    bytes over the measured time, against the measured HBM peak."""
    peak, kind = peaks()
    gbs = alg_bytes / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
    return {"bound": "hbm", "kernel": kernel, "algorithmic_bytes": int(alg_bytes), "achieved": round(gbs, 1),
            "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4), "peak_source": kind, "traffic": traffic}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        """Start sampling every 50 ms; returns once the first sample arrived
        (at most 5 s), so that the sampler is live when the timed region opens."""
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.monotonic()
            while not self.lines and time.monotonic() - t0 < 5:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def mark(self):
        """Open the timed window."""
        self.t_open = time.monotonic()

    def stop(self):
        """Close the window; summarise the samples taken inside it (or, when
        the window was shorter than one sampling period, the first sample
        after it opened)."""
        if self.proc is None:
            return None
        t_close = time.monotonic()
        time.sleep(0.06)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        t_open = getattr(self, "t_open", 0.0)
        inside = [ln for ts, ln in self.lines if t_open <= ts <= t_close]
        if not inside:
            inside = [ln for ts, ln in self.lines if ts >= t_open][:1]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in inside:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm),
                "window_ms": round((t_close - t_open) * 1e3, 1)}


def measured_traffic():
    """DRAM bytes per launch of the numeric rows kernel from the committed ncu
    capture, or None once the kernel sources differ from the captured ones."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "numeric_traffic.json")) as f:
            d = json.load(f)
        h = hashlib.sha256()
        for fn in d["source_files"]:
            with open(os.path.join(ROOT, fn), "rb") as g:
                h.update(g.read())
        return d["dram_bytes_per_launch_full"] if h.hexdigest() == d["source_sha256"] else None
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_model() -> str:
    """The host CPU's model name (lscpu / /proc/cpuinfo), or the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def _trials(fn, trials: int):
    """One warm-up call, then `trials` timed calls: (mean s, min s)."""
    fn()
    ts = []
    for _ in range(trials):
        t0 = time.perf_counter()
        fn()
        ts.append(time.perf_counter() - t0)
    return float(np.mean(ts)), float(np.min(ts))


def cpu_baseline(A, B, budget_rows: int, trials: int = 6):
    """The oracle, as it stands, on the first ``budget_rows`` rows of A: one
    warm-up and ``trials`` timed runs on all host cores, and the same with a
    single thread on a quarter of those rows.  ``value`` is the all-core mean."""
    import gen
    import oracle
    rows = min(budget_rows, A.nrows)

    def head(r):
        end = int(A.rowptr[r])
        return gen.CSR(r, A.ncols, A.rowptr[:r + 1].copy(), A.col[:end], A.val[:end])

    As = head(rows)
    prods = products(As, B)
    cores = oracle.get_threads()
    mean_all, min_all = _trials(lambda: oracle.spgemm(As, B, with_scale=False), trials)
    rows1 = max(1, rows // 4)
    As1 = head(rows1)
    prods1 = products(As1, B)
    oracle.set_threads(1)
    try:
        mean_1, min_1 = _trials(lambda: oracle.spgemm(As1, B, with_scale=False), trials)
    finally:
        oracle.set_threads(cores)
    g = lambda p, t: round(2 * p / t / 1e9, 4)
    return {"value": g(prods, mean_all), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {rows} of {A.nrows} rows ({prods} products), 1 warm-up + {trials} timed runs",
            "all_cores": {"mean": g(prods, mean_all), "best": g(prods, min_all), "threads": cores},
            "single_thread": {"mean": g(prods1, mean_1), "best": g(prods1, min_1), "threads": 1,
                              "sample": f"first {rows1} rows ({prods1} products)"},
            "cpu_model": cpu_model()}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n, A, B = workload(args)
    import gen
    import oracle
    rows = min(1 << 15, A.nrows)
    end = int(A.rowptr[rows])
    As = gen.CSR(rows, A.ncols, A.rowptr[:rows + 1].copy(), A.col[:end], A.val[:end])
    prods = products(As, B)
    for _ in range(max(args.warmup, 0)):
        oracle.spgemm(As, B, with_scale=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.spgemm(As, B, with_scale=False)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    val = 2 * prods / dt / 1e9
    line = {"metric": METRIC, "value": round(val, 4), "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "parallelism": "single"},
            "cpu_baseline": {"value": round(val, 4), "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": f"first {rows} of {n} rows ({prods} products) per step"},
            "e2e": {"value": round(val, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_native(args):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    __graft_entry__.build()
    import paper_2603_21444_gb300 as tsg

    n, A, B = workload(args)
    prods = products(A, B)
    dA = tsg.DeviceCSR.from_host(A)
    dB = tsg.DeviceCSR.from_host(B)
    h = tsg.Handle()
    stream = torch.cuda.current_stream()
    rp, nnz = tsg.symbolic(dA, dB, h)
    C = tsg.DeviceCSR(n, n, rp, torch.empty(nnz, dtype=torch.int32, device="cuda"),
                      torch.empty(nnz, dtype=torch.float64, device="cuda"))

    # each step writes into the same C: symbolic into C.row_ptr, numeric into C.col / C.val
    import ctypes
    from paper_2603_21444_gb300 import _abi
    a_in, b_in = dA.as_in(), dB.as_in()
    c_out = C.as_out()
    nnz_box = ctypes.c_int64()
    L = _abi.lib()
    sptr = ctypes.c_void_p(stream.cuda_stream)

    def step():
        _abi.check(L.spgemm_symbolic(h.ptr, ctypes.byref(a_in), ctypes.byref(b_in), ctypes.c_void_p(c_out.row_ptr),
                                     ctypes.byref(nnz_box), sptr), "symbolic")
        _abi.check(L.spgemm_numeric(h.ptr, _abi.F64, ctypes.byref(a_in), ctypes.byref(b_in), ctypes.byref(c_out),
                                    sptr), "numeric")

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    h.read_timing()
    h.set_timing(True)
    launches0 = h.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    launches = h.launch_count() - launches0
    h.set_timing(False)
    phase_ms, phase_cnt = h.read_timing()
    ms, all_prods = combine_over_ranks(ms, prods, "cuda")
    value = 2 * all_prods / (ms * 1e-3) / 1e9

    # roofline of the dominant kernel (numeric rows): algorithmic bytes per launch / duration
    num_bytes, sym_bytes = algorithmic_bytes(A, B, nnz)
    peak, peak_kind = peaks()
    num_ms = phase_ms[3] / max(phase_cnt[3], 1)
    sym_ms = phase_ms[1] / max(phase_cnt[1], 1)
    achieved = num_bytes / (num_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": "k_num_rows<32, 8, double> (numeric rows, warp team)",
            "achieved": round(achieved, 1),
            "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": measured_traffic() if args.n_log2 == 20 and args.d == 16 else None,
            "peak_source": peak_kind, "algorithmic_bytes": num_bytes, "launch_ms": round(num_ms, 4)}
    # streaming (per-product) model: every B-row gather misses cache -- 4 B
    # per product in the symbolic pass, 4 + 8 B per product in the numeric one
    stream_bytes = prods * (4 + 12)
    roof["streaming_model"] = {"bytes_per_step": stream_bytes,
                               "achieved_gbs": round(stream_bytes / (ms * 1e-3) / 1e9, 1),
                               "frac": round(stream_bytes / (ms * 1e-3) / 1e9 / peak, 4)}
    phases = {"analysis_ms": phase_ms[0] / args.steps, "symbolic_rows_ms": sym_ms, "scan_ms": phase_ms[2] / args.steps,
              "numeric_rows_ms": num_ms, "heavy_ms": phase_ms[4] / args.steps,
              "symbolic_frac_of_hbm": round(sym_bytes / (sym_ms * 1e-3) / 1e9 / peak, 4) if sym_ms > 0 else None}

    single = None
    if rank == 0 and args.extras:
        single = bench_single_pass(tsg, h, dA, dB, prods, nnz, min(args.steps, 20), stream)

    e2e = None
    if not args.no_e2e and rank == 0:
        e2e = e2e_public_api(tsg, A, B, prods, args)

    if rank == 0:
        cb = None
        if not args.no_cpu_baseline and world == 1:
            cb = cpu_baseline(A, B, 1 << 18)
        line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_name(args),
                           "parallelism": "replicas" if world > 1 else "single",
                           "products": prods, "nnz_c": nnz, "l2": "inputs+outputs > L2 (C = "
                           f"{nnz * 12 / 1e9:.2f} GB written per step)"},
                "roofline": roof, "phases": {k: (round(v, 4) if isinstance(v, float) else v)
                                              for k, v in phases.items()},
                "single_pass": single, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
        if args.extras and world == 1:
            extras = {}
            for name in EXTRAS:
                try:
                    extras[name] = extra_fn(name)(tsg, 3)
                except Exception as ex:  # report, keep the main line
                    extras[name] = {"error": f"{type(ex).__name__}: {ex}"}
            line["workloads"] = extras
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def bench_single_pass(tsg, h, dA, dB, prods, nnz, steps, stream):
    """The same product through spgemm_fused: one numeric pass whose row
    offsets come from a decoupled look-back, output buffers preallocated at
    capacity nnz(C); checked against the two-pass result's size."""
    import ctypes

    import torch
    from paper_2603_21444_gb300 import _abi
    C = tsg.DeviceCSR(dA.nrows, dB.ncols, torch.empty(dA.nrows + 1, dtype=torch.int32, device="cuda"),
                      torch.empty(nnz, dtype=torch.int32, device="cuda"),
                      torch.empty(nnz, dtype=torch.float64, device="cuda"))
    a_in, b_in, c_out = dA.as_in(), dB.as_in(), C.as_out()
    box = ctypes.c_int64()
    L = _abi.lib()
    sptr = ctypes.c_void_p(stream.cuda_stream)

    def step():
        _abi.check(L.spgemm_fused(h.ptr, _abi.F64, ctypes.byref(a_in), ctypes.byref(b_in), ctypes.byref(c_out),
                                  ctypes.c_int64(nnz), ctypes.byref(box), sptr), "spgemm_fused")

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    if box.value != nnz:
        return {"error": f"nnz {box.value} != {nnz}"}
    h.read_timing()
    h.set_timing(True)
    ms = _time(step, steps, warmup=0)
    h.set_timing(False)
    phase_ms, phase_cnt = h.read_timing()
    return {"value": round(2 * prods / (ms * 1e-3) / 1e9, 2), "unit": UNIT, "ms_per_step": round(ms, 4),
            "numeric_fused_ms": round(phase_ms[3] / max(phase_cnt[3], 1), 4),
            "analysis_ms": round(phase_ms[0] / max(steps, 1), 4), "steps": steps}


def combine_over_ranks(ms: float, units: float, device: str = "cpu"):
    """(max of the ranks' step times, sum of the ranks' units): the job's
    time is its slowest rank's, its work the work of all ranks.  One rank
    (or no process group) returns its own values."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, units
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def e2e_public_api(tsg, A, B, prods, args):
    """Same metric through the public API with host inputs and output:
    ``spgemm_host`` on page-locked A, B, every step copying both in, sizing,
    computing C in row panels and copying each panel of C back to pinned
    host memory while the next panels run.  The same product through the
    device API with the copies issued one after another is reported beside
    it (``serial_ms_per_step``)."""
    import torch
    hA = tsg.DeviceCSR.from_host(A, device="cpu", pin=True)
    hB = tsg.DeviceCSR.from_host(B, device="cpu", pin=True)
    h = tsg.Handle()
    box = {}

    def step():
        box["C"] = tsg.spgemm_host(hA, hB, h, panels=8, out=box.get("C"))
        return box["C"].nnz

    nnz = step()
    torch.cuda.synchronize()
    steps = min(max(3, args.steps // 4), 10)
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    out = {}

    def serial():
        dA = tsg.DeviceCSR(A.nrows, A.ncols, hA.row_ptr.to("cuda", non_blocking=True),
                           hA.col.to("cuda", non_blocking=True), hA.val.to("cuda", non_blocking=True))
        dB = tsg.DeviceCSR(B.nrows, B.ncols, hB.row_ptr.to("cuda", non_blocking=True),
                           hB.col.to("cuda", non_blocking=True), hB.val.to("cuda", non_blocking=True))
        C = tsg.spgemm(dA, dB, h)
        C2 = box["C"]
        C2.row_ptr.copy_(C.row_ptr, non_blocking=True)
        C2.col.copy_(C.col, non_blocking=True)
        C2.val.copy_(C.val, non_blocking=True)

    serial()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        serial()
    torch.cuda.synchronize()
    dts = (time.perf_counter() - t0) / steps
    h2d = sum(int(t.numel() * t.element_size()) for t in (hA.row_ptr, hA.col, hA.val, hB.row_ptr, hB.col, hB.val))
    d2h = (A.nrows + 1) * 4 + nnz * 12
    h.close()
    return {"value": round(2 * prods / dt / 1e9, 2), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": round(dt * 1e3, 3), "steps": steps,
            "api": "spgemm_host (8 row panels, copies overlapped)", "serial_ms_per_step": round(dts * 1e3, 3)}


def _time(fn, steps, warmup=1, stream=None):
    """Mean ms of fn() over `steps` calls (CUDA events, after warm-up)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def bench_trident(tsg, steps, n_log2=21):
    """ER A, B with n = 2^21 and 32 per row, float64, on the trident grid
    4 x 4 x lambda=4: 256 block products, 64 output blocks of 4 rounds
    (n_log2 < 21: a smaller grid of the same shape, for profiling)."""
    import torch
    import gen
    n, d, q, lam = 1 << n_log2, 32, 4, 4
    A = gen.er(n, n, d, 4)
    B = gen.er(n, n, d, 5)
    prods = products(A, B)
    dA, dB = tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(B)
    del A, B
    h = tsg.Handle()
    t_split = _time(lambda: tsg.TridentPlan(dA, dB, q, lam, h), 1, warmup=1)
    plan = tsg.TridentPlan(dA, dB, q, lam, h)
    out = {"workload": f"ER A*B n=2^{n_log2} d=32 f64, trident 4x4x4 (256 block products, 64 blocks)",
           "products": prods, "partition_ms": round(t_split, 3)}
    # fused, persistent: sized once, numeric replayed from a CUDA graph
    fp = plan.fused_plan()
    # bins one after another, then concurrent (the default)
    fp.set_concurrent_bins(False)
    fp.execute(True)
    out["batched_graph_sequential_bins_ms"] = round(_time(lambda: fp.execute(True), steps), 3)
    fp.set_concurrent_bins(True)
    fp.execute(True)
    torch.cuda.synchronize()
    t_replay = _time(lambda: fp.execute(True), steps)
    out["batched_graph_ms"] = round(t_replay, 3)
    out["batched_graph_gflops"] = round(2 * prods / t_replay / 1e6, 2)
    out["nnz_c"] = int(sum(fp.nnz))
    # compulsory bytes of one replay: every A slice and B tile read once, the
    # 64 output blocks (row_ptr, columns, values) written once
    in_bytes = sum(csr_bytes(T.nrows, T.nnz) for row in plan.A_tiles + plan.B_tiles for T in row)
    out_bytes = sum(csr_bytes(C.nrows, C.nnz) for C in fp.C)
    out["roofline"] = workload_roofline(in_bytes + out_bytes, t_replay,
                                        "fused plan replay (k_num_rows per bin, one CUDA graph)")
    # the per-bin autotuner on the same plan
    tuned = fp.autotune()
    fp.execute(True)
    t_tuned = _time(lambda: fp.execute(True), steps)
    out["batched_graph_autotuned_ms"] = round(t_tuned, 3)
    out["autotune"] = {"num_bins": tuned.num_bins, "bin_upper": list(tuned.bin_upper)[:tuned.num_bins],
                       "bin_kernel": list(tuned.bin_kernel)[:tuned.num_bins],
                       "warps_per_block": tuned.warps_per_block}
    # fused, fresh: sizing + numeric every step
    fresh = lambda: tsg.Plan(plan.As, plan.Bs, plan.group_ptr).execute(False)
    t_fresh = _time(fresh, max(1, steps // 4))
    out["batched_fresh_ms"] = round(t_fresh, 3)
    out["batched_fresh_gflops"] = round(2 * prods / t_fresh / 1e6, 2)
    # fresh adds the sizing pass, which reads the index arrays once more
    idx_bytes = sum(4 * (T.nrows + 1) + 4 * T.nnz for row in plan.A_tiles + plan.B_tiles for T in row)
    out["roofline_fresh"] = workload_roofline(in_bytes + out_bytes + idx_bytes, t_fresh,
                                              "fused plan, sized every call")
    del fp
    plan.fused = None
    torch.cuda.empty_cache()
    # unfused: partials materialised, then one ordered merge per block
    t_unf = _time(lambda: plan.run_unfused(), 1)
    out["unfused_ms"] = round(t_unf, 3)
    plan.partials = None
    torch.cuda.empty_cache()
    # plain: the per-block loop, one product call per round, one merge per block
    t_plain = _time(lambda: plan.run_plain(), 1, warmup=0)
    out["plain_per_block_ms"] = round(t_plain, 3)
    out["plain_per_block_gflops"] = round(2 * prods / t_plain / 1e6, 2)
    out["speedup_batched_fresh_vs_plain"] = round(t_plain / t_fresh, 2)
    out["speedup_batched_graph_vs_plain"] = round(t_plain / t_replay, 2)
    h.close()
    torch.cuda.empty_cache()
    return out


def bench_many(tsg, steps, count=256):
    """256 independent ER products, n log-uniform in [2^10, 2^16], 4..64 per
    row, float64: one plan (one graph launch) against 256 product calls.
    count < 256 takes the first `count` products (profiling runs)."""
    import torch
    import gen
    pairs = gen.er_batch(256)[:count]
    prods = sum(products(a, b) for a, b in pairs)
    As = [tsg.DeviceCSR.from_host(a) for a, _ in pairs]
    Bs = [tsg.DeviceCSR.from_host(b) for _, b in pairs]
    h = tsg.Handle()
    plan = tsg.Plan(As, Bs)
    plan.set_concurrent_bins(False)
    sequential_ms = _time(lambda: plan.execute(True), steps)
    plan.set_concurrent_bins(True)
    default_ms = _time(lambda: plan.execute(True), steps)
    # the block-team bins with their B rows staged in shared memory by TMA
    staged = tsg.default_tune()
    for b in range(staged.num_bins):
        if staged.bin_kernel[b] in (11, 12, 13, 14):
            staged.bin_kernel[b] += 5
    splan = tsg.Plan(As, Bs, tune=staged)
    staged_ms = _time(lambda: splan.execute(True), steps)
    splan.close()
    del splan
    # compulsory bytes of one replay: each A_t, B_t read once, each C_t written once
    alg = sum(csr_bytes(a.nrows, a.nnz) + csr_bytes(b.nrows, b.nnz) for a, b in zip(As, Bs))
    alg += sum(csr_bytes(C.nrows, C.nnz) for C in plan.C)
    nnz_c = int(sum(plan.nnz))
    tuned = plan.autotune()
    plan.execute(True)
    tuned_ms = _time(lambda: plan.execute(True), steps)
    fresh_ms = _time(lambda: tsg.Plan(As, Bs).execute(False), max(1, steps // 4))
    loop_ms = _time(lambda: [tsg.spgemm(a, b, h) for a, b in zip(As, Bs)], 1)
    best = min(default_ms, tuned_ms)
    name = "256 ER products, n=2^U(10,16), d=U{4..64}, f64"
    if count < 256:
        name += f" (first {count})"
    out = {"workload": name, "products": prods, "nnz_c": nnz_c,
           "batched_graph_ms": round(default_ms, 3), "batched_graph_autotuned_ms": round(tuned_ms, 3),
           "batched_graph_sequential_bins_ms": round(sequential_ms, 3),
           "batched_graph_tma_staged_ms": round(staged_ms, 3),
           "roofline": workload_roofline(alg, best, "plan replay (k_num_rows per bin, one CUDA graph)"),
           "autotune": {"num_bins": tuned.num_bins, "bin_upper": list(tuned.bin_upper)[:tuned.num_bins],
                        "bin_kernel": list(tuned.bin_kernel)[:tuned.num_bins],
                        "warps_per_block": tuned.warps_per_block},
           "batched_fresh_ms": round(fresh_ms, 3), "plain_256_calls_ms": round(loop_ms, 3),
           "batched_graph_gflops": round(2 * prods / min(default_ms, tuned_ms) / 1e6, 2),
           "speedup_batched_fresh_vs_plain": round(loop_ms / fresh_ms, 2)}
    plan.close()
    h.close()
    return out


def bench_autograd(tsg, steps):
    """A 2^18 x 2^18, B 2^18 x 2^16, 16 per row, float32 N(0,1); loss =
    sum(C * W): forward and hand-written backward on fixed patterns."""
    import torch
    import gen
    from paper_2603_21444_gb300 import autograd as ag
    A = gen.er(1 << 18, 1 << 18, 16, 5, np.float32, "normal")
    B = gen.er(1 << 18, 1 << 16, 16, 6, np.float32, "normal")
    prods = products(A, B)
    dA, dB = tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(B)
    h = tsg.Handle()
    pat = ag.Pattern(dA, dB, h)
    a = dA.val.clone().requires_grad_(True)
    b = dB.val.clone().requires_grad_(True)
    W = torch.randn(pat.C.nnz, device="cuda", generator=torch.Generator(device="cuda").manual_seed(5))

    def fwd():
        return ag.spgemm_values(a, b, pat)

    def fwd_bwd():
        a.grad = None
        b.grad = None
        (fwd() * W).sum().backward()

    fwd_ms = _time(fwd, steps)
    fb_ms = _time(fwd_bwd, steps)
    c = fwd()
    g = W
    bwd_ms = _time(lambda: ag.backward(dA, dB, pat.C, g, handle=h), steps)
    det_ms = _time(lambda: ag.backward(dA, dB, pat.C, g, deterministic=True, handle=h), max(1, steps // 2))
    fresh_ms = _time(lambda: tsg.spgemm(dA, dB, h), steps)
    h.close()
    del c
    return {"workload": "A 2^18x2^18, B 2^18x2^16, d=16, f32, loss sum(C*W)", "products": prods,
            "nnz_c": pat.C.nnz, "forward_ms": round(fwd_ms, 3), "forward_with_sizing_ms": round(fresh_ms, 3),
            "backward_ms": round(bwd_ms, 3), "backward_deterministic_ms": round(det_ms, 3),
            "fwd_plus_bwd_ms": round(fb_ms, 3), "forward_gflops": round(2 * prods / fwd_ms / 1e6, 2)}


def bench_small(tsg, steps):
    """The small ER case: C = A A, n = 4096, 8 per row, float64 -- launch
    and latency bound, so reported in microseconds per call (symbolic +
    numeric through the C ABI into a preallocated C)."""
    import ctypes

    import torch
    import gen
    from paper_2603_21444_gb300 import _abi
    A = gen.er(4096, 4096, 8, 0)
    prods = products(A, A)
    dA = tsg.DeviceCSR.from_host(A)
    h = tsg.Handle()
    C = tsg.spgemm(dA, dA, h)
    a_in, c_out = dA.as_in(), C.as_out()
    box = ctypes.c_int64()
    L = _abi.lib()
    sptr = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def step():
        _abi.check(L.spgemm_symbolic(h.ptr, ctypes.byref(a_in), ctypes.byref(a_in), ctypes.c_void_p(c_out.row_ptr),
                                     ctypes.byref(box), sptr), "symbolic")
        _abi.check(L.spgemm_numeric(h.ptr, _abi.F64, ctypes.byref(a_in), ctypes.byref(a_in), ctypes.byref(c_out),
                                    sptr), "numeric")

    ms = _time(step, max(steps, 50), warmup=5)
    # the same product sized once and replayed from a CUDA graph (numeric only)
    plan = tsg.Plan([dA], [dA])
    plan.execute(True)
    ms_replay = _time(lambda: plan.execute(True), max(steps, 50), warmup=5)
    plan.close()
    h.close()
    return {"workload": "ER A*A n=4096 d=8 f64 (seed 0)", "products": prods, "nnz_c": C.nnz,
            "us_per_call": round(ms * 1e3, 2), "gflops": round(2 * prods / ms / 1e6, 2),
            "plan_replay_us": round(ms_replay * 1e3, 2)}


def bench_restriction(tsg, steps):
    """C = A R: A the main ER matrix (n = 2^20, 16 per row, float64), R an
    unsmoothed-aggregation restriction operator (n x n/4, one entry per
    row); sized and computed every step."""
    import ctypes

    import torch
    import gen
    from paper_2603_21444_gb300 import _abi
    n = 1 << 20
    A = gen.er(n, n, 16, 0)
    R = gen.aggregation(n, 4, 7)
    prods = products(A, R)
    dA, dR = tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(R)
    h = tsg.Handle()
    C = tsg.spgemm(dA, dR, h)
    a_in, r_in, c_out = dA.as_in(), dR.as_in(), C.as_out()
    box = ctypes.c_int64()
    L = _abi.lib()
    sptr = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def step():
        _abi.check(L.spgemm_symbolic(h.ptr, ctypes.byref(a_in), ctypes.byref(r_in), ctypes.c_void_p(c_out.row_ptr),
                                     ctypes.byref(box), sptr), "symbolic")
        _abi.check(L.spgemm_numeric(h.ptr, _abi.F64, ctypes.byref(a_in), ctypes.byref(r_in), ctypes.byref(c_out),
                                    sptr), "numeric")

    ms = _time(step, max(steps, 10), warmup=3)
    h.close()
    return {"workload": "C = A R, A ER n=2^20 d=16 f64, R aggregation n x n/4 (ratio 4, seed 7)",
            "products": prods, "nnz_c": C.nnz, "ms": round(ms, 4), "gflops": round(2 * prods / ms / 1e6, 2)}


def bench_permutation(tsg, steps):
    """Random relabelling of a banded matrix (Sec. 5, permuted HV15R):
    the permutation kernel's time, the trident imbalance (max / mean nnz per
    process at P = 256, lambda = 4) before and after, and the product A A
    of each on one GPU."""
    import torch
    import gen
    n = 1 << 20
    X = gen.banded(n, [-(n // 4), 0, n // 4], 4, 8)
    dX = tsg.DeviceCSR.from_host(X)
    h = tsg.Handle()
    rp = torch.from_numpy(gen.random_permutation(n, 9)).cuda()
    cp = torch.from_numpy(gen.random_permutation(n, 10)).cuda()
    Y = tsg.permute(dX, rp, cp, h)
    ms_perm = _time(lambda: tsg.permute(dX, rp, cp, h), max(steps, 5), warmup=1)
    moved = 2 * (X.nnz * 12 + 4 * (n + 1)) + 8 * n
    out = {"workload": f"banded n=2^20, bands at 0 and +-n/4, half-width 4 ({X.nnz} nnz), f64; symmetric random "
                       "relabelling of rows and columns",
           "permute_ms": round(ms_perm, 4), "permute_gbs": round(moved / ms_perm / 1e6, 1)}
    from paper_2603_21444_gb300 import volume
    for name, M in (("banded", dX), ("permuted", Y)):
        lo = tsg.trident_loads(M, 8, 4, h)
        loads = np.array(lo, dtype=np.float64)
        out[f"imbalance_{name}_P256"] = round(float(loads.max() / loads.mean()), 3)
        # Alg. 1 volumes per emulated process at P = 256 (A = B = M), against Prop. 1
        s = volume.summarize(volume.trident_volumes(lo, lo, 8, 4), 8, 4)
        model = volume.prop1_volumes(X.nnz, 256, 4)
        out[f"gi_max_over_prop1_{name}"] = round(s["gi"]["max"] / model["total_gi"], 3)
        out[f"li_max_over_prop1_{name}"] = round(s["li"]["max"] / model["total_li"], 3)
        C = tsg.spgemm(M, M, h)
        ms = _time(lambda: tsg.spgemm(M, M, h), max(steps, 3), warmup=1)
        out[f"product_{name}_ms"] = round(ms, 3)
        del C
    out["products"] = products(X, X)
    out["product_banded_gflops"] = round(2 * out["products"] / out["product_banded_ms"] / 1e6, 2)
    out["product_permuted_gflops"] = round(2 * out["products"] / out["product_permuted_ms"] / 1e6, 2)
    h.close()
    return out


def bench_mcl(tsg, steps):
    """Markov clustering on an R-MAT graph (scale 20, edge factor 16, a=0.57,
    b=c=0.19, symmetrised, self-loops, duplicates removed, column-stochastic
    float32): 3 iterations of expansion fused with inflation 2, pruning below
    1e-4, top-1000 per column and renormalisation."""
    import torch
    import gen
    Mt = gen.rmat_stochastic(scale=20, edge_factor=16, seed=3)
    cur = tsg.DeviceCSR.from_host(Mt)
    h = tsg.Handle()
    # one untimed call sizes the handle's workspaces (accumulators, staging)
    tsg.mcl_step(cur, handle=h)
    torch.cuda.synchronize()
    iters = []
    for it in range(3):
        rp = cur.row_ptr.cpu().numpy().astype(np.int64)
        col = cur.col.cpu().numpy()
        prods = int(np.diff(rp)[col].sum())
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        nxt = tsg.mcl_step(cur, handle=h)
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        # compulsory: the iterate read once (it is both factors), the kept
        # entries written once; streaming: 8 B (column + value) per product
        alg = csr_bytes(cur.nrows, int(rp[-1]), 4) + csr_bytes(cur.nrows, nxt.nnz, 4)
        roof = workload_roofline(alg, ms, "k_mcl_rows / k_mcl_rows_bucket / k_mcl_heavy_* (expansion fused with "
                                          "selection) + k_mcl_collect")
        peak = roof["peak"]
        roof["streaming_model"] = {"bytes": 8 * prods, "achieved_gbs": round(8 * prods / ms / 1e6, 1),
                                   "frac": round(8 * prods / ms / 1e6 / peak, 4)}
        paths, ratio = h.mcl_paths()
        iters.append({"iteration": it + 1, "nnz_in": int(rp[-1]), "products": prods, "ms": round(ms, 3),
                      "gflops": round(2 * prods / ms / 1e6, 2), "nnz_out": nxt.nnz,
                      "rows_per_path": {"per_block": paths[0], "window_summed": paths[1], "batched": paths[2]},
                      "pilot_products_per_column": round(ratio, 2), "roofline": roof})
        cur = nxt
    h.close()
    return {"workload": "MCL on R-MAT scale 20 ef 16, f32 (f64 accumulation), 3 iterations", "iterations": iters,
            "total_ms": round(sum(x["ms"] for x in iters), 3)}


EXTRAS = ("small_er", "trident_grid", "many_products", "autograd", "restriction", "permutation",
          "markov_clustering")


def extra_fn(name):
    return {"small_er": bench_small, "trident_grid": bench_trident, "many_products": bench_many,
            "autograd": bench_autograd, "restriction": bench_restriction, "permutation": bench_permutation,
            "markov_clustering": bench_mcl}[name]


def run_only(args):
    """One further workload alone (profiling runs): builds the library, runs
    it once and prints its entry as one JSON line."""
    import torch

    import __graft_entry__
    if args.only not in EXTRAS:
        raise SystemExit(f"--only: unknown workload {args.only!r}; one of {', '.join(EXTRAS)}")
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    __graft_entry__.build()
    import paper_2603_21444_gb300 as tsg
    fn = extra_fn(args.only)
    if args.only == "many_products":
        res = fn(tsg, args.steps, args.many_count)
    elif args.only == "trident_grid":
        res = fn(tsg, args.steps, args.trident_n_log2)
    else:
        res = fn(tsg, args.steps)
    print(json.dumps({"workload_only": args.only, args.only: res}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        run_only(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
