#!/usr/bin/env python3
"""Benchmark: block decomposition P*A = L*E over F2 of a dense n x n
Bernoulli(1/2) matrix (default n = 32768), the workload of Table 4 of the
paper, on synthetic seeded input.

One step = one full decomposition (every kernel of the path: ingest, panel
pivot selection, Y/L multipliers, M4RM trailing updates, factor output) of
an input already resident in HBM.  The metric is effective GF(2) bit-op/s:
bitops = sum over pivots t of 2 (n - t - 1)(m - q_t - 1), the AND+XOR pairs
of plain elimination (q_t = pivot column of pivot t).

Prints ONE JSON line (rank 0).  Under torchrun every rank decomposes its own
matrix (independent problems, no collective on the data path: weak scaling).

--impl reference times the plain CPU oracle on this host's cores on a
bounded sample of the same workload (a prefix of the columns), in the same
unit.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import f2gen  # noqa: E402

PAPER_SECONDS_32768 = 11.498  # Table 4, b = 128 recursive, 3.06 GHz Xeon
METRIC = "decomposition GF(2) bit-op/s (P*A = L*E, dense Bernoulli(1/2))"
UNIT = "bit-op/s"


def bitops(n: int, m: int, pivcols: np.ndarray) -> float:
    t = np.arange(len(pivcols), dtype=np.float64)
    q = np.asarray(pivcols, dtype=np.float64)
    return float(np.sum(2.0 * (n - t - 1) * (m - q - 1)))


TILE_WORDS = 4  # words per column tile of the library's working copy


def rest_launch_bytes(n: int, mu: int, rj: np.ndarray, pairs: bool, lookups: bool = False) -> list:
    """Algorithmic bytes of every wide update of one decomposition (a pair's
    head and body launches together): one read and one write (16 B) of every
    word the update touches.  Panel j's
    wide update (or that of the pair j, j+1, j even) covers the rows that are
    not pivots of the panels it applies and the column tiles after the one
    holding word j+2 (j+3 for a pair); a launch happens when its panels have
    pivots and such tiles exist."""
    Rj = np.concatenate([[0], np.cumsum(rj)])
    out = []
    j = 0
    while j < mu:
        np_ = 2 if (pairs and j + 1 < mu) else 1
        rows = n - Rj[j + np_]
        words = mu - TILE_WORDS * ((j + 1 + np_) // TILE_WORDS + 1)
        if rj[j:j + np_].sum() > 0 and words > 0:
            per_word = 64.0 * np_ if lookups else 16.0
            out.append(per_word * max(rows, 0) * words)
        j += np_
    return out


def smem_roofline(lookup_bytes: float, upd_ms: float, clocks: dict):
    """The update's co-bound: table-lookup bytes per second against the shared
    memory bandwidth of the SMs it runs on (128 B/clk each, all SMs but the
    one kept for the panel kernel, at the SM clock sampled under load)."""
    try:
        import torch
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count - 1
    except Exception:
        return None
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz")
    if not mhz or upd_ms <= 0:
        return None
    peak = 128.0 * sms * mhz * 1e6 / 1e9
    achieved = lookup_bytes / (upd_ms / 1000.0) / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "per_word_bytes": "64 per panel (8 lookups of 8 B, c = 8)"}


def rest_traffic(n: int, m: int, kernel: str = "k_rest"):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    capture of this workload, or None when the kernel source changed since
    the capture (or the capture is of another size)."""
    import hashlib
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", f"{kernel}_32768_traffic.json")))
        src = b"".join(open(os.path.join(ROOT, f), "rb").read() for f in t["sources"])
    except Exception:
        return None
    if t.get("n") != n or t.get("m") != m or hashlib.sha256(src).hexdigest() != t.get("source_sha256"):
        return None
    return float(t["bytes_per_launch"])


def workload_name(n, m):
    return f"decompose {n}x{m} Bernoulli(1/2), L and E, seed 0x{f2gen.BASE_SEED:x}"


def make_input(n: int, m: int, tag: int) -> np.ndarray:
    return f2gen.uniform(n, m, f2gen.BASE_SEED, 1, tag)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ oracle

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model Name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_sample(A_rm: np.ndarray, n: int, m: int, seconds: float, cores: int):
    """Times the oracle on a prefix of the columns sized to ~`seconds`."""
    import oracle

    oracle.build()
    cols = 128
    t0 = time.perf_counter()
    out = oracle.ple(A_rm, m, col_limit=cols, nthreads=cores)
    dt = time.perf_counter() - t0
    if dt < seconds / 4:
        cols = int(min(m, max(cols, cols * seconds / max(dt, 1e-3) * 0.8)))
        t0 = time.perf_counter()
        out = oracle.ple(A_rm, m, col_limit=cols, nthreads=cores)
        dt = time.perf_counter() - t0
    return bitops(n, m, out["pivcols"]) / dt, dt, cols


def run_reference(args):
    import oracle

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n, m = args.n, args.m
    A = make_input(n, m, 0)
    oracle.build()
    cores = oracle.max_threads()
    per_step = max(2.0, args.cpu_seconds / 3)
    for _ in range(args.warmup):
        oracle_sample(A, n, m, per_step / 4, cores)
    vals, cols_used, times = [], None, []
    for _ in range(args.steps):
        v, dt, cols = oracle_sample(A, n, m, per_step, cores)
        vals.append(v)
        times.append(dt)
        cols_used = cols
    value = statistics.median(vals)
    sample = f"oracle PLE on the first {cols_used} of {m} columns of the {n}x{m} input (all {n} rows updated)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.median(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": workload_name(n, m), "n": n, "m": m},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batched

BATCH_METRIC = "batched decomposition matrices/s (P*A = L*E each)"


def batch_matrices(count: int, p: float, seed: int, dev):
    """The batched workload: count matrices, rows and columns uniform in
    [64, 2048], entries Bernoulli(p); every second matrix made rank-deficient
    (its rows after a random r are XORs of two of its first r rows).  Made on
    the GPU with torch's seeded generator (inputs only); returns row-major
    int64 word tensors and their column counts."""
    import torch
    g = torch.Generator(device=dev).manual_seed(seed)
    sizes = torch.randint(64, 2049, (count, 2), generator=g, device=dev).cpu().tolist()
    mats = []
    for i, (n, m) in enumerate(sizes):
        mu = (m + 63) // 64
        bits = torch.rand((n, mu * 64), generator=g, device=dev) < p
        bits[:, m:] = False
        w = (bits.view(n, mu, 64).to(torch.int64) << torch.arange(64, device=dev)).sum(-1)
        if i % 2 == 1:
            r = int(torch.randint(1, min(n, m) + 1, (1,), generator=g, device=dev).item())
            if r < n:
                a = torch.randint(0, r, (n - r,), generator=g, device=dev)
                b = torch.randint(0, r, (n - r,), generator=g, device=dev)
                w[r:] = w[a] ^ w[b]
        mats.append((w, n, m))
    return mats


def run_batched(args):
    import torch

    import paper_1209_5198_gb300 as gf2
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    count = args.batch
    lib = gf2.load()
    stream = torch.cuda.current_stream()
    # the table size per matrix size, measured by the library's autotuner
    tune = {}
    c8_from = gf2.batched_autotune(2048, times=tune)
    results = {}
    for p, seed in ((0.5, 0x1209), (0.1, 0x5198)):
        mats = batch_matrices(count, p, seed, dev)
        As = [gf2.Mat(w.t().contiguous(), n, m) for w, n, m in mats]
        perms = [torch.empty(n, dtype=torch.int32, device=dev) for _, n, _ in mats]
        pivs = [torch.empty(min(n, m), dtype=torch.int32, device=dev) for _, n, m in mats]
        ranks = torch.zeros(count, dtype=torch.int64, device=dev)
        Ls = [gf2.Mat.empty(n, min(n, m), dev) for _, n, m in mats]
        Es = [gf2.Mat.empty(min(n, m), m, dev) for _, n, m in mats]
        ns = [n for _, n, _ in mats]
        ms = [m for _, _, m in mats]
        import ctypes
        wsb = lib.gf2_decompose_batched_workspace_bytes(count, (ctypes.c_int64 * count)(*ns),
                                                        (ctypes.c_int64 * count)(*ms), 1)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)

        def step():
            gf2.gf2_decompose_batched(As, perms, pivs, ranks, Ls, Es, workspace=ws, stream=stream)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_batch = e0.elapsed_time(e1) / args.steps
        # the same batch with 4-bit tables for every matrix (no autotuned split)
        gf2.set_batched_c8_from(1 << 62)
        ws4 = torch.empty(lib.gf2_decompose_batched_workspace_bytes(count, (ctypes.c_int64 * count)(*ns),
                                                                    (ctypes.c_int64 * count)(*ms), 1),
                          dtype=torch.uint8, device=dev)
        step4 = lambda: gf2.gf2_decompose_batched(As, perms, pivs, ranks, Ls, Es, workspace=ws4, stream=stream)
        step4()
        ms_c4 = time_calls(step4, args.steps, stream)
        gf2.set_batched_c8_from(c8_from)
        rk = ranks.cpu().numpy()
        ops = sum(bitops(n, m, pv.cpu().numpy()[: int(r)]) for (_, n, m), pv, r in zip(mats, pivs, rk))
        # the same matrices one plain gf2_decompose call after another
        wsp = torch.empty(lib.gf2_decompose_workspace_bytes(2048, 2048, 1), dtype=torch.uint8, device=dev)
        rk1 = torch.zeros(1, dtype=torch.int64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(count):
            gf2.gf2_decompose(As[i], perms[i], pivs[i], rk1, Ls[i], Es[i], workspace=wsp, stream=stream)
        torch.cuda.synchronize()
        ms_loop = (time.perf_counter() - t0) * 1000
        results[p] = dict(ms=ms_batch, ms_c4=ms_c4, ops=ops, ms_loop=ms_loop,
                          deficient=int(sum(1 for (w, n, m), r in zip(mats, rk) if r < min(n, m))))
    total_ms = sum(r["ms"] for r in results.values())
    total_loop = sum(r["ms_loop"] for r in results.values())
    line = {
        "metric": BATCH_METRIC, "value": 2 * count / (total_ms / 1000), "unit": "matrices/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"batched: 2 batches (p = 0.5, 0.1) of {count} matrices, rows and cols uniform "
                               f"in [64, 2048], every second one rank-deficient; one step = both batches",
                   "per_batch_ms": {str(p): r["ms"] for p, r in results.items()},
                   "c8_from": c8_from,
                   "autotune_ms_4bit_8bit": {str(d): v for d, v in tune.items()},
                   "per_batch_ms_4bit_tables_only": {str(p): r["ms_c4"] for p, r in results.items()},
                   "rank_deficient": {str(p): r["deficient"] for p, r in results.items()}},
        "bitops_per_s": sum(r["ops"] for r in results.values()) / (total_ms / 1000),
        "plain_loop": {"value": 2 * count / (total_loop / 1000), "unit": "matrices/s",
                       "how": "one gf2_decompose call per matrix on the same stream, host clock, one pass"},
        "speedup_vs_plain_loop": total_loop / total_ms,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ product

PRODUCT_METRIC = "GF(2) product bit-op/s (C = A B, square Bernoulli(1/2))"


def rand_words(rows: int, cols: int, g, dev):
    """A rows x cols Bernoulli(1/2) matrix as column blocks of random words
    (cols a multiple of 64), made on the GPU with torch's seeded generator."""
    import torch
    return torch.randint(-(2 ** 63), 2 ** 63 - 1, (cols // 64, rows), dtype=torch.int64, generator=g, device=dev)


def time_calls(fn, steps: int, stream) -> float:
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_wide(args):
    """The wide-panel question (Section 5's wider blocks, Table 4's "rec"
    columns): the trailing update by w = 64 s columns at once is the product
    C ^= Y P with an n x w multiplier matrix Y and w pivot rows P.  Timed
    here with the M4RM kernel alone (C in registers over the inner
    dimension, so C is read and written once per call) at n = m = --n and
    w = 64 .. 1024: the time per 64 columns of w falls while fixed costs per
    call (table builds, C's loads) are amortised and levels off once the
    table lookups (8 of 8 B per output word and 64 columns of w) bound it."""
    import torch

    import paper_1209_5198_gb300 as gf2
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    lib = gf2.load()
    n = args.n
    g = torch.Generator(device=dev).manual_seed(0x1209)
    props = torch.cuda.get_device_properties(0)
    fl = gf2.GF2_MMM_TABLES | gf2.GF2_NOCHECK
    C = gf2.Mat(rand_words(n, n, g, dev), n, n)
    rows = []
    sampler = ClockSampler(0)
    sampler.start()
    for w in (64, 128, 256, 512, 1024):
        Y = gf2.Mat(rand_words(n, w, g, dev), n, w)
        P = gf2.Mat(rand_words(w, n, g, dev), w, n)
        ws = torch.empty(max(1, lib.gf2_mmm_workspace_bytes(n, w, n, fl)), dtype=torch.uint8, device=dev)
        fn = lambda: gf2.gf2_mmm(Y, P, C, accumulate=True, flags=fl, workspace=ws, stream=stream)
        for _ in range(args.warmup):
            fn()
        ms = time_calls(fn, args.steps, stream)
        words = n * (n // 64)
        rows.append({"w": w, "ms": ms, "ms_per_64_columns": ms / (w // 64),
                     "c_gbs": 16.0 * words / (ms / 1000) / 1e9,
                     "lookup_gbs": 8.0 * 8 * (w // 64) * words / (ms / 1000) / 1e9})
    clocks = sampler.stop()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    clk = clocks.get("sm_mhz") or 2070.0
    line = {"metric": "wide-panel trailing update: ms per 64 columns of w (C ^= Y P, M4RM)",
            "value": rows[2]["ms_per_64_columns"], "unit": "ms", "higher_is_better": False,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"C ^= Y P over F2, C {n} x {n}, Y {n} x w, P w x {n}, w = 64..1024 "
                                   "(Bernoulli(1/2)); value = w = 256", "rows": rows,
                       "hbm_peak_gbs": peaks.get("hbm_gbs"),
                       "lookup_peak_gbs": 128.0 * props.multi_processor_count * clk * 1e6 / 1e9},
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_product(args):
    import torch

    import paper_1209_5198_gb300 as gf2
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    lib = gf2.load()
    cutoff = gf2.mmm_autotune(min(32768, max(args.product_sizes)))
    g = torch.Generator(device=dev).manual_seed(0x1209)
    backends = {"m4rm": gf2.GF2_MMM_TABLES, "strassen": 0, "tensor": gf2.GF2_MMM_TENSOR}
    table, main = [], None
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    for n in args.product_sizes:
        A = gf2.Mat(rand_words(n, n, g, dev), n, n)
        B = gf2.Mat(rand_words(n, n, g, dev), n, n)
        outs = {}
        row = {"n": n, "strassen_levels": 0}
        for name, fl in backends.items():
            if name == "tensor" and n > args.tensor_max:
                continue
            C = gf2.Mat.empty(n, n, dev)
            ws = torch.empty(max(1, lib.gf2_mmm_workspace_bytes(n, n, n, fl)), dtype=torch.uint8, device=dev)
            fn = lambda: gf2.gf2_mmm(A, B, C, flags=fl, workspace=ws, stream=stream)
            for _ in range(args.warmup):
                fn()
            steps = args.steps if n <= 32768 else max(1, args.steps // 2)
            if name == "tensor":
                steps = 1
            sampler = None
            if n == 32768 and name == "strassen":
                sampler = ClockSampler(0)
                sampler.start()
                l0 = gf2.launch_count()
            ms = time_calls(fn, steps, stream)
            if sampler:
                row["clocks"] = sampler.stop()
                row["launches_per_step"] = (gf2.launch_count() - l0) / steps
            row[name + "_ms"] = ms
            row[name + "_bitops_per_s"] = 2.0 * n ** 3 / (ms / 1000)
            outs[name] = C.t
        ref = outs["m4rm"]
        row["backends_agree"] = all(bool(torch.equal(ref, t)) for t in outs.values())
        levels, d = 0, n
        while d >= cutoff and levels < 8:
            levels, d = levels + 1, d // 2
        row["strassen_levels"] = levels
        table.append(row)
        if n == 32768:
            main = row
        del A, B, outs
        torch.cuda.empty_cache()
    if main is None:
        main = table[-1]
    n = main["n"]
    # roofline of the M4RM kernel: its shared-memory lookups, n*m*k/64 bytes
    # (8 B per row, output word and 8 bits of the inner dimension)
    clk = (main.get("clocks") or {}).get("sm_mhz") or 2070.0
    lookup_bytes = n ** 3 / 64.0
    achieved = lookup_bytes / (main["m4rm_ms"] / 1000) / 1e9
    peak = 128.0 * sms * clk * 1e6 / 1e9
    # end to end: A and B from pinned host memory, C back, inside the timed region
    Ah = torch.empty((n // 64, n), dtype=torch.int64, pin_memory=True)
    Bh = torch.empty((n // 64, n), dtype=torch.int64, pin_memory=True)
    Ch = torch.empty((n // 64, n), dtype=torch.int64, pin_memory=True)
    Ah.copy_(rand_words(n, n, g, dev))
    Bh.copy_(rand_words(n, n, g, dev))
    Ad, Bd, Cd = torch.empty_like(Ah, device=dev), torch.empty_like(Bh, device=dev), torch.empty_like(Ch, device=dev)
    ws = torch.empty(max(1, lib.gf2_mmm_workspace_bytes(n, n, n, 0)), dtype=torch.uint8, device=dev)

    def e2e_step():
        Ad.copy_(Ah, non_blocking=True)
        Bd.copy_(Bh, non_blocking=True)
        gf2.gf2_mmm(gf2.Mat(Ad, n, n), gf2.Mat(Bd, n, n), gf2.Mat(Cd, n, n), workspace=ws, stream=stream)
        Ch.copy_(Cd, non_blocking=True)

    e2e_step()
    e2e_ms = time_calls(e2e_step, max(1, args.steps // 2), stream)
    cpu = None
    if not args.no_cpu_baseline:
        cpu = product_cpu_sample(n, args.cpu_seconds)
    line = {
        "metric": PRODUCT_METRIC, "value": 2.0 * n ** 3 / (main["strassen_ms"] / 1000), "unit": "bit-op/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": main["strassen_ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"product C = A B, n = k = m = {n}, Bernoulli(1/2) words from torch's seeded "
                               "generator; default backend = M4RM under Strassen-Winograd at the cutoff the "
                               "library's autotuner picked on this GPU", "n": n, "strassen_cutoff": cutoff,
                   "l2": "no flush: A, B and C (3 x n^2/8 bytes) exceed the 129 MB L2 from n = 32768; smaller "
                         "sizes run L2-warm"},
        "sizes": table,
        "roofline": {"kernel": "k_mmm (M4RM product, no recursion)", "bound": "smem", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "alg_bytes_per_launch": lookup_bytes,
                     "peak_source": f"128 B/clk/SM x {sms} SMs x {clk:.0f} MHz (shared-memory bandwidth)"},
        "e2e": {"value": 2.0 * n ** 3 / (e2e_ms / 1000), "unit": "bit-op/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(2 * Ah.numel() * 8), "d2h_bytes_per_step": int(Ch.numel() * 8)},
        "cpu_baseline": cpu,
        "gpu_launches": main.get("launches_per_step"),
        "clocks": main.get("clocks"),
    }
    # the tcgen05 backend against the tensor pipe: the probe of its MMA shape
    # (kind::f8f6f4 128 x 256 x 32 from shared memory) and the measured bf16
    # GEMM rate x 2 (the nominal fp8 / bf16 ratio)
    if main.get("tensor_ms"):
        probe = gf2.tensor_peak(4096)
        tflops = 2.0 * n ** 3 / (main["tensor_ms"] / 1000) / 1e12
        bf16 = measured_peaks().get("bf16_tflops")
        line["tensor_roofline"] = {
            "kernel": "k_umma (tcgen05 kind::f8f6f4, e2m1 operands by TMA, fp32 accumulators in tensor memory)",
            "bound": "tensor", "achieved": tflops, "unit": "TFLOP/s", "peak": probe, "frac": tflops / probe,
            "peak_source": "gf2_tensor_peak probe on this GPU (its MMA shape from shared memory, no loads)",
            "fp8_from_measured_bf16": (2.0 * bf16) if bf16 else None,
            "frac_of_fp8_from_measured_bf16": (tflops / (2.0 * bf16)) if bf16 else None,
            "ms": main["tensor_ms"], "includes": "operand expansion (two kernels) + the tcgen05 kernel"}
    print(json.dumps(line), flush=True)


def measured_peaks() -> dict:
    """The measured peaks of this machine's GPUs ({} when absent)."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def product_cpu_sample(n: int, seconds: float):
    """The oracle's product on the first rows of A (all of B), sized to about
    `seconds`, scaled to bit-op/s."""
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    B = f2gen.uniform(n, n, 0x1209, 1)
    rows = 64
    A = f2gen.uniform(rows, n, 0x1209, 2)
    t0 = time.perf_counter()
    oracle.mmm(A, B, n, n, nthreads=cores)
    dt = time.perf_counter() - t0
    if dt < seconds / 4:
        rows = int(min(n, rows * seconds / max(dt, 1e-3) * 0.8))
        A = f2gen.uniform(rows, n, 0x1209, 2)
        t0 = time.perf_counter()
        oracle.mmm(A, B, n, n, nthreads=cores)
        dt = time.perf_counter() - t0
    return {"value": 2.0 * rows * n * n / dt, "unit": "bit-op/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle product of the first {rows} rows of A with all of B (n = {n}), {dt:.1f} s"}


# ------------------------------------------------------------------ sizes

SIZES_METRIC = "decomposition time and GF(2) bit-op/s across the scale configurations"


def run_sizes(args):
    """The scale configurations of the plain decomposition: square 1024 (the
    single-matrix configuration), 16384, 32768, 65536 Bernoulli(1/2);
    rectangular 16384 x 65536 and 65536 x 16384;
    fixed rank r = n/2 and n - 64 (A = X Y, X n x r and Y r x n Bernoulli(1/2),
    full rank with overwhelming probability, formed with the library's
    product).  Inputs made on the GPU with torch's seeded generator."""
    import torch

    import paper_1209_5198_gb300 as gf2
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    lib = gf2.load()
    g = torch.Generator(device=dev).manual_seed(0x5198)
    cfgs = [(1024, 1024, None), (16384, 16384, None), (32768, 32768, None), (65536, 65536, None), (16384, 65536, None),
            (65536, 16384, None), (16384, 16384, 8192), (16384, 16384, 16320), (32768, 32768, 16384),
            (32768, 32768, 32704)]
    rows = []
    for n, m, r in cfgs:
        if r is None:
            A = gf2.Mat(rand_words(n, m, g, dev), n, m)
        else:
            X = gf2.Mat(rand_words(n, r, g, dev), n, r)  # r is a multiple of 64 here
            Y = gf2.Mat(rand_words(r, m, g, dev), r, m)
            A = gf2.Mat.empty(n, m, dev)
            gf2.gf2_mmm(X, Y, A, flags=gf2.GF2_MMM_TABLES, stream=stream)
            del X, Y
        k = min(n, m)
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        piv = torch.empty(k, dtype=torch.int32, device=dev)
        rk = torch.zeros(1, dtype=torch.int64, device=dev)
        L = gf2.Mat.empty(n, k, dev)
        E = gf2.Mat.empty(k, m, dev)
        ws = torch.empty(lib.gf2_decompose_workspace_bytes(n, m, 1), dtype=torch.uint8, device=dev)
        fn = lambda: gf2.gf2_decompose(A, perm, piv, rk, L, E, workspace=ws, stream=stream)
        for _ in range(max(2, args.warmup)):  # the second call captures the graph
            fn()
        ms = time_calls(fn, 2, stream)
        rank = int(rk.item())
        ops = bitops(n, m, piv.cpu().numpy()[:rank])
        rows.append({"n": n, "m": m, "kind": "fixed rank" if r else "Bernoulli(1/2)", "r_built": r,
                     "rank": rank, "ms": ms, "bitops_per_s": ops / (ms / 1000)})
        if r is None and n == m and n <= 32768:
            # the reduced row echelon form of E (gf2_rref, in place): each
            # timed call starts from a fresh copy of the echelon factor
            E0 = E.t.clone()
            rws = torch.empty(lib.gf2_rref_workspace_bytes(k, m), dtype=torch.uint8, device=dev)
            times = []
            for it in range(2 + 3):
                E.t.copy_(E0)
                t = time_calls(lambda: gf2.gf2_rref(E, piv, workspace=rws, stream=stream), 1, stream)
                if it >= 2:
                    times.append(t)
            rows[-1]["rref_ms"] = min(times)
            del E0, rws
        if n < m:
            # the rank alone: gf2_rank (which ranks the m x n transpose) against
            # the rank-only decomposition of the n x m matrix itself
            rws = torch.empty(lib.gf2_rank_workspace_bytes(n, m), dtype=torch.uint8, device=dev)
            dws = torch.empty(lib.gf2_decompose_workspace_bytes(n, m, 0), dtype=torch.uint8, device=dev)
            f_rank = lambda: gf2.gf2_rank(A, workspace=rws, stream=stream)
            f_direct = lambda: gf2.gf2_decompose(A, perm, piv, rk, None, None, workspace=dws, stream=stream)
            for _ in range(max(2, args.warmup)):
                f_rank()
                f_direct()
            rows[-1]["rank_transposed_ms"] = time_calls(f_rank, 2, stream)
            rows[-1]["rank_direct_ms"] = time_calls(f_direct, 2, stream)
            del rws, dws
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        del A, L, E, ws
        torch.cuda.empty_cache()
    main = next(x for x in rows if x["n"] == 32768 and x["m"] == 32768 and x["r_built"] is None)
    line = {
        "metric": SIZES_METRIC, "value": main["bitops_per_s"], "unit": "bit-op/s", "n_gpus": 1, "steps": 2,
        "warmup": max(2, args.warmup), "ms_per_step": main["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "plain decomposition (L and E) over the scale configurations; value = the "
                               "32768 x 32768 Bernoulli(1/2) case", "configs": rows},
    }
    print(json.dumps(line), flush=True)


SPARSE_METRIC = "decomposition time and GF(2) bit-op/s on the sparse S_n set (i nonzeros per row)"


def run_sparse(args):
    """The paper's sparse low-rank family S_n (Section 7): n x n matrices
    whose every row has exactly i ones at distinct uniform positions
    (f2gen.sparse_rows, seeded; i = 2, 10, 40), n = 16384, 32768, 65536.
    Plain decomposition with L and E, timed like the sizes workload; their
    ranks are below n, so many panels have few pivots (the low-rank path).
    value = the n = 32768, i = 10 case."""
    import torch

    import f2gen
    import paper_1209_5198_gb300 as gf2
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    lib = gf2.load()
    rows = []
    for n in args.sparse_sizes:
        for i in (2, 10, 40):
            A = gf2.Mat.from_rowmajor(f2gen.sparse_rows(n, n, i, f2gen.BASE_SEED, 7), n, device=dev)
            perm = torch.empty(n, dtype=torch.int32, device=dev)
            piv = torch.empty(n, dtype=torch.int32, device=dev)
            rk = torch.zeros(1, dtype=torch.int64, device=dev)
            L = gf2.Mat.empty(n, n, dev)
            E = gf2.Mat.empty(n, n, dev)
            ws = torch.empty(lib.gf2_decompose_workspace_bytes(n, n, 1), dtype=torch.uint8, device=dev)
            fn = lambda: gf2.gf2_decompose(A, perm, piv, rk, L, E, workspace=ws, stream=stream)
            for _ in range(max(2, args.warmup)):  # the second call captures the graph
                fn()
            ms = time_calls(fn, 2, stream)
            rank = int(rk.item())
            ops = bitops(n, n, piv.cpu().numpy()[:rank])
            rows.append({"n": n, "i": i, "rank": rank, "ms": ms, "bitops_per_s": ops / (ms / 1000)})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            del A, L, E, ws
            torch.cuda.empty_cache()
    main = next((x for x in rows if x["n"] == 32768 and x["i"] == 10), rows[-1])
    line = {
        "metric": SPARSE_METRIC, "value": main["bitops_per_s"], "unit": "bit-op/s", "n_gpus": 1, "steps": 2,
        "warmup": max(2, args.warmup), "ms_per_step": main["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"plain decomposition (L and E) of S_n: n x n, i ones per row at distinct uniform "
                               f"positions; value = n {main['n']}, i {main['i']}", "configs": rows},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ F_p

FP_METRIC = "decomposition over F_p: multiply-adds mod p per second (P*A = L*E, uniform residues)"


def run_fp(args):
    """The decomposition over a prime field F_p (the remark after eq.
    (cond:nonsing:Bk)): uniform residues mod p from the seeded generator, n x n
    for n in --fp-sizes, p = 65521 and 2^31 - 1; time per decomposition (L and
    E), and multiply-adds per second counted as sum over pivots t of
    (n - t - 1)(m - q_t).  value = the largest n with p = 65521."""
    import torch

    import f2gen
    import paper_1209_5198_gb300 as gf2
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    lib = gf2.load()
    rows = []
    for n in args.fp_sizes:
        for p in (65521, 2147483647):
            A = torch.from_numpy(f2gen.fp_uniform(n, n, p, f2gen.BASE_SEED, 30).astype(np.int32)).to(dev)
            ws = torch.empty(lib.gf2_fp_decompose_workspace_bytes(n, n), dtype=torch.uint8, device=dev)
            fn = lambda: gf2.fp_decompose(A, p, flags=gf2.GF2_NOCHECK, workspace=ws, stream=stream)
            for _ in range(max(1, args.warmup)):
                out = fn()
            ms = time_calls(fn, 2, stream)
            out = fn()
            torch.cuda.synchronize()
            rank = int(out["rank"].item())
            piv = out["pivcols"].cpu().numpy()[:rank].astype(np.float64)
            t = np.arange(rank, dtype=np.float64)
            madds = float(np.sum((n - t - 1) * (n - piv)))
            rows.append({"n": n, "p": p, "rank": rank, "ms": ms, "madds_per_s": madds / (ms / 1000)})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            del A, ws, out
            torch.cuda.empty_cache()
    main = max((x for x in rows if x["p"] == 65521), key=lambda x: x["n"])
    line = {
        "metric": FP_METRIC, "value": main["madds_per_s"], "unit": "madd/s", "n_gpus": 1, "steps": 2,
        "warmup": max(1, args.warmup), "ms_per_step": main["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32 mod p", "data": "synthetic",
        "config": {"workload": f"decomposition over F_p of n x n uniform residues; value = n {main['n']}, "
                               f"p = {main['p']}", "configs": rows},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving

SERVE_METRIC = "served solves/s (rank + solve requests on resident factors, continuous batching)"


class ServeWorkload:
    """Config 5: `ids` square matrices, n = 2^U with U uniform in [8, 14],
    rounded up to a multiple of 64, entries Bernoulli(1/2) (random words made
    on the GPU with torch's seeded generator, inputs only); `nreq` requests,
    matrix ids Zipf(s = 1.1) over the ids, k uniform in 1..64 right-hand
    sides, B = A X0 (so every right-hand side is consistent; B is formed on
    the GPU with the library's product).  Host buffers (A pinned column
    blocks, B and X per request) stay alive with the object."""

    def __init__(self, nreq: int, ids: int, seed: int):
        import torch

        import paper_1209_5198_gb300 as gf2
        dev = torch.device("cuda", 0)
        rng = np.random.default_rng(seed)
        g = torch.Generator(device=dev).manual_seed(seed)
        self.n = [int(-(-int(round(2.0 ** u)) // 64) * 64) for u in rng.uniform(8, 14, size=ids)]
        self.A, B64 = [], []
        for n in self.n:
            mu = n // 64
            Ad = torch.randint(-(2 ** 63), 2 ** 63 - 1, (mu, n), dtype=torch.int64, generator=g, device=dev)
            X0 = torch.randint(-(2 ** 63), 2 ** 63 - 1, (1, n), dtype=torch.int64, generator=g, device=dev)
            C = gf2.Mat.empty(n, 64, dev)
            gf2.gf2_mmm(gf2.Mat(Ad, n, n), gf2.Mat(X0, n, 64), C)
            Ah = torch.empty((mu, n), dtype=torch.int64, pin_memory=True)
            Ah.copy_(Ad)
            self.A.append(Ah)
            B64.append(C.t[0].cpu().numpy().view(np.uint64).copy())
        zipf = 1.0 / np.arange(1, ids + 1) ** 1.1
        self.key = rng.choice(ids, size=nreq, p=zipf / zipf.sum())
        self.k = rng.integers(1, 65, size=nreq)
        nn = np.array(self.n)[self.key]
        off = np.concatenate([[0], np.cumsum(nn)])
        self.Bpool = np.empty(int(off[-1]), dtype=np.uint64)
        self.Xpool = np.zeros(int(off[-1]), dtype=np.uint64)
        self.req = np.zeros(nreq, dtype=gf2.REQUEST_DTYPE)
        for i in range(nreq):
            kk, n, o = int(self.key[i]), int(nn[i]), int(off[i])
            mask = np.uint64((1 << int(self.k[i])) - 1) if self.k[i] < 64 else ~np.uint64(0)
            np.bitwise_and(B64[kk], mask, out=self.Bpool[o:o + n])
            self.req[i] = (i, kk, n, n, self.A[kk].data_ptr(), n, int(self.k[i]),
                           self.Bpool.ctypes.data + 8 * o, self.Xpool.ctypes.data + 8 * o, 0.0)
        self.nn = nn

    def bytes_per_request(self):
        # right-hand sides in, solutions out; A once per distinct key (a miss)
        h2d = float(np.mean(self.nn) * 8) + sum(self.n[k] ** 2 / 8 for k in set(self.key.tolist())) / len(self.key)
        return h2d, float(np.mean(self.nn) * 8)


def serve_run(w: ServeWorkload, serial: bool, arrivals_us=None, device_bytes: int = 16 << 30):
    """One pass of the request trace through a fresh engine (cold factors).
    Returns (completions, makespan_s, launches, stats)."""
    import paper_1209_5198_gb300 as gf2
    req = w.req.copy()
    w.Xpool[:] = 0
    with gf2.Server(device_bytes, 16384, 16384, max_batch=1024, serial=serial) as s:
        t_first = s.clock_us() + 20000.0  # the engine has the whole trace before the first arrival
        req["arrival_us"] = t_first + (0.0 if arrivals_us is None else np.asarray(arrivals_us))
        l0 = gf2.launch_count()
        s.submit(req)
        done = s.wait_all(len(req), timeout_s=1800)
        launches = gf2.launch_count() - l0
        st = s.stats()
    bad = done[done["status"] != gf2.GF2_OK]
    if len(bad):
        raise RuntimeError(f"{len(bad)} requests failed, first status {int(bad[0]['status'])}")
    makespan = (float(done["done_us"].max()) - t_first) / 1e6
    return done, makespan, launches, st


def latency_ms(done):
    lat = (done["done_us"] - done["arrival_us"]) / 1000.0
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99))


def run_serving(args):
    import torch

    torch.cuda.set_device(0)
    w = ServeWorkload(args.requests, 256, 0x5198)
    rates = [0.25, 0.5, 0.75, 0.9]
    done_sat_serial, span_serial, _, _ = serve_run(w, serial=True)
    cap_serial = len(w.req) / span_serial
    for _ in range(max(0, args.warmup - 1)):
        serve_run(w, serial=False)
    clk = ClockSampler(0)
    clk.start()
    done_sat, span, launches, st = serve_run(w, serial=False)
    clocks = clk.stop()
    verify_serving(w, done_sat, 16)
    cap = len(w.req) / span
    rng = np.random.default_rng(7)
    per_rate = []
    for f in rates:
        lam = f * cap_serial  # requests per second
        arr = np.cumsum(rng.exponential(1e6 / lam, size=len(w.req)))
        d_ours, span_o, _, _ = serve_run(w, serial=False, arrivals_us=arr)
        d_ser, span_s, _, _ = serve_run(w, serial=True, arrivals_us=arr)
        p50, p99 = latency_ms(d_ours)
        s50, s99 = latency_ms(d_ser)
        per_rate.append({"load": f, "offered_per_s": lam, "served_per_s": len(w.req) / span_o,
                         "p50_ms": p50, "p99_ms": p99, "serial_p50_ms": s50, "serial_p99_ms": s99})
    sat_p50, sat_p99 = latency_ms(done_sat)
    h2d, d2h = w.bytes_per_request()
    line = {
        "metric": SERVE_METRIC, "value": cap, "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": span * 1000, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"serving: {len(w.req)} requests, 256 square matrices n = 2^U(8,14) rounded up "
                               "to 64, ids Zipf(1.1), k = 1..64 right-hand sides, B = A X0, cold factors; "
                               "one step = the whole trace, all requests at t = 0 (saturated)",
                   "requests": len(w.req), "distinct_matrices": int(len(set(w.key.tolist()))),
                   "mean_n": float(np.mean(w.nn))},
        "latency_saturated": {"p50_ms": sat_p50, "p99_ms": sat_p99},
        "serial": {"value": cap_serial, "unit": "solves/s",
                   "how": "the same engine with GF2_SERVE_SERIAL: gf2_decompose / gf2_solve one request at a time"},
        "speedup_vs_serial": cap / cap_serial,
        "poisson": per_rate,
        "stats": st,
        "e2e": {"value": cap, "unit": "solves/s", "h2d_bytes_per_step": h2d * len(w.req),
                "d2h_bytes_per_step": d2h * len(w.req)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def verify_serving(w: ServeWorkload, done, count: int):
    """A X = B for `count` sampled requests (host arithmetic: parity of A's
    rows against X, column block by column block)."""
    rng = np.random.default_rng(3)
    small = np.flatnonzero(w.nn <= 4096)  # keeps the host check to a few seconds
    ids = rng.choice(small, size=min(count, len(small)), replace=False)
    for i in ids:
        c = done[done["id"] == i][0]
        kk, n, k = int(w.key[i]), int(w.nn[i]), int(w.k[i])
        assert int(c["consistent"]) == ((1 << k) - 1 if k < 64 else (1 << 64) - 1), i
        A = w.A[kk].numpy().view(np.uint64)  # column blocks (n/64, n)
        o = int(w.req[i]["X"] - w.Xpool.ctypes.data) // 8
        X = w.Xpool[o:o + n]
        B = w.Bpool[o:o + n]
        acc = np.zeros(n, dtype=np.uint64)
        for q in range(n // 64):  # acc[row] ^= XOR of X[64q + t] over the set bits t of A(row, q)
            blk = A[q]
            for t in range(64):
                sel = ((blk >> np.uint64(t)) & np.uint64(1)).astype(bool)
                acc[sel] ^= X[64 * q + t]
        assert np.array_equal(acc, B), f"request {i}: A X != B"


# ------------------------------------------------------------------ ours

def reduce_over_ranks(x: float, op: str, dist, device) -> float:
    """The whole-job value of a per-rank number: the slowest rank's time
    ("max") or the total work ("sum"); x itself on one process."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def job_line_values(per_rank_ms: float, per_rank_ops: float, dist, device):
    """(ms per step, whole-job bit-op/s) under weak scaling: every rank
    decomposes its own matrix; the job takes as long as its slowest rank and
    does the work of all of them."""
    ms = reduce_over_ranks(per_rank_ms, "max", dist, device)
    ops = reduce_over_ranks(per_rank_ops, "sum", dist, device)
    return ms, ops / (ms / 1000.0)


def run_ours(args):
    import torch

    import paper_1209_5198_gb300 as gf2

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    n, m = args.n, args.m
    k = min(n, m)
    A_rm = make_input(n, m, rank)
    A = gf2.Mat.from_rowmajor(A_rm, m, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    piv = torch.empty(k, dtype=torch.int32, device=dev)
    rk = torch.zeros(1, dtype=torch.int64, device=dev)
    L = gf2.Mat.empty(n, k, dev)
    E = gf2.Mat.empty(k, m, dev)
    lib = gf2.load()
    ws = torch.empty(lib.gf2_decompose_workspace_bytes(n, m, 1), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    sched = {"auto": gf2.SCHEDULE_AUTO, "streams": gf2.SCHEDULE_STREAMS, "persistent": gf2.SCHEDULE_PERSISTENT,
             "split": gf2.SCHEDULE_SPLIT}
    opts = gf2.Opts(schedule=sched[args.schedule])
    tuned = None
    if args.schedule == "auto" and not args.no_tune:
        # the library's autotuner times the speed-only options (update width,
        # table size, schedule) on this GPU for this shape; the automatic
        # options of every later call then take its choice
        best = gf2.decompose_autotune(n, m, factors=True, stream=stream)
        tuned = {"panel_w": best.opts.panel_w, "table_c": best.opts.table_c,
                 "schedule": {1: "streams", 2: "persistent", 3: "split"}.get(best.opts.schedule, "auto"),
                 "tuned_ms": round(best.ms, 4), "bucket": [best.bucket_n, best.bucket_m],
                 "device": best.device.decode()}

    def step():
        gf2.gf2_decompose_ex(A, perm, piv, rk, L, E, opts, workspace=ws, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if dist:
            dist.barrier()

    max_over_ranks = lambda x: reduce_over_ranks(x, "max", dist, dev)

    # ---- timed region: K decompositions, nothing else on the stream
    sampler = ClockSampler(dev.index if world == 1 else local)
    sampler.start()
    launches0 = gf2.launch_count()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = gf2.launch_count() - launches0
    clocks = sampler.stop()
    # every step decomposes the same matrix: the operation count comes from
    # the pivots of the last one
    pivh = piv.cpu().numpy()[: int(rk.item())]
    my_ops = bitops(n, m, pivh)
    r = int(rk.item())
    ms, value = job_line_values(ev0.elapsed_time(ev1) / args.steps, my_ops, dist, dev)
    total_ops = value * ms / 1000.0

    # ---- per-kernel-class device time: CUDA events recorded by the library on
    # the launching stream around every launch of one more step
    gf2.timing(True)
    torch.cuda.synchronize()
    step()
    torch.cuda.synchronize()
    per_class = gf2.timing_read()
    gf2.timing(False)
    prof_steps = 1

    # ---- roofline of the dominant kernel (the M4RM trailing update)
    mu = (m + 63) // 64
    blk = pivh // 64
    rj = np.bincount(blk, minlength=mu)
    pairs = os.environ.get("GF2_PAIRS", "1") != "0"
    alg_bytes = float(np.sum(rest_launch_bytes(n, mu, rj, pairs))) * prof_steps
    # the co-bound: shared-memory table lookups, 8 of 8 bytes per updated word
    # and panel (c = 8), against 128 B/clk on each SM the update runs on
    lookup_bytes = float(np.sum(rest_launch_bytes(n, mu, rj, pairs, lookups=True))) * prof_steps
    upd_ms, upd_n = per_class["update"]
    fac_ms, fac_n = per_class.get("factor", (0.0, 0))
    persistent = fac_n > 0
    if persistent:
        # one persistent launch does the whole factorization: its duration
        # is the denominator of the pair updates' bytes
        upd_ms, upd_n = fac_ms, fac_n
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    achieved = alg_bytes / (upd_ms / 1000.0) / 1e9 if upd_ms > 0 else None
    traffic = rest_traffic(n, m, "k_factor" if persistent else "k_rest")
    shares = {c: round(v[0] / max(1e-9, sum(x[0] for x in per_class.values())), 4) for c, v in per_class.items()}

    # ---- end to end through the host-buffer entry point (pinned memory)
    e2e = None
    if not args.no_e2e:
        A_cb = torch.from_numpy(f2gen.to_colblocks(A_rm).view(np.int64)).pin_memory()
        perm_h = torch.empty(n, dtype=torch.int32).pin_memory()
        piv_h = torch.empty(k, dtype=torch.int32).pin_memory()
        rk_h = torch.empty(1, dtype=torch.int64).pin_memory()
        L_h = torch.empty(((k + 63) // 64, n), dtype=torch.int64).pin_memory()
        E_h = torch.empty((mu, k), dtype=torch.int64).pin_memory()
        ws_h = torch.empty(lib.gf2_decompose_host_workspace_bytes(n, m, 1), dtype=torch.uint8, device=dev)
        ptr = lambda t: t.data_ptr()

        def e2e_step():
            st = lib.gf2_decompose_host(n, m, ptr(A_cb), n, ptr(perm_h), ptr(piv_h), ptr(rk_h), ptr(L_h), ptr(E_h),
                                        0, ptr(ws_h), ws_h.numel(), stream.cuda_stream)
            if st:
                raise gf2.Gf2Error(st, "gf2_decompose_host")

        for _ in range(max(2, args.warmup)):  # the second call captures the graph
            e2e_step()
        ke = max(1, min(args.steps, 3))
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ke):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ems = max_over_ranks(e0.elapsed_time(e1) / ke)
        assert int(rk_h.item()) == r and np.array_equal(piv_h.numpy()[:r], pivh)
        e2e = {"value": total_ops / (ems / 1000.0), "unit": UNIT, "ms_per_step": ems,
               "h2d_bytes_per_step": int(A_cb.numel() * 8),
               "d2h_bytes_per_step": int(perm_h.numel() * 4 + piv_h.numel() * 4 + 8 + L_h.numel() * 8 + E_h.numel() * 8)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = oracle.max_threads()
        v, dt, cols = oracle_sample(A_rm, n, m, args.cpu_seconds, cores)
        # one thread, comparable to the paper's single-core timings (Table 4)
        v1, dt1, cols1 = oracle_sample(A_rm, n, m, max(2.0, args.cpu_seconds / 3), 1)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"oracle PLE on the first {cols} of {m} columns of the same {n}x{m} input "
                         f"(all {n} rows updated), {dt:.1f} s",
               "one_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"the same on the first {cols1} columns, {dt1:.1f} s"},
               "cpu_model": cpu_model(), "nproc": os.cpu_count()}

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras = compact_extras(args)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": (PAPER_SECONDS_32768 / (ms / 1000.0)) if (n == m == 32768) else None,
            "dtype": "u64", "data": "synthetic",
            "config": {"workload": workload_name(n, m), "n": n, "m": m, "rank": r, "factors": "L,E",
                       "schedule": args.schedule, "tuned": tuned,
                       "per_rank_matrix": "independent seed per rank",
                       "l2": "no flush: working set (A 128 MiB + W + L + E, ~512 MiB) > 129 MB L2",
                       "vs_baseline_ref": "Table 4 b=128 rec 11.498 s (3.06 GHz Xeon, other machine)"},
            "roofline": {"kernel": ("k_factor (one persistent launch: panel chain, look-ahead and the M4RM pair "
                                    "updates; bytes = the pair updates' read + write of every trailing word)"
                                    if persistent else "k_rest (M4RM trailing update)"), "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "peak_source": peak_src,
                         "alg_bytes_per_launch": alg_bytes / max(1, upd_n),
                         "smem_lookups": smem_roofline(lookup_bytes, upd_ms, clocks),
                         "avg_launch_ms": upd_ms / max(1, upd_n), "launches": upd_n,
                         "time_share": shares},
            "kernel_ms_per_step": {c: v[0] / prof_steps for c, v in per_class.items()},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def compact_extras(args) -> dict:
    """The rest of the headline metric, measured after the decomposition's
    timed region (each with its own clock record):
      serving: a 4000-request trace (the serving workload's generator, 256
        matrices), saturated solves/s of the engine against its serial mode,
        and p50 / p99 at one Poisson load (0.5 of the serial capacity) for
        both;
      batched: one batch of 4096 matrices (rows and columns uniform in
        [64, 2048], Bernoulli(1/2), every second one rank-deficient) in one
        launch against a loop of plain gf2_decompose calls."""
    import torch

    import paper_1209_5198_gb300 as gf2
    out = {}
    dev = torch.device("cuda", 0)
    # ---- serving
    w = ServeWorkload(4000, 256, 0x5198)
    serve_run(w, serial=False)  # warm-up (kernel attributes, graphs)
    clk = ClockSampler(0)
    clk.start()
    done_sat, span, _, st = serve_run(w, serial=False)
    done_ser, span_ser, _, _ = serve_run(w, serial=True)
    cap, cap_ser = len(w.req) / span, len(w.req) / span_ser
    rng = np.random.default_rng(7)
    lam = 0.5 * cap_ser
    arr = np.cumsum(rng.exponential(1e6 / lam, size=len(w.req)))
    d_o, _, _, _ = serve_run(w, serial=False, arrivals_us=arr)
    d_s, _, _, _ = serve_run(w, serial=True, arrivals_us=arr)
    clocks = clk.stop()
    verify_serving(w, done_sat, 8)
    p50, p99 = latency_ms(d_o)
    s50, s99 = latency_ms(d_s)
    out["serving"] = {
        "metric": SERVE_METRIC, "value": cap, "unit": "solves/s",
        "workload": "4000 requests, 256 square matrices n = 2^U(8,14) rounded up to 64, ids Zipf(1.1), "
                    "k = 1..64 right-hand sides, B = A X0, cold factors; saturated = all requests at t = 0",
        "serial": {"value": cap_ser, "unit": "solves/s", "how": "the same engine one request at a time "
                   "(GF2_SERVE_SERIAL: gf2_decompose / gf2_solve, each waited for)"},
        "speedup_vs_serial": cap / cap_ser,
        "poisson_load_0.5": {"offered_per_s": lam, "p50_ms": p50, "p99_ms": p99,
                             "serial_p50_ms": s50, "serial_p99_ms": s99},
        "admitted_in_flight": int(st.get("admitted_in_flight", -1)),
        "clocks": clocks,
    }
    # ---- batched
    lib = gf2.load()
    count = 4096
    mats = batch_matrices(count, 0.5, 0x1209, dev)
    As = [gf2.Mat(wm.t().contiguous(), nn, mm) for wm, nn, mm in mats]
    perms = [torch.empty(nn, dtype=torch.int32, device=dev) for _, nn, _ in mats]
    pivs = [torch.empty(min(nn, mm), dtype=torch.int32, device=dev) for _, nn, mm in mats]
    ranks = torch.zeros(count, dtype=torch.int64, device=dev)
    Ls = [gf2.Mat.empty(nn, min(nn, mm), dev) for _, nn, mm in mats]
    Es = [gf2.Mat.empty(min(nn, mm), mm, dev) for _, nn, mm in mats]
    import ctypes
    wsb = lib.gf2_decompose_batched_workspace_bytes(count, (ctypes.c_int64 * count)(*[a.rows for a in As]),
                                                    (ctypes.c_int64 * count)(*[a.cols for a in As]), 1)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def bstep():
        gf2.gf2_decompose_batched(As, perms, pivs, ranks, Ls, Es, workspace=ws, stream=stream)

    for _ in range(3):
        bstep()
    clk = ClockSampler(0)
    clk.start()
    ms_batch = time_calls(bstep, 5, stream)
    wsp = torch.empty(lib.gf2_decompose_workspace_bytes(2048, 2048, 1), dtype=torch.uint8, device=dev)
    rk1 = torch.zeros(1, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(count):
        gf2.gf2_decompose(As[i], perms[i], pivs[i], rk1, Ls[i], Es[i], workspace=wsp, stream=stream)
    torch.cuda.synchronize()
    ms_loop = (time.perf_counter() - t0) * 1000
    clocks = clk.stop()
    out["batched"] = {
        "metric": BATCH_METRIC, "value": count / (ms_batch / 1000), "unit": "matrices/s",
        "workload": f"one batch of {count} matrices, rows and cols uniform in [64, 2048], Bernoulli(1/2), every "
                    "second one rank-deficient; CUDA events over 5 batches after 3 warm-ups",
        "ms_per_batch": ms_batch,
        "plain_loop": {"value": count / (ms_loop / 1000), "unit": "matrices/s",
                       "how": "one gf2_decompose call per matrix on the same stream, host clock, one pass"},
        "speedup_vs_plain_loop": ms_loop / ms_batch,
        "clocks": clocks,
    }
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--m", type=int, default=None)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the compact serving and batched measurements")
    ap.add_argument("--no-tune", action="store_true", help="skip the decomposition autotuner (library defaults)")
    ap.add_argument("--fp-sizes", type=int, nargs="+", default=[1024, 4096, 8192], help="n of the F_p workload")
    ap.add_argument("--schedule", default="auto", choices=["auto", "streams", "persistent", "split"],
                    help="decomposition schedule (gf2_opts.schedule)")
    ap.add_argument("--workload", default="decompose", choices=["decompose", "batched", "serving", "product", "sizes", "sparse", "fp", "wide"],
                    help="decompose: the headline 32768^2 decomposition; batched: many small matrices in one "
                         "launch; serving: a request stream on resident factors")
    ap.add_argument("--requests", type=int, default=20000, help="requests in the serving trace")
    ap.add_argument("--product-sizes", type=int, nargs="+", default=[8192, 16384, 32768, 65536])
    ap.add_argument("--sparse-sizes", type=int, nargs="+", default=[16384, 32768, 65536])
    ap.add_argument("--tensor-max", type=int, default=32768, help="largest n timed on the tensor-core backend")
    ap.add_argument("--batch", type=int, default=4096, help="matrices per batch (batched workload)")
    args = ap.parse_args()
    args.m = args.m or args.n
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "product":
        run_product(args)
    elif args.workload == "fp":
        run_fp(args)
    elif args.workload == "sparse":
        run_sparse(args)
    elif args.workload == "sizes":
        run_sizes(args)
    elif args.workload == "wide":
        run_wide(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
