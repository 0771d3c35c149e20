"""Benchmark: exact k-clique counting on one GB300 through the C ABI.

Workload (one "step" = one pass of the whole path over one graph):
    Chung-Lu power-law graph, n = 1,000,000, exponent 2.1, mean degree 20,
    plus 2,000 planted cliques of size U[20, 60] (seed 1), counted for
    k = 5, 6, 7, 8, 9.  The step runs kc_upload from device buffers
    (validation, k-core peeling, DAG orientation) and one kc_count per k,
    then frees the graph.
Metric: k-cliques/s = (sum of the five counts) / (time per step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The reference arm times the oracle (plain CPU listing, all host cores) on a
bounded sample of the same workload.  One JSON line is printed by rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "k-cliques/s (exact count, k=5..9 sweep)"
UNIT = "k-cliques/s"
WORKLOAD = "chung_lu_n1e6_g2.1_d20_planted2000x[20,60]_seed1"
KS = (5, 6, 7, 8, 9)
L2_BYTES = 129 * 1024 * 1024
ENUM_TRAFFIC = None


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--ks", type=str, default=",".join(map(str, KS)))
    p.add_argument("--small", action="store_true", help="a small graph (for profiling runs)")
    p.add_argument("--workload", choices=("sweep", "batched", "serve", "rmat", "ablation"), default="sweep",
                   help="sweep: config 2 k=5..9 (default); batched: config 4, 4,096 graphs in one kc_count_batched; "
                        "serve: config 5, Poisson arrivals served by kc_serve_*; rmat: config 3, R-MAT scale 22 k=6 "
                        "listing of a root-range chunk into a device buffer; ablation: memo / pruning / split / "
                        "decomposition variants on configs 2 and 3")
    p.add_argument("--chunk", type=float, default=2 ** 29, help="rmat: about this many cliques in the listed chunk")
    p.add_argument("--rate", type=float, default=2000.0, help="serve: arrivals per second")
    p.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    p.add_argument("--count", type=int, default=4096, help="graphs in the batched workload")
    return p.parse_args()


def _config(workload: str, ks, ws: int) -> dict:
    """The workload as both arms describe it (the GPU arm and the oracle arm)."""
    return {"workload": workload, "ks": list(ks), "parallelism": f"replicas x{ws}",
            "step": "upload (validate + peel + orient) and one exact count per k",
            "l2": "flushed between timed steps (512 MiB write)"}


def _graph(small: bool):
    from paper_2502_00317_gb300 import graphgen as gg

    if small:
        return gg.chung_lu_planted(n=100_000, n_cliques=200, seed=1), "chung_lu_n1e5_planted200_seed1"
    return gg.config_chung_lu(), WORKLOAD


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def _max_over_ranks(ws, x: float) -> float:
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- our arm
def run_ours(a):
    import torch

    from paper_2502_00317_gb300 import kclique as kc

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    ks = tuple(int(x) for x in a.ks.split(","))
    g, workload = _graph(a.small)
    # inputs resident in HBM before the timed region
    d_rowptr = torch.from_numpy(g.rowptr.view(np.int64)).cuda()
    d_col = torch.from_numpy(g.col.view(np.int32)).cuda()
    # pinned host copies for the end-to-end measurement
    h_rowptr = torch.from_numpy(g.rowptr.view(np.int64)).pin_memory()
    h_col = torch.from_numpy(g.col.view(np.int32)).pin_memory()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    ctx = kc.Context(local)
    n = g.n

    def step(host: bool):
        if host:
            h = kc.kc_upload(ctx.h, n, h_rowptr, h_col, kc.KC_HOST_PTRS, stream)
        else:
            h = kc.kc_upload(ctx.h, n, d_rowptr, d_col, kc.KC_DEVICE_PTRS, stream)
        up = ctx.upload_stats()
        counts, stats = [], []
        for k in ks:
            counts.append(ctx.count(h, k, stream))
            stats.append(ctx.stats())
        ctx.free(h)
        return counts, up, stats

    for _ in range(a.warmup):
        counts, _, _ = step(False)
    units = sum(counts)
    build_bytes = None
    try:  # the DAG the GPU builds, for the build's algorithmic bytes (outside the timed region)
        h = kc.kc_upload(ctx.h, n, d_rowptr, d_col, kc.KC_DEVICE_PTRS, stream)
        _, _, orow, ocol = ctx.export_dag(h)
        ctx.free(h)
        build_bytes = build_algorithmic_bytes(orow, ocol, ks)
    except Exception:  # pragma: no cover
        build_bytes = None

    def timed(host: bool):
        times, ups, sts = [], [], []
        for _ in range(a.steps):
            _barrier(ws)
            flush.fill_(1)  # L2 flush between timed steps (outside the timed interval)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c, up, st = step(host)
            e1.record(stream)
            torch.cuda.synchronize()
            assert sum(c) == units, "count changed between steps"
            times.append(e0.elapsed_time(e1))
            ups.append(up)
            sts.append(st)
        return times, ups, sts

    sampler = ClockSampler(local)
    sampler.start()
    times, ups, sts = timed(False)
    clocks = sampler.stop()
    etimes, _, _ = timed(True)
    ms = _max_over_ranks(ws, statistics.mean(times))
    ems = _max_over_ranks(ws, statistics.mean(etimes))
    value = ws * units / (ms / 1e3)
    evalue = ws * units / (ems / 1e3)
    launches = sum(u["launches"] + sum(s["total_launches"] for s in st) for u, st in zip(ups, sts))
    # dominant kernel family: the enumerator (k_enum + k_tasks of every width
    # tier of one kc_count call; the tiers run concurrently on their own
    # streams, so their wall time is the events around the whole family)
    enum_ms = statistics.mean(sum(s["ms_enum"] for s in st) for st in sts)
    enum_launch = statistics.mean(sum(s["enum_launches"] for s in st) for st in sts)
    word_ops = statistics.mean(sum(s["word_ops"] for s in st) for st in sts)
    calls = len(ks)
    peak_ops, peak_note = word_op_peak()
    achieved = (word_ops / calls) / (enum_ms / calls / 1e3) / 1e9 if enum_ms > 0 else None
    roof = {
        "kernel": "enumerator family (k_enum + k_tasks, all width tiers of one kc_count call)",
        "bound": "alu",
        "achieved": round(achieved, 3) if achieved else None,
        "peak": round(peak_ops / 1e9, 1) if peak_ops else None,
        "peak_source": peak_note,
        "unit": "Gword-op/s (word-op = 32-bit AND + POPC of candidate words)",
        "frac": round(achieved * 1e9 / peak_ops, 5) if (achieved and peak_ops) else None,
        # DRAM bytes of the family per kc_count call (dram__bytes_read.sum +
        # dram__bytes_write.sum over its kernels) from an ncu capture of the
        # current kernels; null while no such capture exists
        "traffic": ENUM_TRAFFIC if (not a.small and ks == KS) else None,
        "traffic_unit": "bytes per kc_count call (enumerator family)",
        "word_ops_per_launch": round(word_ops / calls),
        "ms_per_launch": round(enum_ms / calls, 3),
        "enum_launches_per_step": enum_launch,
    }
    # upload stages are HBM-bound: algorithmic bytes of peel + orient per step
    hbm = _peaks().get("hbm_gbs")
    m_und = int(g.rowptr[-1]) // 2
    up_bytes = (8 * (n + 1) + 4 * 2 * m_und) + 4 * 2 * m_und + (8 * (n + 1) + 4 * m_und) + 12 * n
    up_ms = statistics.mean(u["ms_peel"] + u["ms_orient"] for u in ups)
    roof_upload = {"kernel": "k_peel + orient (a2-a3)", "bound": "hbm",
                   "achieved": round(up_bytes / (up_ms / 1e3) / 1e9, 2), "peak": hbm, "unit": "GB/s",
                   "frac": round(up_bytes / (up_ms / 1e3) / 1e9 / hbm, 4) if hbm else None,
                   "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)", "algorithmic_bytes": up_bytes}
    # a5, the per-root bit-matrix build, inside the enumerator kernels: its
    # algorithmic bytes are 4 * sum over the roots of (d+(u) + sum of d+(v) over
    # v in N+(u)) -- every root with out-degree >= k - 1 reads its out-list and
    # each out-neighbour's -- from the DAG the GPU built; its time is the
    # family's event time times the share of warp time spent building
    # (%globaltimer around each build, summed over warps)
    roof_build = None
    if build_bytes is not None:
        share = [s["warp_ns_build"] / s["warp_ns_busy"] if s["warp_ns_busy"] else 0.0 for s in sts[0]]
        t_build = sum(sh * s["ms_enum"] for sh, s in zip(share, sts[0])) / 1e3
        if t_build > 0:
            gbs = sum(build_bytes) / t_build / 1e9
            roof_build = {"kernel": "build_root inside k_enum (a5), all width tiers", "bound": "hbm",
                          "achieved": round(gbs, 2), "peak": hbm, "unit": "GB/s",
                          "frac": round(gbs / hbm, 4) if hbm else None,
                          "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                          "algorithmic_bytes_per_step": int(sum(build_bytes)),
                          "bytes_read_per_step": int(4 * sum(s["build_words"] for s in sts[0])),
                          "build_share_of_warp_time": [round(x, 4) for x in share],
                          "time": "enumerator event time x build share of warp time, summed over the sweep"}
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": ws,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32/u64 (exact integer)",
        "data": "synthetic (seeded generator)",
        "config": _config(workload, ks, ws),
        "counts": counts,
        "units_per_step": units,
        "upload": "device pointers (validate + peel + orient inside the step)",
        "e2e": {"value": evalue, "unit": UNIT, "ms_per_step": ems,
                "h2d_bytes_per_step": int(g.rowptr.nbytes + g.col.nbytes),
                "d2h_bytes_per_step": 8 * len(ks)},
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": roof,
        "roofline_upload": roof_upload,
        "roofline_build": roof_build,
        "step_ms": [round(t, 3) for t in times],
        "stage_ms": {"upload": statistics.mean(u["ms_total"] for u in ups),
                     "peel": statistics.mean(u["ms_peel"] for u in ups),
                     "enum_per_k": [round(statistics.mean(st[i]["ms_enum"] for st in sts), 3) for i in range(len(ks))],
                     "memo_hits_per_k": [sts[0][i]["memo_hits"] for i in range(len(ks))]},
    }
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(g)
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def build_algorithmic_bytes(orow, ocol, ks):
    """Bytes the per-root build must read for each k: 4 * sum over the roots
    with out-degree >= k - 1 of (d+(u) + sum of d+(v) over v in N+(u))."""
    orow = np.asarray(orow, dtype=np.int64)
    d = np.diff(orow)
    nb = np.zeros(d.size, dtype=np.int64)
    nz = d > 0
    if ocol.size:
        sums = np.add.reduceat(d[np.asarray(ocol, dtype=np.int64)], orow[:-1][nz])
        nb[nz] = sums
    return [int(4 * (d[d >= k - 1] + nb[d >= k - 1]).sum()) for k in ks]


def word_op_peak():
    """Measured word-op rate of this GPU (libkc_peak.so: an AND + POPC loop at full occupancy)."""
    import ctypes

    from paper_2502_00317_gb300 import build as b

    try:
        lib = ctypes.CDLL(b.build_peak())
        f = lib.kc_peak_word_ops
        f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                      ctypes.POINTER(ctypes.c_float)]
        rate, per, ms = ctypes.c_double(), ctypes.c_double(), ctypes.c_float()
        st = f(4096, 5, ctypes.byref(rate), ctypes.byref(per), ctypes.byref(ms))
        if st != 0:
            return None, f"kc_peak failed ({st})"
        return rate.value, f"measured: kc_peak_word_ops, best of 5 launches of {ms.value:.2f} ms (burst)"
    except Exception as e:  # pragma: no cover
        return None, f"kc_peak unavailable: {e}"


# The oracle's sample: one root in every n / 4096 of its rank order.  The
# whole k = 5..9 sweep takes it about 40 core-minutes; the sample about 10 s
# on 16 cores, and on the config-2 graph it holds the expected share of the
# cliques (the light periphery and the dense core are both in it).
ORACLE_SAMPLE_ROOTS = 4096


def _oracle_sample_step(og, ks, threads: int):
    """One sampled step of the oracle: for every k, the cliques whose first
    vertex (in the oracle's order) is one of ORACLE_SAMPLE_ROOTS evenly spaced
    ranks, one single-threaded oracle call per root, the calls spread over
    the host cores.  Returns (cliques found, seconds)."""
    from concurrent.futures import ThreadPoolExecutor

    n = og.n
    B = min(ORACLE_SAMPLE_ROOTS, n)
    jobs = [(k, b * n // B, b * n // B + 1) for k in ks for b in range(B)]
    t0 = time.time()
    with ThreadPoolExecutor(max_workers=threads) as ex:  # ctypes releases the GIL
        found = sum(c for c, _ in ex.map(lambda j: og.count(j[0], threads=1, root_lo=j[1], root_hi=j[2]), jobs))
    return found, time.time() - t0


def _sample_fraction(n: int) -> float:
    return min(ORACLE_SAMPLE_ROOTS, n) / max(n, 1)


def _sample_text(ks, tb: float) -> str:
    return (f"k = {list(ks)}, cliques whose first vertex is one of {ORACLE_SAMPLE_ROOTS} evenly spaced ranks of the "
            f"oracle's order, plus that fraction of the oracle's canonicalise+peel+orient ({tb:.1f} s, run once)")


def cpu_baseline(g, ks=KS):
    """The oracle on the host cores, on a bounded sample of the same k = 5..9
    sweep (about 10-30 s): its own preprocessing once, then one sampled step."""
    import oracle

    threads = os.cpu_count() or 1
    t0 = time.time()
    og = oracle.OracleGraph.from_graph(g)
    tb = time.time() - t0
    found, tt = _oracle_sample_step(og, ks, threads)
    sec = tt + _sample_fraction(og.n) * tb  # the sample's share of the preprocessing is charged to it
    return {"value": found / sec, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": _sample_text(ks, tb) + f"; {found} cliques in {tt:.1f} s"}


# ---------------------------------------------------------- reference arm
def run_reference(a):
    """The oracle, as it stands, on the host cores: each step is the sampled
    sweep of cpu_baseline (the whole k = 5..9 sweep would take it most of an
    hour); value = cliques found / (sample time + the sample's share of the
    oracle's preprocessing)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle

    g, workload = _graph(a.small)
    ks = tuple(int(x) for x in a.ks.split(","))
    threads = os.cpu_count() or 1
    t0 = time.time()
    og = oracle.OracleGraph.from_graph(g)
    tb = time.time() - t0
    times, units = [], 0
    for i in range(a.warmup + a.steps):
        found, tt = _oracle_sample_step(og, ks, threads)
        if i >= a.warmup:
            times.append(tt + _sample_fraction(og.n) * tb)
        units = found
    sec = statistics.mean(times)
    value = units / sec
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": ws,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": 1e3 * sec,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32/u64 (exact integer)",
        "data": "synthetic (seeded generator)",
        "config": _config(workload, ks, ws),
        "units_per_step": units,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "each step: " + _sample_text(ks, tb)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _gen_batch_part(args):
    seed, count, lo, hi = args
    from paper_2502_00317_gb300 import graphgen as gg

    return gg.config_batched(seed=seed, count=count)[lo:hi]


def batched_graphs(count: int, seed: int = 3):
    """Config 4's graphs, generated in parallel worker processes (spawned, before any GPU use)."""
    import multiprocessing as mp

    from paper_2502_00317_gb300 import graphgen as gg

    if count <= 256:
        return gg.config_batched(seed=seed, count=count)
    workers = max(1, min(16, os.cpu_count() or 1))
    step = (count + workers * 4 - 1) // (workers * 4)
    parts = [(seed, count, lo, min(count, lo + step)) for lo in range(0, count, step)]
    with mp.get_context("spawn").Pool(workers) as pool:
        out = []
        for part in pool.map(_gen_batch_part, parts):
            out.extend(part)
    return out


def run_batched(a):
    """Config 4: one kc_count_batched over every (graph, k) vs one kc_count per graph."""
    batch = batched_graphs(a.count)  # before the first CUDA call (spawned pool)
    import torch

    from paper_2502_00317_gb300 import kclique as kc

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = kc.Context(local)
    t0 = time.time()
    hs = [ctx.upload_host(g.n, g.rowptr, g.col) for g, _ in batch]
    upload_s = time.time() - t0
    ks = [k for _, k in batch]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")

    def timed(fn, steps):
        out, ts = None, []
        for _ in range(steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return out, ts

    def batched():
        return ctx.count_batched(hs, ks, stream)

    def separate():
        return [ctx.count(h, k, stream) for h, k in zip(hs, ks)]

    # the fixed default launch settings first, then the autotuner's choice for this batch
    for _ in range(a.warmup):
        ref = batched()
    _, tfix = timed(batched, a.steps)
    t1 = time.time()
    tune = ctx.tune(hs, ks)
    tune_s = time.time() - t1
    for _ in range(a.warmup):
        ref2 = batched()
    sampler = ClockSampler(local)
    sampler.start()
    got, tb = timed(batched, a.steps)
    clocks = sampler.stop()
    st = ctx.stats()
    alone, tsep = timed(separate, max(1, min(a.steps, 2)))
    assert got == ref == ref2 == alone, "batched counts differ from per-graph counts"
    ms, ms_sep, ms_fix = statistics.mean(tb), statistics.mean(tsep), statistics.mean(tfix)
    line = {
        "metric": "graphs/s (batched exact k-clique counts)", "value": len(batch) / (ms / 1e3), "unit": "graphs/s",
        "n_gpus": ws, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64 (exact integer)", "data": "synthetic (seeded generator)",
        "config": {"workload": f"batched_{len(batch)}_graphs_er_rgg_n50-20000_k4-8_seed3",
                   "sum_n": int(sum(g.n for g, _ in batch)), "sum_m": int(sum(g.nnz for g, _ in batch) // 2),
                   "cliques": int(sum(got)), "l2": "flushed between timed steps", "resident": "CSRs uploaded once"},
        "per_graph_launches": {"value": len(batch) / (ms_sep / 1e3), "unit": "graphs/s", "ms_per_step": ms_sep},
        "speedup_vs_per_graph": ms_sep / ms,
        "autotune": {"choice": {kk: tune[kk] for kk in ("split_threshold", "warps_small", "warps_large",
                                                         "memo_bytes")},
                     "class_key": tune["key"], "probes": tune["probes"], "tuning_s": tune_s,
                     "probe_ms_default": tune["ms_default"], "probe_ms_tuned": tune["ms_tuned"],
                     "fixed_settings": {"value": len(batch) / (ms_fix / 1e3), "unit": "graphs/s",
                                        "ms_per_step": ms_fix},
                     "speedup_vs_fixed": ms_fix / ms},
        "upload_s_all": upload_s,
        "gpu_launches": st["total_launches"] * a.steps,
        "clocks": clocks,
        "stage_ms": {"bin": st["ms_bin"], "enum": st["ms_enum"], "tiers": st["ms_tier"], "roots": st["roots_total"],
                     "heavy": st["roots_heavy"]},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def _serve_run(kc, ctx, hs, ks_all, arrivals, lanes, max_batch, cap):
    """Submits each request at its arrival time; returns (per-request results, server stats)."""
    kc.kc_serve_start(ctx.h, lanes=lanes, max_batch=max_batch, mem_cap_bytes=cap)
    t0 = time.perf_counter()
    tickets = []
    for (t_arr, gi, k) in arrivals:
        while True:
            dt = t_arr - (time.perf_counter() - t0)
            if dt <= 0:
                break
            time.sleep(min(dt, 0.0005) if dt > 0.0002 else 0)
        tickets.append(kc.kc_serve_submit(ctx.h, hs[gi], k))
    res = [kc.kc_serve_wait(ctx.h, t, 600000) for t in tickets]
    st = kc.kc_serve_stats_get(ctx.h)
    kc.kc_serve_stop(ctx.h)
    return res, st


def run_serve(a):
    """Config 5: Poisson arrivals of config-4 graphs (resident) with k in 4..8."""
    batch = batched_graphs(a.count)
    import torch

    from paper_2502_00317_gb300 import kclique as kc

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    ctx = kc.Context(local)
    hs = [ctx.upload_host(g.n, g.rowptr, g.col) for g, _ in batch]
    rng = np.random.default_rng(5)
    n_req = int(a.rate * a.duration)
    gaps = rng.exponential(1.0 / a.rate, n_req)
    arrivals = list(zip(np.cumsum(gaps).tolist(), rng.integers(0, len(hs), n_req).tolist(),
                        (4 + rng.integers(0, 5, n_req)).tolist()))
    cap = 64 << 30
    # warm the lanes' scratch on a short prefix
    _serve_run(kc, ctx, hs, None, arrivals[: min(200, n_req)], 2, 4096, cap)
    sampler = ClockSampler(local)
    sampler.start()
    res, st = _serve_run(kc, ctx, hs, None, arrivals, 2, 4096, cap)
    clocks = sampler.stop()
    base, bst = _serve_run(kc, ctx, hs, None, arrivals, 1, 1, cap)
    assert all(r["status"] == kc.KC_OK for r in res + base)
    assert [r["count"] for r in res] == [r["count"] for r in base], "served counts depend on the mix"
    line = {
        "metric": "serve p50/p99 latency ms and throughput (req/s)", "value": st["req_per_s"], "unit": "req/s",
        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
        "p50_enumerated_ms": st["p50_enum_ms"], "p99_enumerated_ms": st["p99_enum_ms"],
        "enumerated_requests": sum(1 for r in res if r["enumerated"]), "n_gpus": ws, "steps": 1, "warmup": 1,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64 (exact integer)",
        "data": "synthetic (seeded generator)",
        "config": {"workload": f"serve_poisson_{a.rate:g}rps_{a.duration:g}s_config4_pool{len(hs)}_k4-8",
                   "requests": n_req, "lanes": 2, "max_batch": 4096, "mem_cap_bytes": cap,
                   "resident": "CSRs uploaded once"},
        "serve": st,
        "one_request_per_launch": {"req_per_s": bst["req_per_s"], "p50_ms": bst["p50_ms"], "p99_ms": bst["p99_ms"],
                                   "p50_enumerated_ms": bst["p50_enum_ms"], "p99_enumerated_ms": bst["p99_enum_ms"],
                                   "note": "same arrivals, one lane, batches of one request"},
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_rmat(a):
    """Config 3: R-MAT scale 22, k = 6.  The full listing holds 3.3e14 cliques
    (8 PB of tuples), so the timed step lists one root-range chunk of the
    dense core -- starting at the first rank whose out-degree reaches 512 and
    widened until it holds about --chunk cliques -- into a device buffer with
    its total and checksum (kc_list_range).  Also reported: one full k = 6
    count and the upload, each timed once."""
    from paper_2502_00317_gb300 import graphgen as gg

    g = gg.config_rmat()
    import torch

    from paper_2502_00317_gb300 import kclique as kc

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = kc.Context(local)
    k = 6
    t0 = time.time()
    h = ctx.upload_host(g.n, g.rowptr, g.col, canonicalize=True)
    upload_s = time.time() - t0
    up = ctx.upload_stats()
    info = ctx.info(h)
    _, _, orow, _ = ctx.export_dag(h)
    d = np.diff(orow.astype(np.int64))
    # the chunk: from the first rank of out-degree >= T, widened (doubling,
    # then halving back) until it holds about --chunk cliques; T falls from
    # 512 (16-word roots) while one root alone holds more than 4 chunks
    lo = hi = 0
    total = 0
    for thr in (512, 256, 128, 64, 32, 0):
        if not (d >= thr).any():
            continue
        lo = int(np.argmax(d >= thr))
        _, one, _ = ctx.list_range(h, k, lo, lo + 1, None, 0, stream)
        if one > 4 * a.chunk and thr > 0:
            continue
        w, total = 1, one
        while total < a.chunk and lo + w < info["n"]:
            w = min(2 * w, info["n"] - lo)
            _, total, _ = ctx.list_range(h, k, lo, lo + w, None, 0, stream)
        step = w // 4
        while total > 2 * a.chunk and step >= 1:
            _, t2, _ = ctx.list_range(h, k, lo, lo + w - step, None, 0, stream)
            if t2 >= a.chunk // 2:
                w, total = w - step, t2
            step //= 2
        hi = lo + w
        break
    buf = torch.empty(max(total * k, 1), dtype=torch.int32, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    for _ in range(a.warmup):
        ref = ctx.list_range(h, k, lo, hi, buf, total, stream)
    times = []
    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(a.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        got = ctx.list_range(h, k, lo, hi, buf, total, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        assert got == ref, "listing changed between steps"
        times.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    st = ctx.stats()
    ms = statistics.mean(times)
    hbm = _peaks().get("hbm_gbs")
    write_gbs = 4 * k * total / (ms / 1e3) / 1e9
    torch.cuda.synchronize()
    t1 = time.time()
    full = ctx.count(h, k, stream)
    count_s = time.time() - t1
    cst = ctx.stats()
    line = {
        "metric": "k-cliques/s (k=6 listing with checksum into a device buffer, root-range chunk)",
        "value": total / (ms / 1e3), "unit": "k-cliques/s", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32/u64 (exact integer)", "data": "synthetic (seeded generator)",
        "config": {"workload": "rmat_scale22_ef16_abcd.57.19.19.05_seed2_k6", "ranks": [lo, hi],
                   "out_degree_first_root": int(d[lo]),
                   "chunk_cliques": total, "checksum": ref[2], "buffer_bytes": 4 * k * total,
                   "l2": "flushed between timed steps"},
        "graph": info, "upload_s": upload_s, "upload_stage_ms": up,
        "roofline": {"kernel": "listing family (k_enum + k_tasks, mode list with the trie)", "bound": "hbm",
                     "achieved": round(write_gbs, 2), "peak": hbm, "unit": "GB/s (4k bytes of tuples per clique)",
                     "frac": round(write_gbs / hbm, 4) if hbm else None,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
        "list_stats": {kk: st[kk] for kk in ("ms_enum", "word_ops", "memo_hits", "memo_inserts", "memo_peak",
                                             "roots_total", "roots_heavy")},
        "full_count": {"k": k, "count": full, "seconds": count_s, "word_ops": cst["word_ops"],
                       "memo_hits": cst["memo_hits"], "ms_tier": cst["ms_tier"], "roots_tier": cst["roots_tier"]},
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_ablation(a):
    """NEXT-3 (Sec. VII-C's baseline / memo / memo + pruning comparison, the
    2-plex early termination of Sec. VII-A, and the decomposition of Sec.
    VII-D): each variant counts config 2 for
    k = 5..9 (the memo-off variants up to k = 7) and config 3 for k = 5; per
    count its enumeration time, candidate words intersected and the most trie
    entries stored for one root."""
    import torch

    from paper_2502_00317_gb300 import graphgen as gg
    from paper_2502_00317_gb300 import kclique as kc

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    variants = [("default", {}), ("memo_every_k", {"memo_min_k": 3}), ("no_plex", {"no_plex": True}),
                ("no_prune", {"no_prune": True}),
                ("no_split", {"split_threshold": 0xFFFFFFFF}),
                ("no_memo", {"no_memo": True}), ("baseline", {"no_memo": True, "no_prune": True}),
                ("edge_parallel", {"decomposition": kc.KC_EDGE_PARALLEL}),
                ("edge_parallel_no_memo", {"decomposition": kc.KC_EDGE_PARALLEL, "no_memo": True})]
    out = {}
    for gname, g, ks, canon in (("config2", gg.config_chung_lu(), KS, False),
                                ("config3", gg.config_rmat(), (5,), True)):
        rows = {}
        for vname, opts in variants:
            ctx = kc.Context(local, **opts)
            h = ctx.upload_host(g.n, g.rowptr, g.col, canonicalize=canon)
            per_k = {}
            for k in ks:
                if "no_memo" in opts and k > 7:
                    continue
                ctx.count(h, k)  # warm
                c = ctx.count(h, k)
                st = ctx.stats()
                per_k[k] = {"count": c, "ms_enum": round(st["ms_enum"], 3), "word_ops": st["word_ops"],
                            "memo_hits": st["memo_hits"], "memo_inserts": st["memo_inserts"],
                            "memo_peak": st["memo_peak"], "roots_heavy": st["roots_heavy"]}
            rows[vname] = per_k
            ctx.close()
        out[gname] = rows
    if rank == 0:
        print(json.dumps({"metric": "ablation: enumeration ms, word-ops, trie entries per root", "value": None,
                          "unit": "ms", "n_gpus": ws, "data": "synthetic (seeded generator)",
                          "config": {"workload": "ablation_config2_k5-9_config3_k5"}, "ablation": out}), flush=True)


if __name__ == "__main__":
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "rmat":
        run_rmat(args)
    elif args.workload == "ablation":
        run_ablation(args)
    else:
        run_ours(args)
