#!/usr/bin/env python3
"""Throughput of the exact kNN query path (buffer k-d tree, LazySearch) on GB300.

One step = one ``bkd_query`` over the whole query set of the workload: every
round of FindLeafBatch, buffer insertion and ProcessAllBuffers, the binary64
re-check and fallback, with the tree resident in HBM.  Default workload: n =
2^26 reference points and m = 2^24 queries in R^10 drawn from a 32-component
isotropic Gaussian mixture (stand-in for photometric colour features), k =
10, tree height 16 (65,536 leaves of 1,024 points).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank builds the same tree and answers its own query set
(queries are independent: no data-path collective); rank 0 prints one JSON
line with the whole-job queries/s.  ``--impl reference`` times the binary64
CPU oracle (classical k-d tree, OpenMP on all host cores) on bounded query
samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = ("kNN queries/s (k=10, d=10) FP32 vs BF16-screened; p50/p99 "
          "latency; % roofline")
LEAF_SRC = os.path.join(ROOT, "paper_1512_02831_gb300", "csrc", "k_leaf.cuh")
TRAFFIC_NOTE = os.path.join(ROOT, "profiles",
                            "leaf_pipe_kernel_traffic.txt")
# the two BF16 screen kernels: source file and committed ncu traffic note
SCREEN_SRC = {0: os.path.join(ROOT, "paper_1512_02831_gb300", "csrc",
                              "k_screen_warp.cu"),
              1: os.path.join(ROOT, "paper_1512_02831_gb300", "csrc",
                              "k_screen.cu")}
SCREEN_TRAFFIC_NOTE = {0: os.path.join(ROOT, "profiles",
                                       "screen_warp_kernel_traffic.txt"),
                       1: os.path.join(ROOT, "profiles",
                                       "screen_tcgen05_kernel_traffic.txt")}

WORKLOADS = {"mixture64M": workloads.MIXTURE_64M,
             "uniform64K": workloads.UNIFORM_64K,
             # same distribution, 1/4 of the points, 1/16 of the queries
             # (leaf structure 0.67 GB > L2): the case ncu captures
             "mixture16M": workloads.scaled(workloads.MIXTURE_64M, 1 << 24,
                                            1 << 20, 14),
             # d = 27, k = 50, 64 components, 1% duplicate rows (n = 2^28,
             # m = 2^25, h = 18; ~30 GB of points)
             "d27k50": workloads.MIXTURE_D27,
             # serving: n = 2^30, h = 20 (43 GB of points, resident)
             "serving1G": workloads.MIXTURE_1G}


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS),
                    default="mixture64M")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--latency-seconds", type=float, default=4.0,
                    help="time budget of the per-batch latency sample")
    ap.add_argument("--serving-seconds", type=float, default=10.0,
                    help="length of each serving sample (0: none)")
    ap.add_argument("--serving-rates", type=float, nargs="*",
                    default=[1000.0, 10000.0],
                    help="Poisson arrival rates (batches/s) of the serving "
                         "samples")
    ap.add_argument("--serving-slots", type=int, default=1 << 22,
                    help="query slots per list class of the server")
    ap.add_argument("--serving-defer", type=int, default=0,
                    help="the servers' buffer trigger (BKD_OPT_DEFER_QUERIES: "
                         "a leaf's buffer is processed once it holds this "
                         "many queries or waited 4 rounds; 0: off)")
    ap.add_argument("--serving-backlog", type=int, default=1 << 23,
                    help="unfinished submitted queries above which an "
                         "arriving batch is rejected")
    ap.add_argument("--modes", default="fp32,warp,tcgen05",
                    help="leaf scorings timed: fp32, warp (BF16 screen, "
                         "warp kernel), tcgen05 (BF16 screen, tcgen05 "
                         "kernel)")
    ap.add_argument("--queries", type=int, default=0,
                    help="time the first N queries of the workload's query "
                         "set instead of all m (0: all); the line's config "
                         "then names the sample")
    ap.add_argument("--serving-only", action="store_true",
                    help="build the workload's tree and run only the "
                         "serving samples (one JSON line)")
    ap.add_argument("--autotune", action="store_true",
                    help="run the autotuner (paper_1512_02831_gb300.tune) on "
                         "the workload's tree and print its report")
    ap.add_argument("--autotune-queries", type=int, default=1 << 20,
                    help="query sample the autotuner times")
    ap.add_argument("--streamer", action="store_true",
                    help="measure the chunk streamer (bigger mode) instead")
    ap.add_argument("--streamer-n", type=int, default=0,
                    help="streamer workload: reference points (default: "
                         "the 2^24-point mixture)")
    ap.add_argument("--streamer-m", type=int, default=1 << 20)
    ap.add_argument("--streamer-h", type=int, default=20)
    ap.add_argument("--streamer-resident", action="store_true",
                    help="with --streamer-n: also time the resident tree")
    ap.add_argument("--streamer-modes", default="",
                    help="comma-separated subset of resident, chunks=N, "
                         "point_chunks=N (default: resident unless "
                         "--streamer-n, chunks=1,3,10, point_chunks=3,10)")
    ap.add_argument("--streamer-precision", type=int, default=1,
                    choices=[0, 1],
                    help="leaf scoring of the streamer modes: 1 (default) "
                         "the BF16 warp screen (point-chunk modes, which "
                         "cannot screen, run float32), 0 float32")
    ap.add_argument("--streamer-oracle-rows", type=int, default=32,
                    help="queries of the streamer's oracle sample (its "
                         "cpu_baseline and parity rows; 0: none)")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu),
                 f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                 "-lms", "200"], stdout=open(self.path, "w"),
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                    "note": "nvidia-smi unavailable"}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                smax.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def leaf_traffic_per_launch(acc, launches):
    """DRAM bytes (read + write) of an average float32 leaf-kernel launch,
    scaled from the committed ncu capture of one launch if it was taken on
    the current leaf kernel source: the capture's DRAM bytes per staged
    leaf-structure byte times this run's staged bytes, over its launches."""
    try:
        text = open(TRAFFIC_NOTE).read()
    except OSError:
        return None
    sha = hashlib.sha256(open(LEAF_SRC, "rb").read()).hexdigest()[:16]
    m_sha = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_r = re.search(r"dram_bytes_per_staged_byte:\s*([0-9.e+-]+)", text)
    if not m_sha or not m_r or m_sha.group(1) != sha:
        return None
    return float(m_r.group(1)) * acc["leaf_bytes"] / max(launches, 1)


def screen_traffic_per_launch(acc, launches, kernel):
    """DRAM bytes (read + write) of an average screen launch, scaled from the
    committed ncu capture of one launch if it was taken on the current source
    of that screen kernel: the capture's DRAM bytes per streamed operand byte
    times this run's streamed bytes, over the run's screen launches."""
    try:
        text = open(SCREEN_TRAFFIC_NOTE[kernel]).read()
    except OSError:
        return None
    sha = hashlib.sha256(open(SCREEN_SRC[kernel], "rb").read()).hexdigest()[:16]
    m_sha = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_r = re.search(r"dram_bytes_per_streamed_byte:\s*([0-9.e+-]+)", text)
    if not m_sha or not m_r or m_sha.group(1) != sha:
        return None
    return float(m_r.group(1)) * acc["screen_bytes"] / max(launches, 1)


def cpu_baseline(P, Q, w, seconds: float, seed: int = 7):
    """The binary64 oracle's k-d tree (Sec. 2.3), as it stands, timed on a
    bounded sample of the workload's queries on all host cores."""
    import oracle
    t0 = time.perf_counter()
    tree = oracle.build_tree(P, w.height)
    build_s = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    probe = Q[rng.choice(Q.shape[0], 256, replace=False)]
    t0 = time.perf_counter()
    tree.knn(probe, w.k)
    per_q = (time.perf_counter() - t0) / 256
    s = int(min(Q.shape[0], max(256, seconds / max(per_q, 1e-9))))
    rows = np.sort(rng.choice(Q.shape[0], s, replace=False))
    t0 = time.perf_counter()
    res = tree.knn(Q[rows], w.k)
    dt = time.perf_counter() - t0
    info = {"value": s / dt, "unit": "queries/s",
            "cores": oracle.max_threads(), "kind": "oracle",
            "sample": (f"{s} of {Q.shape[0]} queries (seeded), binary64 "
                       f"classical k-d tree of height {w.height}, OpenMP "
                       f"over queries; tree build {build_s:.1f} s not "
                       f"counted; query phase {dt:.1f} s")}
    return info, rows, res


def l2_note(w) -> str:
    """Whether the timed inputs exceed the 129 MB L2 (no flush needed)."""
    dp = min(c for c in (2, 4, 6, 8, 10, 12, 16, 24, 32) if c >= w.d)
    leaf_gb, q_gb = w.n * dp * 4 / 1e9, w.m * dp * 4 / 1e9
    big = leaf_gb > 0.129 and q_gb > 0.129
    return (f"inputs {'larger' if big else 'not all larger'} than L2 (leaf "
            f"structure {leaf_gb:.2f} GB, queries {q_gb:.2f} GB)"
            + (" - no flush needed" if big else
               " - small case, not a bench line"))


def data_description(w) -> str:
    """The synthetic input of workload w, in words."""
    if w.kind == "uniform":
        return (f"synthetic: seeded uniform [0,1)^{w.d}; per-rank query "
                f"sets")
    dup = (f", {w.duplicates:.0%} of the reference rows exact copies of "
           f"others" if w.duplicates else "")
    return (f"synthetic: seeded Gaussian mixture ({w.components} isotropic "
            f"components, centres U[0,1]^{w.d}, sigma logU[{w.sigma_lo},"
            f"{w.sigma_hi}], Dirichlet(1) weights{dup}); per-rank query sets")


# ---------------------------------------------------- multi-rank bookkeeping
# Queries are independent (Sec. 3.2, multi-many-core querying): every rank
# holds the same tree and answers its own query stream; the job's time is
# the slowest rank's, its work the sum over ranks.
def rank_queries(w, rank: int, m: int = 0) -> np.ndarray:
    """This rank's query set: an independent draw of the workload's query
    distribution (stream = rank); m > 0: the first m queries of it."""
    return w.queries(m if m > 0 else None, stream=rank)


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The maximum of x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, m: int, steps: int, ms_max: float) -> float:
    """Queries per second of the whole job: every rank answered m queries
    per step; the timed region ends with the slowest rank."""
    return world * m * steps / (ms_max / 1000.0)


# ------------------------------------------------------------------- arms
def run_reference(a, w):
    """Reference arm: the oracle on bounded samples of the same workload."""
    import oracle
    P = w.points()
    Q = w.queries()
    tree = oracle.build_tree(P, w.height)
    rng = np.random.default_rng(11)
    probe = Q[rng.choice(Q.shape[0], 256, replace=False)]
    t0 = time.perf_counter()
    tree.knn(probe, w.k)
    per_q = (time.perf_counter() - t0) / 256
    budget = 150.0 / max(1, a.steps + a.warmup)    # seconds per step
    s = int(min(Q.shape[0], max(256, budget / max(per_q, 1e-9))))
    times = []
    for step in range(a.warmup + a.steps):
        rows = rng.choice(Q.shape[0], s, replace=False)
        t0 = time.perf_counter()
        tree.knn(Q[rows], w.k)
        if step >= a.warmup:
            times.append(time.perf_counter() - t0)
    total = float(np.sum(times))
    value = s * a.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "queries/s", "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1000 * total / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": dict(w.describe(), sample_queries_per_step=s),
        "cpu_baseline": {"value": value, "unit": "queries/s",
                         "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": f"{s} seeded queries per step of "
                                   f"{Q.shape[0]}, binary64 k-d tree"},
        "e2e": {"value": value, "unit": "queries/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def latency_sample(bkd, tree, Q, seconds: float, barrier) -> dict:
    """p50 / p99 wall latency of single bkd_query calls on a seeded sequence
    of batches (host buffers, pinned), until `seconds` have passed."""
    import torch
    if seconds <= 0:
        return None
    rng = np.random.default_rng(12345)
    m = Q.shape[0]
    Qh = torch.from_numpy(Q).pin_memory()
    kmax = 50
    oi = torch.empty((1 << 20) * kmax, dtype=torch.int64).pin_memory()
    od = torch.empty((1 << 20) * kmax, dtype=torch.float32).pin_memory()
    lat, sizes, ks = [], [], []
    barrier()
    t_end = time.perf_counter() + seconds
    while time.perf_counter() < t_end and len(lat) < 2000:
        b = int(min(m, np.exp(rng.uniform(0.0, np.log(1 << 20)))))
        k = int(rng.choice([1, 10, 50]))
        s0 = int(rng.integers(0, m - b + 1))
        t0 = time.perf_counter()
        bkd.bkd_query(tree, Qh[s0:s0 + b], k, oi[:b * k].view(b, k),
                      od[:b * k].view(b, k))
        lat.append(time.perf_counter() - t0)
        sizes.append(b)
        ks.append(k)
    lat_ms = np.array(lat) * 1e3
    return {"batches": len(lat), "p50_ms": float(np.percentile(lat_ms, 50)),
            "p99_ms": float(np.percentile(lat_ms, 99)),
            "mean_batch": float(np.mean(sizes)),
            "queries_per_s": float(np.sum(sizes) / np.sum(lat)),
            "p50_ms_batches_le_1024": float(np.percentile(
                lat_ms[np.array(sizes) <= 1024], 50))
            if (np.array(sizes) <= 1024).any() else None,
            "recipe": ("sizes logU[1, 2^20] (capped at m), k uniform in "
                       "{1, 10, 50}, queries sliced from the query set, "
                       "pinned host in / out, one call at a time, seed "
                       "12345")}


def serving_sample(bkd, tree, Q, seconds: float, rate: float,
                   max_batch: int = 1 << 20, slots: int = 1 << 22,
                   backlog: int = 1 << 23, seed: int = 777):
    """Continuous batching (bkd_serve_*) under a seeded Poisson stream of
    batches: `rate` batches/s for `seconds`, sizes log-uniform in [1,
    max_batch], k uniform in {1, 10, 50}, queries from pinned host memory,
    results into device buffers.  The server (k_max 50, `slots` query slots)
    steps continuously; a batch that arrives while the queries submitted
    and not yet completed exceed `backlog` is rejected at the door.
    Latency = completion minus arrival (wall clock); at the end the batches
    still queued or running are counted and dropped."""
    import torch
    if seconds <= 0:
        return None
    rng = np.random.default_rng(seed)
    m = Q.shape[0]
    Qh = torch.from_numpy(Q).pin_memory()
    dev = torch.device("cuda", torch.cuda.current_device())
    srv = bkd.Server(tree, k_max=50, max_queries=slots)
    arrivals, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            break
        b = int(min(m, max_batch, np.exp(rng.uniform(0.0, np.log(max_batch)))))
        arrivals.append((t, b, int(rng.choice([1, 10, 50])),
                         int(rng.integers(0, m - b + 1))))
    live, lat, served, steps = {}, [], 0, 0
    rejected = rejected_q = accepted = 0
    outstanding = 0
    t0 = time.perf_counter()
    nxt = 0
    while nxt < len(arrivals):
        now = time.perf_counter() - t0
        while nxt < len(arrivals) and arrivals[nxt][0] <= now:
            ta, b, k, s0 = arrivals[nxt]
            nxt += 1
            if outstanding + b > backlog:
                rejected += 1
                rejected_q += b
                continue
            oi = torch.empty((b, k), dtype=torch.int64, device=dev)
            od = torch.empty((b, k), dtype=torch.float32, device=dev)
            live[srv.submit(Qh[s0:s0 + b], k, oi, od)] = (ta, b)
            outstanding += b
            accepted += 1
        if not live:
            if nxt < len(arrivals):
                time.sleep(max(0.0, arrivals[nxt][0] - now))
            continue
        pending = srv.step()
        steps += 1
        if pending < len(live):  # some batch completed: find it
            now = time.perf_counter() - t0
            for tk in list(live):
                if srv.status(tk) == bkd.BKD_BATCH_DONE:
                    ta, b = live.pop(tk)
                    srv.result(tk)
                    lat.append(now - ta)
                    served += b
                    outstanding -= b
    wall = time.perf_counter() - t0
    left = len(live)
    srv.close()
    lat_ms = np.array(lat) * 1e3 if lat else np.array([np.nan])
    offered = sum(b for _, b, _, _ in arrivals) / seconds
    return {"rate_batches_per_s": rate, "arrived": len(arrivals),
            "accepted": accepted, "rejected": rejected,
            "rejected_queries": rejected_q, "completed": len(lat),
            "unfinished_at_end": left,
            "p50_ms": float(np.percentile(lat_ms, 50)),
            "p99_ms": float(np.percentile(lat_ms, 99)),
            "served_queries_per_s": served / wall,
            "offered_queries_per_s": offered, "steps": steps,
            "recipe": (f"Poisson arrivals of {rate:.0f} batches/s for "
                       f"{seconds:.1f} s (seed {seed}), sizes logU[1, "
                       f"{max_batch}], k uniform in {{1, 10, 50}}, queries "
                       f"from pinned host memory, results into device "
                       f"buffers; one server (k_max 50, {slots} query "
                       f"slots) stepping continuously; a batch arriving "
                       f"while more than {backlog} submitted queries are "
                       f"unfinished is rejected; latency = completion - "
                       f"arrival over the completed batches; served = "
                       f"queries of completed batches / wall time")}


def run_ours(a, w, rank, world, local_rank):
    import torch
    import paper_1512_02831_gb300 as bkd

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def rank_max(x: float) -> float:
        return max_over_ranks(x, dist, dev)

    P = w.points()
    Q = rank_queries(w, rank, a.queries)
    m, k, d = Q.shape[0], w.k, w.d
    modes = [x.strip() for x in a.modes.split(",") if x.strip()]
    if not set(modes) <= {"fp32", "warp", "tcgen05"} or "fp32" not in modes:
        raise SystemExit("--modes: a subset of fp32,warp,tcgen05 with fp32")
    t0 = time.perf_counter()
    # the point layouts of the BF16 screen kernels timed (warp / mma.sync
    # and tcgen05): each is timed, the fastest configuration is the headline
    kernels = 2 if {"warp", "tcgen05"} <= set(modes) else (
        1 if "tcgen05" in modes else 0)
    tree = bkd.bkd_build(P, w.height, precision=1, screen_kernel=kernels)
    build_s = time.perf_counter() - t0
    if a.serving_defer:
        bkd.bkd_set_option(tree, "defer_queries", a.serving_defer)
    if a.serving_only:
        del P
        # the serving samples alone (the resident tree of the workload)
        serving = [serving_sample(bkd, tree, Q, a.serving_seconds, r,
                                  slots=a.serving_slots,
                                  backlog=a.serving_backlog)
                   for r in a.serving_rates]
        bkd.bkd_free(tree)
        if rank == 0:
            print(json.dumps({"metric": "serving (continuous batching)",
                              "workload": w.name,
                              "config": dict(w.describe(),
                                             tree_build_s=round(build_s, 2),
                                             slots=a.serving_slots,
                                             backlog=a.serving_backlog,
                                             defer_queries=a.serving_defer),
                              "serving": serving}), flush=True)
        return
    Qd = torch.from_numpy(Q).to(dev)
    out_i = torch.empty((m, k), dtype=torch.int64, device=dev)
    out_d = torch.empty((m, k), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    stats_keys = ("rounds", "leaf_visits", "pairs", "resorted", "fallback",
                  "leaf_kernel_ms", "kernel_launches", "leaf_launches",
                  "tail_queries", "tail_visits", "tail_pairs", "tail_ms",
                  "screen_kept", "screen_pairs", "screen_ms", "screen_items",
                  "screen_visits", "find_ms", "bucket_ms", "exact_ms",
                  "screen_bytes", "leaf_bytes", "host_syncs")
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    vis = [v for v in vis.split(",") if v.strip()]
    smi_index = (vis[local_rank] if local_rank < len(vis)
                 and vis[local_rank].strip().isdigit() else local_rank)

    def timed(precision: int, kernel: int = 0) -> dict:
        """W warm-up + K timed bkd_query steps with leaf scoring
        `precision` (0 float32, 1 BF16 screen + float32 rescoring) and, for
        the screen, `kernel` (0 warp / mma.sync, 1 tcgen05)."""
        bkd.bkd_set_option(tree, "precision", precision)
        if precision:
            bkd.bkd_set_option(tree, "screen_kernel", kernel)
        for _ in range(a.warmup):
            bkd.bkd_query(tree, Qd, k, out_i, out_d)
        barrier()
        clocks = Clocks(smi_index)
        clocks.start()
        acc = {s: 0.0 for s in stats_keys}
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        for _ in range(a.steps):
            bkd.bkd_query(tree, Qd, k, out_i, out_d)
            for s in stats_keys:
                acc[s] += bkd.bkd_get_stat(tree, s)
        ev1.record(stream)
        barrier()
        clk = clocks.stop()
        ms = ev0.elapsed_time(ev1)
        ms_max = rank_max(ms)
        return {"acc": acc, "clk": clk, "ms": ms, "ms_max": ms_max,
                "value": whole_job_rate(world, m, a.steps, ms_max),
                "idx": out_i.clone(), "dist": out_d.clone()}

    # runs: 0 float32, 1 warp screen, 2 tcgen05 screen (those asked for)
    runs = {0: timed(0)}
    if "warp" in modes:
        runs[1] = timed(1, 0)
    if "tcgen05" in modes:
        runs[2] = timed(1, 1)
    identical = all(bool(torch.equal(runs[0]["idx"], runs[r]["idx"])
                         and torch.equal(runs[0]["dist"], runs[r]["dist"]))
                    for r in runs if r)
    head = max(runs, key=lambda r: runs[r]["value"])
    acc, clk, ms, ms_max = (runs[head][x] for x in ("acc", "clk", "ms",
                                                     "ms_max"))
    value = runs[head]["value"]
    bkd.bkd_set_option(tree, "precision", 0 if head == 0 else 1)
    if head:
        bkd.bkd_set_option(tree, "screen_kernel", 1 if head == 2 else 0)
    out_i.copy_(runs[head]["idx"])

    # end to end through the same call, host buffers (pinned), copies inside
    Qh = torch.from_numpy(Q).pin_memory()
    oi_h = torch.empty((m, k), dtype=torch.int64).pin_memory()
    od_h = torch.empty((m, k), dtype=torch.float32).pin_memory()
    bkd.bkd_query(tree, Qh, k, oi_h, od_h)
    barrier()
    t0 = time.perf_counter()
    for _ in range(a.e2e_steps):
        bkd.bkd_query(tree, Qh, k, oi_h, od_h)
    barrier()
    e2e_s = rank_max(time.perf_counter() - t0)
    e2e = {"value": whole_job_rate(world, m, a.e2e_steps, e2e_s * 1000.0),
           "unit": "queries/s",
           "h2d_bytes_per_step": int(Q.nbytes),
           "d2h_bytes_per_step": int(oi_h.numel() * 8 + od_h.numel() * 4),
           "buffers": "pinned host, bkd_query copies in and out"}
    same = bool(torch.equal(oi_h, out_i.cpu()))

    # per-batch latency: a seeded sequence of batches (sizes log-uniform in
    # [1, 2^20], k in {1, 10, 50}) through the same public call with pinned
    # host buffers, one after the other on the resident tree
    lat = latency_sample(bkd, tree, Q, a.latency_seconds, barrier)
    serving = [serving_sample(bkd, tree, Q, a.serving_seconds, r,
                              slots=a.serving_slots,
                              backlog=a.serving_backlog)
               for r in a.serving_rates] if a.serving_seconds > 0 else None

    # rooflines: the float32 leaf kernel (from the float32 run) and the BF16
    # screen kernel (from the screened run)
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070)
    peak_ops = 128 * sm_count * sm_max * 1e6 / 1e12      # Top/s
    a0 = runs[0]["acc"]
    leaf_s = a0["leaf_kernel_ms"] / 1000.0
    achieved = 2 * d * a0["pairs"] / leaf_s / 1e12 if leaf_s > 0 else 0.0
    roof_fp32 = {
        "bound": "alu", "kernel": "leaf_pipe_kernel (ProcessAllBuffers, fp32)",
        "achieved": achieved, "peak": peak_ops, "unit": "Top/s",
        "frac": achieved / peak_ops,
        "traffic": leaf_traffic_per_launch(a0, a0["leaf_launches"]),
        "algorithmic_bytes_per_launch": (a0["leaf_bytes"]
                                         / max(a0["leaf_launches"], 1)),
        "staged_bytes_per_step": a0["leaf_bytes"] / a.steps,
        "basis": (f"FP32 pipe operations: 2*d = {2 * d} per scored (query, "
                  f"point) pair (d subtractions + d multiply-adds); peak = "
                  f"128 FP32 lanes x {sm_count} SMs x {sm_max:.0f} MHz "
                  f"(max SM clock of measured peaks), 'of measured'; time = "
                  f"CUDA events around every leaf-kernel launch on its "
                  f"stream"),
        "leaf_share_of_step": leaf_s / (runs[0]["ms"] / 1000.0),
        "flop_view": {"flops_per_pair": 3 * d,
                      "achieved_tflops": 1.5 * achieved,
                      "peak_tflops_fma2": 2 * peak_ops},
    }
    dp = min(c for c in (2, 4, 6, 8, 10, 12, 16, 24, 32) if c >= d)
    peak_bf16 = float(peaks.get("bf16_tflops") or 1900.0)
    peak_hbm = float(peaks.get("hbm_gbs") or 6800.0)

    def roof_screen(run: int) -> dict:
        """Roofline of a BF16 screen kernel from its timed run (1 warp, 2
        tcgen05): HBM-bound on the streamed bf16 point operands."""
        kernel = run - 1
        a1 = runs[run]["acc"]
        # k-halves: d offsets + 2 norm slots (warp kernel; its threshold is
        # compared in the epilogue), + 3 threshold slots (tcgen05)
        kh = (d + 2 + 15) // 16 if kernel == 0 else (d + 5 + 15) // 16
        scr_s = a1["screen_ms"] / 1000.0
        pairs_s = a1["screen_pairs"] / scr_s if scr_s else 0.0
        # algorithmic bytes of the screen: the bf16 operand tiles of every
        # work item's leaf (counted by the kernel) plus, per (query, leaf)
        # visit, the query's padded row and its list bound and id
        scr_bytes = a1["screen_bytes"] + a1["screen_visits"] * (4 * dp + 8)
        # one screen launch per LazySearch round after the first
        scr_launches = max(a1["rounds"] - a.steps, 0)
        scr_gbs = scr_bytes / scr_s / 1e9 if scr_s else 0.0
        scr_tf = 2 * 16 * kh * pairs_s / 1e12
        tensor_view = {"achieved": scr_tf, "peak": peak_bf16,
                       "unit": "TFLOP/s", "frac": scr_tf / peak_bf16,
                       "basis": (f"2 x {16 * kh} flops per screened pair; "
                                 f"peak = measured cuBLAS bf16 burst, 'of "
                                 f"measured'")}
        unit = ("32-point super-tiles x 32 kh B per point, one pass per "
                "work item of <= 32 queries of a leaf" if kernel == 0 else
                "128-point tiles x 32 kh B per point, one pass per work "
                "item of <= 128 queries of a leaf, + the items' query "
                "operand rows")
        return {
            "bound": "hbm",
            "kernel": ("screen_kernel (warp items, mma.sync, in-warp fp32 "
                       "rescore)" if kernel == 0 else
                       "prep + screen + rescore kernels (tcgen05.mma into "
                       "tensor memory, bulk copies, fp32 rescore)"),
            "achieved": scr_gbs, "peak": peak_hbm, "unit": "GB/s",
            "frac": scr_gbs / peak_hbm,
            "traffic": screen_traffic_per_launch(a1, scr_launches, kernel),
            "algorithmic_bytes_per_launch": scr_bytes / max(scr_launches, 1),
            "basis": (f"algorithmic bytes = bf16 operands streamed ({unit}) "
                      f"+ {4 * dp + 8} B per (query, leaf) visit; time = "
                      "CUDA events around every screened round's "
                      "ProcessAllBuffers on its stream; peak = measured HBM "
                      "copy bandwidth, 'of measured'"),
            "bytes_per_step": scr_bytes / a.steps,
            "streamed_operand_bytes_per_step": a1["screen_bytes"] / a.steps,
            "tensor_view": tensor_view,
            "screen_share_of_step": scr_s / (runs[run]["ms"] / 1000.0),
            "pairs_per_s": pairs_s,
            "kept_fraction": (a1["screen_kept"] / a1["screen_pairs"]
                              if a1["screen_pairs"] else None),
        }

    roof_bf16 = roof_screen(1) if 1 in runs else None
    roof_tc = roof_screen(2) if 2 in runs else None
    # DRAM traffic over the algorithmic bytes (re-reads above 1.0)
    for r in (roof_fp32, roof_bf16, roof_tc):
        if r and r.get("traffic") and r.get("algorithmic_bytes_per_launch"):
            r["traffic_over_algorithmic"] = (r["traffic"]
                                             / r["algorithmic_bytes_per_launch"])
    roofline = {0: roof_fp32, 1: roof_bf16, 2: roof_tc}[head]
    names = {0: "fp32 exact path",
             1: "bf16 tensor-core screen (warp kernel) + fp32 rescore",
             2: "bf16 tensor-core screen (tcgen05 kernel) + fp32 rescore"}

    line = {
        "metric": METRIC, "value": value, "unit": "queries/s",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms_max / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16+f32" if head else "f32",
        "data": data_description(w),
        "config": dict(w.describe(), precision=names[head],
                       queries_timed_per_step=m,
                       parallelism=f"replicas x{world}, queries sharded",
                       l2=l2_note(w),
                       tree_build_s=round(build_s, 2)),
        "e2e": e2e,
        "latency": lat,
        "serving": serving,
        "gpu_launches": int(acc["kernel_launches"]),
        "roofline": roofline,
        "roofline_fp32_leaf": roof_fp32,
        "roofline_bf16_screen": roof_bf16,
        "roofline_tcgen05_screen": roof_tc,
        "fp32_vs_bf16": {
            "fp32": {"value": runs[0]["value"],
                     "ms_per_step": runs[0]["ms_max"] / a.steps,
                     "clocks": runs[0]["clk"]},
            "bf16_screened": ({"value": runs[1]["value"],
                               "ms_per_step": runs[1]["ms_max"] / a.steps,
                               "screen_ms_per_step":
                                   runs[1]["acc"]["screen_ms"] / a.steps,
                               "clocks": runs[1]["clk"]}
                              if 1 in runs else None),
            "bf16_screened_tcgen05": ({
                "value": runs[2]["value"],
                "ms_per_step": runs[2]["ms_max"] / a.steps,
                "screen_ms_per_step": runs[2]["acc"]["screen_ms"] / a.steps,
                "clocks": runs[2]["clk"]} if 2 in runs else None),
            "identical_results": identical,
            "headline": names[head]},
        "clocks": clk,
        "path": {"rounds_per_step": acc["rounds"] / a.steps,
                 "leaf_visits_per_query": (acc["leaf_visits"]
                                           + acc["tail_visits"])
                 / (m * a.steps),
                 "tail_queries_per_step": acc["tail_queries"] / a.steps,
                 "tail_visits_per_step": acc["tail_visits"] / a.steps,
                 "tail_ms_per_step": acc["tail_ms"] / a.steps,
                 "pairs_per_step": acc["pairs"] / a.steps,
                 "leaf_kernel_ms_per_step": acc["leaf_kernel_ms"] / a.steps,
                 "leaf_launches_per_step": acc["leaf_launches"] / a.steps,
                 "resorted_per_step": acc["resorted"] / a.steps,
                 "fallback_per_step": acc["fallback"] / a.steps,
                 "screen_pairs_per_step": acc["screen_pairs"] / a.steps,
                 "screen_kept_per_step": acc["screen_kept"] / a.steps,
                 "screen_ms_per_step": acc["screen_ms"] / a.steps,
                 "screen_queries_per_item": (acc["screen_visits"]
                                             / acc["screen_items"]
                                             if acc["screen_items"] else None),
                 "find_leaf_ms_per_step": acc["find_ms"] / a.steps,
                 "host_syncs_per_step": acc["host_syncs"] / a.steps,
                 "bucket_ms_per_step": acc["bucket_ms"] / a.steps,
                 "recheck_fallback_ms_per_step": acc["exact_ms"] / a.steps,
                 "e2e_matches_device_run": same},
    }
    bkd.bkd_free(tree)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        info, rows, ref = cpu_baseline(P, Q, w, a.cpu_seconds)
        line["cpu_baseline"] = info
        got = out_i.cpu().numpy()[rows]
        exempt = ref.gap_exempt(1e-6)
        line["parity_sample"] = {
            "queries": int(len(rows)),
            "index_rows_equal": int((got == ref.idx).all(1).sum()),
            "gap_exempt": int(exempt.sum()),
            "non_exempt_mismatch": int((~exempt & ~(got == ref.idx).all(1))
                                       .sum())}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_streamer(a):
    """Bigger mode: the leaf structure in pinned host memory, streamed through
    two device chunk buffers on a copy stream (the chunk streamer).  Modes:
    resident; leaf-aligned chunks N in {1, 3, 10} (the resident chunks keep
    running while they hold buffered queries); the paper's point chunks N in
    {3, 10} (every chunk with buffered queries streamed every round).  Per
    mode: queries/s, bytes copied and passes over the leaf structure,
    copy-stream bandwidth against a pinned host-to-device copy measured
    here, and equality with the resident tree's results."""
    import torch
    import paper_1512_02831_gb300 as bkd
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if a.streamer_n:
        w = workloads.scaled(workloads.MIXTURE_64M, a.streamer_n,
                             a.streamer_m, a.streamer_h)
    else:
        w = WORKLOADS["mixture16M"]
    t0 = time.perf_counter()
    P, Q = w.points(), w.queries()
    gen_s = time.perf_counter() - t0
    m, k = Q.shape[0], w.k
    Qd = torch.from_numpy(Q).to(dev)
    # host-to-device peak: 1 GiB from pinned memory, best of 5
    src = torch.empty(1 << 28, dtype=torch.float32).pin_memory()
    dst = torch.empty(1 << 28, dtype=torch.float32, device=dev)
    best = 0.0
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, src.numel() * 4 / (e0.elapsed_time(e1) / 1e3) / 1e9)
    del src, dst
    dp = min(c for c in (2, 4, 6, 8, 10, 12, 16, 24, 32) if c >= w.d)
    structure = w.n * dp * 4
    out = {"metric": "chunk streamer (bigger mode)", "workload": w.describe(),
           "h2d_peak_gbs": best, "leaf_structure_gb": structure / 1e9,
           "data_generation_s": round(gen_s, 1), "modes": {}}
    ref = None
    if a.streamer_modes:
        modes = []
        for name in a.streamer_modes.split(","):
            name = name.strip()
            if name == "resident":
                modes.append((name, {}))
            elif name.startswith("chunks="):
                modes.append((name, {"chunks": int(name.split("=")[1])}))
            elif name.startswith("point_chunks="):
                modes.append((name, {"chunks": int(name.split("=")[1]),
                                     "point_chunks": 1}))
            else:
                raise SystemExit(f"--streamer-modes: unknown mode {name}")
    else:
        modes = [("resident", {})] if not a.streamer_n or a.streamer_resident \
            else []
        modes += [(f"chunks={c}", {"chunks": c}) for c in (1, 3, 10)]
        modes += [(f"point_chunks={c}", {"chunks": c, "point_chunks": 1})
                  for c in (3, 10)]
    for name, opts in modes:
        if a.streamer_precision and not opts.get("point_chunks"):
            opts = dict(opts, precision=1)
        t0 = time.perf_counter()
        tree = bkd.bkd_build(P, w.height, **opts)
        build_s = time.perf_counter() - t0
        if w.n <= (1 << 27):
            bkd.bkd_query(tree, Qd, k)  # warm-up (skipped for huge trees)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        idx, dist = bkd.bkd_query(tree, Qd, k)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st = {x: bkd.bkd_get_stat(tree, x)
              for x in ("chunk_bytes", "copy_ms", "rounds", "leaf_kernel_ms",
                        "chunk_visits", "leaf_visits", "mapped_bytes",
                        "host_syncs")}
        shape = bkd.bkd_tree_shape(tree)
        bkd.bkd_free(tree)
        if ref is None:
            ref = (idx.clone(), dist.clone())
        gbs = (st["chunk_bytes"] / (st["copy_ms"] / 1e3) / 1e9
               if st["copy_ms"] > 0 else None)
        out["modes"][name] = {
            "chunked": shape["chunked"], "chunks": shape["chunks"],
            "precision": opts.get("precision", 0),
            "queries_per_s": m / dt, "ms": dt * 1e3, "build_s": build_s,
            "rounds": st["rounds"],
            "copied_gb": st["chunk_bytes"] / 1e9,
            "passes_over_structure": st["chunk_bytes"] / structure,
            "copy_ms": st["copy_ms"], "copy_gbs": gbs,
            "copy_frac_of_h2d_peak": gbs / best if gbs else None,
            "mapped_gb": st["mapped_bytes"] / 1e9,
            "host_syncs": st["host_syncs"],
            "leaf_kernel_ms": st["leaf_kernel_ms"],
            "identical_to_first_mode": bool(torch.equal(idx, ref[0])
                                            and torch.equal(dist, ref[1]))}
        print(json.dumps({name: out["modes"][name]}), flush=True)
    base = out["modes"].get("resident")
    if base:
        for v in out["modes"].values():
            v["q_per_s_ratio_to_resident"] = (v["queries_per_s"]
                                              / base["queries_per_s"])
    if a.streamer_oracle_rows > 0 and ref is not None:
        # cpu_baseline leg: the oracle's brute force (the definition,
        # binary64, all host cores) timed on a seeded sample of the queries;
        # the same rows give the parity of the GPU result
        import oracle
        rng = np.random.default_rng(11)
        rows = np.sort(rng.choice(m, min(m, a.streamer_oracle_rows),
                                  replace=False))
        t0 = time.perf_counter()
        res = oracle.brute_knn(P, Q[rows], k)
        dt = time.perf_counter() - t0
        got = ref[0].cpu().numpy()[rows]
        exempt = res.gap_exempt(1e-6)
        eq = (got == res.idx).all(1)
        out["cpu_baseline"] = {
            "value": len(rows) / dt, "unit": "queries/s",
            "cores": oracle.max_threads(), "kind": "oracle",
            "sample": (f"{len(rows)} of {m} queries (seeded), binary64 brute "
                       f"force over all {w.n} points")}
        out["parity_sample"] = {
            "queries": int(len(rows)), "index_rows_equal": int(eq.sum()),
            "gap_exempt": int(exempt.sum()),
            "non_exempt_mismatch": int((~exempt & ~eq).sum())}
    print(json.dumps(out), flush=True)


def run_autotune(a, w):
    """The autotuner's search on the workload's tree (both screen layouts):
    every candidate's timing (best of 2 after a warm-up, CUDA-synchronous
    wall time of bkd_query on a device-resident query sample), the setting
    it keeps, and that setting's result checked against the default's."""
    import torch
    import paper_1512_02831_gb300 as bkd
    from paper_1512_02831_gb300 import tune
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    P = w.points()
    Q = w.queries(min(w.m, a.autotune_queries))
    tree = bkd.bkd_build(P, w.height, precision=1, screen_kernel=2)
    Qd = torch.from_numpy(Q).to(dev)
    base = bkd.bkd_query(tree, Qd, w.k)
    rep = tune.autotune(tree, Qd, w.k)
    got = bkd.bkd_query(tree, Qd, w.k)
    same = bool(torch.equal(base[0], got[0]) and torch.equal(base[1], got[1]))
    default = {"precision": 1, "screen_kernel": 0, "tail_queries": -1,
               "screen_tile": 32, "round_batch": 0, "screen_ctas": 0}
    dsec = next((t for o, t in rep["timings"] if o == default), None)
    bkd.bkd_free(tree)
    print(json.dumps({"metric": "autotune", "workload": w.describe(),
                      "queries": int(Q.shape[0]), "best": rep["best"],
                      "best_seconds": rep["best_seconds"],
                      "default_seconds": dsec,
                      "best_queries_per_s": Q.shape[0] / rep["best_seconds"],
                      "calls": rep["calls"],
                      "identical_to_default_options": same,
                      "timings": [[o, t] for o, t in rep["timings"]]}),
          flush=True)


def main():
    a = args_()
    w = WORKLOADS[a.workload]
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if a.impl == "reference":
        if rank == 0:
            run_reference(a, w)
        return
    if a.streamer:
        if rank == 0:
            run_streamer(a)
        return
    if a.autotune:
        if rank == 0:
            run_autotune(a, w)
        return
    run_ours(a, w, rank, world, local_rank)


if __name__ == "__main__":
    main()
