"""Benchmark: single-source dense Dijkstra solves per second at n=16384 on GB300.

Workload (default): an undirected graph of n=16384 nodes, each pair an edge with
probability 0.5, int32 weights uniform in [1, 1000] (a 1 GiB int32 adjacency
matrix, larger than the 129 MB L2, so no flush is needed between steps), seed 2.
One step = one complete solve (every phase of the hot path) from a seeded
source; the sources cycle through 64 seeded distinct nodes.

Printed (rank 0, one JSON line): SSSP/s of the device-resident solve (`value`),
the same through the C ABI with host buffers and the matrix copied host->device
every step (`e2e`, the paper's CUDA accounting: memory transfer + kernel), the
roofline of the dominant kernel, the CPU oracle's SSSP/s on the host cores, the
batched and plain-form throughputs, and the SM clocks sampled during the timed
region.  ``--impl reference`` times the CPU oracle instead (bounded sample).

Multi-GPU: one process per GPU (torchrun); every rank solves its own replica of
the workload (independent solves, no collective on the data path) and the
aggregate counts every rank's solves over the slowest rank's time.
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

WORKLOAD = "dense_n16384_p0.5"
METRIC = "SSSP/s (single-source dense Dijkstra, n=16384) and HBM GB/s vs 8 TB/s"
BATCH_WORKLOAD = "multisource_n8192_p0.05_k256"
INF = 2**31 - 1


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.time(), ln.strip()))

    def mark(self):
        self.marks.append(time.time())

    def stop(self) -> dict:
        """Clocks over the window from the first mark (soak start) to the last (end of the timed
        region): the soak and warm-up keep the GPU under the same load, so the window is long
        enough for the 100 ms sampler even when the timed region itself lasts milliseconds."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        t0 = self.marks[0] if self.marks else 0
        t1 = self.marks[-1] if len(self.marks) > 1 else time.time()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            if not (t0 <= ts <= t1):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "window": "soak + warm-up + timed region (the same solve back to back)",
                "window_s": round(t1 - t0, 3), "power_w_max": max(power) if power else None}


def _dist_setup(n_gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("DJ_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
        return dist, rank, world, local
    return None, 0, 1, 0


def _barrier(dist, device=None):
    if dist is not None:
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device])
        else:
            dist.barrier()


def _max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    backend = dist.get_backend()
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if backend == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(per_rank_units: int, world: int, t_max_s: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return per_rank_units * world / t_max_s


def cpu_oracle_rate(W: np.ndarray, sources, budget_s: float):
    """Oracle solves per second on one host core, over a bounded sample (>= 1 solve)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    done = 0
    while True:
        oracle.dijkstra(W, int(sources[done % len(sources)]))
        done += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return done / el, done, el


def run_reference(args):
    """--impl reference: the CPU oracle as it stands, timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import graphgen
    import oracle
    spec = graphgen.WORKLOADS[args.workload]
    e = graphgen.make_graph(spec)
    W = oracle.build_matrix(e.n, e.src, e.dst, e.w, e.directed)
    srcs = graphgen.sources(e.n, 64, spec["seed"])
    for i in range(min(args.warmup, 1)):
        oracle.dijkstra(W, int(srcs[i % 64]))
    # bounded: the K requested solves, or as many as fit in the time budget
    t0 = time.perf_counter()
    done = 0
    while done < args.steps:
        oracle.dijkstra(W, int(srcs[done % 64]))
        done += 1
        if time.perf_counter() - t0 > args.reference_budget_s:
            break
    el = time.perf_counter() - t0
    v = done / el
    line = {"impl": "reference", "metric": METRIC, "value": v,
            "unit": "SSSP/s", "n_gpus": args.gpus, "steps": done, "steps_requested": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / done, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "n": e.n, "p": spec.get("p"), "weights": [spec["wlo"], spec["whi"]],
                       "seed": spec["seed"], "sources": "64 seeded distinct, cycled",
                       "l2": "inputs larger than L2 (1 GiB matrix)", "parallelism": "one host core"},
            "cpu_baseline": {"value": v, "unit": "SSSP/s", "cores": 1, "kind": "oracle",
                             "sample": f"{done} serial Algorithm 1 solves (plain C, 1 thread) at n={e.n}"},
            "e2e": {"value": v, "unit": "SSSP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-budget-s", type=float, default=10.0)
    ap.add_argument("--reference-budget-s", type=float, default=90.0)
    ap.add_argument("--soak-s", type=float, default=1.0, help="untimed load before warm-up (clock sampling)")
    ap.add_argument("--no-extras", action="store_true", help="skip the batch / plain-form / e2e side measurements")
    ap.add_argument("--trace", action="store_true", help="print the per-phase device timeline of one solve and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import graphgen
    import __graft_entry__
    dist, rank, world, local = _dist_setup(args.gpus)
    torch.cuda.set_device(local)
    __graft_entry__.build()
    from paper_2504_03667_gb300 import dj

    spec = graphgen.WORKLOADS[args.workload]
    e = graphgen.make_graph(spec)
    n = e.n
    g = dj.dj_load_edges(n, e.src, e.dst, e.w, e.directed)
    srcs = graphgen.sources(n, 64, spec["seed"])
    stream = torch.cuda.Stream()
    dist_t = torch.empty(n, dtype=torch.int32, device="cuda")
    pred_t = torch.empty(n, dtype=torch.int32, device="cuda")

    def step(i):
        dj.dj_sssp(g, int(srcs[i % 64]), dist_t, pred_t, stream)

    if args.trace:
        return print_trace(dj, torch, g, int(srcs[0]), n, stream)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.25)  # the sampler's first lines
    # untimed soak so the clock sampler sees the GPU under this load
    clocks.mark()
    t_soak = time.time()
    i = 0
    while time.time() - t_soak < args.soak_s:
        step(i)
        i += 1
        if i % 50 == 0:
            stream.synchronize()
    for i in range(args.warmup):
        step(i)
    dj.dj_sync(stream)
    _barrier(dist, local)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(i)
    e1.record(stream)
    e1.synchronize()
    clocks.mark()
    torch.cuda.synchronize()
    _barrier(dist, local)
    dj.dj_sync(stream)
    clock_info = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    t_max = _max_over_ranks(dist, ms_total / 1e3)
    value = aggregate(args.steps, world, t_max)
    ms_per_step = 1e3 * t_max / args.steps
    phases = dj.dj_last_phases()

    # roofline of the dominant kernel (k_sssp_grid): algorithmic bytes = n^2 * 4 per solve
    alg_bytes = n * n * 4
    per_launch_s = (ms_total / 1e3) / args.steps
    achieved = alg_bytes / per_launch_s / 1e9
    peak, peak_kind = _peaks()
    traffic, traffic_note = _traffic(f"k_sssp_grid_dense_n{n}_traffic.txt", n)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": f"{peak_kind} hbm_gbs (STREAM-style copy)",
                "frac_of_8tbs": achieved / 8000.0, "algorithmic_bytes_per_launch": alg_bytes,
                "kernel": "k_sssp_grid", "traffic_note": traffic_note,
                "dram_gbs_from_traffic": (traffic / per_launch_s / 1e9) if traffic else None}

    extras = {}
    if rank == 0 and not args.no_extras:
        extras = side_measurements(dj, torch, graphgen, g, e, srcs, stream)

    cpu = None
    if rank == 0:
        import oracle
        oracle.build()
        W = oracle.build_matrix(n, e.src, e.dst, e.w, e.directed)
        rate, done, el = cpu_oracle_rate(W, srcs, args.cpu_budget_s)
        cpu = {"value": rate, "unit": "SSSP/s", "cores": 1, "kind": "oracle",
               "sample": f"{done} serial Algorithm 1 solves (plain C, 1 thread) of the same n={n} workload in {el:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "SSSP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "p": spec.get("p"), "weights": [spec["wlo"], spec["whi"]],
                       "seed": spec["seed"], "sources": "64 seeded distinct, cycled", "engine": "grid (cooperative)",
                       "mode": "phase-batched exact", "phases_last_solve": phases,
                       "l2": "inputs larger than L2 (1 GiB matrix), no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roofline,
            "hbm_gbs_algorithmic": achieved,
            "cpu_baseline": cpu,
            "clocks": clock_info,
            "gpu_launches": args.steps,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


TRAFFIC_FILES = {"dense_n1024_p0.1": "k_sssp_cluster_dense_n1024_traffic.txt",
                 "sparse_directed_n32768_deg8": "k_sssp_grid_sparse_n32768_traffic.txt"}


def _traffic(fname: str, n: int):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on this kernel source."""
    path = os.path.join(ROOT, "profiles", fname)
    try:
        kv = {}
        for ln in open(path):
            if ":" in ln and not ln.startswith("#"):
                k, v = ln.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_source_hash") != _kernel_hash():
            return None, "kernel changed since the ncu capture"
        per = int(kv["dram_bytes_per_launch"])
        return per, (f"ncu dram__bytes_read+write per launch at n={n} (1-pass capture, mean of the launches in "
                     f"profiles/{fname})")
    except (OSError, KeyError, ValueError):
        return None, "no ncu capture"


def _kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("dj_core.cuh", "dj_solve.cu", "dj_common.cuh"):
        with open(os.path.join(ROOT, "paper_2504_03667_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def print_trace(dj, torch, g, source: int, n: int, stream):
    """Per-phase timeline of one grid-engine solve (CTA 0's %globaltimer stamps)."""
    tr = torch.zeros(8 * 4096, dtype=torch.int64, device="cuda")
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    p = torch.empty_like(d)
    for _ in range(3):
        dj.dj_sssp(g, source, d, p, stream)
    dj.dj_sssp_ex(g, source, d, p, dj.make_solve_opts(engine=dj.DJ_ENGINE_GRID, trace=tr), stream)
    dj.dj_sync(stream)
    phases = dj.dj_last_phases()
    tall = tr.cpu().numpy()
    t = tall.reshape(-1, 8)[: phases + 1]
    names = ["publish_us", "arrive_us", "barrier_wait_us", "decision_us", "relax_us", "commit_us"]
    rows = []
    for i in range(phases):
        d_ = {"phase": i, "candidates": int(t[i, 7]) & 0xFFFFFFFF, "cta0_live_groups": int(t[i, 7]) >> 32}
        for k, nm in enumerate(names):
            d_[nm] = (t[i, k + 1] - t[i, k]) / 1e3
        d_["relax_gbs_upper"] = d_["candidates"] * n * 4 / max(t[i, 5] - t[i, 4], 1)
        rows.append(d_)
    sums = {nm: sum(r[nm] for r in rows) for nm in names}
    print(json.dumps({"phases": phases, "total_us": (t[phases, 4] - t[0, 0]) / 1e3, "sums_us": sums,
                      "prologue_us": (t[0, 0] - tall[-2]) / 1e3, "epilogue_us": (tall[-1] - t[phases, 4]) / 1e3,
                      "candidates_total": int(sum(r["candidates"] for r in rows)), "n": n,
                      "per_phase": rows if phases <= 64 else rows[:8]}), flush=True)


def side_measurements(dj, torch, graphgen, g, e, srcs, stream) -> dict:
    """e2e through host buffers, the batched workload and the plain one-launch-per-solve form."""
    out = {}
    n = e.n
    # e2e: matrix host->device (pinned) + solve + dist/pred device->host, every step, timed with
    # CUDA events on the solve stream (dj_sssp_host synchronises it, so host gaps are included)
    numa = _numa_placement(torch)
    W_host = torch.empty((n, n), dtype=torch.int32, pin_memory=True)
    Wnp = dj.dj_graph_download(g)
    W_host.numpy()[:] = Wnp
    del Wnp
    dh = torch.empty(n, dtype=torch.int32, pin_memory=True)
    ph = torch.empty(n, dtype=torch.int32, pin_memory=True)
    for i in range(2):
        dj.dj_graph_upload(g, W_host, stream)
        dj.dj_sssp_host(g, int(srcs[i]), dh, ph, stream)
    steps = 20
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for i in range(steps):
        dj.dj_graph_upload(g, W_host, stream)
        dj.dj_sssp_host(g, int(srcs[i % 64]), dh, ph, stream)
    a1.record(stream)
    a1.synchronize()
    el = a0.elapsed_time(a1) / 1e3
    # the bare host->device copy of the same pinned matrix, for the link's share of a step
    W_dev = torch.empty((n, n), dtype=torch.int32, device="cuda")
    with torch.cuda.stream(stream):
        W_dev.copy_(W_host, non_blocking=True)
        a0.record(stream)
        for _ in range(3):
            W_dev.copy_(W_host, non_blocking=True)
        a1.record(stream)
    a1.synchronize()
    copy_gbs = 3 * n * n * 4 / (a0.elapsed_time(a1) / 1e3) / 1e9
    del W_dev
    out["e2e"] = {"value": steps / el, "unit": "SSSP/s", "h2d_bytes_per_step": n * n * 4,
                  "d2h_bytes_per_step": 2 * n * 4, "steps": steps, "timer": "CUDA events on the solve stream",
                  "bare_h2d_copy_gbs": copy_gbs, "host_numa": numa,
                  "what": "dj_graph_upload (pinned host matrix) + dj_sssp_host (results to pinned host), per step"}
    del W_host
    # resident-graph e2e: only the source in and dist/pred out per step
    t0 = time.perf_counter()
    for i in range(50):
        dj.dj_sssp_host(g, int(srcs[i % 64]), dh, ph, stream)
    el = time.perf_counter() - t0
    out["e2e_resident_graph"] = {"value": 50 / el, "unit": "SSSP/s", "h2d_bytes_per_step": 0,
                                 "d2h_bytes_per_step": 2 * n * 4}
    # plain form: literal Algorithm 1 (one node per step), one launch per solve, synchronous
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    p = torch.empty_like(d)
    o = dj.make_solve_opts(mode=dj.DJ_MODE_PLAIN)
    dj.dj_sssp_ex(g, int(srcs[0]), d, p, o, stream)
    dj.dj_sync(stream)
    t0 = time.perf_counter()
    reps = 3
    for i in range(reps):
        dj.dj_sssp_ex(g, int(srcs[i]), d, p, o, stream)
        dj.dj_sync(stream)
    el = time.perf_counter() - t0
    out["plain_form_n16384"] = {"value": reps / el, "unit": "SSSP/s",
                                "what": "one node per step (Algorithm 1 literally), one launch per solve, synced"}
    # the other single-solve workloads, each with its own roofline (n^2 * 4 bytes per solve)
    out["dense_n1024_p0.1"] = single_workload(dj, torch, graphgen, "dense_n1024_p0.1", stream, 400)
    out["sparse_directed_n32768_deg8"] = single_workload(dj, torch, graphgen, "sparse_directed_n32768_deg8",
                                                         stream, 16)
    # the paper's own GPU formulation (label-correcting sweeps, Algorithms 3 and 4) rebuilt
    # coalesced, on the same workload: exact dist, a shortest-path-tree pred
    for i in range(3):
        dj.dj_sssp_lc(g, int(srcs[i]), d, p, stream)
    dj.dj_sync(stream)
    l0 = torch.cuda.Event(enable_timing=True)
    l1 = torch.cuda.Event(enable_timing=True)
    lreps = 50
    l0.record(stream)
    for i in range(lreps):
        dj.dj_sssp_lc(g, int(srcs[i % 64]), d, p, stream)
    l1.record(stream)
    dj.dj_sync(stream)
    lms = l0.elapsed_time(l1) / lreps
    out["label_correcting_n16384"] = {"value": 1e3 / lms, "unit": "SSSP/s", "us_per_solve": 1e3 * lms,
                                      "sweeps_last_solve": dj.dj_last_phases(),
                                      "what": "dj_sssp_lc: the paper's sweep-until-no-update CUDA variant, "
                                              "one cooperative launch per solve"}
    # the sparse directed n=32768 workload kept in compressed-row form (no 4 GiB matrix)
    sspec = graphgen.WORKLOADS["sparse_directed_n32768_deg8"]
    se = graphgen.make_graph(sspec)
    sg = dj.dj_load_edges_csr(se.n, se.src, se.dst, se.w, se.directed)
    ssrc = graphgen.sources(se.n, 16, sspec["seed"])
    sd = torch.empty(se.n, dtype=torch.int32, device="cuda")
    sp = torch.empty_like(sd)
    for i in range(3):
        dj.dj_sssp(sg, int(ssrc[i]), sd, sp, stream)
    dj.dj_sync(stream)
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for i in range(16):
        dj.dj_sssp(sg, int(ssrc[i]), sd, sp, stream)
    c1.record(stream)
    dj.dj_sync(stream)
    cms = c0.elapsed_time(c1) / 16
    out["sparse_n32768_compressed_rows"] = {"value": 1e3 / cms, "unit": "SSSP/s", "us_per_solve": 1e3 * cms,
                                            "graph_bytes": dj.dj_graph_get_info(sg)["bytes"],
                                            "dense_matrix_bytes": se.n * se.n * 4,
                                            "what": "dj_load_edges_csr + dj_sssp, 16 seeded sources"}
    sg.free()
    # batched workload: 256 sources of one n=8192 graph in one persistent launch
    bspec = graphgen.WORKLOADS[BATCH_WORKLOAD]
    be = graphgen.make_graph(bspec)
    bg = dj.dj_load_edges(be.n, be.src, be.dst, be.w, be.directed)
    bs = graphgen.sources(be.n, bspec["k"], bspec["seed"])
    k = len(bs)
    D = torch.empty((k, be.n), dtype=torch.int32, device="cuda")
    P = torch.empty_like(D)
    b = dj.dj_batch_create([bg] * k, bs, list(D), list(P))
    tune = dj.dj_batch_autotune(b, stream)
    for _ in range(2):
        dj.dj_batch_launch(b, stream)
    dj.dj_sync(stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record(stream)
    for _ in range(reps):
        dj.dj_batch_launch(b, stream)
    e1.record(stream)
    e1.synchronize()
    dj.dj_sync(stream)
    batch_ms = e0.elapsed_time(e1) / reps
    batch_rate = k / (batch_ms / 1e3)
    # plain form on the batch graph: one plain launch per solve, synchronous
    d2 = torch.empty(be.n, dtype=torch.int32, device="cuda")
    p2 = torch.empty_like(d2)
    o = dj.make_solve_opts(mode=dj.DJ_MODE_PLAIN)
    dj.dj_sssp_ex(bg, int(bs[0]), d2, p2, o, stream)
    dj.dj_sync(stream)
    t0 = time.perf_counter()
    reps2 = 5
    for i in range(reps2):
        dj.dj_sssp_ex(bg, int(bs[i]), d2, p2, o, stream)
        dj.dj_sync(stream)
    plain_rate = reps2 / (time.perf_counter() - t0)
    # and the fast single-solve kernel, one launch per solve, synchronous
    t0 = time.perf_counter()
    for i in range(20):
        dj.dj_sssp(bg, int(bs[i]), d2, p2, stream)
        dj.dj_sync(stream)
    single_rate = 20 / (time.perf_counter() - t0)
    out["batch"] = {"workload": BATCH_WORKLOAD, "value": batch_rate, "unit": "SSSP/s", "ms_per_batch": batch_ms,
                    "solves_per_batch": k, "autotune": tune,
                    "hbm_gbs_algorithmic": k * be.n * be.n * 4 / (batch_ms / 1e3) / 1e9,
                    "plain_form_value": plain_rate, "vs_plain_form": batch_rate / plain_rate,
                    "phase_single_launch_value": single_rate, "vs_phase_single_launch": batch_rate / single_rate,
                    "cpu_baseline": batch_cpu_baseline(be, bs)}
    b.free()
    # the same 256 solves on the lockstep multi-source engine (all sources advance phase by phase
    # together, each row block read once per phase for every source that settles it)
    lb = dj.dj_batch_create([bg] * k, bs, list(D), list(P), engine=dj.DJ_BATCH_ENGINE_LOCKSTEP)
    for _ in range(2):
        dj.dj_batch_launch(lb, stream)
    dj.dj_sync(stream)
    e0.record(stream)
    for _ in range(reps):
        dj.dj_batch_launch(lb, stream)
    e1.record(stream)
    e1.synchronize()
    dj.dj_sync(stream)
    lms = e0.elapsed_time(e1) / reps
    out["batch_lockstep"] = {"workload": BATCH_WORKLOAD, "value": k / (lms / 1e3), "unit": "SSSP/s",
                             "ms_per_batch": lms, "phases": dj.dj_last_phases(),
                             "vs_cluster_engine": (k / (lms / 1e3)) / batch_rate,
                             "what": "dj_batch_create(engine=DJ_BATCH_ENGINE_LOCKSTEP); not the default: slower "
                                     "than the cluster engine here (bound by instruction issue)"}
    lb.free()
    bg.free()
    out["serve"] = serving_measurement(dj, torch, graphgen, stream)
    return out


def serving_measurement(dj, torch, graphgen, stream) -> dict:
    """64 resident graphs (n log-uniform in [512, 16384], p uniform in [0.01, 0.5]),
    10000 Poisson requests: saturation throughput, then latency at ~70 % load."""
    spec = graphgen.WORKLOADS["serving_64graphs_10000req"]
    probe = graphgen.serving_trace(spec["graphs"], spec["requests"], 1.0, spec["seed"])
    graphs = []
    t0 = time.perf_counter()
    for gi in range(spec["graphs"]):
        e = graphgen.bernoulli(int(probe.graph_n[gi]), float(probe.graph_p[gi]), spec["wlo"], spec["whi"],
                               int(probe.graph_seed[gi]))
        graphs.append(dj.dj_load_edges(e.n, e.src, e.dst, e.w, False))
        del e
    setup_s = time.perf_counter() - t0
    resident = sum(int(dj.dj_graph_get_info(g)["bytes"]) for g in graphs)
    opts = dj.make_serve_opts(max_slots=512)
    # saturation: every request already waiting at t = 0
    zero = np.zeros(spec["requests"])
    sat = dj.dj_serve(graphs, probe.req_graph, probe.req_source, zero, opts=opts)
    rate = 0.7 * sat["solves_per_s"]
    tr = graphgen.serving_trace(spec["graphs"], spec["requests"], rate, spec["seed"])
    live = dj.dj_serve(graphs, tr.req_graph, tr.req_source, tr.req_arrival_s, opts=opts)
    # the plain form on a sample of the same requests: one literal-Algorithm-1 launch each, synchronous
    o = dj.make_solve_opts(mode=dj.DJ_MODE_PLAIN)
    sample = list(range(0, spec["requests"], spec["requests"] // 16))[:16]
    bufs = {}
    t_plain = 0.0
    for r in sample:
        g = graphs[int(tr.req_graph[r])]
        n = int(dj.dj_graph_get_info(g)["n"])
        if n not in bufs:
            bufs[n] = (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"))
        d, p = bufs[n]
        t1 = time.perf_counter()
        dj.dj_sssp_ex(g, int(tr.req_source[r]), d, p, o, stream)
        dj.dj_sync(stream)
        t_plain += time.perf_counter() - t1
    plain_rate = len(sample) / t_plain
    # the fast single-solve path on the same sample: one dj_sssp launch per request, synchronous
    for r in sample[:2]:
        g = graphs[int(tr.req_graph[r])]
        d, p = bufs[int(dj.dj_graph_get_info(g)["n"])]
        dj.dj_sssp(g, int(tr.req_source[r]), d, p, stream)
    dj.dj_sync(stream)
    t_single = 0.0
    for r in sample:
        g = graphs[int(tr.req_graph[r])]
        d, p = bufs[int(dj.dj_graph_get_info(g)["n"])]
        t1 = time.perf_counter()
        dj.dj_sssp(g, int(tr.req_source[r]), d, p, stream)
        dj.dj_sync(stream)
        t_single += time.perf_counter() - t1
    single_rate = len(sample) / t_single
    for g in graphs:
        g.free()
    cpu = serve_cpu_baseline(graphgen, spec, tr)
    return {"workload": "serving_64graphs_10000req", "graphs": spec["graphs"], "requests": spec["requests"],
            "resident_bytes": resident, "setup_s": setup_s,
            "saturation_solves_per_s": sat["solves_per_s"],
            "rate_per_s": rate, "solves_per_s": live["solves_per_s"], "p50_us": live["p50_us"],
            "p90_us": live["p90_us"], "p99_us": live["p99_us"], "max_us": live["max_us"],
            "deferred_requests": live["rejected"], "kernel_launches": live["kernel_launches"],
            "plain_form_value": plain_rate, "vs_plain_form": live["solves_per_s"] / plain_rate,
            "plain_form_sample": f"{len(sample)} requests of the trace, one plain launch each, synchronous",
            "phase_single_launch_value": single_rate, "vs_phase_single_launch": live["solves_per_s"] / single_rate,
            "phase_single_launch_sample": f"the same {len(sample)} requests, one dj_sssp launch each, synchronous",
            "cpu_baseline": cpu}


def single_workload(dj, torch, graphgen, name: str, stream, reps: int) -> dict:
    """One of the single-source workloads: `reps` back-to-back dj_sssp solves (default engine and
    mode, sources cycling through 16 seeded distinct nodes), timed with CUDA events on the solve
    stream, and its roofline against n^2 * 4 algorithmic bytes per solve."""
    spec = graphgen.WORKLOADS[name]
    e = graphgen.make_graph(spec)
    n = e.n
    g = dj.dj_load_edges(n, e.src, e.dst, e.w, e.directed)
    del e
    srcs = [graphgen.workload_source(spec)] + [int(x) for x in graphgen.sources(n, 15, spec["seed"] + 100)]
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    p = torch.empty_like(d)
    for i in range(5):
        dj.dj_sssp(g, srcs[i % 16], d, p, stream)
    dj.dj_sync(stream)
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for i in range(reps):
        dj.dj_sssp(g, srcs[i % 16], d, p, stream)
    c1.record(stream)
    dj.dj_sync(stream)
    s_per = c0.elapsed_time(c1) / 1e3 / reps
    # latency of one solve on its own: events around a single call, the stream idle before it
    lat = []
    for i in range(20):
        c0.record(stream)
        dj.dj_sssp(g, srcs[i % 16], d, p, stream)
        c1.record(stream)
        c1.synchronize()
        lat.append(c0.elapsed_time(c1) * 1e3)
    # small solves: the same calls captured once into a CUDA graph and replayed, which takes the
    # per-launch cost of stream launches (and the host's per-call work) out of the loop
    graph_us = None
    if n < 4096:
        D = torch.empty((16, n), dtype=torch.int32, device="cuda")
        P = torch.empty_like(D)
        K = 200
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=stream):
            for i in range(K):
                dj.dj_sssp(g, srcs[i % 16], D[i % 16], P[i % 16], stream)
        with torch.cuda.stream(stream):
            for _ in range(3):
                cg.replay()
            c0.record(stream)
            for _ in range(10):
                cg.replay()
            c1.record(stream)
        dj.dj_sync(stream)
        graph_us = c0.elapsed_time(c1) * 1e3 / (10 * K)
        del cg
    # phases of one solve from the workload's own source
    dj.dj_sssp(g, srcs[0], d, p, stream)
    dj.dj_sync(stream)
    phases = dj.dj_last_phases()
    info = dj.dj_graph_get_info(g)
    g.free()
    peak, peak_kind = _peaks()
    achieved = n * n * 4 / s_per / 1e9
    traffic, traffic_note = _traffic(TRAFFIC_FILES[name], n) if name in TRAFFIC_FILES else (None, "no ncu capture")
    out = {"value": 1.0 / s_per, "unit": "SSSP/s", "us_per_solve": 1e6 * s_per, "solves_timed": reps,
            "latency_us_alone": statistics.median(lat),
            "phases_first_source": phases if phases >= 0 else None,
            "engine": "grid" if (n >= 4096 or (n >= 2560 and info["entries"] * 4 >= n * n)) else "cluster",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "algorithmic_bytes_per_launch": n * n * 4,
                         "peak_kind": f"{peak_kind} hbm_gbs", "traffic": traffic, "traffic_note": traffic_note},
            "timer": "CUDA events over back-to-back dj_sssp calls (launch overhead included)"}
    if graph_us is not None:
        out["graph_replay_us_per_solve"] = graph_us
        out["graph_replay_note"] = ("200 dj_sssp calls captured into one CUDA graph, replayed 10 times "
                                    "(CUDA events): the rate without the per-launch cost of stream launches")
    return out


def _numa_placement(torch) -> dict:
    """NUMA node of the GPU (sysfs) and of the CPUs this process allocates pinned memory from."""
    out = {"gpu_node": None, "process_nodes": None}
    try:
        q = subprocess.run(["nvidia-smi", "-i", str(torch.cuda.current_device()), "--query-gpu=pci.bus_id",
                            "--format=csv,noheader"], capture_output=True, text=True, timeout=20).stdout.strip()
        dom, rest = q.split(":", 1)  # nvidia-smi prints an 8-digit domain, sysfs a 4-digit one
        bus = f"{int(dom, 16):04x}:{rest}".lower()
        with open(f"/sys/bus/pci/devices/{bus}/numa_node") as f:
            out["gpu_node"] = int(f.read().strip())
    except Exception:
        pass
    try:
        cpus = os.sched_getaffinity(0)
        nodes = set()
        base = "/sys/devices/system/node"
        for nd in os.listdir(base):
            if not nd.startswith("node"):
                continue
            with open(os.path.join(base, nd, "cpulist")) as f:
                spec = f.read().strip()
            ids = set()
            for part in spec.split(","):
                if "-" in part:
                    a, b = part.split("-")
                    ids.update(range(int(a), int(b) + 1))
                elif part:
                    ids.add(int(part))
            if ids & cpus:
                nodes.add(int(nd[4:]))
        out["process_nodes"] = sorted(nodes)
    except Exception:
        pass
    return out


def batch_cpu_baseline(be, bs) -> dict:
    """The oracle over independent solves of the batch workload on every host core (one serial
    Algorithm 1 per thread at a time), on a bounded sample of the 256 sources."""
    import oracle
    oracle.build()
    W = oracle.build_matrix(be.n, be.src, be.dst, be.w, be.directed)
    cores = os.cpu_count() or 1
    k = min(len(bs), 4 * cores)
    t0 = time.perf_counter()
    _, _, used = oracle.dijkstra_many_threads(W, np.asarray(bs[:k], dtype=np.int32), cores)
    el = time.perf_counter() - t0
    return {"value": k / el, "unit": "SSSP/s", "cores": used, "kind": "oracle",
            "sample": f"{k} of the 256 sources, serial Algorithm 1 per thread on {used} threads, {el:.1f} s"}


def serve_cpu_baseline(graphgen, spec, tr) -> dict:
    """The oracle over independent requests of the serving trace on every host core: the first
    3 x cores requests (their graphs built beforehand, as the GPU's are resident), one serial
    Algorithm 1 per thread at a time."""
    import concurrent.futures as cf
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    R = min(len(tr.req_graph), 3 * cores)
    mats = {}
    for r in range(R):
        gi = int(tr.req_graph[r])
        if gi not in mats:
            e = graphgen.bernoulli(int(tr.graph_n[gi]), float(tr.graph_p[gi]), spec["wlo"], spec["whi"],
                                   int(tr.graph_seed[gi]))
            mats[gi] = oracle.build_matrix(e.n, e.src, e.dst, e.w, False)
            del e
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda r: oracle.dijkstra(mats[int(tr.req_graph[r])], int(tr.req_source[r])), range(R)))
    el = time.perf_counter() - t0
    del mats
    return {"value": R / el, "unit": "solves/s", "cores": min(cores, R), "kind": "oracle",
            "sample": f"the trace's first {R} requests ({len(set(int(x) for x in tr.req_graph[:R]))} graphs), "
                      f"serial Algorithm 1 per thread on {min(cores, R)} threads, {el:.1f} s"}


if __name__ == "__main__":
    main()
