#!/usr/bin/env python3
"""Benchmark of the temporal edge-map (earliest arrival / latest departure) on GB300.

One step = one batch of the workload's queries answered by the batched edge-map on the
device-resident graph.  The default workload is the largest single-GPU one: the 2^26-vertex,
2^31-edge skewed R-MAT graph with Zipf(1.2) departure times and 16-bit durations, 64
earliest-arrival + 64 latest-departure queries over the full window (the 64-way batch).  The
graph build (ingest, sort, index) is timed separately.

Prints one JSON line (rank 0).  Beside the timed steps it reports the same queries one per
launch and end to end through host memory; with the extras (default at N = 1) also the
2^28-edge batched workload (256 random windows), the served stream on that graph at 1k-100k
queries/s, and the medium workload's batched, fastest-path, shortest-duration and temporal-BFS
figures.  The CPU baseline is the oracle on a bounded sample of the same graph (the queries
over its most recent departures), on one host core and on every host core.
`--impl reference` times that oracle sample instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "GTEPS & % HBM peak, batched vs one-query launch; served queries/s, p50/p99 ms"
UNIT = "GTEPS"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", type=int, default=5)
    p.add_argument("--lanes", type=int, default=0, help="0: autotune")
    p.add_argument("--shape", default="", help="lanes,warp_max_edges,chunk_edges,dense_div,relax_mode,blocks_per_sm"
                                               "[,concurrent[,block_edges]] (fixes the whole launch shape; no autotuning)")
    p.add_argument("--tune-sample", type=int, default=0, help="queries the autotuner times (0: 32 on the largest "
                                                              "workload, all otherwise)")
    p.add_argument("--no-single", action="store_true", help="skip the one-query-per-launch comparison")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the batched/served and medium-graph extras")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-fastest", action="store_true")
    p.add_argument("--no-duration", action="store_true")
    p.add_argument("--fastest-queries", type=int, default=16)
    p.add_argument("--serve-rates", default="")
    p.add_argument("--serve-queries", type=int, default=400)
    p.add_argument("--serve-slots", type=int, default=16)
    p.add_argument("--serve-slice", type=int, default=0, help="edge-map rounds per server launch (0: default)")
    p.add_argument("--scale", type=int, default=0,
                   help="run the workload's graph at 2^scale vertices, same edge factor and laws (small cases "
                        "for profiling; not a bench line of the named configuration)")
    p.add_argument("--cpu-sample-edges", type=int, default=1 << 26,
                   help="edges of the oracle baseline's sample (the most recent departures)")
    return p.parse_args()


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per edge-map launch of the timed
# step, from one ncu capture of that step (its command and per-launch figures are summarised
# under profiles/).  Keyed by workload, lanes, relax_mode, launches in flight, block_edges and a
# hash of the kernel sources: another shape, or any change to the kernels, reports null.
MEASURED_TRAFFIC = {}
KERNEL_NAME = {3: "stream_kernel"}
KERNEL_SOURCES = ("paper_2401_02563_gb300/csrc/edgemap_kernel.cuh", "paper_2401_02563_gb300/csrc/stream_kernel.cuh",
                  "paper_2401_02563_gb300/csrc/grid_sync.cuh", "paper_2401_02563_gb300/csrc/common.cuh")


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.file:
            return None
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---- algorithmic bytes (edge records + atomic words + init/readout) ------------------------

def launch_groups(queries, lanes):
    """The library's packing: queries grouped by kind in order, `lanes` at a time."""
    groups = []
    for kind in (0, 1):
        idx = [i for i, q in enumerate(queries) if q.kind == kind]
        groups += [idx[c:c + lanes] for c in range(0, len(idx), lanes)]
    return groups


def union_admissible(torch, el, queries, groups, labels_dev, chunk=1 << 25):
    """For each launch group, |union over its lanes of the edges usable under the final
    labels|, counted on the device in edge chunks (measurement only, outside the timed
    region): each chunk is uploaded once for all groups."""
    INF = 0xFFFFFFFF
    totals = [0] * len(groups)
    for c0 in range(0, el.m, chunk):
        c1 = min(el.m, c0 + chunk)
        src = torch.from_numpy(el.src[c0:c1].astype(np.int64)).cuda()
        dst = torch.from_numpy(el.dst[c0:c1].astype(np.int64)).cuda()
        t = torch.from_numpy(el.t[c0:c1].astype(np.int64)).cuda()
        tau = t + torch.from_numpy(el.lam[c0:c1].astype(np.int64)).cuda()
        for gi, group in enumerate(groups):
            anyadm = torch.zeros(c1 - c0, dtype=torch.bool, device="cuda")
            for i in group:
                q = queries[i]
                lab = labels_dev[i].to(torch.int64) & INF
                if q.kind == 0:
                    au = lab[src]
                    thr = au + (q.strict * (src != q.vertex)).to(torch.int64)
                    anyadm |= (au != INF) & (t >= thr) & (tau <= q.tw)
                else:
                    lv = lab[dst]
                    lim = lv - (q.strict * (dst != q.vertex)).to(torch.int64)
                    anyadm |= (lv != INF) & (tau <= lim) & (t >= q.ta)
            totals[gi] += int(anyadm.sum().item())
        del src, dst, t, tau
    return totals


def serve_stream(el, span, count, seed):
    """Served query mix: 70% earliest arrival / 30% latest departure, uniform vertices
    (with an out- / in-edge), window length log-uniform from 2^10 to the whole span."""
    kinds = [synth.EA if synth.u01(synth.draw(seed, q, 220)) < 0.7 else synth.LD for q in range(count)]
    v_ea = synth.pick_vertices(el, count, seed, True, False)
    v_ld = synth.pick_vertices(el, count, seed ^ 0x1D, False, True)
    wins = synth.log_uniform_windows(count, seed, span, 10.0, math.log2(span))
    return [synth.Query(k, v_ea[q] if k == synth.EA else v_ld[q], ta, tw)
            for q, (k, (ta, tw)) in enumerate(zip(kinds, wins))]


def measure_serving(torch, kx, g, el, span, rates, per_rate, slots, slice_rounds=0):
    """Open-loop Poisson arrivals at each rate through kairos_serve_submit/poll; latency is
    the server's submit-to-completion time.  The same stream is also answered one query
    per launch (kairos_earliest_arrival / kairos_latest_departure, FIFO) for comparison."""
    import threading
    n = el.n
    pool = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(256)]
    res = {"slots_per_kind": slots, "rounds_per_slice": slice_rounds or 2, "queries_per_rate": per_rate, "rates": []}
    server = kx.kairos_serve_create(g.handle, max_slots=slots, rounds_per_slice=slice_rounds)
    try:
        for ri, rate in enumerate(rates):
            qs = serve_stream(el, span, per_rate, 0x5E7E + ri)
            arrive = synth.poisson_arrivals(per_rate, rate, 0xA77 + ri)
            lat = [None] * per_rate
            tickets = [None] * per_rate
            free = list(range(len(pool)))
            lock = threading.Condition()
            done_at = [0.0]

            def poller():
                for i in range(per_rate):
                    with lock:
                        while tickets[i] is None:
                            lock.wait()
                        t, buf = tickets[i]
                    info = kx.kairos_serve_poll(server, t, -1)
                    lat[i] = info.latency_ms
                    with lock:
                        free.append(buf)
                        lock.notify_all()
                done_at[0] = time.perf_counter()

            th = threading.Thread(target=poller)
            th.start()
            t0 = time.perf_counter()
            for i, q in enumerate(qs):
                while time.perf_counter() - t0 < arrive[i]:
                    pass
                with lock:
                    while not free:
                        lock.wait()
                    buf = free.pop()
                t = kx.kairos_serve_submit(server, q, pool[buf])
                with lock:
                    tickets[i] = (t, buf)
                    lock.notify_all()
            th.join()
            wall = done_at[0] - t0
            lat_arr = np.array(lat)
            res["rates"].append({"offered_qps": rate, "served_qps": per_rate / wall,
                                 "p50_ms": float(np.percentile(lat_arr, 50)),
                                 "p99_ms": float(np.percentile(lat_arr, 99))})
    finally:
        kx.kairos_serve_destroy(server)
    # one query per launch, FIFO, on the last stream: service time per query and the
    # queueing latency the same arrivals would see
    row = pool[0]
    t_serv = []
    for q in qs:
        t1 = time.perf_counter()
        (g.earliest_arrival if q.kind == 0 else g.latest_departure)(q.vertex, q.ta, q.tw, row)
        t_serv.append(time.perf_counter() - t1)
    finish, lat1 = 0.0, []
    for a_i, s_i in zip(arrive, t_serv):
        start = max(a_i, finish)
        finish = start + s_i
        lat1.append((finish - a_i) * 1e3)
    res["one_query_per_launch"] = {"qps_capacity": len(qs) / sum(t_serv),
                                   "p50_ms_at_last_rate": float(np.percentile(lat1, 50)),
                                   "p99_ms_at_last_rate": float(np.percentile(lat1, 99))}
    return res


def measure_fastest(torch, kx, g, el, ta, tw, count):
    """Fastest-path queries (kairos_fastest_path) from `count` seeded sources with an out-edge,
    window [ta, tw], device output.  Lane work (relaxed edges over all start-time lanes)
    comes from one untimed pass with statistics; the timed pass runs without them."""
    srcs = synth.pick_vertices(el, count, 0xFA57, True, False)
    out = torch.empty(el.n, dtype=torch.int32, device="cuda")
    starts = relaxed = launches = 0
    for s in srcs:
        st = g.fastest_path(s, ta, tw, out, 0, True)
        starts += st.start_times
        relaxed += st.relaxed_edges
        launches += st.launches
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in srcs:
        g.fastest_path(s, ta, tw, out)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"queries": count, "queries_per_s": count / dt, "ms_per_query": dt * 1e3 / count,
            "start_times_per_query": starts / count, "launches_per_query": launches / count,
            "lane_gteps": relaxed / dt / 1e9, "window": [int(ta), int(tw)], "sources": "0xFA57 draw",
            "lanes": g.tuning().lanes, "sources_list": srcs[:4]}


def measure_duration(torch, kx, g, el, ta, tw, count):
    """Shortest-duration queries (kairos_shortest_duration) from `count` seeded sources with an
    out-edge, window [ta, tw], device output; the first call's one-time reverse-slot build is
    timed separately."""
    srcs = synth.pick_vertices(el, count, 0x5D57, True, False)
    out = torch.empty(el.n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.shortest_duration(srcs[0], ta, tw, out)
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    rounds = examined = 0
    t0 = time.perf_counter()
    for s in srcs:
        st = g.shortest_duration(s, ta, tw, out)
        rounds += st.rounds
        examined += st.examined_edges
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    b_rounds = 0
    t0 = time.perf_counter()
    for s in srcs:  # temporal BFS: the same computation with unit costs
        b_rounds += g.temporal_bfs(s, ta, tw, out).rounds
    torch.cuda.synchronize()
    bdt = time.perf_counter() - t0
    return {"queries": count, "queries_per_s": count / dt, "ms_per_query": dt * 1e3 / count,
            "rounds_per_query": rounds / count, "examined_edges_per_s": examined / dt,
            "first_call_ms": first_s * 1e3, "window": [int(ta), int(tw)], "sources": "0x5D57 draw",
            "temporal_bfs": {"queries_per_s": count / bdt, "ms_per_query": bdt * 1e3 / count,
                             "rounds_per_query": b_rounds / count}}


def replica_reduce(step_ms, te_step, world, device):
    """Across replicas: the slowest rank's step time and the total traversed edges.  Replicas
    hold the whole graph and answer their own query shard, so this is the only exchange."""
    if world <= 1:
        return step_ms, te_step
    import torch
    import torch.distributed as dist
    t = torch.tensor([step_ms], dtype=torch.float64, device=device)
    e = torch.tensor([te_step], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), int(e.item())


# ---- the oracle baseline on a bounded sample ------------------------------------------------

def host_description():
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                info["cpu_model"] = line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemTotal:"):
                    info["ram_gib"] = round(int(line.split()[1]) / (1 << 20), 1)
    except Exception:
        pass
    return info


class CpuSample:
    """A bounded sample of the workload for the oracle: the queries over the graph's most
    recent departures.  T is the departure time above which about `edges` edges depart (to
    4096 time units); every query of the sample has the window [T, KAIROS_TIME_MAX], so the
    edges departing before T are usable in none of them and the oracle runs on the sub-graph
    of the others, with labels identical to those of the same queries on the whole graph.
    Queries: earliest arrival from, and latest departure towards, seeded vertices with an
    edge in the sub-graph."""

    def __init__(self, el, edges, count=64, seed=0xC9A5):
        hist = np.bincount(el.t >> 12)
        above = np.cumsum(hist[::-1])[::-1]  # above[b]: edges departing at or after b * 4096
        b = int(np.searchsorted(-above, -min(edges, el.m), side="right")) - 1
        self.T = max(b, 0) << 12
        idx = np.flatnonzero(el.t >= self.T)
        self.sub = synth.EdgeList(el.n, el.src[idx], el.dst[idx], el.t[idx], el.lam[idx], None)
        del idx
        vs_out = synth.pick_vertices(self.sub, count // 2, seed, True, False)
        vs_in = synth.pick_vertices(self.sub, count // 2, seed ^ 0x1D, False, True)
        self.queries = [q for pair in zip([synth.Query(synth.EA, v, self.T, synth.C_MIRROR) for v in vs_out],
                                          [synth.Query(synth.LD, v, self.T, synth.C_MIRROR) for v in vs_in])
                        for q in pair]
        self.describe = (f"the {self.sub.m} edges departing at or after t = {self.T} (the most recent of the "
                         f"{el.m}); queries with window [{self.T}, 2^32 - 2], alternating EA and LD from seeded "
                         f"vertices; labels equal those of the same queries on the whole graph")


class CpuBaselineJob(threading.Thread):
    """The oracle, as it stands, on a CpuSample: the time-order sort (timed separately), then
    one-pass scans on one host core for about `budget_s` seconds of scanning.  Runs beside the
    GPU measurement (the oracle's C scans release the interpreter lock); `ncore()` then runs
    the same scans on every host core at once, one independent single-threaded scan per
    thread."""

    def __init__(self, el, edges, budget_s=12.0):
        super().__init__(daemon=True)
        self.el, self.edges, self.budget_s = el, edges, budget_s
        self.result, self.error = None, None
        self.ready = threading.Event()  # the sample is built (the whole edge list is no longer needed)

    def run(self):
        try:
            import oracle
            self.sample = CpuSample(self.el, self.edges)
            self.el = None
            self.ready.set()
            t0 = time.perf_counter()
            self.orc = oracle.Oracle(self.sample.sub)
            sort_s = time.perf_counter() - t0
            te, scan_s, done = 0, 0.0, 0
            while scan_s < self.budget_s and done < 10 * len(self.sample.queries):
                q = self.sample.queries[done % len(self.sample.queries)]
                t1 = time.perf_counter()
                lab = self.orc.query(q)
                scan_s += time.perf_counter() - t1
                te += self.orc.admissible(q, lab)
                done += 1
            self.result = {"te": te, "scan_s": scan_s, "queries": done, "sort_s": sort_s}
        except Exception as e:  # reported in the JSON line, never fatal to the GPU figures
            self.error = repr(e)
            self.ready.set()

    def ncore(self, threads):
        from concurrent.futures import ThreadPoolExecutor
        qs = self.sample.queries
        per = max(1, self.result["queries"] // threads + 1)  # about the one-core sample's length each

        def work(k):
            te = 0
            for j in range(per):
                q = qs[(k * per + j) % len(qs)]
                te += self.orc.admissible(q, self.orc.query(q))
            return te

        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=threads) as ex:
            te = sum(ex.map(work, range(threads)))
        wall = time.perf_counter() - t0
        return {"value": te / wall / 1e9, "queries": per * threads, "wall_s": wall}

    def report(self):
        if self.error:
            return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: " + self.error}
        r = self.result
        host = host_description()
        out = {"value": r["te"] / r["scan_s"] / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{r['queries']} one-pass scans on 1 host core over {self.sample.describe}; "
                         f"time-order sort ({r['sort_s']:.1f} s) excluded as preprocessing",
               "queries_per_s": r["queries"] / r["scan_s"], "host": host}
        n = host.get("nproc") or 1
        nc = self.ncore(n)
        out["ncore"] = {"value": nc["value"], "unit": UNIT, "cores": n,
                        "sample": f"{nc['queries']} scans of the same sample, {n} independent single-threaded "
                                  f"scans at once (one per host core)", "wall_s": nc["wall_s"]}
        return out


def reference_arm(args, rank, world):
    """--impl reference: the CPU oracle on this machine's host cores, one EA and one LD query of
    the bounded sample per step."""
    if rank != 0:
        return
    import oracle
    w = synth.WORKLOADS[args.workload]
    el = synth.rmat(w.graph)
    sample = CpuSample(el, min(args.cpu_sample_edges, 1 << 24) if args.workload == 5 else args.cpu_sample_edges)
    del el
    orc = oracle.Oracle(sample.sub)
    qs = sample.queries

    def step(k):
        te = 0
        for q in (qs[(2 * k) % len(qs)], qs[(2 * k + 1) % len(qs)]):
            te += orc.admissible(q, orc.query(q))
        return te

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    te = 0
    for k in range(args.steps):
        te += step(args.warmup + k)
    dt = time.perf_counter() - t0
    val = te / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"{w.name}: {w.description}", "queries_per_step": 2,
                       "l2": "host run (no device caches)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"1 EA + 1 LD query per step over {sample.describe}; single-threaded "
                                       f"one-pass scans; time-order sort excluded", "host": host_description()},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- GPU measurements ------------------------------------------------------------------------

def tune(torch, kx, g, queries, args, theta_default, tune_sample, min_lanes=1):
    """Install the launch shape: fixed by --shape / --lanes, else the autotuner (and, where the
    workload fixes no index threshold, the threshold sweep first, on `tune_sample` queries) on
    the whole query set, over lane widths of at least min_lanes."""
    if args.shape:
        f = [int(x) for x in args.shape.split(",")]
        ln, wm, ch, dd, rm, bp = f[:6]
        g.set_tuning(lanes=ln, warp_max_edges=wm, chunk_edges=ch, dense_div=dd, relax_mode=rm, blocks_per_sm=bp,
                     concurrent=f[6] if len(f) > 6 else 1, block_edges=f[7] if len(f) > 7 else 0)
        return None
    if args.lanes:
        g.set_tuning(lanes=args.lanes, relax_mode=3 if args.lanes == 64 else 0)
        return None
    sample = queries
    if tune_sample and tune_sample < len(queries):  # both kinds, evenly
        ea = [q for q in queries if q.kind == 0]
        ld = [q for q in queries if q.kind == 1]
        k = tune_sample // (2 if ea and ld else 1)
        sample = ea[:k] + ld[:k]
    sweep = None
    if theta_default == kx.KAIROS_NO_INDEX:
        # no fixed cutoff: the index threshold is tuned too (swept 16..4096), in a frontier shape
        g.set_tuning(lanes=16, relax_mode=0, concurrent=1, block_edges=0)
        best, ms = g.autotune_index(sample)
        sweep = {"best": best, "ms_by_threshold": ms, "sample_queries": len(sample)}
    g.autotune(queries, min_lanes=min_lanes)
    return sweep


def measure_batched(torch, kx, g, el, queries, args, world, dist, stream, steps, warmup, roofline=True):
    """Timed steps of the batch on the resident graph (device outputs), the exact per-query
    counts from one untimed statistics pass, and the roofline of the edge-map."""
    Q, n = len(queries), el.n
    R = 10 if el.lam.dtype == np.uint16 else 12
    out = torch.empty((Q, n), dtype=torch.int32, device="cuda")
    stats = g.batch(queries, out, want_stats=True)
    for _ in range(warmup):
        g.batch(queries, out, want_stats=False)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kernel_ms = 0.0
    with Clocks(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        for _ in range(steps):
            g.batch(queries, out, want_stats=False)
            kernel_ms += g.last_kernel_ms()
        ev1.record(stream)
        torch.cuda.synchronize()
    step_ms = ev0.elapsed_time(ev1) / steps
    te_step = sum(s.relaxed_edges for s in stats)  # identical every step: exact integer counts
    tuning = g.tuning()
    groups = launch_groups(queries, tuning.lanes)
    scanned_step = sum(stats[grp[0]].scanned_edges for grp in groups)  # one count per launch
    res = {"step_ms": step_ms, "te_step": te_step, "scanned_step": scanned_step, "queries": Q,
           "kernel_ms": kernel_ms / steps, "clocks": clk.summary(), "n_launch": len(groups), "tuning": tuning,
           "rounds": [stats[grp[0]].rounds for grp in groups], "out": out, "stats": stats}
    if roofline:
        U = union_admissible(torch, el, queries, groups, out)
        bytes_step = sum(u * R + 4 * sum(stats[i].relaxed_edges for i in grp) + 8 * len(grp) * n
                         for u, grp in zip(U, groups))
        res["bytes_step"] = bytes_step
        res["union_step"] = sum(U)
    return res


def measure_single(torch, g, queries, stream):
    n = g.n
    row = torch.empty(n, dtype=torch.int32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for q in queries[:2]:
        (g.earliest_arrival if q.kind == 0 else g.latest_departure)(q.vertex, q.ta, q.tw, row)
    torch.cuda.synchronize()
    e0.record(stream)
    for q in queries:
        (g.earliest_arrival if q.kind == 0 else g.latest_departure)(q.vertex, q.ta, q.tw, row)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def measure_e2e(torch, g, queries, te_step, steps):
    """The same batch through the C ABI into the caller's page-locked host buffer: every
    label row crosses to the host inside the timed region."""
    Q, n = len(queries), g.n
    host_t = torch.empty((Q, n), dtype=torch.int32, pin_memory=True)
    host = host_t.numpy().view(np.uint32)
    g.batch(queries, host, want_stats=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        g.batch(queries, host, want_stats=False)
    e2e_s = (time.perf_counter() - t0) / steps
    del host, host_t
    return {"value": te_step / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": Q * 16,
            "d2h_bytes_per_step": Q * n * 4, "ms_per_step": e2e_s * 1e3,
            "note": "queries in, every label row copied to page-locked host memory"}


def selectivity_accuracy(kx, g, el, cutoffs=(1024, 2048, 4096, 8192), percents=(1, 2, 3, 4, 5, 10, 20),
                         theta_permille=200):
    """The estimator-accuracy measure of Sec. 6.5 on the forward lists: histograms for every
    vertex of degree >= the smallest cutoff (built on the device), then for each window
    [T_X, end] over the most recent X% of departures the decision of Eq. 3 at theta_sel = 20%
    from the histogram estimate against the decision from the exact count, per cutoff."""
    deg = np.bincount(el.src, minlength=el.n)
    t0 = time.perf_counter()
    kx.kairos_selectivity_build(g.handle, min(cutoffs))
    build_s = time.perf_counter() - t0
    verts = np.flatnonzero(deg >= min(cutoffs)).astype(np.int32)
    tsort = np.sort(el.t)
    table = []
    for pct in percents:
        T = int(tsort[min(len(tsort) - 1, int(len(tsort) * (1.0 - pct / 100.0)))])
        est, ex = kx.kairos_selectivity_estimate(g.handle, 0, verts, T, 0xFFFFFFFE, 0xFFFFFFFE)
        d = deg[verts].astype(np.uint64)
        agree = (np.uint64(1000) * est <= np.uint64(theta_permille) * d) == \
                (np.uint64(1000) * ex <= np.uint64(theta_permille) * d)
        for c in cutoffs:
            sel_c = deg[verts] >= c
            table.append({"percent": pct, "cutoff": c, "vertices": int(sel_c.sum()),
                          "accuracy": float(agree[sel_c].mean()) if sel_c.any() else None})
    kx.kairos_selectivity_build(g.handle, kx.KAIROS_NO_INDEX)  # drop them again
    return {"theta_sel": theta_permille / 1000, "histogram_build_s": build_s, "table": table}


def tuning_dict(t):
    return {"lanes": t.lanes, "warp_max_edges": t.warp_max_edges, "chunk_edges": t.chunk_edges,
            "blocks_per_sm": t.blocks_per_sm, "relax_mode": t.relax_mode, "dense_div": t.dense_div,
            "concurrent": max(1, t.concurrent), "block_edges": t.block_edges, "select_permille": t.select_permille}


def extra_batched_and_served(torch, kx, args, stream):
    """The 2^28-edge graph: workload 3 (256 random-window EA queries, batched vs one per
    launch) and workload 4 (the served stream at 1k-100k queries/s)."""
    w3 = synth.WORKLOADS[3]
    el = synth.rmat(w3.graph)
    qs = synth.workload_queries(3, el)
    res = {"workload": f"{w3.name}: {w3.description}"}
    with torch.cuda.stream(stream):
        g = kx.Graph.from_edges(el, stream=stream)
        g.index(16)
        sweep = tune(torch, kx, g, qs, args, w3.theta, 64, min_lanes=8)
        b = measure_batched(torch, kx, g, el, qs, args, 1, None, stream, 3, 2, roofline=False)
        s_ms = measure_single(torch, g, qs, stream)
        res.update({"gteps": b["te_step"] / (b["step_ms"] / 1e3) / 1e9, "queries_per_s": len(qs) / (b["step_ms"] / 1e3),
                    "ms_per_step": b["step_ms"], "one_query_per_launch_qps": len(qs) / (s_ms / 1e3),
                    "batched_vs_single_qps": s_ms / b["step_ms"], "tuning": tuning_dict(b["tuning"]),
                    "index_threshold_sweep": sweep})
        del b
        torch.cuda.empty_cache()
        res["selectivity_accuracy"] = selectivity_accuracy(kx, g, el)
        if not args.no_serve:
            w4 = synth.WORKLOADS[4]
            rates = [float(x) for x in (args.serve_rates or "1000,3000,10000,30000,100000").split(",") if x]
            res["served"] = measure_serving(torch, kx, g, el, w4.graph.t_span, rates, args.serve_queries,
                                            args.serve_slots, args.serve_slice)
            res["served"]["workload"] = f"{w4.name}: {w4.description}"
        g.close()
    return res


def extra_medium(torch, kx, args, stream):
    """The 2^25-edge medium graph: the batch of 128 full-window queries, and the other path
    queries (fastest paths, shortest durations, temporal BFS)."""
    w2 = synth.WORKLOADS[2]
    el = synth.rmat(w2.graph)
    qs = synth.workload_queries(2, el)
    res = {"workload": f"{w2.name}: {w2.description}"}
    with torch.cuda.stream(stream):
        g = kx.Graph.from_edges(el, stream=stream)
        g.index(w2.theta)
        tune(torch, kx, g, qs, args, w2.theta, 0)
        b = measure_batched(torch, kx, g, el, qs, args, 1, None, stream, 5, 3, roofline=True)
        s_ms = measure_single(torch, g, qs, stream)
        peak, _ = peaks()
        la_ms = b["kernel_ms"] / b["n_launch"]
        res.update({"gteps": b["te_step"] / (b["step_ms"] / 1e3) / 1e9, "queries_per_s": len(qs) / (b["step_ms"] / 1e3),
                    "ms_per_step": b["step_ms"], "one_query_per_launch_qps": len(qs) / (s_ms / 1e3),
                    "batched_vs_single_qps": s_ms / b["step_ms"], "tuning": tuning_dict(b["tuning"]),
                    "hbm_frac": b["bytes_step"] / b["n_launch"] / (la_ms / 1e3) / 1e9 / peak})
        del b
        torch.cuda.empty_cache()
        res["selectivity_accuracy"] = selectivity_accuracy(kx, g, el)
        if not args.no_fastest:
            res["fastest"] = measure_fastest(torch, kx, g, el, qs[0].ta, qs[0].tw, args.fastest_queries)
        if not args.no_duration:
            res["shortest_duration"] = measure_duration(torch, kx, g, el, qs[0].ta, qs[0].tw, args.fastest_queries)
        g.close()
    return res


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch
    import paper_2401_02563_gb300 as kx

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = synth.WORKLOADS[args.workload]
    spec = w.graph
    if args.scale:
        spec = synth.scaled(w.graph, args.scale, w.graph.m >> max(0, w.graph.scale - args.scale))
        args.no_extras = True
    t0 = time.perf_counter()
    el = synth.rmat(spec)
    gen_s = time.perf_counter() - t0
    queries = synth.workload_queries(args.workload, el, shard=rank)
    Q, n, m = len(queries), el.n, el.m
    R = 10 if el.lam.dtype == np.uint16 else 12
    # the oracle baseline (rank 0, N = 1) runs beside the GPU measurement on one host core
    cpu_job = None
    if not args.no_cpu and world == 1:
        cpu_job = CpuBaselineJob(el, args.cpu_sample_edges)
        cpu_job.start()
    stream = torch.cuda.Stream()
    tune_sample = args.tune_sample or (32 if args.workload == 5 else 0)

    with torch.cuda.stream(stream):
        g = kx.Graph.from_edges(el, stream=stream)
        theta = w.theta if w.theta != kx.KAIROS_NO_INDEX else 16
        g.index(theta)
        info = g.info()
        theta_sweep = tune(torch, kx, g, queries, args, w.theta, tune_sample,
                           min_lanes=16 if args.workload == 5 else 1)
        theta_now = (theta_sweep or {}).get("best", theta)
        b = measure_batched(torch, kx, g, el, queries, args, world, dist, stream, args.steps, args.warmup)
        step_ms, te_all = replica_reduce(b["step_ms"], b["te_step"], world, "cuda")
        if dist:
            dist.barrier()
        value = te_all / (step_ms / 1e3) / 1e9
        tuning = b["tuning"]
        launch_ms = b["kernel_ms"] / b["n_launch"]
        achieved = b["bytes_step"] / b["n_launch"] / (launch_ms / 1e3) / 1e9
        peak, peak_kind = peaks()
        del b["out"]
        torch.cuda.empty_cache()
        single = None
        if not args.no_single:
            s_ms = measure_single(torch, g, queries, stream)
            single = {"gteps": b["te_step"] / (s_ms / 1e3) / 1e9, "queries_per_s": Q / (s_ms / 1e3), "ms_per_batch": s_ms}
        e2e = None if args.no_e2e else measure_e2e(torch, g, queries, te_all, max(2, min(args.steps, 5)))
        graph_launches = g.info().graph_launches
        sel_acc = selectivity_accuracy(kx, g, el) if (world == 1 and not args.no_extras) else None
        # the oracle's sample queries on the GPU too (whole graph, same windows), for the same work
        sample_gpu = None
        if cpu_job is not None:
            cpu_job.ready.wait()
            if cpu_job.error is None:
                sq = cpu_job.sample.queries
                so = torch.empty((len(sq), n), dtype=torch.int32, device="cuda")
                sst = g.batch(sq, so, want_stats=True)
                g.batch(sq, so, want_stats=False)
                sample_gpu = {"gteps": sum(x.relaxed_edges for x in sst) / (g.last_kernel_ms() / 1e3) / 1e9,
                              "queries": len(sq), "kernel_ms": g.last_kernel_ms()}
                del so
        g.close()
        torch.cuda.empty_cache()
    del el
    extras = {}
    if world == 1 and not args.no_extras and args.workload == 5:
        extras["batched_and_served"] = extra_batched_and_served(torch, kx, args, stream)
        torch.cuda.empty_cache()
        extras["medium"] = extra_medium(torch, kx, args, stream)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if cpu_job is not None:
        cpu_job.join()
        cpu = cpu_job.report()
        cpu["gpu_same_sample"] = sample_gpu
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"{w.name}: {w.description}" + (f" (scaled to 2^{args.scale} vertices)" if args.scale else ""),
                   "vertices": n, "edges": m, "queries_per_step": Q,
                   "index_threshold": theta_now, **tuning_dict(tuning), "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2 (graph {2 * (m * R + 8 * n) / 1e9:.1f} GB)"},
        "queries_per_s": world * Q / (step_ms / 1e3),
        "relaxed_edges_per_step": b["te_step"], "scanned_edges_per_step": b["scanned_step"],
        "union_admissible_per_step": b["union_step"], "rounds_per_launch": b["rounds"],
        "generate_s": gen_s, "build_ms": info.build_ms, "index_ms": info.index_ms, "graph_launches": graph_launches,
        "single_launch": single,
        "index_threshold_sweep": theta_sweep,
        "batched_vs_single_qps": (Q / (step_ms / 1e3)) / single["queries_per_s"] if single else None,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": MEASURED_TRAFFIC.get((args.workload, tuning.lanes, tuning.relax_mode,
                                                      max(1, tuning.concurrent), tuning.block_edges, kernel_hash())),
                     "peak_kind": peak_kind, "kernel": KERNEL_NAME.get(tuning.relax_mode, "edgemap_kernel"),
                     "kernel_hash": kernel_hash(), "launches_per_step": b["n_launch"], "avg_launch_ms": launch_ms,
                     "algorithmic_bytes_per_step": b["bytes_step"]},
        "selectivity_accuracy": sel_acc,
        "extras": extras or None,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps * b["n_launch"],
        "clocks": b["clocks"],
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
