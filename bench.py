#!/usr/bin/env python
"""Benchmark: coarsening throughput of the GB300 partitioner on the 2^26-node
Erdos-Renyi graph (671,088,640 undirected edges, unit weights, k = 128,
eps = 0.03, seed 1), printed as one JSON line.

A step is one full gp_partition call (validation, coarsening with
sparsification, initial partitioning, uncoarsening with refinement) on the
device-resident graph.  `value` is coarsening edges/s: input edges divided
by the device time of the coarsening phase (CUDA events on the library's
stream inside each step), summed over the timed steps.  `e2e` is the same
graph through gp_partition_host from pinned host memory: input copies,
partition and the copy of the block ids back are all in its timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

With N > 1 (launched by torchrun) every rank partitions its own replica of
the graph (the method does not shard one graph); value sums all ranks' edges
over the slowest rank's time.  `--impl reference` times the CPU oracle of
the same method (single-threaded C) on a bounded sample of the workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("coarsening edges/s and HBM GB/s (% of GB300 peak); batched graphs/s, served p50/p99 ms")
WORKLOAD = dict(name="erdos_renyi_n2^26_m671088640_k128", n=1 << 26, m=671_088_640, k=128, eps=0.03,
                seed=1)
SMALL = dict(name="erdos_renyi_n2^20_m10485760_k128", n=1 << 20, m=10_485_760, k=128, eps=0.03, seed=1)
# bounded CPU sample of the same workload family (same degree, same k)
CPU_SAMPLE = dict(name="erdos_renyi_n2^21_m20971520_k128", n=1 << 21, m=20_971_520, k=128, seed=1)
FALLBACK_HBM_GBS = 6800.0
# profile classes of the coarsening phase (the rest belong to initial partitioning and uncoarsening,
# or are shared: sort, scan, round_setup)
COARSEN_CLASSES = ("lp_rate", "lp_accept", "lp_overflow", "lp_apply", "lp_small", "two_hop", "relabel", "contract",
                   "contract_aux", "sparsify")
# ncu DRAM traffic per algorithmic byte, by class, with the sources the counters were taken on
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def workload_of(args):
    if args.scale:
        n = 1 << args.scale
        return dict(name=f"erdos_renyi_n2^{args.scale}_m{10 * n}_k128", n=n, m=10 * n, k=128, eps=0.03,
                    seed=1)
    return SMALL if args.small else WORKLOAD


def max_over_ranks(values):
    """Element-wise maximum over all ranks (the slowest rank's times); a no-op on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def source_digest(files):
    import hashlib
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_ratio(cls):
    """DRAM bytes per algorithmic byte of `cls` from a committed ncu summary, or None when that
    summary is missing or was taken on sources that have changed since."""
    if not os.path.exists(TRAFFIC_FILE):
        return None, "no ncu summary"
    with open(TRAFFIC_FILE) as f:
        d = json.load(f).get(cls)
    if not d:
        return None, "no ncu summary for this class"
    if source_digest(d["sources"]) != d["digest"]:
        return None, "kernel changed since the ncu capture"
    return d["dram_bytes"] / d["algorithmic_bytes"], d["capture"]


def gather_floor(ctx, st, rates):
    """Lower bound (ms per step) of the label reads of the clustering LP and of the
    coarse-id reads of contraction: per level, the rated entries (every node with
    neighbours is rated once per round of 8 sub-rounds) and the contracted entries,
    each a random 4-byte read from an n_i-word array, at the measured random-read
    rate for that array size."""
    def rate(n):
        b = max(4, 4 * int(n))
        if b not in rates:
            rates[b] = ctx.measure_random_reads(b, 1 << 26)
        return rates[b]
    lp = contract = 0.0
    for L in st.levels_list():
        entries = 2 * L["m"]
        r = rate(L["n"])
        lp += entries * L["lp_subrounds"] / 8.0 / r
        contract += entries / r
    return 1000 * lp, 1000 * contract


# ------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu_index), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------- inputs

def make_graph(w, rank: int, world: int):
    """Rank 0 draws the graph; other ranks read it from a shared file."""
    import numpy as np
    import graphgen as gg
    if world == 1:
        t = time.time()
        g = gg.er(w["n"], w["m"], w["seed"])
        log(f"[bench] generated {w['name']} in {time.time() - t:.1f}s")
        return g
    import torch.distributed as dist
    shared = os.path.join(tempfile.gettempdir(), f"gpbench_{w['name']}_{os.environ.get('MASTER_PORT', '0')}")
    if rank == 0:
        g = gg.er(w["n"], w["m"], w["seed"])
        os.makedirs(shared, exist_ok=True)
        np.save(os.path.join(shared, "xadj.npy"), g.xadj)
        np.save(os.path.join(shared, "adjncy.npy"), g.adjncy)
    dist.barrier()
    if rank != 0:
        xadj = np.load(os.path.join(shared, "xadj.npy"), mmap_mode="r")
        adj = np.load(os.path.join(shared, "adjncy.npy"), mmap_mode="r")
        g = gg.Graph(w["n"], np.asarray(xadj), np.asarray(adj), np.ones(w["n"], np.int32),
                     np.ones(len(adj), np.int32), w["name"])
    dist.barrier()
    if rank == 0:
        for f in ("xadj.npy", "adjncy.npy"):
            os.unlink(os.path.join(shared, f))
        os.rmdir(shared)
    return g


# ---------------------------------------------------------------- CPU arm

def cpu_sample_run(steps: int = 1):
    """Times the oracle's coarsening phase on the bounded CPU sample."""
    import graphgen as gg
    import oracle as orc
    g = gg.er(CPU_SAMPLE["n"], CPU_SAMPLE["m"], CPU_SAMPLE["seed"])
    times = []
    for _ in range(steps):
        t = time.perf_counter()
        orc.coarsen_only(g, CPU_SAMPLE["k"], CPU_SAMPLE["seed"])
        times.append(time.perf_counter() - t)
    return g.m, times


def cpu_baseline_obj(m, times):
    return {"value": m / statistics.mean(times), "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": (f"coarsening phase (Alg. 1) of the single-threaded C oracle on "
                       f"{CPU_SAMPLE['name']} (same degree and k as the workload), "
                       f"{len(times)} run(s), {statistics.mean(times):.2f} s each, host cpu "
                       f"{os.cpu_count()} cores available, 1 used")}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        cpu_sample_run(1)
    m, times = cpu_sample_run(args.steps)
    cb = cpu_baseline_obj(m, times)
    w = workload_of(args)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "edges/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": w["name"], "k": w["k"], "eps": w["eps"], "seed": w["seed"],
                       "sample": CPU_SAMPLE["name"], "parallelism": "replicas"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "edges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm

def run_gpu(args, world, rank, local):
    import numpy as np
    import torch
    import paper_2504_17615_gb300 as gp
    from paper_2504_17615_gb300 import build as gpbuild

    w = workload_of(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    gpbuild.build()
    g = make_graph(w, rank, world)
    n, m2 = g.n, g.m2
    ctx = gp.Context(local)
    stream = ctx.stream
    t0 = time.time()
    dg = gp.DeviceGraph.from_host(g)
    torch.cuda.synchronize()
    log(f"[bench] rank {rank}: uploaded n={n} m={g.m} in {time.time() - t0:.1f}s")
    blocks = torch.empty(n, dtype=torch.int32, device="cuda")

    def step():
        return ctx.gp_partition(dg, w["k"], w["eps"], w["seed"], blocks=blocks)

    for i in range(args.warmup):
        _, cut, st = step()
        log(f"[bench] warmup {i}: {st.ms_total:.1f} ms (coarsen {st.ms_coarsen:.1f}) cut={cut} "
            f"levels={st.levels}")
    gpu_index = local
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if cvd and cvd.split(",")[local].strip().isdigit():
        gpu_index = int(cvd.split(",")[local])
    clocks = ClockSampler(gpu_index)
    clocks.start()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = gp.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = []
    for _ in range(args.steps):
        _, cut, st = step()
        stats.append((st.ms_coarsen, st.ms_initial, st.ms_uncoarsen, st.ms_total, cut, st.levels))
    hierarchy = [[L["n"], L["m"], L["n_next"], L["m_coarse"], L["m_hat"], L["triggered"], L["m_next"]]
                 for L in st.levels_list()] + [[st.n_coarsest]]
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = gp.launch_count() - launches0
    clk = clocks.stop()
    step_ms = ev0.elapsed_time(ev1)
    # per-class CUDA events bracket the launches of a second pass over the same steps, so that
    # their host cost stays out of the timed steps above
    ctx.profile_reset()
    ctx.profile(True)
    torch.cuda.synchronize()
    pv0, pv1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pv0.record(stream)
    for _ in range(args.steps):
        step()
    pv1.record(stream)
    torch.cuda.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read()
    profiled_ms = pv0.elapsed_time(pv1) / args.steps
    # Sec. 5 diagnostic of the level-1 clustering (outside the timed steps)
    U1 = st.U
    cmap1, nc1, _ = ctx.gp_coarsen(dg, U1, 1, w["seed"])
    mod = ctx.gp_modularity(dg, cmap1, nc1).as_dict()
    L1 = st.levels_list()[0] if st.levels else None
    if L1:
        mod["kept_edge_fraction"] = L1["m_coarse"] / L1["m"]
        mod["what"] = ("Q_C, alpha_C and Lemma 2's bound 1 - Q_C - alpha_C for the level-1 clustering; "
                       "kept_edge_fraction = coarse edges / input edges before sparsification")
    coarsen_ms = sum(s[0] for s in stats)
    step_ms, coarsen_ms = max_over_ranks([step_ms, coarsen_ms])
    value = world * g.m * args.steps / (coarsen_ms / 1000.0)

    # roofline of the dominant kernel class of the coarsening phase (by device time in the
    # timed region), plus the achieved bandwidth of every class with algorithmic bytes
    peak, peak_kind = measured_peaks()
    dom = max((k for k in COARSEN_CLASSES if prof.get(k, {}).get("bytes", 0) > 0), key=lambda k: prof[k]["ms"])
    dom_ms = prof[dom]["ms"]
    achieved = prof[dom]["bytes"] / (dom_ms / 1000.0) / 1e9 if dom_ms > 0 else 0.0
    per_launch = prof[dom]["bytes"] / max(prof[dom]["launches"], 1)
    ratio, traffic_src = traffic_ratio(dom)
    traffic = args.traffic if args.traffic is not None else (ratio * per_launch if ratio else None)
    roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
            if peak_kind == "measured" else "fallback", "traffic": traffic, "traffic_source": traffic_src,
            "launches": prof[dom]["launches"], "ms": dom_ms, "algorithmic_bytes": prof[dom]["bytes"],
            "algorithmic_bytes_per_launch": per_launch,
            "classes": {k: {"achieved_gbs": v["bytes"] / (v["ms"] / 1000.0) / 1e9, "frac": v["bytes"] / (v["ms"] / 1000.0) / 1e9 / peak,
                            "ms": v["ms"], "launches": v["launches"]}
                        for k, v in prof.items() if v["bytes"] > 0 and v["ms"] > 0}}

    # the random-read bound of the gather-heavy classes (measured on this GPU, per level)
    rates = {}
    lp_floor, ct_floor = gather_floor(ctx, st, rates)
    per_step = lambda k: prof[k]["ms"] / args.steps
    roof["random_read_bound"] = {
        "what": "time the label / coarse-id reads alone take at the measured random 4-byte read rate "
                "for each level's array size (entries rated per level = 2m x sub-rounds / 8)",
        "lp_rate": {"floor_ms": lp_floor, "ms": per_step("lp_rate"), "frac": lp_floor / per_step("lp_rate")},
        "contract": {"floor_ms": ct_floor, "ms": per_step("contract"), "frac": ct_floor / per_step("contract")},
        "reads_per_s_by_array_bytes": {str(k): v for k, v in sorted(rates.items())}}

    # end to end through the host entry point from pinned memory
    e2e = None
    if not args.no_e2e:
        hx = torch.from_numpy(np.ascontiguousarray(g.xadj, dtype=np.int32)).pin_memory()
        ha = torch.from_numpy(g.adjncy).pin_memory()
        hv = torch.from_numpy(np.ascontiguousarray(g.vwgt)).pin_memory()
        hw = torch.from_numpy(np.ascontiguousarray(g.adjwgt)).pin_memory()
        hb = torch.empty(n, dtype=torch.int32).pin_memory()
        ctx.gp_partition_host(n, m2, hx, ha, hv, hw, w["k"], w["eps"], w["seed"], blocks=hb)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.steps):
            ctx.gp_partition_host(n, m2, hx, ha, hv, hw, w["k"], w["eps"], w["seed"], blocks=hb)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t
        e2e_s = max_over_ranks([e2e_s])[0]
        e2e = {"value": world * g.m * args.steps / e2e_s, "unit": "edges/s",
               "what": "gp_partition_host: H2D of the CSR, full partition, D2H of the block ids",
               "ms_per_step": 1000 * e2e_s / args.steps,
               "h2d_bytes_per_step": 4 * ((n + 1) + 2 * m2 + n), "d2h_bytes_per_step": 4 * n}

    if rank != 0:
        return 0
    # the batched and served forms on bounded samples of their mixes (one GPU only)
    batched = served = None
    if world == 1 and not args.no_batch_serve:
        batched = batch_summary(gp, args.batch_count, args.batch_nmax, args.batch_workers, 1, 1)
        served = serve_summary(gp, args.serve_count, args.serve_mmax, args.serve_workers)
    cb = None
    if not args.no_cpu_baseline:
        m_s, times = cpu_sample_run(1)
        cb = cpu_baseline_obj(m_s, times)
    mean = lambda i: statistics.mean(s[i] for s in stats)
    line = {"metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": w["name"], "n": w["n"], "m": w["m"], "k": w["k"], "eps": w["eps"],
                       "seed": w["seed"], "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs (CSR 10.7 GB) larger than L2, no flush",
                       "value_is": "input edges / coarsening-phase device time"},
            "partition_edges_per_s": world * g.m * args.steps / (step_ms / 1000.0),
            "phases_ms": {"coarsen": mean(0), "initial": mean(1), "uncoarsen": mean(2), "total": mean(3)},
            "cut": stats[-1][4], "levels": stats[-1][5], "ip_cut": st.ip_cut,
            "rebalance_moves": st.rebalance_moves, "n_coarsest": st.n_coarsest,
            "hierarchy": {"columns": ["n", "m", "n_next", "m_coarse", "m_hat", "triggered", "m_next"],
                          "levels": hierarchy},
            "batched": batched, "served": served,
            "roofline": roof, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": launches // max(args.steps, 1),
            "gpu_launches_total": launches, "clocks": clk, "modularity_level1": mod,
            "kernel_classes_from": "a second pass over the same steps with per-class CUDA events "
                                   f"({profiled_ms:.1f} ms per step with the events)",
            "kernel_classes": {k: v for k, v in prof.items() if v["launches"]}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_level1(args):
    """Level 1 of Alg. 1 alone (LP clustering with 2-hop and isolated nodes, contraction, and
    sparsification when it triggers) on the workload graph: the profiling case for ncu."""
    import torch
    import paper_2504_17615_gb300 as gp
    from paper_2504_17615_gb300 import build as gpbuild
    w = workload_of(args)
    gpbuild.build()
    g = make_graph(w, 0, 1)
    ctx = gp.Context(0)
    dg = gp.DeviceGraph.from_host(g)
    U = max(1, g.n // (160 * w["k"]))
    m = g.m2 // 2

    def step():
        cmap, nc, _ = ctx.gp_coarsen(dg, U, 1, w["seed"])
        cg = ctx.gp_contract(dg, cmap, nc)
        m_c = cg.m2 // 2
        m_hat = min(m // 2, (m * nc) // (2 * g.n))  # tau_e = tau_d = 1/2
        if m_c > 4 * m_hat:  # rho = 4
            sg, _ = ctx.gp_sparsify(cg, m_hat, 2, w["seed"])
            sg.release()
        cg.release()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.profile_reset()
    ctx.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(ctx.stream)
    for _ in range(args.steps):
        step()
    ev1.record(ctx.stream)
    torch.cuda.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read()
    ms = ev0.elapsed_time(ev1) / args.steps
    print(json.dumps({"metric": "level-1 edges/s (clustering, contraction, sparsification)",
                      "value": m / (ms / 1000.0), "unit": "edges/s", "ms_per_step": ms, "steps": args.steps,
                      "warmup": args.warmup, "config": {"workload": w["name"], "U": U},
                      "kernel_classes": {k: v for k, v in prof.items() if v["launches"]}}), flush=True)
    ctx.close()
    return 0


def batch_mix(count, nmax, seed, place=None):
    """Independent graphs of the batched workload: n log-uniform in [1e3, nmax], the generator
    uniform over ER (average degree 8..32), 2D grid, 3D grid and R-MAT (edge factor 8), unit
    weights, k uniform over {2, 4, ..., 64}, eps 0.03, a seed per graph.  `place` (optional) maps
    each host graph to what is kept (e.g. its device copy), so that the host copies of a large
    batch need not all be held at once."""
    import numpy as np
    import graphgen as gg
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(nmax))))
        kind = int(rng.integers(0, 4))
        if kind == 0:
            g = gg.er(n, n * int(rng.integers(4, 17)), int(rng.integers(1, 1 << 30)))
        elif kind == 1:
            s2 = max(2, int(np.sqrt(n)))
            g = gg.grid2d(s2, s2)
        elif kind == 2:
            s3 = max(2, int(round(n ** (1 / 3))))
            g = gg.grid3d(s3, s3, s3)
        else:
            g = gg.rmat(max(10, int(round(np.log2(n)))), 8, seed=int(rng.integers(1, 1 << 30)))
        jobs.append((place(g) if place else g, int(2 ** rng.integers(1, 7)), 0.03, int(rng.integers(1, 1 << 30))))
    return jobs


def batch_summary(gp, count, nmax, workers, warmup, steps, serial=True):
    """Batched form on the same graphs: one gp_partition call after another (serial), the per-graph
    path of gp_partition_batch alone (host worker threads, engine off), and gp_partition_batch with
    the batched engine after gp_batch_autotune has picked its CTA size and the engine/per-graph split
    on this batch.  graphs/s of each (best of `steps` passes after `warmup`), and whether the results
    agree item by item."""
    import torch
    t = time.time()
    ctx = gp.Context(0)
    jobs = batch_mix(count, nmax, 1, place=lambda g: (gp.DeviceGraph.from_host(g), g.m))
    dev = [(dg, k, e, sd) for (dg, _), k, e, sd in jobs]
    torch.cuda.synchronize()
    log(f"[bench] generated and uploaded {len(jobs)} graphs in {time.time() - t:.1f}s")

    def timed(fn):
        best, out = None, None
        for rep in range(warmup + steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if rep >= warmup:
                best = dt if best is None else min(best, dt)
        return best, out

    res = {}
    if serial:
        ts, ser = timed(lambda: [ctx.gp_partition(dg, k, e, sd)[:2] for dg, k, e, sd in dev])
        res["serial"] = ser
    ctx.batch_set_tuning(engine=0)
    tw, wrk = timed(lambda: ctx.gp_partition_batch(dev, workers=workers))
    t0 = time.perf_counter()
    tun = ctx.batch_autotune(dev, workers=workers)
    tune_s = time.perf_counter() - t0
    te, eng = timed(lambda: ctx.gp_partition_batch(dev, workers=workers, details=True))
    n_engine = sum(1 for r in eng if r[2])
    ref = res.get("serial", wrk)
    same = all(c1 == c2 == c3 and torch.equal(b1, b2) and torch.equal(b1, b3)
               for (b1, c1), (b2, c2), (b3, c3, _, _) in zip(ref, wrk, eng))
    ctx.batch_set_tuning()
    ctx.close()
    out = {"graphs_per_s": len(jobs) / te, "worker_path_graphs_per_s": len(jobs) / tw,
           "speedup_vs_worker_path": tw / te, "identical_results": same, "graphs": len(jobs),
           "engine_items": n_engine, "edges": sum(m for (_, m), _, _, _ in jobs), "workers": workers,
           "tuning": tun.as_dict(), "tune_s": tune_s,
           "timing": f"best of {steps} pass(es) after {warmup}, host wall clock around each pass "
                     "(tuning outside the timed passes)",
           "workload": f"{len(jobs)} graphs, n log-uniform in [1e3, {nmax:g}], ER deg 8-32 / 2D grid / 3D grid / "
                       "R-MAT ef 8, k in {2..64}, eps 0.03 (C4 mix)"}
    if serial:
        out.update({"serial_graphs_per_s": len(jobs) / ts, "speedup": ts / te})
    return out


def run_batch(args):
    import paper_2504_17615_gb300 as gp
    from paper_2504_17615_gb300 import build as gpbuild
    gpbuild.build()
    out = batch_summary(gp, args.batch_count, args.batch_nmax, args.batch_workers, args.warmup, args.steps,
                        serial=not args.batch_no_serial)
    out.update({"metric": "batched graphs/s", "value": out["graphs_per_s"], "unit": "graphs/s",
                "steps": args.steps, "warmup": args.warmup, "config": {"workload": out["workload"]}})
    print(json.dumps(out), flush=True)
    return 0


def serve_mix(count, mmax, seed):
    """Requests of the served workload: edge counts log-uniform in [1e4, mmax], the generator
    uniform over ER (average degree 8..32), 2D grid, 3D grid and R-MAT (edge factor 8), unit
    weights, k uniform over {2, 8, 32, 128}, eps 0.03, a seed per request."""
    import numpy as np
    import graphgen as gg
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = float(np.exp(rng.uniform(np.log(1e4), np.log(mmax))))
        kind = int(rng.integers(0, 4))
        if kind == 0:
            d = int(rng.integers(8, 33))
            n = max(64, int(2 * m / d))
            g = gg.er(n, int(m), int(rng.integers(1, 1 << 30)))
        elif kind == 1:
            s2 = max(2, int(np.sqrt(m / 2)))
            g = gg.grid2d(s2, s2)
        elif kind == 2:
            s3 = max(2, int(round((m / 3) ** (1 / 3))))
            g = gg.grid3d(s3, s3, s3)
        else:
            g = gg.rmat(max(8, int(round(np.log2(m / 8)))), 8, seed=int(rng.integers(1, 1 << 30)))
        out.append((g, int(rng.choice([2, 8, 32, 128])), 0.03, int(rng.integers(1, 1 << 30))))
    return out


def serve_run(gp, reqs, arrivals, workers, budget):
    """Submits request i at arrivals[i] seconds; returns (latencies ms, wall seconds, results)."""
    import threading
    srv = gp.Server(0, workers=workers, hbm_budget=budget)
    tickets = [None] * len(reqs)
    t0 = time.perf_counter()

    def submitter():
        for i, (r, a) in enumerate(zip(reqs, arrivals)):
            d = a - (time.perf_counter() - t0)
            if d > 0:
                time.sleep(d)
            tickets[i] = srv.submit(*r)

    th = threading.Thread(target=submitter)
    th.start()
    lat, res = [], []
    for i in range(len(reqs)):
        while tickets[i] is None:
            time.sleep(0.0005)
        blocks, cut, resp = srv.wait(tickets[i])
        lat.append(resp.total_ms)
        res.append((blocks.copy(), cut))
    th.join()
    wall = time.perf_counter() - t0
    srv.close()
    return lat, wall, res


def serve_summary(gp, count, mmax, workers):
    """Served form: a Poisson stream of requests through the library's request loop.  The
    capacity with `workers` workers is measured closed-loop (all requests at once); then Poisson
    arrivals at 70% of it (sustained load) and at 150% of it (saturated), each served with `workers`
    workers and with one worker (the plain one-request-at-a-time path) on the same arrivals."""
    import numpy as np
    t = time.time()
    reqs = serve_mix(count, mmax, 2)
    log(f"[bench] generated {len(reqs)} requests in {time.time() - t:.1f}s")
    budget = 96 << 30
    _, closed1, _ = serve_run(gp, reqs, [0.0] * len(reqs), 1, budget)
    _, closedw, _ = serve_run(gp, reqs, [0.0] * len(reqs), workers, budget)
    out = {"requests": len(reqs), "edges": sum(r[0].m for r in reqs), "hbm_budget_bytes": budget,
           "capacity_graphs_per_s": {"workers_1": len(reqs) / closed1, f"workers_{workers}": len(reqs) / closedw},
           "workload": f"{len(reqs)} requests, m log-uniform in [1e4, {mmax:g}], ER / 2D grid / 3D grid / R-MAT, "
                       "k in {2, 8, 32, 128}, eps 0.03, Poisson arrivals (C5 mix)"}
    same = True
    for name, lam in (("sustained", 0.7 * len(reqs) / closedw), ("saturated", 1.5 * len(reqs) / closedw)):
        arrivals = np.cumsum(np.random.default_rng(3).exponential(1.0 / lam, len(reqs))).tolist()
        rec = {"arrival_rate_per_s": lam}
        res = {}
        for w in (1, workers):
            lat, wall, r = serve_run(gp, reqs, arrivals, w, budget)
            res[w] = r
            rec[f"workers_{w}"] = {"graphs_per_s": len(reqs) / wall, "p50_ms": float(np.percentile(lat, 50)),
                                   "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(np.mean(lat))}
            log(f"[bench] serve {name} workers={w}: {len(reqs) / wall:.1f} graphs/s p50 "
                f"{rec[f'workers_{w}']['p50_ms']:.1f} ms p99 {rec[f'workers_{w}']['p99_ms']:.1f} ms")
        same = same and all(c1 == c2 and np.array_equal(b1, b2) for (b1, c1), (b2, c2) in zip(res[1], res[workers]))
        out[name] = rec
    out["identical_results"] = same
    return out


def run_serve(args):
    import paper_2504_17615_gb300 as gp
    from paper_2504_17615_gb300 import build as gpbuild
    gpbuild.build()
    out = serve_summary(gp, args.serve_count, args.serve_mmax, args.serve_workers)
    out.update({"metric": "served graphs/s and p50/p99 latency",
                "value": out["sustained"][f"workers_{args.serve_workers}"]["graphs_per_s"], "unit": "graphs/s",
                "config": {"workload": out["workload"]}})
    print(json.dumps(out), flush=True)
    return 0


def run_report(args):
    """Per-level nodes and edges of the hierarchy with each sparsifier (Sec. 4.2; the synthetic
    analogue of the paper's edges-per-level figure), with cut and phase times."""
    import torch
    import paper_2504_17615_gb300 as gp
    from paper_2504_17615_gb300 import build as gpbuild
    w = workload_of(args)
    gpbuild.build()
    g = make_graph(w, 0, 1)
    ctx = gp.Context(0)
    dg = gp.DeviceGraph.from_host(g)
    out = {"report": "hierarchy by sparsifier", "config": {"workload": w["name"], "k": w["k"], "eps": w["eps"],
                                                        "seed": w["seed"]}, "modes": {}}
    names = {gp.GP_SPARSIFY_NONE: "none", gp.GP_SPARSIFY_TWEIGHT: "t_weight", gp.GP_SPARSIFY_UNIFORM: "uniform",
             gp.GP_SPARSIFY_TWEIGHT_EXACT: "t_weight_exact"}
    for mode, name in names.items():
        cfg = gp.default_config(sparsifier=mode)
        ctx.gp_partition(dg, w["k"], w["eps"], w["seed"], cfg)  # warm-up
        torch.cuda.synchronize()
        _, cut, st = ctx.gp_partition(dg, w["k"], w["eps"], w["seed"], cfg)
        levels = [{"n": L["n"], "m": L["m"], "m_coarse": L["m_coarse"], "m_hat": L["m_hat"],
                   "triggered": L["triggered"], "m_next": L["m_next"]} for L in st.levels_list()]
        out["modes"][name] = {"cut": cut, "ms_total": st.ms_total, "ms_coarsen": st.ms_coarsen,
                              "levels": levels, "n_coarsest": st.n_coarsest,
                              "edges_summed_over_levels": sum(L["m"] for L in levels)}
        log(f"[bench] report {name}: cut={cut} total {st.ms_total:.1f} ms coarsen {st.ms_coarsen:.1f} ms")
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--small", action="store_true", help="2^20-node graph (quick checks)")
    ap.add_argument("--scale", type=int, default=None,
                    help="ER graph with 2^S nodes and average degree 20 instead (profiling cases)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch-serve", action="store_true",
                    help="leave the batched and served summaries out of the default line")
    ap.add_argument("--batch", action="store_true",
                    help="batched form: many independent graphs, serial calls against gp_partition_batch")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-nmax", type=float, default=1e5)
    ap.add_argument("--batch-workers", type=int, default=8)
    ap.add_argument("--batch-no-serial", action="store_true",
                    help="batched form: leave out the one-call-after-another pass (large batches)")
    ap.add_argument("--serve", action="store_true",
                    help="served form: Poisson request stream through the request loop, p50/p99 latency")
    ap.add_argument("--serve-count", type=int, default=128)
    ap.add_argument("--serve-mmax", type=float, default=1e8)
    ap.add_argument("--serve-workers", type=int, default=8)
    ap.add_argument("--report", action="store_true",
                    help="per-level hierarchy of the workload with each sparsifier (no timing contract)")
    ap.add_argument("--level1", action="store_true",
                    help="time level 1 of Alg. 1 alone on the workload graph (profiling case)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the dominant kernel, if measured")
    args = ap.parse_args()
    if args.warmup < 3:
        log("[bench] warning: fewer than 3 warm-up steps")
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.level1:
        return run_level1(args)
    if args.report:
        return run_report(args)
    if args.batch:
        return run_batch(args)
    if args.serve:
        return run_serve(args)
    return run_gpu(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
