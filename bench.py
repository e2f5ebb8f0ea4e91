"""Benchmark of the exact k-clique counter on synthetic workloads.

Default workload: R-MAT scale 20 (1,048,576 vertices, edge factor 16,
a/b/c/d = .57/.19/.19/.05, seed 0), symmetrised and deduplicated, u32 CSR.
One step = the whole hot path on that graph: degeneracy orientation on the
device (kc_graph_create from a device-resident CSR) followed by the counts of
the plan (default: k = 4 vertex-centric, then k = 4 edge-centric, both with
the graph-orientation traversal of Fig. 2).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank counts its
own replica of the workload (weak scaling); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2104_13209_gb300 import synth  # noqa: E402

CACHE = os.path.join(ROOT, "paper_2104_13209_gb300", "_build", "cache")
PROFILES = os.path.join(ROOT, "profiles")
L2_FLUSH_BYTES = 512 << 20   # larger than the 129 MB L2
POPC_PER_SM_CLK = 16         # population count results per SM per clock (CUDA arithmetic throughput table)
ISSUE_PER_SM_CLK = 4         # warp instructions issued per SM per clock (four schedulers)
METRIC = "k-clique count time & cliques/s (k=4/7/10); batched/served queries/s, p99 vs plain"


_T0 = time.perf_counter()


def log(msg: str):
    """Progress of the run, on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:8.1f}s] {msg}", file=sys.stderr, flush=True)


def workload_graph(scale=20, ef=16, seed=0):
    os.makedirs(CACHE, exist_ok=True)
    path = os.path.join(CACHE, f"rmat{scale}_ef{ef}_s{seed}.npz")
    if os.path.exists(path):
        z = np.load(path)
        return synth.CSRGraph(int(z["n"]), z["row_ptr"], z["col_idx"], f"RMAT{scale}-ef{ef}s{seed}")
    g = synth.rmat(scale, ef, seed=seed)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, n=g.n, row_ptr=g.row_ptr, col_idx=g.col_idx)
    os.replace(tmp, path)
    return g


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over the ranks of the default process group (x itself
    when there is one rank): the slowest replica sets the time."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job throughput of `world` replicas that each process
    units_per_rank units: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds


def parse_plan(s: str):
    """'4vc,7pv' -> [(4, 'vc'), ...]."""
    out = []
    for tok in s.split(","):
        tok = tok.strip()
        k = int("".join(ch for ch in tok if ch.isdigit()))
        sch = "".join(ch for ch in tok if ch.isalpha()) or "vc"
        out.append((k, sch))
    return out


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU baseline: the oracle, as it stands, on a bounded sample of roots
# ----------------------------------------------------------------------------
def oracle_sample_rate(g, k: int, budget_s: float, dag=None, stride: int | None = None):
    """cliques/s of the oracle's Fig. 2 traversal on a uniform sample of roots
    (every stride-th root with out-degree >= k - 1; the stride is calibrated to
    about budget_s of work unless given)."""
    from oracle import oracle as O

    if dag is None:
        dag = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    drp, dci = dag[0], dag[1]
    d = np.diff(drp.astype(np.int64))
    roots = np.nonzero(d >= k - 1)[0].astype(np.uint32)
    threads = O.default_threads()

    def run(st):
        sample = roots[::st]
        t = time.perf_counter()
        c = O.count_orient(drp, dci, k, roots=sample, threads=threads).total
        return c, time.perf_counter() - t, int(sample.size)

    if stride is None:
        stride = 1 << 14
        while True:
            c, dt, ns = run(stride)
            if dt >= budget_s * 0.25 or stride == 1:
                break
            stride = max(1, int(stride * max(dt, 1e-3) / budget_s))
        if dt < budget_s * 0.5 and stride > 1:
            stride = max(1, int(stride * dt / budget_s))
    c, dt, ns = run(stride)
    return {"count": c, "seconds": dt, "roots": ns, "stride": stride, "threads": threads,
            "rate": c / dt if dt > 0 else None}


def run_reference(a, g, plan, world, rank):
    """--impl reference: the CPU oracle timed on this host's cores on bounded samples."""
    if rank != 0:
        return
    from oracle import oracle as O

    t0 = time.perf_counter()
    dag = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    orient_s = time.perf_counter() - t0
    k = plan[0][0]
    per_step = max(2.0, 60.0 / max(1, a.steps + a.warmup))
    stride = oracle_sample_rate(g, k, per_step, dag)["stride"]
    for _ in range(a.warmup):
        oracle_sample_rate(g, k, per_step, dag, stride)
    cnt, secs, info = 0, 0.0, None
    for _ in range(a.steps):
        info = oracle_sample_rate(g, k, per_step, dag, stride)
        cnt += info["count"]
        secs += info["seconds"]
    value = cnt / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "cliques/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * secs / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": g.name, "n": g.n, "edges": g.num_edges, "orientation": "degeneracy",
                   "plan": [f"k={kk} {sch}" for kk, sch in plan],
                   "traversal": f"graph orientation (Fig. 2), CPU oracle, k = {k} (both splits count the same)"},
        "cpu_baseline": {"value": value, "unit": "cliques/s", "cores": info["threads"], "kind": "oracle",
                         "sample": f"every {info['stride']}-th root with out-degree >= {k - 1} "
                                   f"({info['roots']} roots), orientation {orient_s:.1f}s untimed"},
        "e2e": {"value": value, "unit": "cliques/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2104_13209_gb300", "csrc", f)
                  for f in ("kc_count.cu", "kc_dfs.cuh", "kc_bitmap.cuh", "kc_common.cuh")]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def traffic_record() -> dict:
    """Counters of the count kernel from profiles/traffic.json (DRAM bytes
    and warp instructions per launch), if the kernel's sources are unchanged
    since they were taken; else {}."""
    path = os.path.join(PROFILES, "traffic.json")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        rec = json.load(f)
    if rec.get("kernel_source_sha256_16") != kernel_source_hash():
        return {}
    return rec


def algorithmic_bytes(drp, dci, k: int) -> float:
    """HBM bytes the vertex-centric bitmap build must read for size-k counts:
    for every root v with out-degree >= k - 1, its own DAG row and the DAG
    row of every out-neighbour (4 bytes per entry)."""
    d = np.diff(drp.astype(np.int64))
    roots = d >= k - 1
    src = np.repeat(np.arange(d.size), d)
    return float(4 * (d[roots].sum() + d[dci.astype(np.int64)][roots[src]].sum()))


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def measured_hbm_gbs() -> float:
    return float(measured_peaks()["hbm_gbs"])


def device_rates(dev_index: int) -> dict:
    """SM count (device attribute) and the maximum SM clock (the measured
    peaks record, else nvidia-smi), and the integer-pipe and issue peaks
    derived from them."""
    import torch

    sms = torch.cuda.get_device_properties(dev_index).multi_processor_count
    mhz = measured_peaks().get("sm_max_mhz")
    src = "MEASURED_PEAKS.json sm_max_mhz"
    if not mhz:
        try:
            out = subprocess.run(["nvidia-smi", "-i", str(dev_index), "--query-gpu=clocks.max.sm",
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
            mhz = float(out.stdout.strip().splitlines()[0])
            src = "nvidia-smi clocks.max.sm"
        except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
            mhz, src = 2070.0, "nominal maximum"
    hz = float(mhz) * 1e6
    return {"sms": sms, "sm_hz": hz, "clock_source": src,
            "alu_tops": 2.0 * sms * POPC_PER_SM_CLK * hz / 1e12,
            "issue_ginst": sms * ISSUE_PER_SM_CLK * hz / 1e9,
            "alu_note": f"derived: {sms} SMs x {POPC_PER_SM_CLK} popc/clk x {hz / 1e9:.2f} GHz x 2 ops "
                        "(AND + POPC) per word",
            "issue_note": f"derived: {sms} SMs x {ISSUE_PER_SM_CLK} warp instructions/clk x {hz / 1e9:.2f} GHz"}


def measured_l2_read_gbs(dev) -> float:
    """Bandwidth of the L2: a 24 MiB buffer copied into another (both
    resident in the 129 MB L2), read plus written bytes, 50 copies per
    timing, best of 8 (a lower bound of the peak: a plain vectorised copy)."""
    import torch

    x = torch.ones(6 << 20, dtype=torch.float32, device=dev)
    y = torch.empty_like(x)
    for _ in range(5):
        y.copy_(x)
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(8):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(50):
            y.copy_(x)
        e1.record()
        e1.synchronize()
        best = max(best, 50 * 2 * x.numel() * 4 / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


def run_ours(a, g, plan, world, rank, local_rank):
    import torch

    from paper_2104_13209_gb300 import build, kclique

    build.build()
    kclique.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    rp_d = torch.from_numpy(g.row_ptr.view(np.int32)).to(dev)
    ci_d = torch.from_numpy(g.col_idx.view(np.int32)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    results = torch.zeros((len(plan), kclique.RESULT_BYTES), dtype=torch.uint8, device=dev)
    n, nnz = g.n, int(g.row_ptr[-1])

    def step(timing):
        """One pass of the hot path; timing: list to which (label, ms) pairs are appended."""
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G = kclique.Graph(rp_d, ci_d, n=n, orient="degeneracy", validate=False, stream=stream)
            e1.record(stream)
            evs = [("orient", e0, e1)]
            for i, (k, sch) in enumerate(plan):
                c0 = torch.cuda.Event(enable_timing=True)
                c1 = torch.cuda.Event(enable_timing=True)
                c0.record(stream)
                G.count_async(k, results[i], scheme=sch, stream=stream)
                c1.record(stream)
                evs.append((f"k{k}{sch}", c0, c1))
            stream.synchronize()
            G.close()
        for lab, x0, x1 in evs:
            timing.append((lab, x0.elapsed_time(x1)))

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.fill_(1)
        stream.synchronize()

    log("main workload: warm-up")
    for _ in range(a.warmup):
        step([])
        flush_l2()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    launches0 = kclique.launch_count()
    timings = []
    with ClockSampler(local_rank) as clk:
        t_wall0 = time.perf_counter()
        for _ in range(a.steps):
            flush_l2()
            step(timings)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    launches = kclique.launch_count() - launches0
    if world > 1:
        dist.barrier()
    res = [kclique.parse_result(bytes(results[i].cpu().numpy())) for i in range(len(plan))]
    step_ms = sum(ms for _, ms in timings) / a.steps
    per_label = {}
    for lab, ms in timings:
        per_label[lab] = per_label.get(lab, 0.0) + ms / a.steps
    total_cliques = sum(r.total for r in res)
    step_ms = max_over_ranks(step_ms, dev)

    log("main workload: timed steps done; end-to-end steps")
    # end to end through the public API from pinned host memory
    rp_h = torch.from_numpy(g.row_ptr.view(np.int32)).pin_memory()
    ci_h = torch.from_numpy(g.col_idx.view(np.int32)).pin_memory()
    rp_np = rp_h.numpy().view(np.uint32)
    ci_np = ci_h.numpy().view(np.uint32)

    def e2e_step():
        G = kclique.Graph(rp_np, ci_np, n=n, orient="degeneracy", validate=True, stream=stream)
        tot = 0
        for k, sch in plan:
            tot += G.count(k, scheme=sch, stream=stream).total
        G.close()
        return tot

    for _ in range(max(1, a.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    e2e_times = []
    for _ in range(a.steps):
        flush_l2()
        t0 = time.perf_counter()
        tot = e2e_step()
        e2e_times.append(time.perf_counter() - t0)
        assert tot == total_cliques, "end-to-end count differs from the device-resident count"
    e2e_s = max_over_ranks(float(np.mean(e2e_times)), dev)

    # roofline of the dominant kernel (the first count of the plan): the
    # slower of its algorithmic CSR bytes at HBM bandwidth and its AND + POPC
    # word operations at the population-count pipe's peak (the model's two
    # terms), with the terms that show its actual limiter beside them: the
    # same bytes at the measured L2 read bandwidth (the DAG stays resident in
    # L2) and its issued warp instructions at the issue peak (ncu counters)
    k0, s0 = plan[0]
    lab0 = f"k{k0}{s0}"
    t_cnt = per_label[lab0] / 1e3
    with torch.cuda.stream(stream):
        G = kclique.Graph(rp_d, ci_d, n=n, orient="degeneracy", validate=False, stream=stream)
        drp, dci, _, _ = G.export()
    b_alg = algorithmic_bytes(drp, dci, k0)
    ops = 2.0 * res[0].words            # one AND + one POPC per 32-bit bitmap word
    rates = device_rates(local_rank)
    peak_hbm = measured_hbm_gbs()
    peak_alu = rates["alu_tops"]
    peak_l2 = measured_l2_read_gbs(dev)
    t_hbm = b_alg / (peak_hbm * 1e9)
    t_alu = ops / (peak_alu * 1e12)
    rec = traffic_record()
    terms = {"hbm": {"bytes": b_alg, "achieved_gbs": b_alg / t_cnt / 1e9, "peak_gbs": peak_hbm,
                     "roof_ms": 1e3 * t_hbm},
             "alu": {"ops": ops, "achieved_tops": ops / t_cnt / 1e12, "peak_tops": peak_alu, "roof_ms": 1e3 * t_alu,
                     "peak_note": rates["alu_note"]},
             "l2": {"bytes": b_alg, "achieved_gbs": b_alg / t_cnt / 1e9, "peak_gbs": peak_l2,
                    "roof_ms": 1e3 * b_alg / (peak_l2 * 1e9),
                    "peak_note": "measured here: a 48 MiB L2-resident buffer read by a reduction (lower bound)"}}
    if rec.get("warp_inst_per_launch"):
        inst = float(rec["warp_inst_per_launch"])
        terms["issue"] = {"warp_inst": inst, "achieved_ginst_s": inst / t_cnt / 1e9,
                          "peak_ginst_s": rates["issue_ginst"], "roof_ms": 1e3 * inst / (rates["issue_ginst"] * 1e9),
                          "peak_note": rates["issue_note"], "source": "profiles/traffic.json (ncu)"}
    if t_hbm >= t_alu:
        roof = {"bound": "hbm", "achieved": terms["hbm"]["achieved_gbs"], "peak": peak_hbm, "unit": "GB/s"}
    else:
        roof = {"bound": "alu", "achieved": terms["alu"]["achieved_tops"], "peak": peak_alu, "unit": "Tops/s"}
    limiter = max(terms, key=lambda x: terms[x]["roof_ms"] / (1e3 * t_cnt) if x != "hbm" else 0.0)
    roof.update({"frac": roof["achieved"] / roof["peak"], "traffic": rec.get("dram_bytes_per_launch"),
                 "kernel": f"k_count_orient ({lab0})", "kernel_ms": 1e3 * t_cnt, "terms": terms,
                 "closest_term": limiter,
                 "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if roof["bound"] == "hbm"
                 else "derived from unit counts and clock"})

    # the deep sizes of the same configuration: one count of size k_deep
    # (edge-centric, the choice for k >= 6), after a k = 5 count that loads
    # the same kernel
    deep = None
    log("roofline terms measured")
    if a.deep_k:
        log(f"k = {a.deep_k} sub-record")
        kd = a.deep_k
        rr = torch.zeros(kclique.RESULT_BYTES, dtype=torch.uint8, device=dev)
        G.set_time_limit(a.deep_limit)  # an unfinished count reports KC_E_TIMEOUT in "status"
        with torch.cuda.stream(stream):
            G.count_async(5, rr, scheme="ec", stream=stream)
        stream.synchronize()
        launches_d0 = kclique.launch_count()
        with ClockSampler(local_rank) as clk_d:
            with torch.cuda.stream(stream):
                d0 = torch.cuda.Event(enable_timing=True)
                d1 = torch.cuda.Event(enable_timing=True)
                d0.record(stream)
                if a.deep_pivot:
                    G.count_async(kd, rr, pivot=True, stream=stream)
                else:
                    G.count_async(kd, rr, scheme="ec", stream=stream)
                d1.record(stream)
            stream.synchronize()
        rd = kclique.parse_results(bytes(rr.cpu().numpy()), 1)[0]  # a timed-out count reports its status
        dms = d0.elapsed_time(d1)
        ok = rd.status == kclique.KC_OK
        deep = {"k": kd, "traversal": "pivot (fixed k)" if a.deep_pivot else "orientation, edge-centric",
                "status": kclique.status_name(rd.status), "count": str(rd.total) if ok else None,
                "ms": dms, "time_limit_s": a.deep_limit, "cliques_per_s": rd.total / (dms / 1e3) if ok else None,
                "gpu_launches": kclique.launch_count() - launches_d0, "clocks": clk_d.summary()}
        if a.deep_pivot:
            deep["tree_nodes"] = rd.words
            deep["tree_nodes_per_s"] = rd.words / (dms / 1e3)
        else:
            dops = 2.0 * rd.words
            deep["roofline"] = {"bound": "alu", "achieved": dops / (dms / 1e3) / 1e12, "peak": peak_alu,
                                "unit": "Tops/s", "frac": dops / (dms / 1e3) / 1e12 / peak_alu,
                                "kernel": "k_count_deep<EC> (one launch)", "ops": dops, "peak_note": rates["alu_note"]}
    G.close()

    clocks = clk.summary()
    value = replica_throughput(total_cliques, step_ms / 1e3, world)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "cliques/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": step_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int64",
        "data": "synthetic",
        "config": {
            "workload": g.name, "n": n, "edges": g.num_edges, "orientation": "degeneracy",
            "plan": [f"k={k} {sch}" for k, sch in plan], "counts": [str(r.total) for r in res],
            "step_ms_parts": {k: round(v, 3) for k, v in per_label.items()},
            "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
            "wall_s_timed_region": t_wall, "parallelism": f"replicas x{world}",
        },
        "e2e": {"value": replica_throughput(total_cliques, e2e_s, world), "unit": "cliques/s",
                "h2d_bytes_per_step": 4 * (n + 1) + 4 * nnz,
                "d2h_bytes_per_step": kclique.RESULT_BYTES * len(plan)},
        "roofline": roof,
        "clocks": clocks,
        "gpu_launches": launches,
    }
    if deep is not None:
        line[f"k{deep['k']}"] = deep
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        log("CPU baseline (oracle)")
        cb = oracle_sample_rate(g, k0, a.cpu_budget)
        line["cpu_baseline"] = {"value": cb["rate"], "unit": "cliques/s", "cores": cb["threads"], "kind": "oracle",
                                "sample": f"k={k0}: every {cb['stride']}-th root with out-degree >= {k0 - 1} "
                                          f"({cb['roots']} roots, {cb['seconds']:.1f} s)"}
    return line


# ----------------------------------------------------------------------------
# the planted-community power-law graph: fixed-k totals and per-vertex counts
# ----------------------------------------------------------------------------
def chunglu_graph(seed=0):
    """Chung-Lu, 4,000,000 vertices, exponent 2.1, mean degree 30, with 2,000
    planted communities of 40-200 vertices at intra-edge probability 0.9."""
    os.makedirs(CACHE, exist_ok=True)
    path = os.path.join(CACHE, f"chunglu4m_c2000_s{seed}.npz")
    if os.path.exists(path):
        z = np.load(path)
        return synth.CSRGraph(int(z["n"]), z["row_ptr"], z["col_idx"], str(z["name"]))
    g = synth.chung_lu_planted(4_000_000, 2.1, 30.0, ncomm=2000, size_min=40, size_max=200, p_in=0.9, seed=seed)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, n=g.n, row_ptr=g.row_ptr, col_idx=g.col_idx, name=g.name)
    os.replace(tmp, path)
    return g


def run_chunglu(a, world, rank, local_rank):
    """One degeneracy orientation, then the k-clique totals (orientation
    traversal) for each k of --chunglu-k and the per-vertex counts for each
    k of --chunglu-pv-k, every count under --chunglu-limit seconds.  The
    per-vertex counts are checked by the identity sum_v c_k(v) = k * c_k."""
    import torch

    from paper_2104_13209_gb300 import build, kclique

    log("planted-community graph: generating")
    g = chunglu_graph()
    log(f"planted-community graph: {g.n} vertices, {g.num_edges} edges")
    build.build()
    kclique.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    rp_d = torch.from_numpy(g.row_ptr.view(np.int32)).to(dev)
    ci_d = torch.from_numpy(g.col_idx.view(np.int32)).to(dev)
    ks = [int(x) for x in str(a.chunglu_k).split(",") if x]
    pks = [int(x) for x in str(a.chunglu_pv_k).split(",") if x]
    rec = {"workload": g.name, "n": g.n, "edges": g.num_edges, "time_limit_s": a.chunglu_limit, "totals": {},
           "per_vertex": {}}
    rates = device_rates(local_rank)
    launches0 = kclique.launch_count()
    with ClockSampler(local_rank) as clk:
        with torch.cuda.stream(stream):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G = kclique.Graph(rp_d, ci_d, n=g.n, orient="degeneracy", validate=False, stream=stream)
            e1.record(stream)
        stream.synchronize()
        rec["orient_ms"] = e0.elapsed_time(e1)
        rec["d_max"] = G.info()["d_max"]
        G.set_time_limit(a.chunglu_limit)
        rr = torch.zeros(kclique.RESULT_BYTES, dtype=torch.uint8, device=dev)
        for k in ks:
            with torch.cuda.stream(stream):
                c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                c0.record(stream)
                G.count_async(k, rr, scheme="ec", stream=stream)
                c1.record(stream)
            stream.synchronize()
            r = kclique.parse_results(bytes(rr.cpu().numpy()), 1)[0]
            ms = c0.elapsed_time(c1)
            ops = 2.0 * r.words
            rec["totals"][str(k)] = {
                "status": kclique.status_name(r.status), "count": str(r.total) if r.status == kclique.KC_OK else None,
                "ms": ms, "cliques_per_s": r.total / (ms / 1e3) if r.status == kclique.KC_OK else None,
                "flags": r.flags,
                "roofline": {"bound": "alu", "achieved": ops / (ms / 1e3) / 1e12, "peak": rates["alu_tops"],
                             "unit": "Tops/s", "frac": ops / (ms / 1e3) / 1e12 / rates["alu_tops"],
                             "kernel": "k_count_deep<EC> (one launch)" if k >= 5 else "k_count_orient<EC>",
                             "ops": ops, "peak_note": rates["alu_note"]}}
            log(f"planted-community graph: k = {k} total {r.total} in {ms:.0f} ms ({kclique.status_name(r.status)})")
        for k in pks:
            t0 = time.perf_counter()
            try:
                tot, pv, fl = G.count_per_vertex(k, pivot=False, stream=stream)
                dt = time.perf_counter() - t0
                s = int(pv.astype(object).sum())
                rec["per_vertex"][str(k)] = {
                    "status": "KC_OK", "ms": 1e3 * dt, "total": str(tot), "flags": fl,
                    "sum_equals_k_times_total": s == k * tot, "vertices_in_a_clique": int(np.count_nonzero(pv)),
                    "max": str(int(pv.max())),
                    "timed": "host clock around the synchronous call (per-vertex array copied to the host inside)"}
            except kclique.KCError as e:
                rec["per_vertex"][str(k)] = {"status": kclique.status_name(e.status),
                                             "ms": 1e3 * (time.perf_counter() - t0)}
            log(f"planted-community graph: per-vertex k = {k}: {rec['per_vertex'][str(k)]['status']}")
        G.close()
    rec["clocks"] = clk.summary()
    rec["gpu_launches"] = kclique.launch_count() - launches0
    return rec


# ----------------------------------------------------------------------------
# the paper's ablation (Section 4.3, Figs. 6 and 7) on the R-MAT workload
# ----------------------------------------------------------------------------
def run_ablation(a, g, world, rank, local_rank):
    """Binary-encoded bitmaps against sorted lists (schemes vc/ec against
    vc-list/ec-list), every sub-warp width of the bitmap traversal, and the
    per-SM split of each count's work units (load balance, max / mean over
    the SMs), each count timed alone with CUDA events after an L2 flush."""
    import torch

    from paper_2104_13209_gb300 import build, kclique

    build.build()
    kclique.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    rp_d = torch.from_numpy(g.row_ptr.view(np.int32)).to(dev)
    ci_d = torch.from_numpy(g.col_idx.view(np.int32)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    rr = torch.zeros(kclique.RESULT_BYTES, dtype=torch.uint8, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    with torch.cuda.stream(stream):
        G = kclique.Graph(rp_d, ci_d, n=g.n, orient="degeneracy", validate=False, stream=stream)
    stream.synchronize()
    G.set_time_limit(a.deep_limit)

    def one(k, scheme, subwarp=0):
        with torch.cuda.stream(stream):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G.count_async(k, rr, scheme=scheme, subwarp=subwarp, stream=stream)
            e1.record(stream)
        stream.synchronize()
        r = kclique.parse_results(bytes(rr.cpu().numpy()), 1)[0]
        w = G.last_sm_work()[:sms].astype(np.float64)
        mean = float(w.mean()) if w.size else 0.0
        return {"k": k, "scheme": scheme, "subwarp": subwarp, "status": kclique.status_name(r.status),
                "count": str(r.total), "ms": e0.elapsed_time(e1), "work_units": r.words,
                "sm_work_max_over_mean": float(w.max()) / mean if mean > 0 else None,
                "sm_work_cv": float(w.std()) / mean if mean > 0 else None}

    log("ablation: warm-up")
    for scheme in ("vc", "ec", "vc-list", "ec-list"):
        one(3, scheme)
    runs = []
    for k in (3, 4):
        for scheme in ("vc", "ec", "vc-list", "ec-list"):
            runs.append(one(k, scheme))
            log(f"ablation: k = {k} {scheme}: {runs[-1]['ms']:.2f} ms")
    sweep = []
    for scheme in ("vc", "ec"):
        for sw in (1, 2, 4, 8, 16, 32):
            sweep.append(one(4, scheme, sw))
    G.close()
    by = {(r["k"], r["scheme"]): r for r in runs}
    ratios = {f"k{k}_{s}": by[(k, s + "-list")]["ms"] / by[(k, s)]["ms"] for k in (3, 4) for s in ("vc", "ec")}
    best = {s: min(x["ms"] for x in sweep if x["scheme"] == s) for s in ("vc", "ec")}
    worst = {s: max(x["ms"] for x in sweep if x["scheme"] == s) for s in ("vc", "ec")}
    return {"metric": METRIC, "workload": g.name, "orientation": "degeneracy", "runs": runs,
            "list_over_bitmap_time": ratios, "subwarp_sweep_k4": sweep,
            "subwarp_best_over_worst": {s: worst[s] / best[s] for s in ("vc", "ec")},
            "l2": f"flushed before each count ({L2_FLUSH_BYTES >> 20} MiB write)", "sms": sms}


# ----------------------------------------------------------------------------
# batched and serving workloads (many small graphs; a stream of queries)
# ----------------------------------------------------------------------------
def run_batch(a, world, rank, local_rank):
    """4,096 ego networks of BA(500k, 20), k uniform in 3..8: one captured
    CUDA graph of persistent launches against one launch per query."""
    import torch

    from paper_2104_13209_gb300 import build, kclique, workloads

    log("batched workload: generating the ego networks")
    egos, ks = workloads.ego_batch()
    log("batched workload: generated")
    build.build()
    kclique.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    nq = len(egos)
    gid = np.arange(nq)
    B = kclique.Batch(egos)
    tune_path = os.path.join(CACHE, f"tune_ego{nq}.json")
    os.makedirs(CACHE, exist_ok=True)
    if os.path.exists(tune_path):
        with open(tune_path) as f:
            tune = kclique.tune_from_list(json.load(f))
    else:
        log("batched workload: tuning")
        tune = B.tune(gid, ks, sample=256, stream=stream)
        with open(tune_path, "w") as f:
            json.dump(kclique.tune_to_list(tune), f)
    res = torch.zeros(nq * kclique.RESULT_BYTES, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ex = B.capture(gid, ks, res, tune=tune)

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        stream.synchronize()
        ms = []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.mean(ms))

    launches0 = kclique.launch_count()
    with ClockSampler(local_rank) as clk:
        step_ms = timed(lambda: ex.launch(stream), a.steps, a.warmup)
    launches = kclique.launch_count() - launches0
    got = kclique.parse_results(bytes(res.cpu().numpy()), nq)
    total = sum(r.total for r in got)
    words = sum(r.words for r in got)
    assert all(r.status == kclique.KC_OK for r in got)

    def per_query():
        for i in range(nq):
            B.count_async(gid[i:i + 1], ks[i:i + 1], res[i * kclique.RESULT_BYTES:(i + 1) * kclique.RESULT_BYTES],
                          tune=tune, stream=stream)

    log("batched workload: one launch sequence per query")
    plain_ms = timed(per_query, 1, 1)
    # end to end through the public call from host arrays, results read back
    e2e = []
    for _ in range(max(1, a.warmup)):
        B.count(gid, ks, tune=tune, stream=stream)
    for _ in range(a.steps):
        t0 = time.perf_counter()
        r2 = B.count(gid, ks, tune=tune, stream=stream)
        e2e.append(time.perf_counter() - t0)
    assert [r.total for r in r2] == [r.total for r in got]
    rates = device_rates(local_rank)
    peak = rates["alu_tops"]
    achieved = 2.0 * words / (step_ms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": nq / (step_ms / 1e3), "unit": "queries/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"batched: {nq} radius-1 ego networks of BA(500000, m=20), 50-5000 vertices, "
                               "k uniform in 3..8, degeneracy orientation",
                   "cliques": str(total), "launch": "one captured CUDA graph of persistent batched launches",
                   "tune": kclique.tune_to_list(tune), "l2": "flushed between timed steps"},
        "plain": {"value": nq / (plain_ms / 1e3), "unit": "queries/s", "ms_per_step": plain_ms,
                  "launch": "one batched launch sequence per query"},
        "e2e": {"value": nq / float(np.mean(e2e)), "unit": "queries/s", "h2d_bytes_per_step": nq * 56,
                "d2h_bytes_per_step": nq * kclique.RESULT_BYTES},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "k_count_batch (whole step)", "peak_note": rates["alu_note"]},
        "clocks": clk.summary(), "gpu_launches": launches,
    }
    if not a.no_cpu_baseline:
        from oracle import oracle as O

        t0 = time.perf_counter()
        done = 0
        while done < nq and time.perf_counter() - t0 < a.cpu_budget:
            h = egos[done]
            O.count(h.row_ptr, h.col_idx, int(ks[done]), threads=O.default_threads())
            done += 1
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": done / dt, "unit": "queries/s", "cores": O.default_threads(),
                                "kind": "oracle", "sample": f"the first {done} queries ({dt:.1f} s)"}
    return line


def run_serve(a, world, rank, local_rank):
    """The 64-graph pool under a Poisson query stream: the continuous-batching
    server against the same stream served one launch per query."""
    from paper_2104_13209_gb300 import workloads

    log("serving workload: generating the pool")
    gs = workloads.serve_pool()  # worker processes are spawned before any CUDA use
    log("serving workload: generated")
    import torch

    from paper_2104_13209_gb300 import build, kclique

    build.build()
    kclique.load()
    torch.cuda.set_device(local_rank)
    ts, gq, kq, pq = workloads.query_stream(a.rate, a.serve_seconds, len(gs))
    out = {}
    for mode in a.serve_modes.split(","):
        # both modes share the admission policy: each graph's cost profile
        # (measured as it is added, under the time limit) picks the traversal
        # and refuses the shapes that run out of time in both; they differ in
        # batching and overlap only
        S = kclique.Server(hbm_budget=200 << 30, max_batch=256, slots=4, serial=(mode == "plain"),
                           auto_traversal=True, refuse_expensive=True)
        S.set_time_limit(a.time_limit)
        log(f"serving ({mode}): adding and profiling the pool")
        t_add = time.perf_counter()
        for h in gs:
            S.add_graph(h)
        t_add = time.perf_counter() - t_add
        log(f"serving ({mode}): warm-up")
        for i in range(min(16, len(ts))):  # warm-up: the batched kernels once
            S.poll(S.submit(int(gq[i]), int(kq[i]), bool(pq[i])), -1)
        log(f"serving ({mode}): stream")
        launches0 = S.stats()["launches"]
        tickets = []
        t0 = time.perf_counter()
        for i in range(len(ts)):
            d = t0 + ts[i] - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets.append(S.submit(int(gq[i]), int(kq[i]), bool(pq[i])))
        rs = [S.poll(t, -1) for t in tickets]
        wall = time.perf_counter() - t0
        log(f"serving ({mode}): {len(rs)} queries answered in {wall:.1f} s")
        ok = [r for r in rs if r["status"] == kclique.KC_OK]
        lat = np.array([r["t_done_ms"] - r["t_submit_ms"] for r in ok]) if ok else np.zeros(1)
        span = (max(r["t_done_ms"] for r in rs) - min(r["t_submit_ms"] for r in rs)) / 1e3
        out[mode] = {"queries": len(rs), "completed": len(ok), "qps": len(ok) / span,
                     "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "mean_ms": float(lat.mean()), "latency_over": "completed queries",
                     "timeouts": int(sum(r["status"] == kclique.KC_E_TIMEOUT for r in rs)),
                     "refused": int(sum(r["status"] == kclique.KC_E_REFUSED for r in rs)),
                     "errors": int(sum(r["status"] not in (kclique.KC_OK, kclique.KC_E_TIMEOUT, kclique.KC_E_REFUSED)
                                       for r in rs)),
                     "launches": S.stats()["launches"] - launches0, "wall_s": wall, "add_and_profile_s": t_add,
                     "totals": [r["total"] if r["status"] == kclique.KC_OK else None for r in rs]}
        S.close()
    modes = list(out)
    mismatch = 0
    if len(modes) == 2:
        for x, y in zip(out[modes[0]]["totals"], out[modes[1]]["totals"]):
            if x is not None and y is not None and x != y:
                mismatch += 1
    main_mode = modes[0]
    line = {
        "metric": METRIC, "value": out[main_mode]["qps"], "unit": "queries/s", "n_gpus": world, "steps": 1,
        "warmup": 1, "ms_per_step": 1e3 * out[main_mode]["wall_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"serving: pool of {len(gs)} graphs (16 ER, 24 R-MAT 14-18, 24 Chung-Lu 100k-1M), "
                               f"Poisson {a.rate:g} req/s for {a.serve_seconds:g} s, k uniform 3..12, pivot p=0.5 "
                               "(the server picks the traversal from each graph's cost profile)",
                   "time_limit_s": a.time_limit, "max_batch": 256, "slots": 4},
        "latency_ms": {"p50": out[main_mode]["p50_ms"], "p99": out[main_mode]["p99_ms"]},
        "served": {m: {k: v for k, v in out[m].items() if k != "totals"} for m in modes},
        "mismatches": mismatch,
    }
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plan", default="4vc,4ec")
    ap.add_argument("--scale", type=int, default=20)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="rmat", choices=["rmat", "batch", "serve", "chunglu", "ablation"])
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--serve-seconds", type=float, default=0.5)
    ap.add_argument("--time-limit", type=float, default=0.25)
    ap.add_argument("--serve-modes", default="batched,plain")
    ap.add_argument("--sub", default="batch,serve",
                    help="sub-records of the default line: batch, serve, chunglu (one GPU only; empty: none)")
    ap.add_argument("--deep-k", type=int, default=7,
                    help="also time one count of this size on the same graph (0: skip)")
    ap.add_argument("--deep-limit", type=float, default=120.0,
                    help="time limit (s) of that count")
    ap.add_argument("--deep-pivot", action="store_true", help="count that size by the pivoting traversal")
    ap.add_argument("--chunglu-k", default="7,8", help="sizes of the planted-community totals")
    ap.add_argument("--chunglu-limit", type=float, default=180.0, help="time limit (s) of each planted-community count")
    ap.add_argument("--chunglu-pv-k", default="7", help="sizes of the planted-community per-vertex counts")
    a = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    if a.workload == "batch" and a.impl == "ours":
        print(json.dumps(run_batch(a, world, rank, local_rank)), flush=True)
        return
    if a.workload == "serve" and a.impl == "ours":
        print(json.dumps(run_serve(a, world, rank, local_rank)), flush=True)
        return
    if a.workload == "chunglu" and a.impl == "ours":
        print(json.dumps(run_chunglu(a, world, rank, local_rank)), flush=True)
        return
    g = workload_graph(a.scale)
    if a.workload == "ablation" and a.impl == "ours":
        print(json.dumps(run_ablation(a, g, world, rank, local_rank)), flush=True)
        return
    plan = parse_plan(a.plan)
    if a.impl == "reference":
        run_reference(a, g, plan, world, rank)
    else:
        line = run_ours(a, g, plan, world, rank, local_rank)
        # the batched and serving workloads of the same metric, as sub-records
        # of the one line (one GPU only: they are not replicated)
        subs = [x for x in a.sub.split(",") if x] if world == 1 else []
        if "batch" in subs:
            b = run_batch(a, world, rank, local_rank)
            line["batched"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "config", "plain", "e2e",
                                                 "roofline", "clocks", "gpu_launches", "cpu_baseline") if k in b}
        if "serve" in subs:
            sv = run_serve(a, world, rank, local_rank)
            line["served"] = {k: sv[k] for k in ("value", "unit", "config", "latency_ms", "served", "mismatches")}
        if "chunglu" in subs:
            line["planted_community"] = run_chunglu(a, world, rank, local_rank)
        if rank == 0:
            print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
