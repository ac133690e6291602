#!/usr/bin/env python
"""Benchmark of the s-line-graph build (the s-overlap hot path).

One step builds the canonical edge list of L_s for s = 2 and s = 8 on the
hypergraph H and on its dual H* (four slg_build calls) for the power-law
Chung-Lu workload (|E| = 1M hyperedges, |V| = 2M vertices, ~21M incidences,
hyperedge sizes Zipf(2.1) capped at 10^4, vertex weights power law 2.3).
Throughput is reported in wedges/s, a wedge being one upper-triangle path
e -> v -> f with |e|, |f| >= s (the exact work of the walk), summed over the
four builds.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank builds its own independent instance of the
workload (seed + rank): weak scaling, no collective on the data path.
``--impl reference`` times the CPU oracle (plain C, all host cores) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "L_s(H) build ms & wedges/s at s=2,8: batched/tiled vs plain GPU kernel, bit-exact"
UNIT = "wedges/s"
S_VALUES = (2, 8)
SIDES = (False, True)
WORKLOAD = "chung_lu_1m"
WORKLOAD_TEXT = ("Chung-Lu power-law hypergraph |E|=1M, |V|=2M, ~21M int32 incidences, "
                 "sizes Zipf(2.1) capped 1e4 (mean ~21), vertex weights power law 2.3; "
                 "builds L_s(H) and L_s(H*) at s=2 and s=8 per step")
CPU_SAMPLE_STRIDE = 16      # oracle baseline, context figure: every 16th row of each build
CPU_FULL_BUILD = (False, 8)  # the build the oracle times in full: L_8(H), 1.6e9 wedges
CPU_FULL_REPS = 2           # full timed oracle builds in the GPU arm's cpu_baseline


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--algo", choices=["binned", "plain", "spgemm"], default="binned")
    ap.add_argument("--relabel", choices=["none", "asc", "desc"], default="none",
                    help="degree-ordered relabelling of the rows before the walk")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the plain-kernel and SpGEMM comparison builds")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the dense-core (tiled) and batched comparisons")
    ap.add_argument("--no-handle", action="store_true",
                    help="each build validates and maps the input itself (no slg_graph "
                         "handle per step)")
    ap.add_argument("--scale", type=float, default=1.0, help="workload scale (testing)")
    ap.add_argument("--builds", default="all",
                    help="comma list of builds to run, e.g. 'H:8,H*:2' (profiling)")
    ap.add_argument("--mode", choices=["headline", "batch", "serve", "core", "sweep", "ablation",
                                       "post", "table", "atomics"],
                    default="headline",
                    help="headline: the Chung-Lu build (default); batch: many hypergraphs "
                         "in one captured pipeline vs sequential builds; serve: Poisson "
                         "query stream; core: planted dense core with and without the "
                         "tensor-core tile path")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-max", type=int, default=200_000)
    ap.add_argument("--queries", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--core-scale", type=float, default=1.0)
    ap.add_argument("--ablation-scale", type=float, default=0.25)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(units: float, ms: float, world: int, device=None):
    """Whole-job units (sum over ranks) and the slowest rank's time (max)."""
    if world == 1:
        return units, ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    m = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(t.item()), float(m.item())


def make_workload(rank: int, scale: float):
    import hypergen
    c = dict(hypergen.CONFIGS[WORKLOAD])
    c.pop("kind")
    c["seed"] = c["seed"] + rank
    if scale != 1.0:
        c["m"] = int(c["m"] * scale)
        c["n"] = int(c["n"] * scale)
    return hypergen.chung_lu(name=WORKLOAD, **c)


_ONLY = None


def jobs():
    all_jobs = [(dual, s) for dual in SIDES for s in S_VALUES]
    if _ONLY is None:
        return all_jobs
    return [j for j in all_jobs if j in _ONLY]


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", self.gpu_id], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
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
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- roofline --

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def walk_bytes(st, b):
    """Algorithmic bytes of the bin-b walk kernel in one build: per row its
    list entry, CSR offsets, count and staging offset (24 B); per incidence
    its tail bounds (8 B); per wedge the far end's id (4 B); per pair its
    staged (j, w) (8 B)."""
    return (24 * st["rows_bin"][b] + 8 * st["incid_bin"][b] + 4 * st["wedges_bin"][b]
            + 8 * st["pairs_bin"][b])


# kernels of slg_graph_create: two validation passes, the CSR->CSC map, the
# status copy and the dual map's inversion
GRAPH_CREATE_LAUNCHES = 5

WALK_KERNELS = ["k_walk_warp", "k_walk_cta<256,2048>", "k_walk_cta<256,8192>",
                "k_walk_giant", "k_walk_sparse"]
NBINS = len(WALK_KERNELS)


def recorded_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if
    it was taken on the current walk source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = os.path.join(ROOT, "paper_2010_11448_gb300", "csrc", "slg_walk.cu")
    if not os.path.exists(path):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for ln in open(path):
        kv = dict(x.split("=", 1) for x in ln.split() if "=" in x)
        if kv.get("kernel") == kernel and kv.get("src_sha") == sha and \
                kv.get("workload") == WORKLOAD:
            return float(kv["bytes_per_launch"])
    return None


# ---------------------------------------------------------------- CPU leg --

def cpu_oracle_full(h, reps: int):
    """The oracle as it stands, all host cores, on one whole build of the
    step (L_8(H): every row, no sampling, no scaling); returns (wedges/s of
    the fastest rep, seconds per rep, cores, wedges, sample text)."""
    import oracle
    cores = os.cpu_count() or 1
    dual, s = CPU_FULL_BUILD
    m, n, off, idx = oracle.side(h, dual)
    W = oracle.wedges(m, n, off, idx, s)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.line_graph(m, n, off, idx, s, threads=cores)
        times.append(time.perf_counter() - t0)
    sample = (f"one whole build of the step, L_{s}({'H*' if dual else 'H'}) ({W} wedges, every "
              f"row), timed in full; fastest of {reps}")
    return W / min(times), times, cores, W, sample


def cpu_oracle_rate(h, stride: int):
    """The oracle as it stands, all host cores, every `stride`-th row of each
    of the four builds; returns (wedges/s, seconds, cores, sample text).  A
    context figure only: the fixed per-call work (the oracle's own transpose)
    is scaled with the sampled rows."""
    import numpy as np

    import oracle
    cores = os.cpu_count() or 1
    total_w = 0
    total_t = 0.0
    for dual, s in jobs():
        m, n, off, idx = oracle.side(h, dual)
        rows = np.arange(0, m, stride, dtype=np.int32)
        t0 = time.perf_counter()
        oracle.line_graph(m, n, off, idx, s, rows=rows, threads=cores)
        total_t += (time.perf_counter() - t0) * stride   # extrapolated to all rows
        total_w += oracle.wedges(m, n, off, idx, s)
    sample = (f"every {stride}th row of each of the 4 builds (s=2,8 on H and H*); time "
              f"scaled by {stride} to the full build")
    return total_w / total_t, total_t / stride, cores, sample


def gpu_local_cpus(dev):
    """Host CPUs attached to the GPU's NUMA node (from sysfs), or None."""
    try:
        import torch
        p = torch.cuda.get_device_properties(dev)
        bus = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        base = f"/sys/bus/pci/devices/{bus}"
        node = int(open(os.path.join(base, "numa_node")).read().strip())
        path = (f"/sys/devices/system/node/node{node}/cpulist" if node >= 0
                else os.path.join(base, "local_cpulist"))
        cpus = set()
        for part in open(path).read().strip().split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        return cpus or None
    except Exception:
        return None


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, all host cores.  A
    step is one whole build of the benchmark's step, L_8(H), every row (a
    bounded sample of the four-build step; nothing is scaled)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    h = make_workload(0, args.scale)
    dual, s = CPU_FULL_BUILD
    m, n, off, idx = oracle.side(h, dual)
    W = oracle.wedges(m, n, off, idx, s)
    cores = os.cpu_count() or 1

    def step():
        oracle.line_graph(m, n, off, idx, s, threads=cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    step_s = dt / args.steps
    value = W / step_s
    sample = (f"each step is one whole build of the step's four, L_{s}({'H*' if dual else 'H'}) "
              f"({W} wedges, every row, nothing scaled)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "int32", "data": "synthetic",
           "config": {"workload": WORKLOAD_TEXT, "m": h.m, "n": h.n, "nnz": h.nnz,
                      "s": list(S_VALUES), "sides": ["H", "H*"],
                      "reference_step": f"L_{s}({'H*' if dual else 'H'}) in full"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# --------------------------------------------------------------- GPU leg --

def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import oracle
    import paper_2010_11448_gb300 as slg
    from paper_2010_11448_gb300 import build_lib
    build_lib.build()
    slg.load()

    h = make_workload(rank, args.scale)
    dh = slg.to_device(h, dev)
    algo = args.algo
    rl = None if args.relabel == "none" else args.relabel
    J = jobs()
    caps, wedges = {}, {}
    for dual, s in J:
        caps[(dual, s)] = slg.count(dh, s, dual, algo=algo)
        wedges[(dual, s)] = slg.wedges(dh, s, dual)
    outs = {k: slg._outputs(caps[k], False, dev) for k in J}
    W_step = sum(wedges.values())
    P_step = sum(caps.values())

    stats_acc = {"launches": 0, "ms_walk": [0.0] * NBINS, "bytes_walk": [0.0] * NBINS,
                 "launch_walk": [0] * NBINS, "ms_other": 0.0}

    # one step validates the input and maps its incidences once (an slg_graph
    # handle made and released inside the step) and runs the four builds
    # through it; relabelled builds map their renumbered side themselves
    use_handle = not args.no_handle and rl is None and algo != "spgemm"

    def step(record):
        g = slg.Graph(dh) if use_handle else None
        if g is not None and record:
            stats_acc["launches"] += GRAPH_CREATE_LAUNCHES
        for dual, s in J:
            if g is not None:
                g.build(s, dual=dual, algo=algo, out=outs[(dual, s)])
            else:
                slg.build(dh, s, dual=dual, algo=algo, out=outs[(dual, s)], relabel=rl)
            if record:
                st = slg.last_stats()
                stats_acc["launches"] += st["kernel_launches"]
                if st["profiled"]:
                    for b in range(NBINS):
                        stats_acc["ms_walk"][b] += st["ms_walk"][b]
                        stats_acc["bytes_walk"][b] += walk_bytes(st, b)
                        stats_acc["launch_walk"][b] += 1
                    stats_acc["ms_other"] += (st["ms_plan"] + st["ms_scan"] + st["ms_gather"] +
                                              st["ms_relabel"] + st["ms_order"])
        if g is not None:
            g.close()

    for _ in range(max(args.warmup, 0)):
        step(False)
    slg.set_profiling(True)
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_id) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step(True)
        e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    slg.set_profiling(False)
    ms = e0.elapsed_time(e1)
    units, ms_max = aggregate(W_step * args.steps, ms, world, dev)
    value = units / (ms_max / 1e3)

    # roofline of the dominant kernel (largest share of walk time)
    b = int(np.argmax(stats_acc["ms_walk"]))
    n_l = max(stats_acc["launch_walk"][b], 1)
    t_l = stats_acc["ms_walk"][b] / n_l / 1e3
    bytes_l = stats_acc["bytes_walk"][b] / n_l
    peak, peak_kind = peaks()
    achieved = bytes_l / t_l / 1e9 if t_l > 0 else 0.0
    roofline = {"bound": "hbm", "kernel": WALK_KERNELS[b], "achieved": achieved,
                "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_kind, "traffic": recorded_traffic(WALK_KERNELS[b]),
                "algorithmic_bytes_per_launch": bytes_l, "ms_per_launch": t_l * 1e3,
                "walk_ms_share": {WALK_KERNELS[i]: stats_acc["ms_walk"][i] / max(ms, 1e-9)
                                  for i in range(NBINS)}}

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
              "dtype": "int32", "data": "synthetic",
              "config": {"workload": WORKLOAD_TEXT, "m": h.m, "n": h.n, "nnz": h.nnz,
                         "s": list(S_VALUES), "sides": ["H", "H*"], "algo": algo,
                         "relabel": args.relabel,
                         "wedges_per_step": W_step, "pairs_per_step": P_step,
                         "l2": "inputs (CSR+CSC 168 MB) larger than the 129 MB L2; no flush",
                         "parallelism": f"independent instance per rank x{world}",
                         "input_checks": ("validated and mapped once per step (slg_graph "
                                          "handle), shared by its four builds" if use_handle
                                          else "validated and mapped by every build")},
              "build_ms": None, "roofline": roofline, "clocks": clk.summary(),
              "gpu_launches": stats_acc["launches"]}

    # per-build ms (one more profiled pass, untimed)
    per = {}
    for dual, s in J:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        slg.build(dh, s, dual=dual, algo=algo, out=outs[(dual, s)], relabel=rl)
        per[f"{'H*' if dual else 'H'} s={s}"] = (time.perf_counter() - t0) * 1e3
    result["build_ms"] = per

    # the same builds with the plain per-hyperedge kernel and the filtered
    # SpGEMM (one run each, outside the timed region; outputs compared)
    if algo == "binned" and not args.no_compare:
        comp = {}
        for other in ("plain", "spgemm"):
            ms_o, same = {}, True
            for dual, s in J:
                o2 = slg._outputs(caps[(dual, s)], False, dev)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r2 = slg.build(dh, s, dual=dual, algo=other, out=o2)
                torch.cuda.synchronize()
                ms_o[f"{'H*' if dual else 'H'} s={s}"] = (time.perf_counter() - t0) * 1e3
                r1 = slg.build(dh, s, dual=dual, out=outs[(dual, s)])
                same = same and all(torch.equal(a, b) for a, b in zip(r1, r2))
                del o2, r2
            comp[other] = {"build_ms": ms_o, "identical": same,
                           "step_ms": sum(ms_o.values()),
                           "binned_speedup": sum(ms_o.values()) / sum(per.values())}
        result["comparison"] = comp

    # end to end through the C ABI with host buffers (pinned): one
    # slg_build_host_many call per step copies the hypergraph in once, builds
    # the four line graphs and returns each in compressed row form (row_ptr,
    # j, w), the copy back of one build overlapping the next build; the host
    # side is allocated and driven from the CPUs local to the GPU when the
    # system says which
    if not args.no_e2e:
        host_cpus = gpu_local_cpus(dev)
        saved_affinity = os.sched_getaffinity(0) if host_cpus else None
        if host_cpus:
            os.sched_setaffinity(0, host_cpus)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).pin_memory()

        class HostH:
            pass
        hh = HostH()
        hh.m, hh.n = h.m, h.n
        hh.e_off, hh.e_idx, hh.v_off, hh.v_idx = (pin(h.e_off), pin(h.e_idx), pin(h.v_off),
                                                  pin(h.v_idx))
        # the largest outputs first, so that their copies overlap later builds
        order = sorted(J, key=lambda k: -caps[k])

        def queries(csr):
            # the row form also takes the weights as uint16 (exact: the library
            # fails the query if a weight is above 65,535)
            qs = []
            for dual, s in order:
                cap = caps[(dual, s)]
                q = {"s": s, "dual": dual, "algo": algo, "capacity": cap, "w16": csr,
                     "out_j": torch.empty(cap, dtype=torch.int32).pin_memory(),
                     "out_w": torch.empty(cap, dtype=torch.int16 if csr else torch.int32
                                          ).pin_memory()}
                if csr:
                    q["row_ptr"] = torch.empty((h.n if dual else h.m) + 1,
                                               dtype=torch.int64).pin_memory()
                else:
                    q["out_i"] = torch.empty(cap, dtype=torch.int32).pin_memory()
                qs.append(q)
            return qs

        def e2e_rate(qs):
            res = slg.build_host_many(hh, qs)  # warm
            assert all(st == 0 for st, _ in res), res
            torch.cuda.synchronize()
            k2 = max(1, min(args.steps, 3))
            t0 = time.perf_counter()
            bad = []
            for _ in range(k2):
                bad += [r for r in slg.build_host_many(hh, qs) if r[0] != 0]
            torch.cuda.synchronize()
            assert not bad, bad
            dt = (time.perf_counter() - t0) * 1e3
            u2, dt_max = aggregate(W_step * k2, dt, world, dev)
            return u2 / (dt_max / 1e3), k2, dt / k2

        qs = queries(True)
        v_csr, k2, ms_csr = e2e_rate(qs)
        d2h_csr = sum(8 * (q["row_ptr"].shape[0]) + 6 * q["capacity"] for q in qs)
        del qs
        qs = queries(False)
        v_tri, _, ms_tri = e2e_rate(qs)
        # context for the host leg: the plain device-to-host copy rate into
        # the same page-locked arrays
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for q, (dual, s) in zip(qs, order):
            for a, b in zip((q["out_i"], q["out_j"], q["out_w"]), outs[(dual, s)]):
                a.copy_(b, non_blocking=True)
        torch.cuda.synchronize()
        d2h_gbs = 12 * P_step / (time.perf_counter() - t0) / 1e9
        in_bytes = 4 * (h.m + 1 + h.n + 1 + 2 * h.nnz)
        result["e2e"] = {"value": v_csr, "unit": UNIT,
                         "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": d2h_csr,
                         "steps": k2, "ms_per_step": ms_csr,
                         "api": "slg_build_host_many: one upload per step, four builds, each "
                                "copied back in compressed row form (int64 row_ptr, int32 j, "
                                "uint16 w: SLG_W16) while the next one builds",
                         "triples": {"value": v_tri, "ms_per_step": ms_tri,
                                     "d2h_bytes_per_step": 12 * P_step},
                         "d2h_copy_gbs": d2h_gbs,
                         "host_cpus": (f"{min(host_cpus)}-{max(host_cpus)}" if host_cpus
                                       else "any")}
        if saved_affinity:
            os.sched_setaffinity(0, saved_affinity)
        del qs, hh

    # the metric's batched and tiled arms (untimed by the step clock; each
    # compared with its sequential / walk-only counterpart on this GPU)
    if not args.no_extras:
        del outs
        torch.cuda.empty_cache()
        result["tiled"] = core_comparison(torch, slg, 1.0, (2, 8))
        result["tiled"]["workload"] = ("web-shaped hypergraph |E|=4M, |V|=10M, lognormal(2,1.5) "
                                       "sizes capped 1e5, planted core 4096 x 8192 at 0.3")
        result["tile_kernel"] = tile_roofline(torch, slg)
        result["batched"] = batch_comparison(torch, slg, 512, 200_000, 5, 2)
        result["batched"]["workload"] = ("512 Chung-Lu hypergraphs, |E| log-uniform 1k-200k, "
                                         "|V| = 2|E|, own s ~ U{2..32}; one captured launch")

    if rank == 0 and not args.no_cpu:
        oracle.build()
        rate, times, cores, w_full, sample = cpu_oracle_full(h, CPU_FULL_REPS)
        srate, ssecs, _, ssample = cpu_oracle_rate(h, CPU_SAMPLE_STRIDE)
        result["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores,
                                  "kind": "oracle", "sample": sample,
                                  "seconds": times,
                                  "sampled_all_builds": {"value": srate, "sample": ssample,
                                                         "seconds": ssecs}}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# --------------------------------------------------------------- other modes --

def _setup_gpu():
    import torch
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    import paper_2010_11448_gb300 as slg
    from paper_2010_11448_gb300 import build_lib
    build_lib.build()
    slg.load()
    return torch, slg


def batch_comparison(torch, slg, count: int, max_m: int, steps: int, warmup: int):
    """Batched form: `count` Chung-Lu hypergraphs (m log-uniform in
    [1e3, max_m], n = 2m), each with its own s ~ U{2..32}, built by one
    captured pipeline (one CUDA-graph launch for the whole union) vs the same
    builds one call at a time (binned, and the plain per-hyperedge kernel);
    the batched lists equal the sequential ones member by member."""
    import hypergen
    t0 = time.perf_counter()
    members = hypergen.batch(count, seed=100, m_lo=1000, m_hi=max_m,
                             workers=min(16, os.cpu_count() or 1))
    gen_s = time.perf_counter() - t0
    dhs = [slg.to_device(h) for h, _ in members]
    ss = [s for _, s in members]
    W = sum(slg.wedges(d, s) for d, s in zip(dhs, ss))
    t0 = time.perf_counter()
    plan = slg.Plan(dhs, ss)
    plan_s = time.perf_counter() - t0
    info = plan.info()
    st = torch.cuda.current_stream()
    for _ in range(max(warmup, 1)):
        plan.execute()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        plan.execute()
    e1.record(st)
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1) / steps
    res = plan.results()
    pairs = sum(int(r[0].shape[0]) for r in res)
    caps = [slg.count(d, s) for d, s in zip(dhs, ss)]
    outs = [slg.alloc_outputs(c) for c in caps]
    seq = {}
    for algo in ("binned", "plain"):
        slg.build(dhs[0], ss[0], algo=algo, out=outs[0])  # warm
        torch.cuda.synchronize()
        t = time.perf_counter()
        for d, s, o in zip(dhs, ss, outs):
            slg.build(d, s, algo=algo, out=o)
        torch.cuda.synchronize()
        seq[algo] = (time.perf_counter() - t) * 1e3
    same = all(torch.equal(r[1], o[1][:c]) and torch.equal(r[2], o[2][:c])
               for r, o, c in zip(res, outs, caps))
    out = {"members": len(dhs), "incidences": int(sum(d.nnz for d in dhs)),
           "union_rows": int(sum(d.m for d in dhs)), "wedges": int(W), "pairs": pairs,
           "batched_ms": batched_ms, "batched_wedges_per_s": W / (batched_ms / 1e3),
           "sequential_binned_ms": seq["binned"], "sequential_plain_ms": seq["plain"],
           "speedup_vs_plain": seq["plain"] / batched_ms,
           "speedup_vs_sequential_binned": seq["binned"] / batched_ms,
           "bit_identical_to_sequential": bool(same), "plans": 1,
           "autotuned": dict(zip(["warp", "cta_small", "cta_large", "sparse_max", "sparse_min",
                                  "dense_ratio"], info["bins"])),
           "kernels_per_launch": info["launches"], "plan_s": plan_s, "generate_s": gen_s,
           "steps": steps}
    del plan, res, outs, dhs
    torch.cuda.empty_cache()
    return out


def run_batch(args):
    """--mode batch: the batched-form comparison alone."""
    torch, slg = _setup_gpu()
    out = {"mode": "batch", "metric": "batched L_s build: one captured launch vs sequential"}
    out.update(batch_comparison(torch, slg, args.batch_count, args.batch_max, args.steps,
                                args.warmup))
    print(json.dumps(out), flush=True)
    return 0


def run_serve(args):
    """Serving form: a resident pool of 16 Chung-Lu hypergraphs (the headline
    recipe scaled 0.05x-1x, geometric), a Poisson stream of queries (graph
    U{0..15}, s U{1..64}, side Bernoulli(0.5)) at `rate` per second."""
    import numpy as np
    # lists of very different sizes come and go: let torch's allocator grow
    # and shrink its segments instead of keeping fragments
    os.environ.setdefault("PYTORCH_ALLOC_CONF", "expandable_segments:True")
    torch, slg = _setup_gpu()
    import hypergen
    from paper_2010_11448_gb300.serve import Server
    scales = np.geomspace(0.05, 1.0, 16)
    c = dict(hypergen.CONFIGS[WORKLOAD])
    graphs = [hypergen.chung_lu(int(c["m"] * sc), int(c["n"] * sc), seed=200 + k)
              for k, sc in enumerate(scales)]
    dhs = [slg.to_device(h) for h in graphs]
    rng = np.random.default_rng(5)
    n = args.queries
    gaps = rng.exponential(1.0 / args.rate, size=n)
    qs_spec = [(int(rng.integers(0, 16)), int(rng.integers(1, 65)), bool(rng.integers(0, 2)))
               for _ in range(n)]
    runs = {}
    for name, reuse, warm in (("walk_every_query", False, False), ("base_lists", True, False),
                              ("base_lists_warm", True, True)):
        srv = Server(dhs, slots=4, memory_budget=96 << 30, reuse=reuse, cache_bytes=48 << 30,
                     base_s=2, max_result_bytes=48 << 30)
        warm_s = srv.warm() if warm else 0.0
        t0 = time.perf_counter()
        due = t0
        queries = []
        for gap, spec in zip(gaps, qs_spec):
            due += gap
            now = time.perf_counter()
            if due > now:
                time.sleep(due - now)
            queries.append(srv.submit(*spec))
        for q in queries:
            if not q.wait(900):
                raise RuntimeError(f"serving: query {q.gid}/{q.s}/{q.dual} did not complete")
        wall = time.perf_counter() - t0
        srv.close()
        slg.release_memory()
        runs[name] = Server.summary(queries, wall)
        if warm:
            runs[name]["warm_s"] = warm_s
        del srv, queries
        torch.cuda.empty_cache()
    torch.cuda.empty_cache()
    # the same queries one at a time through the plain kernel (first 40)
    k = min(40, n)
    lat = []
    for gid, s, dual in qs_spec[:k]:
        torch.cuda.synchronize()
        t = time.perf_counter()
        slg.build(dhs[gid], s, dual=dual, algo="plain")
        torch.cuda.synchronize()
        lat.append((time.perf_counter() - t) * 1e3)
    lat = np.array(lat)
    out = {"mode": "serve", "metric": "s-line-graph queries: latency and throughput",
           "rate_per_s": args.rate, "slots": 4, **runs,
           "plain_one_at_a_time": {"queries": k, "p50_ms": float(np.percentile(lat, 50)),
                                   "p99_ms": float(np.percentile(lat, 99)),
                                   "queries_per_s": k / (lat.sum() / 1e3)}}
    print(json.dumps(out), flush=True)
    return 0


def fp8_peak_tflops(torch):
    """Dense FP8 (e4m3) tensor throughput of this GPU, measured with
    torch._scaled_mm (cuBLASLt) on 8192^3, best of 10 (burst).  Falls back to
    twice the measured bf16 peak (the nominal FP8 / BF16 ratio)."""
    try:
        M = N = K = 8192
        a = torch.randn(M, K, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(N, K, device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.ones((), device="cuda")

        def f():
            return torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        for _ in range(3):
            f()
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            f()
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        del a, b
        return 2.0 * M * N * K / (best / 1e3) / 1e12, \
            "measured: torch._scaled_mm fp8 e4m3 8192^3 (cuBLASLt), best of 10"
    except Exception as exc:  # noqa: BLE001
        p = os.path.join(ROOT, "MEASURED_PEAKS.json")
        bf16 = json.load(open(p))["bf16_tflops"] if os.path.exists(p) else 1900.0
        return 2.0 * bf16, f"bf16 peak x 2 (nominal fp8/bf16); _scaled_mm failed: {exc}"


def tile_roofline(torch, slg, rows: int = 4096, cols: int = 8192, density: float = 0.3):
    """The tensor-core tile kernel alone on the planted core's shape (rows x
    cols 0/1 at `density`, FP8 0x38 = 1): CUDA-event ms (best of 5), FLOP/s of
    the upper-triangle tiles it computes, against the FP8 peak; the counts
    are checked against an FP32 product (exact below 2^24)."""
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    A01 = (torch.rand(rows, cols, device="cuda", generator=g) < density)
    A = A01.to(torch.uint8) * 0x38
    slg.set_profiling(True)
    best = 1e30
    C = None
    for _ in range(6):
        C = slg.tile_overlap(A)
        best = min(best, slg.last_stats()["ms_tile"])
    slg.set_profiling(False)
    nt = rows // 128
    tasks = nt * (nt + 1) // 2
    flops = 2.0 * 128 * 128 * cols * tasks
    ref = (A01.float() @ A01.float().t()).to(torch.int32)
    upper = torch.triu(torch.ones(nt, nt, dtype=torch.bool, device="cuda")).repeat_interleave(
        128, 0).repeat_interleave(128, 1)
    exact = bool(torch.equal(C[upper], ref[upper]))
    peak, src = fp8_peak_tflops(torch)
    achieved = flops / (best / 1e3) / 1e12
    del A, A01, C, ref, upper
    torch.cuda.empty_cache()
    return {"kernel": "k_tile_overlap", "shape": [rows, cols], "density": density,
            "tiles": tasks, "ms": best, "bound": "tensor", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "peak_source": src,
            "flops": flops, "exact_vs_fp32_product": exact}


def core_comparison(torch, slg, scale: float = 1.0, s_list=(2, 8, 32)):
    """Dense core: the lognormal web-shaped hypergraph (4M x 10M, sizes
    lognormal(2, 1.5) capped 1e5) with a planted core of 4096 hyperedges x
    8192 vertices at density 0.3; builds on H and H* with and without the
    tensor-core tile path (identical output)."""
    import hypergen
    t0 = time.perf_counter()
    h = hypergen.lognormal_web(int(4_000_000 * scale), int(10_000_000 * scale), seed=2)
    gen_s = time.perf_counter() - t0
    dh = slg.to_device(h)
    rows = {}
    for dual in (False, True):
        for s in s_list:
            n = slg.count(dh, s, dual, tensor=True)
            o = slg.alloc_outputs(n)
            res = {}
            for tensor in (True, False):
                slg.build(dh, s, dual=dual, out=o, tensor=tensor)   # warm
                slg.set_profiling(True)
                torch.cuda.synchronize()
                t = time.perf_counter()
                i, j, w = slg.build(dh, s, dual=dual, out=o, tensor=tensor)
                torch.cuda.synchronize()
                ms = (time.perf_counter() - t) * 1e3
                slg.set_profiling(False)
                st = slg.last_stats()
                res["tile" if tensor else "walk"] = {"ms": ms, "wedges_walked": st["wedges"],
                                                     "core": [st["core_rows"], st["core_cols"]],
                                                     "tile_kernel_ms": st["ms_tile"]}
                if tensor:
                    ref = (i.clone(), j.clone(), w.clone())
                else:
                    res["identical"] = bool(torch.equal(ref[0], i) and torch.equal(ref[1], j)
                                            and torch.equal(ref[2], w))
            res["pairs"] = n
            res["speedup"] = res["walk"]["ms"] / res["tile"]["ms"]
            rows[f"{'H*' if dual else 'H'} s={s}"] = res
            del o, ref, i, j, w
    out = {"m": h.m, "n": h.n, "nnz": h.nnz, "generate_s": gen_s, "builds": rows}
    del dh
    torch.cuda.empty_cache()
    return out


def run_core(args):
    """--mode core: the dense-core comparison and the tile kernel's roofline."""
    torch, slg = _setup_gpu()
    out = {"mode": "core", "metric": "dense-core tile path vs wedge walk, build ms"}
    out.update(core_comparison(torch, slg, args.core_scale))
    out["tile_kernel"] = tile_roofline(torch, slg)
    print(json.dumps(out), flush=True)
    return 0


SWEEP_S = (2, 3, 4, 6, 8, 12, 16)


def run_sweep(args):
    """s-sweep on the headline workload: L_s for s in SWEEP_S on H and H*,
    from one walk at s = 2 plus filters (slg_build_sweep), against one
    independent build per threshold (same outputs, checked)."""
    torch, slg = _setup_gpu()
    h = make_workload(0, args.scale)
    dh = slg.to_device(h)
    rows = {}
    for dual in (False, True):
        caps = [slg.count(dh, s, dual) for s in SWEEP_S]
        outs = [slg.alloc_outputs(c) for c in caps]
        ind = [slg.alloc_outputs(c) for c in caps]

        def sweep():
            return slg.build_sweep(dh, SWEEP_S, dual=dual, outs=outs)

        def separate():
            return [slg.build(dh, s, dual=dual, out=o) for s, o in zip(SWEEP_S, ind)]
        res = {}
        for name, fn in (("sweep", sweep), ("separate", separate)):
            fn()
            best = None
            for _ in range(3):
                torch.cuda.synchronize()
                t = time.perf_counter()
                fn()
                torch.cuda.synchronize()
                ms = (time.perf_counter() - t) * 1e3
                best = ms if best is None or ms < best else best
            res[name + "_ms"] = best
        a, b = sweep(), separate()
        res["identical"] = all(torch.equal(x, y) for p, q in zip(a, b) for x, y in zip(p, q))
        res["pairs"] = dict(zip([str(s) for s in SWEEP_S], caps))
        res["speedup"] = res["separate_ms"] / res["sweep_ms"]
        rows["H*" if dual else "H"] = res
    print(json.dumps({"mode": "sweep", "metric": "L_s for s in " + str(list(SWEEP_S)) +
                      ": one walk + filters vs one build per s, ms",
                      "workload": WORKLOAD_TEXT, "sides": rows}), flush=True)
    return 0


ABLATION = [("f0 all heuristics", dict(unweighted=True)),
            ("f1 degree pruning", dict()),
            ("f2 visited skip only", dict(prune=False)),
            ("f3 short-circuit only", dict(prune=False, unweighted=True)),
            ("f4 none (filtered SpGEMM)", dict(algo="spgemm"))]


def run_ablation(args):
    """GPU analogue of the heuristic ablation of Section V (Table 3, Fig. 6):
    build ms and wedges walked per variant at s = 2, 4, 6, 8 on H and H* of the
    Chung-Lu workload scaled by --ablation-scale; every variant's pair list is
    checked against f1's."""
    torch, slg = _setup_gpu()
    h = make_workload(0, args.ablation_scale)
    dh = slg.to_device(h)
    rows = {}
    for dual in (False, True):
        for s in (2, 4, 6, 8):
            n = slg.count(dh, s, dual)
            ref = slg.build(dh, s, dual=dual)
            res = {}
            for name, kw in ABLATION:
                out = slg.alloc_outputs(n, unweighted=kw.get("unweighted", False))
                slg.build(dh, s, dual=dual, out=out, **kw)
                best = None
                for _ in range(2):
                    torch.cuda.synchronize()
                    t = time.perf_counter()
                    got = slg.build(dh, s, dual=dual, out=out, **kw)
                    torch.cuda.synchronize()
                    ms = (time.perf_counter() - t) * 1e3
                    best = ms if best is None or ms < best else best
                same = torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1]) and (
                    got[2] is None or torch.equal(got[2], ref[2]))
                res[name] = {"ms": best, "wedges": slg.last_stats()["wedges"], "same": same}
                del out, got
            rows[f"{'H*' if dual else 'H'} s={s}"] = res
            del ref
    print(json.dumps({"mode": "ablation", "metric": "build ms per heuristic variant",
                      "m": h.m, "n": h.n, "nnz": h.nnz, "scale": args.ablation_scale,
                      "builds": rows}), flush=True)
    return 0


def run_post(args):
    """After the edge list, on the headline workload: ID squeezing, the
    symmetric adjacency of the squeezed list and the s-connected components,
    for L_s at s = 2, 8 on H and H* (ms, best of 3)."""
    torch, slg = _setup_gpu()
    h = make_workload(0, args.scale)
    dh = slg.to_device(h)
    rows = {}

    def best(fn):
        b = None
        for _ in range(3):
            torch.cuda.synchronize()
            t = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t) * 1e3
            b = ms if b is None or ms < b else b
        return b, r
    for dual in (False, True):
        R = h.n if dual else h.m
        for s in (2, 8):
            i, j, w = slg.build(dh, s, dual=dual)
            t_sq, (si, sj, old) = best(lambda: slg.squeeze(i, j, R))
            V = int(old.shape[0])
            t_adj, _ = best(lambda: slg.adjacency(si, sj, w, V))
            t_cc, (lab, k) = best(lambda: slg.components(i, j, R))
            _, k2 = slg.components(si, sj, V)
            rows[f"{'H*' if dual else 'H'} s={s}"] = {
                "pairs": int(i.shape[0]), "ids": V, "components": k,
                "components_squeezed_agree": k == k2, "squeeze_ms": t_sq,
                "adjacency_ms": t_adj, "components_ms": t_cc}
            del i, j, w, si, sj, old, lab
    print(json.dumps({"mode": "post", "metric": "ID squeezing, adjacency, s-connected "
                      "components after the build, ms", "workload": WORKLOAD_TEXT,
                      "builds": rows}), flush=True)
    return 0


def run_table(args):
    """Per-config table: for the small config and the headline workload,
    each side and threshold (s = 1 of the headline workload streamed in row
    ranges of at most 4e8 pairs, checked against the closed form):
    sizes, W_s, pairs, ms of the binned build (and
    of the plain kernel and the filtered SpGEMM at s = 2, 8 on the headline
    workload), wedges/s, the walk's algorithmic GB/s, and a bit-exact check
    against the oracle (all rows of the small config; every 97th row plus
    the 64 largest of the headline workload)."""
    import numpy as np
    import hypergen
    import oracle
    torch, slg = _setup_gpu()
    peak, _ = peaks()
    out = {}

    def timed(fn, reps=3):
        if reps > 1:
            fn()
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t) * 1e3
            best = ms if best is None or ms < best else best
        return best, r

    for cname, svals, extra_s in (("uniform_2k", (1, 2, 3), ()),
                                  (WORKLOAD, (2, 4, 8, 16), (2, 8))):
        h = hypergen.config(cname) if cname != WORKLOAD else make_workload(0, 1.0)
        dh = slg.to_device(h)
        for dual in (False, True):
            if cname == WORKLOAD:  # L_1: billions of pairs, built in row ranges
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                P1 = slg.count(dh, 1, dual)
                count_ms = (time.perf_counter() - t0) * 1e3
                _, n1, _, idx1 = oracle.side(h, dual)
                d = np.bincount(idx1, minlength=n1).astype(np.int64)
                for _ in slg.build_stream(dh, 1, 400_000_000, dual=dual):
                    pass  # untimed warm-up pass
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                tp, tw, chunks = 0, 0, 0
                for _, _, i1, _, w1 in slg.build_stream(dh, 1, 400_000_000, dual=dual):
                    tp += int(i1.shape[0])
                    tw += int(w1.sum(dtype=torch.int64))
                    chunks += 1
                torch.cuda.synchronize()
                st_ms = (time.perf_counter() - t0) * 1e3
                out[f"{cname} {'H*' if dual else 'H'} s=1"] = {
                    "pairs": int(P1), "count_ms": count_ms, "streamed_ms": st_ms,
                    "chunks": chunks, "streamed_pairs_per_s": tp / (st_ms / 1e3),
                    "weights_equal_closed_form": tw == int((d * (d - 1) // 2).sum()),
                    "pairs_equal_count": tp == P1}
            m, n, off, idx = oracle.side(h, dual)
            sizes = np.diff(off)
            degs = np.bincount(idx, minlength=n)
            for sv in svals:
                P = slg.count(dh, sv, dual)
                o = slg.alloc_outputs(P)
                slg.set_profiling(True)
                ms, res = timed(lambda: slg.build(dh, sv, dual=dual, out=o))
                st = slg.last_stats()
                slg.set_profiling(False)
                W = st["wedges"]
                walk_ms = sum(st["ms_walk"])
                wbytes = sum(walk_bytes(st, b) for b in range(NBINS))
                if cname == "uniform_2k":
                    rows = None
                    sel = res
                else:
                    big = np.argsort(-sizes, kind="stable")[:64]
                    rows = np.unique(np.concatenate([np.arange(0, m, 97), big])).astype(np.int32)
                    keep = torch.isin(res[0], torch.from_numpy(rows).to(res[0].device))
                    sel = tuple(x[keep] for x in res)
                i, j, w = (x.cpu().numpy() for x in sel)
                want = oracle.canonical(*oracle.line_graph(m, n, off, idx, sv, rows=rows,
                                                           threads=os.cpu_count() or 1))
                got = np.stack([i, j, w], 1).astype(np.int64)
                row = {"nnz": int(h.nnz), "max_size": int(sizes.max()), "max_degree": int(degs.max()),
                       "W_s": int(W), "pairs": int(P), "binned_ms": ms,
                       "wedges_per_s": W / (ms / 1e3), "pairs_per_s": P / (ms / 1e3),
                       "walk_GBps_algorithmic": wbytes / (walk_ms / 1e3) / 1e9 if walk_ms else None,
                       "walk_frac_of_peak": (wbytes / (walk_ms / 1e3) / 1e9 / peak) if walk_ms else None,
                       "bit_exact": bool(np.array_equal(got, want)),
                       "checked_rows": "all" if rows is None else int(rows.size)}
                if sv in extra_s:
                    o2 = slg.alloc_outputs(P)
                    for algo in ("plain", "spgemm"):
                        ms_a, ra = timed(lambda: slg.build(dh, sv, dual=dual, algo=algo, out=o2),
                                         reps=1)
                        row[algo + "_ms"] = ms_a
                        row[algo + "_same"] = all(torch.equal(a, b) for a, b in zip(ra, res))
                        o2[0].fill_(-1)
                    del o2
                out[f"{cname} {'H*' if dual else 'H'} s={sv}"] = row
                del o, res
                torch.cuda.empty_cache()
    print(json.dumps({"mode": "table", "metric": "per-config build table", "peak_GBps": peak,
                      "rows": out}), flush=True)
    return 0


def run_atomics(args):
    """Shared-memory atomic throughput on random slots (the ceiling of the
    per-row hash tables): compiles csrc/micro/shared_atomics.cu with nvcc
    for sm_103a and runs it."""
    import tempfile
    from paper_2010_11448_gb300 import build_lib
    src = os.path.join(ROOT, "paper_2010_11448_gb300", "csrc", "micro", "shared_atomics.cu")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "shared_atomics")
        subprocess.run([build_lib.nvcc(), *build_lib.ARCH, "-O3", "-o", exe, src], check=True)
        r = subprocess.run([exe], check=True, capture_output=True, text=True)
    rows = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    clock_ghz, sms = 2.07, 152
    for x in rows:
        x["ops_per_s"] = x["ops_per_cycle_per_sm"] * sms * clock_ghz * 1e9
    print(json.dumps({"mode": "atomics", "metric": "shared-memory ops per SM cycle, random "
                      "slots of a 64 KB table", "rows": rows}), flush=True)
    return 0


def main():
    global _ONLY
    args = parse()
    if args.builds != "all":
        _ONLY = set()
        for tok in args.builds.split(","):
            side, sv = tok.split(":")
            _ONLY.add((side.strip() == "H*", int(sv)))
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "core":
        return run_core(args)
    if args.mode == "sweep":
        return run_sweep(args)
    if args.mode == "ablation":
        return run_ablation(args)
    if args.mode == "post":
        return run_post(args)
    if args.mode == "table":
        return run_table(args)
    if args.mode == "atomics":
        return run_atomics(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
