#!/usr/bin/env python
"""Benchmark of the semi-naive fixpoint engine.

Workload (one "step" = every hot-path step, load + fixpoint, on both programs):
  * same generation on a seeded random tree of 50,000 nodes (branching U{1..4}):
        sg(x,y) :- parent(p,x), parent(p,y), x != y.
        sg(x,y) :- parent(a,x), sg(a,b), parent(b,y).
  * transitive closure on a seeded Chung-Lu power-law digraph (gamma 2.1) of
    20,000 nodes and 100,000 edges:
        path(x,y) :- edge(x,y).      path(x,z) :- path(x,y), edge(y,z).
  unit semiring, u32 ids; metric = derived tuples (|sg| + |path|) per second.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
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

from paper_2503_21937_gb300 import workloads as W  # noqa: E402

METRIC = "derived tuples/s (fixpoint)"
UNIT = "tuples/s"
WORKLOAD = "same-generation 50k-node random tree + transitive closure 20k-node/100k-edge power-law graph (unit semiring)"
SG_NODES, TC_NODES, TC_EDGES = 50_000, 20_000, 100_000


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash(unit: str = "pjoin.cu"):
    """Hash of the translation unit that holds the join emission kernels and
    of every local header it includes (recursively): the sources the ncu
    counters in profiles/ were taken on."""
    import re
    d = os.path.join(ROOT, "paper_2503_21937_gb300", "csrc")
    seen, todo = set(), [unit]
    while todo:
        f = todo.pop()
        if f in seen or not os.path.exists(os.path.join(d, f)):
            continue
        seen.add(f)
        with open(os.path.join(d, f)) as fh:
            todo += re.findall(r'#include "([^"]+)"', fh.read())
    h = hashlib.sha256()
    for f in sorted(seen):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, outputs_per_launch: float):
    """DRAM bytes per launch of `kernel` at the benchmark's size, from the
    committed ncu summary: DRAM bytes per join output measured on the small
    profile cases (one kernel, a few launches), times this workload's join
    outputs per launch.  None when the summary was taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except Exception:
        return None
    if t.get("source_hash") != kernel_source_hash():
        return None
    k = t.get("kernels", {}).get(kernel)
    if k is None or not outputs_per_launch:
        return None
    return k["dram_bytes_per_output"] * outputs_per_launch


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_inputs(sg_nodes=SG_NODES, tc_nodes=TC_NODES, tc_edges=TC_EDGES):
    parent, child, _ = W.random_tree(sg_nodes)
    s, d = W.chung_lu_power_law(tc_nodes, tc_edges)
    return {"sg": (W.SG_PROGRAM, {"parent": np.stack([parent, child])}),
            "tc": (W.TC_PROGRAM, {"edge": np.stack([s, d])})}


def cpu_info() -> dict:
    """Host cores and CPU model of the machine the CPU baselines run on."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware") and model is None:
                    model = line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


def cpu_oracle_sample():
    """The oracle (single thread) on the reduced instances of the benchmark's
    generators: same generation on a 5,000-node tree and transitive closure on a
    2,000-node / 10,000-edge power-law graph, one run each."""
    import oracle
    oracle.build()
    inputs = make_inputs(sg_nodes=5000, tc_nodes=2000, tc_edges=10000)
    t0 = time.perf_counter()
    derived = 0
    for name, (prog, rels) in inputs.items():
        res = oracle.run(prog, {k: (v,) for k, v in rels.items()})
        derived += res.relation("sg" if name == "sg" else "path").cols.shape[1]
    dt = time.perf_counter() - t0
    return {"value": derived / dt, "unit": UNIT, "cores": 1, "kind": "oracle", **cpu_info(),
            "sample": f"same generation on a 5,000-node random tree + transitive closure on a 2,000-node/10,000-edge "
                      f"power-law graph (reduced instances of the benchmark's generators), naive FP64 std::map oracle, "
                      f"single thread, {derived} derived tuples in {dt:.1f} s"}


def _bfs_count(args):
    """Reachable (source, target) pairs from a range of sources (one BFS each)."""
    lo, hi, s, d, n = args
    import numpy as np
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import breadth_first_order
    g = csr_matrix((np.ones(len(s)), (s, d)), shape=(n, n))
    gt = g.T.tocsr()
    tot = 0
    for src in range(lo, hi):
        order = breadth_first_order(g, src, directed=True, return_predecessors=False)
        tot += len(order) - 1
        preds = gt.indices[gt.indptr[src]:gt.indptr[src + 1]]
        if np.isin(preds, order).any():  # a cycle leads back to the source
            tot += 1
    return tot


def cpu_checkers(andersen: bool = False) -> dict:
    """Full-size textbook computations of the benchmark's relations on the host:
    the same-generation closed form (sum over tree levels of n_d (n_d - 1)), the
    transitive closure by one BFS per source on every host core, the oracle on
    the 1,000-node / 3,000-edge Erdos-Renyi closure, and (optionally, under a
    minute) Andersen points-to as a boolean sparse-matrix fixpoint."""
    import multiprocessing as mp
    import numpy as np
    out = {}
    parent, child, depth = W.random_tree(SG_NODES)
    t0 = time.perf_counter()
    counts = np.bincount(depth)
    n_sg = int(sum(int(c) * (int(c) - 1) for c in counts[1:]))
    dt = time.perf_counter() - t0
    out["sg_50k_closed_form"] = {"tuples": n_sg, "s": dt, "cores": 1}
    s, d = W.chung_lu_power_law(TC_NODES, TC_EDGES)
    cores = os.cpu_count() or 1
    step = (TC_NODES + 4 * cores - 1) // (4 * cores)
    jobs = [(lo, min(lo + step, TC_NODES), s, d, TC_NODES) for lo in range(0, TC_NODES, step)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        n_tc = sum(pool.map(_bfs_count, jobs))
    dt = time.perf_counter() - t0
    out["tc_20k_parallel_bfs"] = {"tuples": n_tc, "s": dt, "cores": cores, "tuples_per_s": n_tc / dt}
    import oracle
    oracle.build()
    a, b = W.erdos_renyi(1000, 3000)
    t0 = time.perf_counter()
    n_er = oracle.run(W.TC_PROGRAM, {"edge": ((a, b),)}).relation("path").cols.shape[1]
    dt = time.perf_counter() - t0
    out["er_tc_1k_oracle"] = {"tuples": n_er, "s": dt, "cores": 1, "tuples_per_s": n_er / dt}
    if andersen:
        sys.path.insert(0, ROOT)
        from tests import pins
        A = W.andersen_program(200_000, 1_000_000)
        t0 = time.perf_counter()
        n_pt = pins.andersen_sparse(A["addr"], A["assign"], A["load"], A["store"], 200_000).nnz
        dt = time.perf_counter() - t0
        out["andersen_200k_sparse_fixpoint"] = {"tuples": int(n_pt), "s": dt, "cores": 1, "tuples_per_s": n_pt / dt}
    return out


def side_leg(name: str, fn):
    """Run one of the secondary measurements (per-config lines, batched,
    pathfinder, CPU checkers).  They are taken after the headline; if one of
    them fails, the JSON line still carries the headline and reports the
    failure in that leg's place instead of being lost."""
    try:
        return fn()
    except Exception as exc:  # reported in the line, with the traceback on stderr
        import traceback
        traceback.print_exc(file=sys.stderr)
        return {"error": f"{name}: {type(exc).__name__}: {exc}"}


def max_over_ranks(ms: float, dist=None, device: str = "cuda") -> float:
    """The job's time: the slowest rank's (all_reduce MAX); `ms` itself when
    there is one process."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step: float, steps: int, world: int, job_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the job's time."""
    return units_per_rank_step * steps * world / (job_ms / 1000.0)


def base_config(world: int = 1) -> dict:
    """The workload description both arms report."""
    return {"workload": WORKLOAD, "sg_tree_nodes": SG_NODES, "tc_nodes": TC_NODES, "tc_edges": TC_EDGES,
            "semiring": "unit", "parallelism": "replicas" if world > 1 else "1 GPU",
            "l2": "flushed between timed steps (256 MiB write)"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    inputs = make_inputs(sg_nodes=1500, tc_nodes=500, tc_edges=2500)

    def step():
        n = 0
        for name, (prog, rels) in inputs.items():
            res = oracle.run(prog, {k: (v,) for k, v in rels.items()})
            n += res.relation("sg" if name == "sg" else "path").cols.shape[1]
        return n

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    tot = sum(step() for _ in range(args.steps))
    dt = time.perf_counter() - t0
    v = tot / dt
    sample = ("per step: same generation on a 1,500-node random tree + transitive closure on a 500-node/"
              "2,500-edge power-law graph (reduced instances of the benchmark's generators)")
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": base_config(),
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                                       **cpu_info()},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------------------
# batched differentiable reasoning: one launch for 512 samples vs a loop
# ---------------------------------------------------------------------------
BATCH_PROGRAM = W.REACH_PROGRAM + W.KIN_PROGRAM


def _batched_tensors(B, sel=None):
    """Device tensors of the batched instance, restricted to sample `sel`
    (ids kept) when given."""
    import torch

    def pick(sids):
        return np.ones(len(sids), bool) if sel is None else sids == sel

    e, st, f, c = B["edge"], B["start"], B["fact"], B["comp"]
    me, ms, mf, mc = pick(e[3]), pick(st[2]), pick(f[4]), pick(c[4])
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a).astype(np.int32)).cuda()
    F = lambda a: torch.from_numpy(np.ascontiguousarray(a).astype(np.float32)).cuda()
    return {"edge": (T(np.stack([e[0][me], e[1][me]])), F(e[2][me]), T(e[3][me])),
            "start": (T(st[0][ms][None, :]), None, T(st[2][ms])),
            "fact": (T(np.stack([f[0][mf], f[1][mf], f[2][mf]])), F(f[3][mf]), T(f[4][mf])),
            "comp": (T(np.stack([c[0][mc], c[1][mc], c[2][mc]])), None, T(c[4][mc]))}


def batched_fwd_bwd(n_samples=512, reps=3):
    """Forward + backward (torch.autograd) samples/s of the batched workload in
    one engine run, with the device-driven and the host-driven iteration loop,
    against the same API called once per sample for every sample.  Engines are
    reused across calls (the binding keeps idle engines per program and size
    class); the first call of each setting is an untimed warm-up."""
    import torch
    from paper_2503_21937_gb300.autograd import LAST_STATS, fixpoint
    B = W.batched_instance(n_samples)
    full = _batched_tensors(B)
    singles = [_batched_tensors(B, i) for i in range(n_samples)]

    def fwd_bwd(inp, semiring, options):
        ins = {k: (v[0], v[1].clone().requires_grad_(True) if v[1] is not None else None, v[2]) for k, v in inp.items()}
        out = fixpoint(BATCH_PROGRAM, ins, semiring, outputs=["reach", "kin"], options=options)
        stats = dict(LAST_STATS)
        loss = out["reach"][1].sum() + out["kin"][1].sum()
        loss.backward()
        return stats

    res = {}
    for semiring in ("diff_add_mult", "diff_max_min"):
        r = {}
        for name, opts in (("device_driven", {"driver": 1}), ("host_driven", {"driver": 0})):
            fwd_bwd(full, semiring, opts)
            torch.cuda.synchronize()
            t, st = [], None
            for _ in range(reps):
                t0 = time.perf_counter()
                st = fwd_bwd(full, semiring, opts)
                torch.cuda.synchronize()
                t.append(time.perf_counter() - t0)
            r[name] = {"samples_per_s": round(n_samples / min(t), 1), "ms": round(1e3 * min(t), 2),
                       "iterations": st["iterations"], "device_iterations": st["device_iterations"],
                       "graph_launches": st["graph_launches"], "host_syncs_per_run": st["host_syncs"],
                       "host_syncs_per_device_iteration": round(st["graph_launches"] / st["device_iterations"], 4)
                       if st["device_iterations"] else None}
        fwd_bwd(singles[0], semiring, {})
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for sgl in singles:
            fwd_bwd(sgl, semiring, {})
        torch.cuda.synchronize()
        loop = n_samples / (time.perf_counter() - t0)
        best = max(r.values(), key=lambda x: x["samples_per_s"])["samples_per_s"]
        res[semiring] = {**r, "per_sample_loop_samples_per_s": round(loop, 1),
                         "speedup_device_driven_vs_loop": round(r["device_driven"]["samples_per_s"] / loop, 1),
                         "speedup_best_vs_loop": round(best / loop, 1)}
    return {"metric": "batched fwd+bwd samples/s vs per-sample (same GB300)", "samples": n_samples,
            "per_sample_loop": f"all {n_samples} samples, one fixpoint + backward call each, engines reused",
            "workload": "512 samples: grid reachability (side U{8..48}) + 20-relation kinship composition, f32 tags, "
                        "torch.autograd backward of sum(tags)", "results": res}


# ---------------------------------------------------------------------------
# the other configurations: throughput lines (device time, median of 5 runs
# after a warm-up run on the same engine) with the dominant kernel's roofline
# ---------------------------------------------------------------------------
def _roofline(prof: dict, peak: float, peak_kind: str):
    # phases of the device-driven loop carry no bytes; kernels timed one by one do
    kern = {k: v for k, v in prof.items() if v["bytes"] > 0 and v["ms"] > 0}
    if not kern:
        return None
    name, v = max(kern.items(), key=lambda kv: kv[1]["ms"])
    ach = (v["bytes"] / v["launches"]) / (v["ms"] / v["launches"] / 1e3) / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(ach / peak, 4), "peak_source": peak_kind, "share": round(v["ms"] / sum(x["ms"] for x in kern.values()), 3)}


def config_legs(runs: int = 5) -> dict:
    import torch
    from paper_2503_21937_gb300 import Engine
    peak, peak_kind = load_peaks()
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a).astype(np.int32)).cuda()
    F = lambda a: torch.from_numpy(np.ascontiguousarray(a).astype(np.float32)).cuda()
    a, b = W.erdos_renyi(1000, 3000)
    g = W.grid_reach_instance(64)
    gs, gd, gp = g["edge"]
    A = W.andersen_program(200_000, 1_000_000)
    cases = {
        "er_tc_1k_3k_unit": (W.TC_PROGRAM, {"edge": (T(np.stack([a, b])), None)}, "unit", ["path"], None),
        "grid_64_diff_max_min_fwd_bwd": (W.REACH_PROGRAM, {"edge": (T(np.stack([gs, gd])), F(gp)),
                                                           "start": (T(np.zeros((1, 1))), None)},
                                         "diff_max_min", ["reach"], "edge"),
        "grid_64_diff_add_mult_fwd_bwd": (W.REACH_PROGRAM, {"edge": (T(np.stack([gs, gd])), F(gp)),
                                                            "start": (T(np.zeros((1, 1))), None)},
                                          "diff_add_mult", ["reach"], "edge"),
        "andersen_200k_1m_unit": (W.ANDERSEN_PROGRAM, {k: (T(np.stack([v[0], v[1]])), None) for k, v in A.items()},
                                  "unit", ["pt"], None),
    }
    out = {}
    for name, (prog, ins, sr, heads, grad_rel) in cases.items():
        e = Engine()
        e.program(prog)

        def one(profile=False, driver=1):
            e.reset()
            e.set_option("profile", 1 if profile else 0)
            e.set_option("driver", driver)
            for rel, (c, p) in ins.items():
                e.load(rel, c, p)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            st = e.run(sr)
            if grad_rel:
                n = e.size(heads[0])
                gin = {grad_rel: torch.zeros(ins[grad_rel][0].shape[1], device="cuda")}
                e.backward(heads[0], torch.ones(n, device="cuda"), gin)
            ev1.record()
            ev1.synchronize()
            return st, ev0.elapsed_time(ev1)

        one()
        times, st = [], None
        for _ in range(runs):
            st, ms = one()
            times.append(ms)
        ms = statistics.median(times)
        e.profile_reset()
        one(profile=True, driver=0)  # per-kernel timing on the host-driven loop
        prof = e.profile()
        e.close()
        out[name] = {"semiring": sr, "derived": st["derived"], "candidates": st["candidates"],
                     "iterations": st["iterations"], "device_iterations": st["device_iterations"],
                     "ms": round(ms, 3), "derived_tuples_per_s": st["derived"] / (ms / 1e3),
                     "candidate_tuples_per_s": st["candidates"] / (ms / 1e3),
                     "timed": "fixpoint + backward" if grad_rel else "fixpoint",
                     "roofline": _roofline(prof, peak, peak_kind)}
    return out


# ---------------------------------------------------------------------------
# small cases for ncu captures (a few GB on the device at most)
# ---------------------------------------------------------------------------
def parse_options(pairs):
    """--option KEY=VALUE strings as (key, int value) pairs."""
    out = []
    for kv in pairs:
        k, v = kv.split("=")
        out.append((k, int(v)))
    return out


def profile_case(name, options=()):
    import torch
    from paper_2503_21937_gb300 import Engine, build
    build.build()
    e = Engine()
    for k, v in options:
        e.set_option(k, v)
    if name == "sort_u32_2e26":  # one sort of 2^26 random 30-bit keys (4 LSD passes)
        keys = W.stream(7001).below(1 << 26, 1 << 30)
        k = torch.from_numpy(keys.view(np.int32)).cuda()
        e.prim_sort(k, None, key_bits=30)
        torch.cuda.synchronize()
        ok = bool(torch.all(k[1:].to(torch.int64) >= k[:-1].to(torch.int64)).item())
        print(json.dumps({"case": name, "n": 1 << 26, "sorted": ok}))
    elif name == "tc_8k":  # transitive closure of an 8,000-node / 40,000-edge power-law graph
        s, d = W.chung_lu_power_law(8000, 40000, seed_index=3)
        e.program(W.TC_PROGRAM)
        e.load("edge", torch.from_numpy(np.stack([s, d]).astype(np.int32)).cuda())
        print(json.dumps({"case": name, **e.run("unit")}))
    else:  # same generation on a 20,000-node random tree
        parent, child, _ = W.random_tree(20000, seed_index=2)
        e.program(W.SG_PROGRAM)
        e.load("parent", torch.from_numpy(np.stack([parent, child]).astype(np.int32)).cuda())
        print(json.dumps({"case": name, **e.run("unit")}))
    e.close()


# ---------------------------------------------------------------------------
# the engine arm
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=1, help="extra steps with per-kernel CUDA-event timing")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched fwd+bwd measurement")
    ap.add_argument("--no-configs", action="store_true", help="skip the per-configuration throughput lines")
    ap.add_argument("--no-pathfinder", action="store_true",
                    help="skip the end-to-end training-step sweep over Pathfinder grid sides")
    ap.add_argument("--cpu-andersen", action="store_true",
                    help="also time the full-size Andersen sparse-matrix checker on the host (about two minutes)")
    ap.add_argument("--option", action="append", default=[], metavar="KEY=VALUE",
                    help="engine option applied to every engine (repeatable)")
    ap.add_argument("--profile-case", choices=["sort_u32_2e26", "tc_8k", "sg_20k"],
                    help="run one small case once (for ncu captures) and exit")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args.profile_case, parse_options(args.option))
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    from paper_2503_21937_gb300 import Engine, build
    build.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    inputs = make_inputs()
    dev = {name: {k: torch.from_numpy(v.astype(np.int32)).cuda() for k, v in rels.items()}
           for name, (_, rels) in inputs.items()}
    engines = {}
    with torch.cuda.stream(stream):
        for name, (prog, rels) in inputs.items():
            e = Engine(stream=stream.cuda_stream)
            e.program(prog)
            for k, v in parse_options(args.option):
                e.set_option(k, v)
            engines[name] = e
    heads = {"sg": "sg", "tc": "path"}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")

    def step(profile=False):
        st_all = {}
        for name, e in engines.items():
            e.reset()
            e.set_option("profile", 1 if profile else 0)
            for rel, t in dev[name].items():
                e.load(rel, t)
            st_all[name] = e.run("unit")
        return st_all

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times, derived, launches, iters, cands = [], [], 0, {}, {}
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.fill_(1)  # L2 flush between timed steps (256 MiB write), outside the timed interval
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = step()
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
            derived.append(sum(s["derived"] for s in st.values()))
            launches += sum(s["kernel_launches"] for s in st.values())
            iters = {k: s["iterations"] for k, s in st.items()}
            cands = {k: s["candidates"] for k, s in st.items()}
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(times), dist)
    value = job_throughput(derived[0], args.steps, world, total_ms)

    # per-kernel CUDA-event timing on extra steps (not part of the timed value)
    prof = {}
    by_workload = {}
    with torch.cuda.stream(stream):
        for _ in range(args.profile_steps):
            step(profile=True)
    for wname, e in engines.items():
        by_workload[wname] = {k: round(v["ms"], 3) for k, v in sorted(e.profile().items(), key=lambda kv: -kv[1]["ms"])
                              if v["ms"] >= 0.05}
        for k, v in e.profile().items():
            p = prof.setdefault(k, {"launches": 0, "ms": 0.0, "bytes": 0.0})
            for f in p:
                p[f] += v[f]
        e.profile_reset()
        e.set_option("profile", 0)
    peak, peak_kind = load_peaks()
    tot_k = sum(v["ms"] for v in prof.values()) or 1.0
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 4), "share": round(v["ms"] / tot_k, 4),
                   "GBps": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] > 0 else None,
                   "frac": round(v["bytes"] / (v["ms"] / 1e3) / 1e9 / peak, 4) if v["ms"] > 0 else None}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"]) if prof else None
    roofline = None
    if dom:
        name, v = dom
        per_launch_bytes = v["bytes"] / v["launches"]
        per_launch_s = v["ms"] / v["launches"] / 1e3
        ach = per_launch_bytes / per_launch_s / 1e9
        outs = sum(cands.values()) / max(v["launches"], 1) if name == "join_emit" else 0
        traffic = ncu_traffic(name, outs)
        roofline = {"kernel": name, "bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(ach / peak, 4), "peak_source": peak_kind,
                    "algorithmic_bytes_per_launch": per_launch_bytes, "traffic": traffic,
                    # the same launch time against the DRAM bytes ncu measured (scaled from the small cases)
                    "traffic_frac": round(traffic / per_launch_s / 1e9 / peak, 4) if traffic else None}

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        host_in = {name: {k: torch.from_numpy(v.astype(np.int32)).pin_memory() for k, v in rels.items()}
                   for name, (_, rels) in inputs.items()}
        h2d = sum(t.numel() * 4 for rels in host_in.values() for t in rels.values())
        outs = {}
        d2h = 0
        e2e_ms = []
        with torch.cuda.stream(stream):
            for it in range(args.steps + 1):
                t0 = time.perf_counter()
                nbytes = 0
                for name, e in engines.items():
                    e.reset()
                    for rel, t in host_in[name].items():
                        e.load(rel, t.numpy().view(np.uint32))
                    e.run("unit")
                    h = heads[name]
                    n = e.size(h)
                    if h not in outs or outs[h].shape[1] < n:
                        outs[h] = torch.empty((2, n), dtype=torch.int32).pin_memory()
                    e.read_into(h, outs[h].numpy())
                    nbytes += n * 2 * 4
                dt = (time.perf_counter() - t0) * 1e3
                if it > 0:  # first pass allocates the pinned output buffers
                    e2e_ms.append(dt)
                d2h = nbytes
        e2e = {"value": derived[0] / (statistics.mean(e2e_ms) / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": statistics.mean(e2e_ms)}

    configs = None
    if not args.no_configs:
        configs = side_leg("configs", config_legs)
    batched = None
    if not args.no_batched:
        batched = side_leg("batched", batched_fwd_bwd)
    pathfinder = None
    if not args.no_pathfinder:
        def pathfinder_leg():
            from paper_2503_21937_gb300 import pathfinder as PF
            return {"metric": "training-step samples/s (CNN edge predictor -> batched differentiable fixpoint -> "
                              "BCE -> backward -> Adam), synthetic Pathfinder-like grids",
                    "by_side": PF.sweep(semiring="diff_max_min"),
                    "by_side_diff_top1_proofs": PF.sweep(semiring="diff_top1_proofs")}
        pathfinder = side_leg("pathfinder", pathfinder_leg)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample()
        cpu["checkers"] = side_leg("checkers", lambda: cpu_checkers(andersen=args.cpu_andersen))
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {**base_config(world), "derived_per_step": derived[0], "iterations": iters,
                           "join_outputs": cands, "engine_options": args.option},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "kernels": kernels, "kernels_by_workload": by_workload, "configs": configs,
                "batched": batched, "pathfinder": pathfinder}
        print(json.dumps(line))
    for e in engines.values():
        e.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
