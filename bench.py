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


def kernel_source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2503_21937_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """dram bytes per launch for `kernel` from the committed ncu summary, or None
    when the summary was taken on different kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except Exception:
        return None
    if t.get("source_hash") != kernel_source_hash():
        return None
    k = t.get("kernels", {}).get(kernel)
    return None if k is None else k.get("dram_bytes_per_launch_full_size")


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


def cpu_oracle_sample(budget_s: float = 20.0):
    """Time the oracle on reduced instances of the same generators."""
    import oracle
    oracle.build()
    inputs = make_inputs(sg_nodes=2000, tc_nodes=600, tc_edges=3000)
    t0 = time.perf_counter()
    derived = 0
    reps = 0
    while True:
        for name, (prog, rels) in inputs.items():
            res = oracle.run(prog, {k: (v,) for k, v in rels.items()})
            head = "sg" if name == "sg" else "path"
            derived += res.relation(head).cols.shape[1]
        reps += 1
        if time.perf_counter() - t0 > budget_s / 2 or reps >= 5:
            break
    dt = time.perf_counter() - t0
    return {"value": derived / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} x (same generation on a 2,000-node random tree + transitive closure on a "
                      f"600-node/3,000-edge power-law graph), naive FP64 std::map oracle, single thread, "
                      f"{dt:.1f} s"}


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
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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


def batched_fwd_bwd(n_samples=512, loop_samples=32, reps=3):
    """Forward + backward (torch.autograd) samples/s of the batched workload in
    one engine launch, against the same API called once per sample."""
    import torch
    from paper_2503_21937_gb300.autograd import fixpoint
    B = W.batched_instance(n_samples)
    full = _batched_tensors(B)
    singles = [_batched_tensors(B, i) for i in range(loop_samples)]

    def fwd_bwd(inp, semiring):
        ins = {k: (v[0], v[1].clone().requires_grad_(True) if v[1] is not None else None, v[2]) for k, v in inp.items()}
        out = fixpoint(BATCH_PROGRAM, ins, semiring, outputs=["reach", "kin"])
        loss = out["reach"][1].sum() + out["kin"][1].sum()
        loss.backward()
        return out

    res = {}
    for semiring in ("diff_add_mult", "diff_max_min"):
        fwd_bwd(full, semiring)
        torch.cuda.synchronize()
        t = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fwd_bwd(full, semiring)
            torch.cuda.synchronize()
            t.append(time.perf_counter() - t0)
        batched = n_samples / min(t)
        fwd_bwd(singles[0], semiring)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in singles:
            fwd_bwd(s, semiring)
        torch.cuda.synchronize()
        loop = loop_samples / (time.perf_counter() - t0)
        res[semiring] = {"batched_samples_per_s": round(batched, 1), "per_sample_loop_samples_per_s": round(loop, 1),
                         "speedup": round(batched / loop, 1), "batched_ms": round(1e3 * min(t), 2)}
    return {"metric": "batched fwd+bwd samples/s vs per-sample (same GB300)", "samples": n_samples,
            "loop_sample_subset": loop_samples,
            "workload": "512 samples: grid reachability (side U{8..48}) + 20-relation kinship composition, f32 tags, "
                        "torch.autograd backward of sum(tags)", "results": res}


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
        roofline = {"kernel": name, "bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(ach / peak, 4), "peak_source": peak_kind,
                    "algorithmic_bytes_per_launch": per_launch_bytes, "traffic": ncu_traffic(name)}

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

    batched = None
    if not args.no_batched:
        batched = batched_fwd_bwd()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {**base_config(world), "derived_per_step": derived[0], "iterations": iters,
                           "join_outputs": cands, "engine_options": args.option},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "kernels": kernels, "kernels_by_workload": by_workload, "batched": batched}
        print(json.dumps(line))
    for e in engines.values():
        e.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
