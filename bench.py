"""Throughput of the multi-species TreePM step on GB300 (one JSON line).

A step is one kick-drift-kick step (Sec. 2.1.1) of the whole hot path:
kick, FP64 drift + wrap, Morton+type keys and radix sort, canonical octree,
per-species monopoles, PM long-range force (CIC, cuFFT, D x D kernels,
interpolation), the short-range group walk, kick. Steps replay a captured
CUDA graph through ng_step.

metric: particle-node interactions per second, where the interactions are
those of the per-particle Barnes-Hut walk (ng_count_interactions, the
algorithm's unit of work: one (accepted node, species with mass) term or
one body of an opened leaf) on the canonical tree with leaf size 8, counted
on the positions at the start and at the end of the timed region and
averaged. The timed walk may run on a tree with another leaf size (the
autotuner's choice); the count does not follow it.

e2e: the same metric through ng_step_host with pinned host buffers (the
copies in and out inside the timed region), run after the timed region on
the state the simulation has reached by then; its interactions are counted
the same way on the positions at the start and at the end of its own steps.

roofline: the dominant kernel is the walk, bound by the FP32 pipe; achieved
= 23 flop x per-particle-walk interactions on the walk's own tree / average
walk duration (CUDA events around ng_tree_force on the launching stream);
the same on the leaf-8 tree of the metric is given beside it; peak = SMs x
128 lanes x 2 flop x SM clock (the maximum clock; the same at the median
clock sampled during the run is given beside it).

hbm: per-stage milliseconds of one sort + tree + force evaluation
(ng_stage_times: CUDA events on the context's stream), the stage's
algorithmic bytes and their fraction of the measured copy bandwidth.

--impl reference: the FP64 CPU checker timed on the host cores for a
bounded sample of the same workload (per-particle tree walk of a random
sample of targets on the full tree).
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

FLOP_PER_INTERACTION = 23
DEFAULT_WORKLOAD = "clustered16m_d4_yukawa"
# The unit of work is counted on the canonical tree with this leaf size (the
# library's default), whatever leaf size the timed walk runs with: the count
# of the per-particle walk grows with the leaf size, the work to be done does not.
REF_LEAF = 8
# Walk shape (leaf size, group cell) of served requests: requests of 2^17
# bodies or more, whose walks fill the GPU and bound the saturated serving
# loop, take leaf 32 / cell 128 (their 10-step integrations, timed one at a
# time: 643 ms summed at leaf 8 / cell 32, 598 ms at 32 / 128); smaller ones
# keep the library default.
SERVE_LARGE_N = 1 << 17
SERVE_LARGE_SHAPE = (32, 128)
SERVE_SMALL_SHAPE = (8, 32)


def job_totals(units, ms, world):
    """Whole-job totals of a replicas run: the units every rank processed
    (summed) and the timed region of the slowest rank (maximum). Ranks run
    independent problems, so this is the only exchange; world == 1 returns the
    inputs. Works with any initialised process group (NCCL here, gloo in the
    tests), the tensors living on the group's device."""
    if world <= 1:
        return float(units), float(ms)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend() == "nccl" else torch.device("cpu")
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def walk_traffic(workload, n_override, leaf, cell):
    """DRAM bytes (read + write) of one walk launch, from the ncu capture recorded in
    profiles/ for this workload and walk configuration; None unless that capture was
    taken of the walk and tree sources as they are now (the SHA-256 of ng_walk.cu
    followed by ng_tree.cu is recorded beside it)."""
    import hashlib
    import re
    if workload != DEFAULT_WORKLOAD or n_override is not None:
        return None
    try:
        text = open(os.path.join(ROOT, "profiles", "k_walk_clustered16m_d4_yukawa_dram.md")).read()
        csrc = os.path.join(ROOT, "paper_1502_07442_gb300", "csrc")
        src = b"".join(open(os.path.join(csrc, f), "rb").read() for f in ("ng_walk.cu", "ng_tree.cu"))
    except OSError:
        return None
    sha = hashlib.sha256(src).hexdigest()
    for line in text.splitlines():
        m = re.search(r"traffic: leaf=(\d+) cell=(\d+) read=(\d+) write=(\d+) "
                      r"source_sha256=([0-9a-f]{64})", line)
        if m and int(m[1]) == leaf and int(m[2]) == cell and m[5] == sha:
            return int(m[3]) + int(m[4])
    return None


def measured_peaks():
    """Measured peaks of this GPU model (MEASURED_PEAKS.json beside this
    file), else a copy bandwidth measured earlier on the same model."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            m = json.load(fh)
        return float(m["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def stage_bytes(n, D, mesh, passes=8):
    """Algorithmic DRAM bytes of the memory-bound stages of one force
    evaluation (reads + writes of the arrays each stage must touch once):
    keys 24 B position + 1 B species read, 8 B key + 4 B index written; each
    radix pass (8 for a full sort, fewer when the step's tree stops at a level
    cap) 8 B key read by the histogram, 12 B key + index read and 12 B written
    by the scatter; type-major order 4 B index written,
    then one 32 B radix pass; deposit 33 B per body read plus the D mesh
    clears; FFTs and k-space one read and one write of the D real meshes or
    half spectra; interpolation 24 B position + 1 B species + 4 B index read,
    12 B acceleration written, and one read of the D potential meshes. The
    gather of a step (ng_step keeps the state in the previous step's sorted
    order) reads and writes 24 B position, 12 B velocity, 4 B mass, 1 B
    species, 4 B caller index and reads the 4 B permutation."""
    real = 4 * D * mesh ** 3
    spec = 8 * D * mesh * mesh * (mesh // 2 + 1)
    b = {"keys": 37 * n, "radix": passes * 32 * n, "gather": (2 * 45 + 4) * n, "type_order": 36 * n,
         "interp": 41 * n + real}
    if mesh > 0:
        b.update(deposit=33 * n + real, fft_fwd=real + spec, kspace=2 * spec, fft_inv=spec + real)
    return b


def hbm_block(times, n, D, mesh, passes=8):
    peak, src = measured_peaks()
    out = {"peak_gbs": peak, "peak_source": f"{src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
           "radix_passes": passes}
    for k, nbytes in stage_bytes(n, D, mesh, passes).items():
        ms = times.get(k, 0.0)
        if ms > 0:
            gbs = nbytes / (ms / 1e3) / 1e9
            out[k] = {"ms": round(ms, 4), "bytes": int(nbytes), "gbs": round(gbs, 1),
                      "frac": round(gbs / peak, 4)}
    for k in ("octree", "monopoles", "groups", "walk"):
        if times.get(k, 0.0) > 0:
            out[k] = {"ms": round(times[k], 4), "bound": "latency / FP64" if k != "walk" else "FP32"}
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--n", type=int, default=None, help="override N (smaller test runs)")
    ap.add_argument("--acc64", action="store_true",
                    help="the FP64-accumulated walk variant (per-body sums in FP64)")
    ap.add_argument("--species", type=int, default=None,
                    help="override the species count D (the paper's 1/D scaling)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-tune", action="store_true", help="skip the leaf/group autotuner")
    ap.add_argument("--leaf", type=int, default=None,
                    help="leaf size (with --cell: fixed walk configuration, no autotuning)")
    ap.add_argument("--cell", type=int, default=None, help="group cell size (with --leaf)")
    return ap.parse_args()


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()

    def summary(self):
        rows = []
        try:
            with open(self.f.name) as fh:
                for line in fh:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


ARM_PARTS = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1",
             "0xd49": "Arm Neoverse N2", "0xd8e": "Arm Neoverse N3", "0xd84": "Arm Neoverse V3"}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                v = line.split(":", 1)[1].strip()
                return ARM_PARTS.get(v.lower(), v)
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_leg(w, seconds, tag, threads=0):
    """The FP64 checker on host cores: per-particle walk of random targets on the
    full tree; rate = interactions / walk seconds (tree build timed apart)."""
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    prm = w["params"]
    op = oracle.make_params(prm["D"], prm["G"], box=prm["box"], eps=prm["eps"], rs=prm["rs"],
                            rcut=prm["rcut"], theta=prm["theta"], leaf_size=REF_LEAF,
                            pm_mesh=prm["pm_mesh"], law=prm["law"], ya=prm["ya"], yl=prm["yl"])
    default_threads = oracle.set_threads(0)
    cores = oracle.set_threads(threads)
    n = w["pos"].shape[1]
    rng = np.random.Generator(np.random.PCG64(4242))
    probe = rng.choice(n, size=min(n, 2000), replace=False)
    _, cnt, tb, tw = oracle.tree_walk_timed(op, w["pos"], w["type"], w["mass"], probe)
    rate = cnt.sum() / max(tw, 1e-9)
    per_target = tw / probe.size
    m = int(min(n, max(probe.size, seconds / max(per_target, 1e-9))))
    tgt = rng.choice(n, size=m, replace=False)
    _, cnt, tb2, tw2 = oracle.tree_walk_timed(op, w["pos"], w["type"], w["mass"], tgt)
    rate = cnt.sum() / tw2
    oracle.set_threads(default_threads)
    return {"value": float(rate), "unit": "interactions/s", "cores": int(cores), "kind": "oracle",
            "cpu": f"{cpu_model()} ({os.cpu_count()} logical cores)",
            "sample": f"{tag}: FP64 per-particle tree walk of {m} random targets of {n} bodies "
                      f"on the leaf-{REF_LEAF} tree (tree build {tb2:.1f} s timed apart, walk "
                      f"{tw2:.1f} s)"}, float(tw2)


def run_reference(args, w, ws, rank):
    if rank != 0:
        return
    vals = []
    info = None
    budget = max(3.0, 150.0 / max(1, args.steps + args.warmup))
    for s in range(args.warmup + args.steps):
        info, _ = cpu_leg(w, budget, "reference step")
        if s >= args.warmup:
            vals.append(info["value"])
    v = float(np.mean(vals))
    info["value"] = v
    print(json.dumps({
        "impl": "reference", "metric": "particle-node interactions/s", "value": v,
        "unit": "interactions/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w, args), "cpu_baseline": info,
        "e2e": {"value": v, "unit": "interactions/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def workload_config(w, args):
    prm = w["params"]
    return {"workload": w["name"], "n": int(w["pos"].shape[1]), "D": int(prm["D"]),
            "laws": "newton+yukawa" if int(np.max(prm["law"])) else "newton",
            "pm_mesh": int(prm["pm_mesh"]), "theta": float(prm["theta"]),
            "leaf_size": int(prm["leaf_size"]), "dt": float(w["dt"]),
            "step": "KDK: kick, drift, sort, octree, monopoles, PM, group walk, kick",
            "l2": "inputs larger than L2 (particle state and tree >> 129 MB, no flush)",
            "parallelism": f"replicas{args.gpus}",
            "accumulation": "fp64 per-body sums" if prm.get("accumulate_fp64") else "fp32"}


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.workload == "batch64":
        return bench_batch(args, ws, rank, local)
    if args.workload == "serve2000":
        return bench_serve(args, ws, rank, local)
    from paper_1502_07442_gb300 import inputs
    w = inputs.workload(args.workload, n=args.n, seed=None if rank == 0 else 1002 + 7919 * rank,
                        species=args.species)
    if args.impl == "reference":
        return run_reference(args, w, ws, rank)

    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1502_07442_gb300 import binding as ng

    dev = torch.device("cuda", local)
    n = int(w["pos"].shape[1])
    pos = torch.from_numpy(w["pos"]).to(dev)
    typ = torch.from_numpy(w["type"]).to(dev)
    mass = torch.from_numpy(w["mass"]).to(dev)
    vel = torch.from_numpy(w["vel"]).to(dev)
    acc = torch.zeros((3, n), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    tuned = None
    if args.leaf is not None and args.cell is not None:
        w["params"] = dict(w["params"], leaf_size=args.leaf, group_cell=args.cell)
        tuned = {"leaf_size": args.leaf, "group_cell": args.cell, "fixed": True}
    elif not args.no_tune:
        from paper_1502_07442_gb300 import autotune
        best, trials = autotune.tune(w["params"], pos, typ, mass, stream=stream)
        w["params"] = dict(w["params"], leaf_size=best["leaf_size"], group_cell=best["group_cell"])
        tuned = {"leaf_size": best["leaf_size"], "group_cell": best["group_cell"],
                 "trials": len(trials), "build_plus_walk_ms": round(best["ms"], 2)}
    if args.acc64:
        w["params"] = dict(w["params"], accumulate_fp64=1)
    sim = ng.Simulation(ng.params_from_workload(w["params"]), stream)
    dt = float(w["dt"])

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # warm-up: the first call computes the initial force and captures the step graph
    ng.ng_step(sim.ctx, pos, vel, typ, mass, acc, False, args.warmup, dt)
    ref = ng.Simulation(ng.params_from_workload(dict(w["params"], leaf_size=REF_LEAF)), stream)

    def algorithmic():
        # per-particle walk count on the reference tree of the current positions
        ng.ng_build_tree(ref.ctx, pos, typ, mass)
        return ng.ng_count_interactions(ref.ctx)

    count0 = algorithmic()
    l0 = ng.ng_launch_count(sim.ctx)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(stream)
        ng.ng_step(sim.ctx, pos, vel, typ, mass, acc, True, args.steps, dt)
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1)
    launches = ng.ng_launch_count(sim.ctx) - l0
    clocks = clk.summary()
    count1 = algorithmic()
    count_tuned_leaf = ng.ng_count_interactions(sim.ctx)
    count = 0.5 * (count0 + count1)
    # every rank integrates its own simulation: sum the units, take the slowest clock
    job_count, ms = job_totals(count, ms, ws)
    job_n, _ = job_totals(n, ms, ws)
    value = job_count * args.steps / (ms / 1e3)

    # dominant kernel: the walk alone, events on the launching stream
    walk_ms = []
    for _ in range(3):
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        ng.ng_tree_force(sim.ctx, acc)
        a1.record(stream)
        torch.cuda.synchronize()
        walk_ms.append(a0.elapsed_time(a1))
    executed = ng.ng_tree_force(sim.ctx, acc, count=True)
    walk = float(np.mean(walk_ms))
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = nsm * 128 * 2 * 2070e6 / 1e12
    achieved = FLOP_PER_INTERACTION * count1 / (walk / 1e3) / 1e12
    achieved_own = FLOP_PER_INTERACTION * count_tuned_leaf / (walk / 1e3) / 1e12
    med = clocks.get("sm_mhz") or 2070.0
    # per-stage times of one step as ng_step runs it (CUDA events on the
    # context's stream), best of three, for the HBM fractions
    best = {}
    for _ in range(3):
        t = ng.ng_stage_times(sim.ctx, pos, vel, typ, mass, acc, dt)
        best = {k: min(v, best.get(k, v)) for k, v in t.items()}
    hbm = hbm_block(best, n, int(w["params"]["D"]), int(w["params"]["pm_mesh"]),
                    ng.ng_sort_passes(sim.ctx))
    roofline = {"bound": "alu", "achieved": round(achieved_own, 3), "peak": round(peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved_own / peak, 4),
                "frac_basis": "23 flop x per-particle walk interactions on the walk's own tree "
                              "(the algorithmic count on the same tree)",
                "achieved_leaf8": round(achieved, 3),
                "frac_leaf8": round(achieved / peak, 4),
                "frac_leaf8_basis": f"23 flop x per-particle interactions on the leaf-{REF_LEAF} "
                                    "tree (the count of the metric's value)",
                "traffic": walk_traffic(args.workload,
                                        args.n if args.species is None and not args.acc64 else -1,
                                        int(w["params"]["leaf_size"]),
                                        int(w["params"].get("group_cell", 0) or 32)),
                "kernel": "k_walk", "walk_ms": round(walk, 3),
                "peak_at_median_clock": round(nsm * 128 * 2 * med * 1e6 / 1e12, 2),
                "frac_at_median_clock": round(achieved_own / (nsm * 128 * 2 * med * 1e6 / 1e12), 4),
                "executed_interactions": int(executed),
                # over-opening of the group walk: both counts on the walk's own tree
                "executed_over_algorithmic": round(executed / count_tuned_leaf, 3),
                "peak_source": "FP32 pipe: SMs x 128 x 2 flop x 2070 MHz (derived)"}

    # end to end through the public call with host buffers
    e2e = None
    if not args.no_e2e:
        hp = {k: t.cpu().pin_memory() for k, t in dict(pos=pos, vel=vel, typ=typ, mass=mass,
                                                       acc=acc).items()}
        h2d = sum(t.numel() * t.element_size() for t in hp.values())
        d2h = sum(hp[k].numel() * hp[k].element_size() for k in ("pos", "vel", "acc"))
        ksteps = max(1, min(args.steps, 3))
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # one untimed call sizes the context's device copies and captures the step
        # graph for them (two steps: the first runs eagerly, the second is captured)
        ng.ng_step_host(sim.ctx, hp["pos"], hp["vel"], hp["typ"], hp["mass"], hp["acc"], True, 2, dt)
        # the unit of work of these steps, counted like the timed region's: the
        # bodies have moved on since, so their steps hold more interactions
        pos.copy_(hp["pos"])
        ecount0 = algorithmic()
        # the host link's rate on these pinned buffers (boxes differ): every
        # input to the device, then the outputs back (the same values, so the
        # host state is unchanged)
        dt_ = dict(pos=pos, vel=vel, typ=typ, mass=mass, acc=acc)
        link = {"h2d_gbs": 0.0, "d2h_gbs": 0.0}
        for _ in range(3):                                     # best of three passes
            for name, keys, nbytes in (("h2d_gbs", ("pos", "vel", "typ", "mass", "acc"), h2d),
                                       ("d2h_gbs", ("pos", "vel", "acc"), d2h)):
                g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                g0.record(stream)
                for k in keys:
                    if name == "h2d_gbs":
                        dt_[k].copy_(hp[k], non_blocking=True)
                    else:
                        hp[k].copy_(dt_[k], non_blocking=True)
                g1.record(stream)
                torch.cuda.synchronize()
                rate = round(nbytes / (g0.elapsed_time(g1) / 1e3) / 1e9, 1)
                link[name] = max(link[name], rate)
        barrier()
        f0.record(stream)
        for _ in range(ksteps):
            # host arrays in, one step, host arrays out: all inside the C call
            ng.ng_step_host(sim.ctx, hp["pos"], hp["vel"], hp["typ"], hp["mass"], hp["acc"],
                            True, 1, dt)
        f1.record(stream)
        barrier()
        ems = f0.elapsed_time(f1)
        pos.copy_(hp["pos"])
        ecount, ems = job_totals(0.5 * (ecount0 + algorithmic()), ems, ws)
        e2e = {"value": ecount * ksteps / (ems / 1e3), "unit": "interactions/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": ems / ksteps, "interactions_per_step": ecount, "host_link": link}
    ref.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu, _ = cpu_leg(w, args.cpu_seconds, "cpu baseline")
        one, _ = cpu_leg(w, max(2.0, args.cpu_seconds / 3), "one core", threads=1)
        cpu["one_core"] = {"value": one["value"], "sample": one["sample"]}

    sim.close()
    if rank == 0:
        line = {"metric": "particle-node interactions/s", "value": value,
                "unit": "interactions/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic", "config": workload_config(w, args),
                "interactions_per_step": count,
                "count_basis": f"per-particle walk (theta {w['params']['theta']}) on the canonical "
                               f"tree with leaf size {REF_LEAF}",
                "interactions_per_step_at_walk_leaf": int(count_tuned_leaf),
                "particles_per_s": job_n * args.steps / (ms / 1e3),
                "roofline": roofline, "hbm": hbm, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": int(launches), "autotune": tuned}
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def bench_batch(args, ws, rank, local):
    """64 independent simulations (N log-uniform in [2^12, 2^18], D uniform in
    1..6, Newtonian couplings in [0.5, 1.5], PM 64^3) advanced together: each
    batch step is one captured graph with one persistent walk launch per
    species-count class."""
    import torch
    from paper_1502_07442_gb300 import binding as ng, inputs
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    specs = inputs.batch_specs(seed=1003 + 7919 * rank)
    state = []
    params = []
    counts = []
    for sp in specs:
        x = dict(pos=torch.from_numpy(sp["pos"]).to(dev), vel=torch.from_numpy(sp["vel"]).to(dev),
                 typ=torch.from_numpy(sp["type"]).to(dev), mass=torch.from_numpy(sp["mass"]).to(dev))
        x["acc"] = torch.zeros((3, sp["type"].size), dtype=torch.float32, device=dev)
        state.append(x)
    # walk leaf size and group cell: the three fastest for the largest
    # simulation alone, then timed on batch steps of all of them
    big = max(range(len(specs)), key=lambda i: specs[i]["type"].size)
    tuned = {"leaf_size": 8, "group_cell": 32, "tuned_on_n": int(specs[big]["type"].size)}
    if not args.no_tune:
        from paper_1502_07442_gb300 import autotune
        _, trials = autotune.tune(specs[big]["params"], state[big]["pos"], state[big]["typ"],
                                  state[big]["mass"])
        short = [(t["leaf_size"], t["group_cell"]) for t in sorted(trials, key=lambda t: t["ms"])[:3]]
        best, btrials = autotune.tune_batch([sp["params"] for sp in specs], state, short)
        tuned.update(leaf_size=best["leaf_size"], group_cell=best["group_cell"], trials=len(trials),
                     batch_trials={f"{t['leaf_size']}/{t['group_cell']}": round(t["ms"], 3)
                                   for t in btrials})
    for sp in specs:
        params.append(ng.params_from_workload(sp["params"], leaf_size=tuned["leaf_size"],
                                              group_cell=tuned["group_cell"]))
    b = ng.ng_batch_create(params)
    L = lambda k: [x[k] for x in state]
    ng.ng_batch_step(b, L("pos"), L("vel"), L("typ"), L("mass"), L("acc"), False, args.warmup, 1e-3)
    # algorithmic interactions per simulation at the start of the timed region
    for x, sp in zip(state, specs):
        s = ng.Simulation(ng.params_from_workload(sp["params"], leaf_size=REF_LEAF))
        ng.ng_build_tree(s.ctx, x["pos"], x["typ"], x["mass"])
        counts.append(ng.ng_count_interactions(s.ctx))
        s.close()
    torch.cuda.synchronize()
    l0 = ng.ng_batch_launch_count(b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    with Clocks(local) as clk:
        e0.record()
        ng.ng_batch_step(b, L("pos"), L("vel"), L("typ"), L("mass"), L("acc"), True, args.steps, 1e-3)
        e1.record()
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    # every rank advances its own 64 simulations: sum the units, slowest clock
    job_count, ms = job_totals(sum(counts), ms, ws)
    nbodies, _ = job_totals(sum(x["typ"].numel() for x in state), ms, ws)
    line = {"metric": "particle-node interactions/s", "value": job_count * args.steps / (ms / 1e3),
            "unit": "interactions/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch64", "simulations": len(specs), "bodies": int(nbodies),
                       "n_range": [int(min(x["typ"].numel() for x in state)),
                                   int(max(x["typ"].numel() for x in state))],
                       "pm_mesh": 64, "walk_launches_per_step": ng.ng_batch_walk_launches(b),
                       "step": "one graph: per-simulation sort/tree/PM on 32 worker streams, one walk launch",
                       "autotune": tuned},
            "particles_per_s": nbodies * args.steps / (ms / 1e3), "clocks": clk.summary(),
            "gpu_launches": int(ng.ng_batch_launch_count(b) - l0)}
    ng.ng_batch_destroy(b)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def bench_serve(args, ws, rank, local):
    """2000 requests (Poisson, 200 req/s; half force evaluations, half 10-step
    integrations; N log-uniform in [2^10, 2^20]; D uniform in 1..6; Newtonian
    couplings in [0.5, 1.5]; PM mesh clamp(next_pow2(N^(1/3)), 32, 128);
    120 GB byte budget). Reports the saturated throughput of the serving loop
    with 16 slots against one-at-a-time solves (plain calls, a context per
    request; the serving loop with one slot), and p50/p99 latency on the
    Poisson trace at 200 requests/s and at 150 requests/s (below capacity)."""
    import torch
    from paper_1502_07442_gb300 import binding as ng, inputs
    torch.cuda.set_device(local)
    nreq = 2000 if args.n is None else int(args.n)
    rng = inputs.rng_for(1004 + 7919 * rank)
    pool = []
    for k in range(96):                      # distinct inputs, reused round-robin
        n = inputs.log_uniform_int(rng, 10, 20)
        D = int(rng.integers(1, 7))
        sub = inputs.rng_for(1004000 + k)
        pos = inputs.clustered(n, sub, nspheres=max(1, n // 4096))
        typ = inputs.species_uniform(n, D, sub)
        coup = inputs.newton_couplings(D, sub)
        mesh = inputs.serve_mesh(n)
        rs = 1.25 / mesh
        prm = dict(D=D, G=coup["G"], law=coup["law"], ya=coup["ya"], yl=coup["yl"], box=1.0,
                   eps=0.02 / n ** (1 / 3), rs=rs, rcut=4.5 * rs, theta=0.5, pm_mesh=mesh)
        # walk shape by request size (the plain calls and the serving loop
        # both take it from the request's parameters)
        shape = SERVE_LARGE_SHAPE if n >= SERVE_LARGE_N else SERVE_SMALL_SHAPE
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        pool.append(dict(n=n, params=ng.params_from_workload(prm, leaf_size=shape[0],
                                                             group_cell=shape[1]),
                         pos=pin(pos), typ=pin(typ),
                         mass=pin(np.full(n, 1.0 / n, np.float32)),
                         acc=torch.zeros((3, n), dtype=torch.float32).pin_memory(),
                         pos_out=torch.zeros((3, n), dtype=torch.float64).pin_memory(),
                         vel_out=torch.zeros((3, n), dtype=torch.float32).pin_memory()))
    kinds = rng.integers(0, 2, nreq)
    gaps = rng.exponential(1.0, nreq)            # unit-rate Poisson gaps, scaled per leg

    def trace(rate):
        g = gaps / rate
        return np.cumsum(g) - g[0]

    def requests():
        reqs = (ng.NgRequest * nreq)()
        for k in range(nreq):
            e = pool[k % len(pool)]
            reqs[k] = ng.make_request(int(kinds[k]), e["params"], e["pos"], e["typ"], e["mass"],
                                      nsteps=10 if kinds[k] else 0, dt=1e-3,
                                      pos_out=e["pos_out"], vel_out=e["vel_out"], acc_out=e["acc"])
        return reqs

    def run(slots, arr):
        s = ng.ng_serve_create(slots, 120 << 30)
        warm = requests()
        wres = (ng.NgResult * len(pool))()
        ng.ng_serve(s, (ng.NgRequest * len(pool))(*[warm[k] for k in range(len(pool))]), wres,
                    None, 600.0)                                   # grow every slot's buffers
        reqs, res = requests(), (ng.NgResult * nreq)()
        t0 = time.perf_counter()
        ng.ng_serve(s, reqs, res, arr, 1800.0)
        wall = time.perf_counter() - t0
        first_err = ng.lib().ng_serve_last_error(s)
        ng.ng_serve_destroy(s)
        lat = np.array([r.t_done - r.t_submit for r in res])
        bad = [(k, r.status) for k, r in enumerate(res) if r.status != 0]
        if bad:
            print(f"serve: {len(bad)} of {nreq} requests failed; first {bad[:5]}; "
                  f"{(first_err or b'').decode()}", file=sys.stderr, flush=True)
        return wall, lat, not bad

    def plain():
        # one request at a time through the plain calls, as a caller without
        # the serving loop writes it: create a context for the request's
        # parameters, copy in, ng_step (nsteps = 0 is one force evaluation),
        # copy out, destroy
        dev = torch.device("cuda", local)
        stream = torch.cuda.current_stream()
        ok = True
        t0 = time.perf_counter()
        for k in range(nreq):
            e = pool[k % len(pool)]
            n = e["n"]
            sim = ng.Simulation(e["params"], stream)
            pos = e["pos"].to(dev, non_blocking=True)
            typ = e["typ"].to(dev, non_blocking=True)
            mass = e["mass"].to(dev, non_blocking=True)
            vel = torch.zeros((3, n), dtype=torch.float32, device=dev)
            acc = torch.empty((3, n), dtype=torch.float32, device=dev)
            try:
                ng.ng_step(sim.ctx, pos, vel, typ, mass, acc, False, 10 if kinds[k] else 0, 1e-3)
            except ng.NgError as err:
                print(f"plain request {k} (n={n}, kind={int(kinds[k])}) failed: {err}",
                      file=sys.stderr, flush=True)
                ok = False
                break
            e["acc"].copy_(acc, non_blocking=True)
            if kinds[k]:
                e["pos_out"].copy_(pos, non_blocking=True)
                e["vel_out"].copy_(vel, non_blocking=True)
            torch.cuda.synchronize()
            sim.close()
        return time.perf_counter() - t0, ok

    def leg(name, fn, *a):
        # a failed leg reports where it failed and ends the process at once
        # (no unwinding through CUDA buffers of a context that has faulted)
        t = time.perf_counter()
        print(f"serve leg {name}: start", file=sys.stderr, flush=True)
        try:
            r = fn(*a)
        except Exception:
            import traceback
            traceback.print_exc()
            sys.stderr.flush()
            os._exit(3)
        print(f"serve leg {name}: {time.perf_counter() - t:.1f} s", file=sys.stderr, flush=True)
        return r

    wpl, okpl = leg("plain", plain)                                # plain calls, one at a time
    w1, _, ok1 = leg("one-slot", run, 1, None)                     # serving loop, one slot
    wk, _, okk = leg("saturated", run, 16, None)                   # continuous batching, saturated
    wp, lat, okp = leg("poisson200", run, 16, trace(200.0))        # the workload's arrival rate
    wq, latq, okq = leg("poisson150", run, 16, trace(150.0))       # below the saturated capacity
    line = {"metric": "requests/s (served, saturated)", "value": nreq / wk, "unit": "requests/s",
            "n_gpus": ws, "steps": 1, "warmup": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serve2000", "requests": nreq, "rate_per_s": 200, "slots": 16,
                       "budget_bytes": 120 << 30, "mix": "50% force, 50% 10-step KDK",
                       "n_range_log2": [10, 20],
                       "walk_shape": {"n_from": SERVE_LARGE_N, "large": list(SERVE_LARGE_SHAPE),
                                      "small": list(SERVE_SMALL_SHAPE)}},
            "one_at_a_time": {"plain_calls_requests_per_s": nreq / wpl,
                              "serving_one_slot_requests_per_s": nreq / w1},
            "speedup_vs_plain_calls": wpl / wk, "speedup_vs_one_slot": w1 / wk,
            "poisson": {"rate_per_s": 200,
                        "p50_latency_ms": float(np.percentile(lat, 50) * 1e3),
                        "p99_latency_ms": float(np.percentile(lat, 99) * 1e3),
                        "throughput_requests_per_s": nreq / wp},
            "poisson_below_capacity": {"rate_per_s": 150,
                                       "p50_latency_ms": float(np.percentile(latq, 50) * 1e3),
                                       "p99_latency_ms": float(np.percentile(latq, 99) * 1e3),
                                       "throughput_requests_per_s": nreq / wq},
            "all_ok": bool(okpl and ok1 and okk and okp and okq)}
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
