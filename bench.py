"""Throughput of the multi-species TreePM step on GB300 (one JSON line).

A step is one kick-drift-kick step (Sec. 2.1.1) of the whole hot path:
kick, FP64 drift + wrap, Morton+type keys and radix sort, canonical octree,
per-species monopoles, PM long-range force (CIC, cuFFT, D x D kernels,
interpolation), the short-range group walk, kick. Steps replay a captured
CUDA graph through ng_step.

metric: particle-node interactions per second, where the interactions are
those of the per-particle Barnes-Hut walk (ng_count_interactions, the
algorithm's unit of work: one (accepted node, species with mass) term or
one body of an opened leaf), counted on the positions at the start and at
the end of the timed region and averaged.

roofline: the dominant kernel is the walk, bound by the FP32 pipe; achieved
= 23 flop x per-particle-walk interactions / average walk duration (CUDA
events around ng_tree_force on the launching stream); peak = SMs x 128
lanes x 2 flop x SM clock (the maximum clock; the same at the median clock
sampled during the run is given beside it).

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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--n", type=int, default=None, help="override N (smaller test runs)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
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


def cpu_leg(w, seconds, tag):
    """The FP64 checker on host cores: per-particle walk of random targets on the
    full tree; rate = interactions / walk seconds (tree build timed apart)."""
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    prm = w["params"]
    op = oracle.make_params(prm["D"], prm["G"], box=prm["box"], eps=prm["eps"], rs=prm["rs"],
                            rcut=prm["rcut"], theta=prm["theta"], leaf_size=prm["leaf_size"],
                            pm_mesh=prm["pm_mesh"], law=prm["law"], ya=prm["ya"], yl=prm["yl"])
    cores = oracle.set_threads(0)
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
    return {"value": float(rate), "unit": "interactions/s", "cores": int(cores), "kind": "oracle",
            "sample": f"{tag}: FP64 per-particle tree walk of {m} random targets of {n} bodies "
                      f"(tree build {tb2:.1f} s timed apart, walk {tw2:.1f} s)"}, float(tw2)


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
            "parallelism": f"replicas{args.gpus}"}


def main():
    args = parse()
    ws, rank, local = dist_env()
    from paper_1502_07442_gb300 import inputs
    w = inputs.workload(args.workload, n=args.n, seed=None if rank == 0 else 1002 + 7919 * rank)
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
    sim = ng.Simulation(ng.params_from_workload(w["params"]), stream)
    dt = float(w["dt"])

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # warm-up: the first call computes the initial force and captures the step graph
    ng.ng_step(sim.ctx, pos, vel, typ, mass, acc, False, args.warmup, dt)
    count0 = ng.ng_count_interactions(sim.ctx)
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
    count1 = ng.ng_count_interactions(sim.ctx)
    count = 0.5 * (count0 + count1)
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = count * args.steps * ws / (ms / 1e3)

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
    med = clocks.get("sm_mhz") or 2070.0
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": "k_walk", "walk_ms": round(walk, 3),
                "peak_at_median_clock": round(nsm * 128 * 2 * med * 1e6 / 1e12, 2),
                "frac_at_median_clock": round(achieved / (nsm * 128 * 2 * med * 1e6 / 1e12), 4),
                "executed_interactions": int(executed),
                "executed_over_algorithmic": round(executed / count1, 3),
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
        f0.record(stream)
        for _ in range(ksteps):
            pos.copy_(hp["pos"], non_blocking=True)
            vel.copy_(hp["vel"], non_blocking=True)
            typ.copy_(hp["typ"], non_blocking=True)
            mass.copy_(hp["mass"], non_blocking=True)
            acc.copy_(hp["acc"], non_blocking=True)
            ng.ng_step(sim.ctx, pos, vel, typ, mass, acc, True, 1, dt)
            hp["pos"].copy_(pos, non_blocking=True)
            hp["vel"].copy_(vel, non_blocking=True)
            hp["acc"].copy_(acc, non_blocking=True)
        f1.record(stream)
        barrier()
        ems = f0.elapsed_time(f1)
        if ws > 1:
            t = torch.tensor([ems], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ems = float(t.item())
        e2e = {"value": count * ksteps * ws / (ems / 1e3), "unit": "interactions/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": ems / ksteps}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu, _ = cpu_leg(w, args.cpu_seconds, "cpu baseline")

    sim.close()
    if rank == 0:
        line = {"metric": "particle-node interactions/s", "value": value,
                "unit": "interactions/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic", "config": workload_config(w, args),
                "interactions_per_step": count, "particles_per_s": n * args.steps * ws / (ms / 1e3),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": int(launches)}
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
