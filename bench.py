#!/usr/bin/env python3
"""Benchmark of the dynamic-bonding MD step (particle-steps/s incl. the bond sweep).

Workload (default): the 10^6-particle colloid-linker gel — 200k C (sigma 1,
valence 4) + 800k L (sigma 0.5, valence 2) placed without overlap at packing
fraction 0.25, C-L harmonic bonds (k 100, r0 0.9, r_max 1.2, eps 6 kT, P_on^0 1),
WCA, Langevin gamma 1, dt 0.005, kT 1, one bond sweep per step.  The headline is
the FP32-force / FP64-integration ("mixed") path; the all-FP64 path is timed
beside it.  Under torchrun each rank runs its own replica (seed + rank): weak
scaling, no data-path collective.

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload (the only other place this script executes oracle code).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "particle-steps/s incl. dynamic-bond update, 1M particles; mixed/batched vs plain"
UNIT = "particle-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="snap", choices=["snap", "reference"])
    ap.add_argument("--n-c", type=int, default=200_000)
    ap.add_argument("--n-l", type=int, default=800_000)
    ap.add_argument("--profile-steps", type=int, default=50)
    ap.add_argument("--fp64-steps", type=int, default=200)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--batch-replicas", type=int, default=256,
                    help="replicas of the batched telechelic sweep leg (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--input-cache", default="",
                    help="directory to keep the generated coordinates between invocations")
    return ap.parse_args()


def workload_config(args, n):
    return {
        "workload": f"colloid-linker gel: {args.n_c} C (sigma 1, valence 4) + {args.n_l} L "
                    "(sigma 0.5, valence 2), packing fraction 0.25, C-L harmonic k=100 r0=0.9 "
                    "r_max=1.2, eps=6 kT, WCA, Langevin gamma=1 dt=0.005 kT=1, sweep every step",
        "n_particles": n,
        "precision": "FP32 pair/bond forces; FP64 positions, integration, sweep cut-off and acceptance",
        "l2": "no flush: per-step working set (~0.35 GB) exceeds the 126 MB L2",
        "seed": 20260921,
    }


def build_batch(args):
    from synth import telechelic_sweep
    procs = max(1, min(16, (os.cpu_count() or 1)))
    if args.input_cache:
        import pickle
        p = Path(args.input_cache) / f"telechelic_sweep_{args.batch_replicas}.pkl"
        if p.exists():
            return pickle.loads(p.read_bytes())
        reps = telechelic_sweep(n_replicas=args.batch_replicas, processes=procs)
        p.parent.mkdir(parents=True, exist_ok=True)
        p.write_bytes(pickle.dumps(reps))
        return reps
    return telechelic_sweep(n_replicas=args.batch_replicas, processes=procs)


def build_system(args, seed):
    from synth import colloid_linker
    if args.input_cache:
        import pickle
        p = Path(args.input_cache) / f"colloid_linker_{args.n_c}_{args.n_l}_{seed}.pkl"
        if p.exists():
            return pickle.loads(p.read_bytes())
        s = colloid_linker(seed=seed, n_c=args.n_c, n_l=args.n_l, eta=0.25)
        p.parent.mkdir(parents=True, exist_ok=True)
        p.write_bytes(pickle.dumps(s))
        return s
    return colloid_linker(seed=seed, n_c=args.n_c, n_l=args.n_l, eta=0.25)


# ----------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in Path(self.path).read_text().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def force_traffic_from_profile(n, nbar):
    """DRAM bytes per launch of the force kernel from the committed ncu summary,
    if it was taken on the current kernel source; scaled to this launch."""
    prof = ROOT / "profiles" / "force_kernel_colloid_linker.txt"
    if not prof.exists():
        return None
    src = (ROOT / "paper_2609_21204_b300" / "csrc" / "md.cu").read_bytes()
    sha = hashlib.sha256(src).hexdigest()[:16]
    kv = {}
    for line in prof.read_text().splitlines():
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("md_cu_sha256_16") != sha:
        return None
    try:
        per_particle = float(kv["dram_bytes_per_particle"])
    except (KeyError, ValueError):
        return None
    return per_particle * n


# ----------------------------------------------------------------- snap arm
def run_snap(args):
    # the batched leg's inputs are generated first, in a spawned pool, before any GPU call
    batch = build_batch(args) if args.batch_replicas > 0 else None
    import torch
    import torch.distributed as dist
    import paper_2609_21204_b300 as snap

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev_index = torch.cuda.current_device()

    def barrier():
        if world > 1:
            dist.barrier()

    def max_all(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def sum_all(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        _run_snap_on_stream(args, torch, dist, snap, rank, world, dev_index, barrier, max_all,
                            sum_all, stream, batch)
    if world > 1:
        dist.destroy_process_group()


def _run_batched(args, torch, snap, batch, barrier, max_all, sum_all, stream):
    """Batched sweep leg: all replicas in one context (one graph launch per
    20 steps), launch shape and skin from the autotuner."""
    from paper_2609_21204_b300 import autotune
    tune = autotune.autotune(batch, precision="mixed", steps=40, warmup=20)
    sim = snap.from_system(batch, precision="mixed", block_size=tune["block_size"],
                           skin=tune["skin"])
    nb = sum(s.n for s in batch)
    sim.step(args.warmup)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.batch_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t = max_all(e0.elapsed_time(e1) / 1e3)
    st = sim.stats()
    sim.close()
    return {"workload": f"{len(batch)} telechelic replicas (N log-uniform in [2k, 50k], "
                        f"eps U[2,10] kT, kT U[0.8,1.2]), {nb} particles in one context",
            "value": sum_all(float(nb)) * args.batch_steps / t, "unit": UNIT,
            "ms_per_step": t * 1e3 / args.batch_steps, "steps": args.batch_steps,
            "particles": nb, "replicas": len(batch), "n_bonds": st["n_bonds"],
            "autotune": {k: tune[k] for k in ("block_size", "skin", "cached", "key")}}


def _run_snap_on_stream(args, torch, dist, snap, rank, world, dev_index, barrier, max_all, sum_all,
                        stream, batch=None):
    s = build_system(args, 20260921 + rank)
    n = s.n
    K, W = args.steps, args.warmup
    sim = snap.from_system(s, precision="mixed", block_size=args.block)

    sim.step(W)
    st0 = sim.stats()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(dev_index)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    t = e0.elapsed_time(e1) / 1e3
    st1 = sim.stats()
    t_max = max_all(t)
    n_all = sum_all(float(n))
    value = n_all * K / t_max

    # per-phase times over an instrumented window right after the timed region
    ph = sim.step_profiled(args.profile_steps)
    st2 = sim.stats()
    nbar = st2["nlist_entries"] / n
    force_ms = ph["force"]
    # algorithmic bytes of the force kernel per particle: own pos4 16, replica id 4,
    # count 4, 4 per neighbour index, static + dynamic slots 2 x (16 + 4), force 16
    bytes_pp = 16 + 4 + 4 + 4 * nbar + 40 + 16
    alg_bytes = bytes_pp * n
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (force_ms / 1e3) / 1e9
    traffic = force_traffic_from_profile(n, nbar)
    sweep_pairs = st2["scanned"] + st2["break_tested"]
    bond_pairs_per_s = sweep_pairs / (ph["sweep"] / 1e3) if ph["sweep"] > 0 else None

    # kernels launched per step: 10 neighbour-list kernels (early exits between
    # rebuilds), 1 + 5 per reaction for the sweep, force, integrate, step end
    kernels_per_step = 10 + (1 + 5 * len(s.reactions)) + 3

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": t_max * 1e3 / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": workload_config(args, n),
        "gpu_launches": kernels_per_step * K,
        "clocks": clk,
        "phases_ms_per_step": {k: round(v, 5) for k, v in ph.items()},
        "bond_update_pairs_per_s": bond_pairs_per_s,
        "sweep": {"scanned_nlist_entries": st2["scanned"], "break_tested": st2["break_tested"],
                  "proposals": st2["proposals"], "formed": st2["formed"], "broken": st2["broken"],
                  "n_bonds": st2["n_bonds"], "mean_neighbours": nbar,
                  "nlist_builds_in_timed_region": st1["nlist_builds"] - st0["nlist_builds"]},
        "roofline": {"kernel": "k_force<float> (pair + bond forces)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_kind, "traffic": traffic,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "launch_ms": force_ms},
    }
    if not args.no_fp64:
        sim.close()
        sim64 = snap.from_system(s, precision="fp64", block_size=args.block)
        sim64.step(W)
        barrier()
        torch.cuda.synchronize()
        K64 = args.fp64_steps
        e0.record(stream)
        sim64.step(K64)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = max_all(e0.elapsed_time(e1) / 1e3)
        v64 = n_all * K64 / t64
        ph64 = sim64.step_profiled(max(5, args.profile_steps // 5))
        out["fp64_plain"] = {"value": v64, "ms_per_step": t64 * 1e3 / K64, "steps": K64,
                             "phases_ms_per_step": {k: round(v, 5) for k, v in ph64.items()}}
        out["speedup_mixed_vs_fp64_plain"] = value / v64
        sim64.close()
        sim = snap.from_system(s, precision="mixed", block_size=args.block)
        sim.step(W)
    if batch is not None:
        sim.close()
        out["batched"] = _run_batched(args, torch, snap, batch, barrier, max_all, sum_all, stream)
        sim = snap.from_system(s, precision="mixed", block_size=args.block)
        sim.step(W)
    if not args.no_e2e:
        # end to end through the C ABI with host buffers: upload the state, one
        # step, read positions back — every step
        pos = np.ascontiguousarray(sim.positions())
        vel = np.ascontiguousarray(sim.velocities())
        E = args.e2e_steps
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(E):
            sim.set_positions(pos, vel)
            sim.step(1)
            pos = sim.positions()
        torch.cuda.synchronize()
        te = max_all(time.perf_counter() - t0)
        out["e2e"] = {"value": n_all * E / te, "unit": UNIT, "h2d_bytes_per_step": 48 * n,
                      "d2h_bytes_per_step": 24 * n, "steps": E,
                      "what": "per step: snap_set_positions (positions+velocities from host), "
                              "snap_step(1), snap_get_positions (to host)"}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        o = oracle.OracleSystem(s)
        t0 = time.perf_counter()
        o.run(args.cpu_steps)
        tc = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": n * args.cpu_steps / tc, "unit": UNIT, "cores": 1,
                               "kind": "oracle",
                               "sample": f"{args.cpu_steps} full MD steps (sweep, forces, Langevin) "
                                         f"of the same {n}-particle gel, single thread, FP64"}
    if rank == 0:
        print(json.dumps(out), flush=True)


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle
    K, W = args.steps, args.warmup
    # bounded sample of the same workload: same composition and packing
    # fraction, sized so that W + K oracle steps take about a minute
    rate = 2.5e5
    n_s = int(min(args.n_c + args.n_l, max(2000, 60.0 * rate / max(1, K + W))))
    n_c = max(1, n_s // 5)
    n_l = n_s - n_c
    from synth import colloid_linker
    s = colloid_linker(seed=20260921, n_c=n_c, n_l=n_l, eta=0.25)
    o = oracle.OracleSystem(s)
    o.run(W)
    t0 = time.perf_counter()
    o.run(K)
    t = time.perf_counter() - t0
    value = s.n * K / t
    cfg = workload_config(args, args.n_c + args.n_l)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": K, "warmup": W, "ms_per_step": t * 1e3 / K, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": cfg,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"each step: one full MD step of a {s.n}-particle sample "
                                      f"({n_c} C + {n_l} L, same packing fraction) on one core"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_snap(args)


if __name__ == "__main__":
    main()
