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
    ap.add_argument("--equil-steps", type=int, default=2000,
                    help="untimed steps from the bond-free start before the warm-up, so that every "
                         "timed window sees the gel in its saturated (push-mode) state")
    ap.add_argument("--profile-steps", type=int, default=50)
    ap.add_argument("--fp64-steps", type=int, default=200)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--block", type=int, default=0,
                    help="threads per block of the particle kernels (0 with --skin 0: autotuned)")
    ap.add_argument("--skin", type=float, default=0.0,
                    help="neighbour-list skin (0 with --block 0: autotuned)")
    ap.add_argument("--subcells", type=int, default=-1,
                    help="list build's sub-cells along x per cell (0 automatic, 1/2/4/8; with --block/--skin)")
    ap.add_argument("--batch-replicas", type=int, default=256,
                    help="replicas of the batched telechelic sweep leg (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--learned-events", type=int, default=1_000_000,
                    help="formation events logged for training the proposal network (0: skip the leg)")
    ap.add_argument("--learned-epochs", type=int, default=10)
    ap.add_argument("--mh-steps", type=int, default=500)
    ap.add_argument("--no-small-legs", dest="small_legs", action="store_false",
                    help="skip the A+B association and telechelic network legs")
    ap.add_argument("--competing-n", type=int, default=262144,
                    help="particles of the four-reaction soup leg (0: skip the leg)")
    ap.add_argument("--competing-steps", type=int, default=1000)
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


def build_system(args, seed, rho=None):
    from synth import colloid_linker
    kw = dict(seed=seed, n_c=args.n_c, n_l=args.n_l)
    kw.update(dict(rho=rho, eta=None) if rho is not None else dict(eta=0.25))
    if args.input_cache:
        import pickle
        tag = f"rho{rho}" if rho is not None else "eta0.25"
        p = Path(args.input_cache) / f"colloid_linker_{args.n_c}_{args.n_l}_{seed}_{tag}.pkl"
        if p.exists():
            return pickle.loads(p.read_bytes())
        s = colloid_linker(**kw)
        p.parent.mkdir(parents=True, exist_ok=True)
        p.write_bytes(pickle.dumps(s))
        return s
    return colloid_linker(**kw)


# ----------------------------------------------------------------- clocks
class _Nvml:
    """The few read-only NVML queries the clock sampler needs, through the
    driver's libnvidia-ml with ctypes (no Python package required)."""
    CLOCK_SM = 1
    # clock-event reason bits (NVML's public constants)
    REASONS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, dev):
        import ctypes
        self.C = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit")
        self.h = ctypes.c_void_p()
        ok = False
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(int(dev)).uuid)
            uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
            ok = self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) == 0
        except Exception:
            ok = False
        if not ok and self.lib.nvmlDeviceGetHandleByIndex_v2(int(dev), ctypes.byref(self.h)) != 0:
            raise RuntimeError("nvmlDeviceGetHandle")
        self.get_reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def sample(self):
        C = self.C
        sm, smax, r = C.c_uint(), C.c_uint(), C.c_ulonglong()
        if (self.lib.nvmlDeviceGetClockInfo(self.h, self.CLOCK_SM, C.byref(sm)) != 0 or
                self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.CLOCK_SM, C.byref(smax)) != 0 or
                self.get_reasons(self.h, C.byref(r)) != 0):
            raise RuntimeError("nvml query")
        return float(sm.value), float(smax.value), {k for k, b in self.REASONS.items() if r.value & b}

    def close(self):
        self.lib.nvmlShutdown()


class Clocks:
    """SM clocks and clock-event reasons sampled during the timed region: NVML
    every 2 ms from a host thread (the GPU runs the queued steps while the host
    waits), with one sample when sampling starts and one when it stops, so
    that even a timed region of a few milliseconds has samples; nvidia-smi
    -lms 200 when NVML cannot be loaded.  Read-only queries."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None
        self.nvml = None
        self.thread = None
        self.samples = []

    def start(self):
        try:
            import threading
            self.nvml = _Nvml(self.dev)
            self.samples = [self.nvml.sample()]
            self.stop_flag = threading.Event()

            def loop():
                while not self.stop_flag.wait(0.002):
                    try:
                        self.samples.append(self.nvml.sample())
                    except Exception:
                        return
            self.thread = threading.Thread(target=loop, daemon=True)
            self.thread.start()
            return
        except Exception:
            self.nvml = None
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
        sm, smax, reasons = [], [], set()
        if self.nvml is not None:
            self.stop_flag.set()
            self.thread.join(timeout=5)
            try:
                self.samples.append(self.nvml.sample())
            except Exception:
                pass
            for a, b, r in self.samples:
                sm.append(a)
                smax.append(b)
                reasons |= r
            try:
                self.nvml.close()
            except Exception:
                pass
            source = "nvml"
        elif self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()
            for line in Path(self.path).read_text().splitlines():
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(self.NAMES, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            os.unlink(self.path)
            source = "nvidia-smi"
        else:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "source": source}


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def inside_cut_fraction(s, pos, nbar):
    """Fraction of force-list entries whose pair lies inside its WCA cut at
    these positions (pairs counted with a k-d tree; nbar = entries per particle)."""
    try:
        from scipy.spatial import cKDTree
        box = np.asarray(s.box, dtype=np.float64)
        p = np.mod(pos, box)
        sig = np.asarray(s.sigma, dtype=np.float64)
        rc = 0.5 * (sig[:, None] + sig[None, :]) * 2.0 ** (1.0 / 6.0)
        pairs = cKDTree(p, boxsize=box).query_pairs(float(rc.max()), output_type="ndarray")
        d = p[pairs[:, 0]] - p[pairs[:, 1]]
        d -= box * np.rint(d / box)
        r2 = (d * d).sum(1)
        t = np.asarray(s.types)
        inside = int((r2 < rc[t[pairs[:, 0]], t[pairs[:, 1]]] ** 2).sum())
        return 2.0 * inside / (nbar * len(p))
    except Exception:
        return None


def fp64_dgemm_tflops(torch):
    """FP64 rate of this GPU: cuBLAS DGEMM of two 8192^2 matrices, best of 3."""
    try:
        a = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
        b = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
        torch.matmul(a, b)
        best = None
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        del a, b
        return 2.0 * 8192 ** 3 / best / 1e12
    except Exception:
        return None


def md_traffic_from_profile(n):
    """DRAM bytes per launch of the fused force + Langevin kernel from the
    committed ncu summary, if it was taken on the current kernel sources;
    scaled to this launch by the particle count."""
    prof = ROOT / "profiles" / "step_md_kernel_colloid_linker.txt"
    if not prof.exists():
        return None
    csrc = ROOT / "paper_2609_21204_b300" / "csrc"
    kv = {}
    for line in prof.read_text().splitlines():
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    for f in ("md.cu", "integrate.cuh"):
        sha = hashlib.sha256((csrc / f).read_bytes()).hexdigest()[:16]
        if kv.get(f.replace(".", "_") + "_sha256_16") != sha:
            return None
    try:
        per_particle = float(kv["dram_bytes_per_particle"])
    except (KeyError, ValueError):
        return None
    return per_particle * n


# ----------------------------------------------------------------- ranks
class RankGroup:
    """What the ranks of one bench run share: a barrier and the max / sum of a
    number over ranks (NCCL tensors on the GPU, gloo on the host).  With one
    rank every call is the identity.  The snap arm shards whole replicas: each
    rank runs its own system (rank_seed) and no data crosses ranks."""

    def __init__(self, dist, world, device):
        self.dist, self.world, self.device = dist, world, device

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def _reduce(self, x, op):
        if self.world == 1:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max_all(self, x):
        return self._reduce(x, self.dist.ReduceOp.MAX)

    def sum_all(self, x):
        return self._reduce(x, self.dist.ReduceOp.SUM)

    def throughput(self, n_local, steps, seconds_local):
        """Whole-job particle-steps per second: every rank's particles over the
        slowest rank's time."""
        return self.sum_all(float(n_local)) * steps / self.max_all(seconds_local)


def run_leg(out, key, world, fn):
    """Run one secondary leg of the benchmark into out[key].  With one rank a
    leg that raises is recorded as {"error": ...} so that the headline line
    still prints; with several ranks the error propagates (a rank that skipped
    the rest of a leg would leave the others waiting in a collective)."""
    try:
        out[key] = fn()
    except Exception as e:   # noqa: BLE001 - recorded in the JSON line, not hidden
        if world > 1:
            raise
        out[key] = {"error": f"{type(e).__name__}: {e}"}


def rank_seed(base, rank):
    """Seed of the system a rank runs (replica r uses seed + r)."""
    return base + rank


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

    group = RankGroup(dist, world, "cuda")
    barrier, max_all, sum_all = group.barrier, group.max_all, group.sum_all

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
                           skin=tune["skin"], list_block=tune.get("list_block"),
                           list_subcells=tune.get("list_subcells"))
    nb = sum(s.n for s in batch)
    sim.step(args.warmup)
    sim.prepare()
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
    sim_subcells = sim.list_subcells()
    sim.close()
    return {"workload": f"{len(batch)} telechelic replicas (N log-uniform in [2k, 50k], "
                        f"eps U[2,10] kT, kT U[0.8,1.2]), {nb} particles in one context",
            "value": sum_all(float(nb)) * args.batch_steps / t, "unit": UNIT,
            "ms_per_step": t * 1e3 / args.batch_steps, "steps": args.batch_steps,
            "particles": nb, "replicas": len(batch), "n_bonds": st["n_bonds"],
            "autotune": dict({k: tune.get(k) for k in ("block_size", "skin", "list_block", "list_subcells",
                                                        "cached", "key")}, subcells_in_use=sim_subcells),
            "vs_oracle": _smallest_replicas_vs_oracle(snap, batch)}


def _smallest_replicas_vs_oracle(snap, batch):
    """Bonded fraction of chain ends of the 8 smallest replicas, from a fresh
    batched run of all replicas with the sampling of the stored FP64 oracle
    runs of those replicas alone (tests/golden/telechelic_sweep_smallest8.json,
    written by the oracle), as z-scores with both error bars."""
    gold = json.loads((ROOT / "tests" / "golden" / "telechelic_sweep_smallest8.json").read_text())
    offs = np.concatenate([[0], np.cumsum([s.n for s in batch])])
    sim = snap.from_system(batch, precision="mixed")
    sim.step(gold["burn_in"])
    idx = [g["replica"] for g in gold["runs"]]
    series = {r: [] for r in idx}
    for _ in range((gold["steps"] - gold["burn_in"]) // gold["every"]):
        sim.step(gold["every"])
        b = sim.bonds()
        for r in idx:
            series[r].append(int(((b[:, 0] >= offs[r]) & (b[:, 0] < offs[r + 1])).sum()))
    sim.close()
    out = []
    nb = gold["blocks"]
    for g in gold["runs"]:
        f = np.array(series[g["replica"]], dtype=np.float64) / g["n_ends"]
        se = float(f.reshape(nb, -1).mean(1).std(ddof=1) / math.sqrt(nb))
        z = (f.mean() - g["bonded_fraction"]) / math.sqrt(se ** 2 + g["bonded_fraction_se"] ** 2 + 1e-12)
        out.append({"replica": g["replica"], "n": g["n"], "eps": round(g["eps"], 3),
                    "bonded_fraction": float(f.mean()), "se": se,
                    "oracle": g["bonded_fraction"], "oracle_se": g["bonded_fraction_se"], "z": float(z)})
    return {"replicas": out, "max_abs_z": max(abs(x["z"]) for x in out),
            "what": "bonded fraction of chain ends, steps %d-%d, mixed precision vs FP64 oracle" %
                    (gold["burn_in"], gold["steps"])}


def _run_assoc_ab(args, torch, snap, max_all, sum_all, stream):
    """A+B association (500 A + 500 B at number density 0.1, eps 5 kT, window
    r <= 1.3, 10^4 steps): graph-launched steps per second on the small system,
    and the bonded fraction against the stored FP64 oracle runs of the same
    seeds (tests/golden/assoc_ab_observables.json)."""
    from synth import assoc_ab
    gold = json.loads((ROOT / "tests" / "golden" / "assoc_ab_observables.json").read_text())
    steps, burn, every, nb = gold["steps"], gold["burn_in"], gold["every"], gold["blocks"]
    fr, se2, t_tot = [], [], 0.0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for g in gold["runs"]:
        s = assoc_ab(seed=g["seed"])
        sim = snap.from_system(s, precision="mixed")
        n_a = int((s.types == 0).sum())
        sim.prepare()
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step(steps)                   # the timed 10^4 steps
        e1.record(stream)
        torch.cuda.synchronize()
        t_tot += e0.elapsed_time(e1) / 1e3
        sim.close()
        sim = snap.from_system(s, precision="mixed")   # the same run again, sampled like the oracle's
        sim.step(burn)
        f = []
        for _ in range((steps - burn) // every):
            sim.step(every)
            f.append(sim.stats()["n_bonds"] / n_a)
        sim.close()
        f = np.array(f)
        fr.append(f.mean())
        se2.append((f.reshape(nb, -1).mean(1).std(ddof=1) / math.sqrt(nb)) ** 2)
    m, se = float(np.mean(fr)), float(math.sqrt(sum(se2)) / len(fr))
    mo = float(np.mean([g["bonded_fraction"] for g in gold["runs"]]))
    seo = float(math.sqrt(sum(g["bonded_fraction_se"] ** 2 for g in gold["runs"])) / len(gold["runs"]))
    t = max_all(t_tot)
    n = 1000 * len(gold["runs"])
    return {"workload": "A+B association: 500 A + 500 B at number density 0.1, harmonic k=100 r0=1.1, "
                        "r_max=1.3, eps=5 kT, valence 1, 10^4 steps, %d seeds" % len(gold["runs"]),
            "value": sum_all(float(n)) * steps / t, "unit": UNIT, "steps_per_s": len(gold["runs"]) * steps / t,
            "ms_per_step": t * 1e3 / (len(gold["runs"]) * steps),
            "bonded_fraction": m, "bonded_fraction_se": se, "oracle_bonded_fraction": mo, "oracle_se": seo,
            "z_vs_oracle": (m - mo) / math.sqrt(se ** 2 + seo ** 2),
            "closed_form_ideal": 0.8110,
            "note": "the ideal closed form neglects bonds carried past r_max, which break but cannot form"}


def _run_telechelic(args, torch, snap, max_all, sum_all, stream):
    """Telechelic network (2000 chains x 12 + 4000 crosslinkers, FP32 forces /
    FP64 integration): steps per second over 10^4 steps, and the bonded
    fraction of chain ends over steps 500-1000 against the stored FP64 oracle
    run (tests/golden/telechelic_network.json)."""
    from synth import telechelic
    gold = json.loads((ROOT / "tests" / "golden" / "telechelic_network.json").read_text())
    s = telechelic()
    sim = snap.from_system(s, precision="mixed")
    sim.step(gold["from"])
    f = []
    for _ in range((gold["steps"] - gold["from"]) // gold["every"]):
        sim.step(gold["every"])
        f.append(sim.stats()["n_bonds"] / gold["n_ends"])
    f = np.array(f)
    se = float(f.reshape(gold["blocks"], -1).mean(1).std(ddof=1) / math.sqrt(gold["blocks"]))
    sim.prepare()
    K = 10_000
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    t = max_all(e0.elapsed_time(e1) / 1e3)
    sim.close()
    return {"workload": "telechelic network: 2000 chains x 12 beads (FENE k=30 R0=1.5 + WCA) + 4000 X "
                        "(valence 3), ends S valence 1, bead density 0.3, S-X harmonic k=100 r0=1.0 "
                        "r_max=1.25, eps=8 kT",
            "value": sum_all(float(s.n)) * K / t, "unit": UNIT, "ms_per_step": t * 1e3 / K, "steps": K,
            "bonded_fraction_500_1000": float(f.mean()), "se": se,
            "oracle": gold["bonded_fraction"], "oracle_se": gold["bonded_fraction_se"],
            "z_vs_oracle": float((f.mean() - gold["bonded_fraction"]) /
                                 math.sqrt(se ** 2 + gold["bonded_fraction_se"] ** 2))}


def _run_competing(args, torch, snap, barrier, max_all, sum_all, stream):
    """Four reactions competing for shared sites (App. A, the mobile version of
    the Eq. Z test): A-B, A-C, D-B, D-C, valence 1, in a WCA soup; four sweep
    passes per step in an order redrawn every sweep.  Reports throughput and
    the mass-action cross ratio n_AB n_DC / (n_AC n_DB) against
    K_AB K_DC / (K_AC K_DB)."""
    from synth import four_reaction_soup
    eps = (0.5, 1.5, 1.0, 2.5)
    s = four_reaction_soup(seed=20260921, n=args.competing_n, rho=0.3, eps=eps)
    sim = snap.from_system(s, precision="mixed", block_size=128, skin=0.4)
    sim.step(max(args.warmup, 200))
    sim.prepare()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.competing_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t = max_all(e0.elapsed_time(e1) / 1e3)
    per_rx = np.zeros(4)
    for _ in range(50):   # bond counts per reaction, sampled after the timed region
        sim.step(20)
        per_rx += np.bincount(sim.bonds()[:, 2], minlength=4)
    per_rx /= 50
    sim.close()
    ab, ac, db, dc = per_rx
    return {"workload": f"four-reaction soup: {s.n} particles, A, B, C, D in equal numbers (valence 1, "
                        f"sigma 1) at number density 0.3, reactions A-B, A-C, D-B, D-C with eps {list(eps)} kT, "
                        "harmonic k=100 r0=1.1 r_max=1.3, WCA, Langevin gamma=1 dt=0.005 kT=1",
            "value": sum_all(float(s.n)) * args.competing_steps / t, "unit": UNIT,
            "ms_per_step": t * 1e3 / args.competing_steps, "steps": args.competing_steps,
            "mean_bonds_per_reaction": per_rx.tolist(),
            "cross_ratio": float(ab * dc / (ac * db)) if min(ac, db) > 0 else None,
            "cross_ratio_mass_action": math.exp(eps[0] + eps[3] - eps[1] - eps[2])}


def _segment_metrics(y, off, lab):
    """held-out listwise cross-entropy and top-1 accuracy of logits y, and of
    a uniform choice, over candidate sets off[e]..off[e+1]."""
    n = np.diff(off)
    seg = np.repeat(np.arange(len(n)), n)
    mx = np.maximum.reduceat(y, off[:-1])
    z = np.exp(y - mx[seg])
    lse = np.log(np.add.reduceat(z, off[:-1])) + mx
    ce = float(np.mean(lse - y[off[:-1] + lab]))
    top = np.maximum.reduceat(y, off[:-1])
    hit = float(np.mean(y[off[:-1] + lab] >= top))
    return {"cross_entropy": ce, "top1": hit, "uniform_cross_entropy": float(np.mean(np.log(n))),
            "uniform_top1": float(np.mean(1.0 / n)), "mean_candidates": float(n.mean())}


def _run_learned(args, torch, snap, rank, stream):
    """Learned-proposal leg on the dense gel (number density 0.8): log the
    plain method's formation events, train the BF16 network on the device,
    then run Langevin dynamics with Metropolis-Hastings bond moves under the
    uniform and the learned proposal from the same state."""
    s = build_system(args, rank_seed(20260921 + 7, rank), rho=0.8)
    sim = snap.from_system(s, precision="mixed", block_size=args.block)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    sim.step(args.warmup)
    sim.prepare()
    K = args.mh_steps
    t_plain = timed(lambda: sim.step(K))
    # log formation events of plain sweeps
    cap = args.learned_events
    sim.log_events(cap)
    logged, log_steps = 0, 0
    while logged < cap and log_steps < 20 * K:
        sim.step(50)
        log_steps += 50
        logged = sim.stats()["events_logged"]
    feat, off, lab = sim.get_events(clear=True)
    sim.log_events(0)
    E = len(lab)
    Et = int(0.9 * E)
    dX = torch.from_numpy(feat).cuda()
    doff = torch.from_numpy(off).cuda()
    dlab = torch.from_numpy(lab).cuda()
    mlp = snap.Mlp(snap.mlp_init_weights(seed=1), stream=stream.cuda_stream)
    losses = None

    def train():
        nonlocal losses
        losses = mlp.train(dX.data_ptr(), int(off[Et]), doff.data_ptr(), dlab.data_ptr(), Et,
                           epochs=args.learned_epochs, batch_events=4096, lr=1e-3, seed=2)
    t_train = timed(train)
    rows_h = int(off[E] - off[Et])
    yh = torch.empty(max(rows_h, 1), device="cuda")
    t_fwd = timed(lambda: mlp.forward(dX.data_ptr() + 4 * 12 * int(off[Et]), rows_h, yh.data_ptr()))
    held = _segment_metrics(yh[:rows_h].cpu().numpy().astype(np.float64),
                            (off[Et:] - off[Et]).astype(np.int64), lab[Et:].astype(np.int64))
    rows_train = int(off[Et]) * args.learned_epochs
    # forward 2 (16x64 + 64x64 + 64) flops per row; backward twice that
    flops_row = 3 * 2 * (16 * 64 + 64 * 64 + 64)
    state = sim.get_state()
    mh = {}
    for mode, name in ((1, "uniform"), (2, "learned")):
        sim.set_state(state)
        sim.set_mh(mode, mlp if mode == 2 else None, eps_u=0.05)
        sim.step(50)
        sim.prepare()
        st0 = sim.stats()
        h0 = sim.lifetime_hist()
        t_mh = timed(lambda: sim.step(K))
        series = []
        for _ in range(20):
            sim.step(50)
            series.append(sim.stats()["n_bonds"])
        st1 = sim.stats()
        hist = (sim.lifetime_hist() - h0).astype(np.float64)
        d = {k: st1["mh_" + k] - st0["mh_" + k]
             for k in ("form_attempts", "form_accepts", "break_attempts", "break_accepts")}
        ser = np.array(series, float)
        blocks = ser.reshape(10, -1).mean(1)
        mh[name] = {"ms_per_step": t_mh * 1e3 / K,
                    "value": s.n * K / t_mh,
                    "accepted_per_attempt": (d["form_accepts"] + d["break_accepts"]) /
                                            max(1, d["form_attempts"] + d["break_attempts"]),
                    **d, "n_bonds_mean": float(ser.mean()),
                    "n_bonds_se": float(blocks.std(ddof=1) / math.sqrt(len(blocks))),
                    "mean_lifetime_steps": float((hist * np.arange(len(hist))).sum() / max(1.0, hist.sum())),
                    "broken_bonds": int(hist.sum()), "_hist": hist}
        sim.set_mh(0)
    hu, hl = mh["uniform"].pop("_hist"), mh["learned"].pop("_hist")
    hell = None
    if hu.sum() > 0 and hl.sum() > 0:
        hell = float(np.sqrt(0.5 * np.sum((np.sqrt(hu / hu.sum()) - np.sqrt(hl / hl.sum())) ** 2)))
    sim.close()
    mlp.close()
    return {"workload": f"dense colloid-linker gel, {s.n} particles at number density 0.8 "
                        "(types, bonds and eps as the headline gel)",
            "plain_ms_per_step": t_plain * 1e3 / K,
            "events": E, "events_train": Et, "log_steps": log_steps,
            "train": {"epochs": args.learned_epochs, "batch_events": 4096, "seconds": t_train,
                      "rows_per_s": rows_train / t_train, "tflops": rows_train * flops_row / t_train / 1e12,
                      "loss_first_epoch": float(losses[0]), "loss_last_epoch": float(losses[-1])},
            "forward_rows_per_s": rows_h / t_fwd if t_fwd > 0 else None,
            "held_out": held, "mh": mh, "lifetime_hellinger_uniform_vs_learned": hell,
            "eps_u": 0.05}


def _run_snap_on_stream(args, torch, dist, snap, rank, world, dev_index, barrier, max_all, sum_all,
                        stream, batch=None):
    s = build_system(args, rank_seed(20260921, rank))
    n = s.n
    K, W = args.steps, args.warmup
    # a fixed untimed equilibration (bonds form from the bond-free start); its
    # end state is where the launch shape and skin are tuned and timing starts
    E = args.equil_steps
    eq = snap.from_system(s, precision="mixed", block_size=args.block or 128, skin=args.skin or 0.5)
    eq.step(E)
    state = eq.get_state()
    eq_check = None
    if rank == 0 and not args.no_cpu_baseline:
        # the equilibrated state and the GPU's forces there, both precisions, for the
        # comparison with the FP64 oracle in the CPU-baseline leg
        eq_check = dict(pos=eq.positions(), vel=eq.velocities(), bonds=eq.bonds(), step=eq.stats()["step"],
                        f_mixed=eq.forces())
        e64 = snap.from_system(s, precision="fp64", block_size=args.block or 128, skin=args.skin or 0.5)
        e64.set_state(state)
        eq_check["f_fp64"] = e64.forces()
        e64.close()
        e1 = snap.from_system(s, precision="mixed", block_size=args.block or 128, skin=args.skin or 0.5)
        e1.set_state(state)
        e1.bond_update()                  # one sweep at the equilibrated state, step counter unchanged
        eq_check["bonds_after_sweep"] = e1.bonds()
        eq_check["sweep_stats"] = e1.stats()
        e1.close()
    eq.close()
    if args.block or args.skin or args.subcells >= 0:
        tune = {"block_size": args.block or 128, "skin": args.skin or s.skin, "cached": None,
                "key": "set by flags", "list_subcells": max(args.subcells, 0)}
    else:
        from paper_2609_21204_b300 import autotune
        tune = autotune.autotune(s, precision="mixed", blocks=(128, 256), skins=(0.3, 0.35, 0.4, 0.45, 0.5, 0.6),
                                 steps=200, warmup=40, state=state)

    def make(precision):
        return snap.from_system(s, precision=precision, block_size=tune["block_size"], skin=tune["skin"],
                                list_block=tune.get("list_block"), list_subcells=tune.get("list_subcells"))

    sim = make("mixed")
    subcells = sim.list_subcells()
    # the equilibrated state, the warm-up, then the step graphs of both buffer
    # parities are captured and uploaded so that no capture falls inside the
    # timed region
    sim.set_state(state)
    sim.step(W)
    sim.prepare()
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
    reb = [sim.rebuild_profiled() for _ in range(3)]
    rebuild_ms = {k: round(float(np.mean([r[k] for r in reb])), 5) for k in reb[0]}
    st2 = sim.stats()
    nbar = st2["nlist_entries"] / n
    md_ms = ph["md"]
    # algorithmic bytes per particle of the fused force + Langevin kernel (mixed
    # precision, one system: no replica ids).  Force part: own pos4 16, count 4,
    # 4 per neighbour index, dynamic slots 16 + 4 (static slots 16 + 4 when there
    # are static bonds).  Langevin part: tag 4, velocity 16, FP64 position 24 and
    # reference position 16 read; FP64 position 24, velocity 16 and the new
    # relative coordinate 16 written.  Neighbours' coordinates are the same pos4
    # array and count once.
    bytes_pp = (16 + 4 + 4 * nbar + 20 + (20 if len(s.static_bonds) else 0)) + (4 + 16 + 24 + 16) + (24 + 16 + 16)
    alg_bytes = bytes_pp * n
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (md_ms / 1e3) / 1e9
    traffic = md_traffic_from_profile(n)
    sweep_pairs = st2["scanned"] + st2["break_tested"]
    bond_pairs_per_s = sweep_pairs / (ph["sweep"] / 1e3) if ph["sweep"] > 0 else None
    # algorithmic bytes of one sweep: per particle the availability pass (type 4, occupancy 4,
    # availability 1), the breaking draws (partner slots 16, reactions 4, tag 4) and the apply
    # phase (break bits 4, formed partner 4, best key 8 + 8, proposal 4, push key 16, slots 16);
    # per neighbour entry scanned by a free site: index 4, availability 1, coordinates 16
    sweep_bytes = (9 + 24 + 60) * n + 21 * st2["scanned"]
    sweep_gbs = sweep_bytes / (ph["sweep"] / 1e3) / 1e9 if ph["sweep"] > 0 else None

    # kernels launched: per step the rebuild condition (which also ends the step
    # before it), the sweep (begin + 4 per reaction: proposals and break draws,
    # resolution, acceptance, apply) and the fused force + Langevin kernel; one
    # step end per 20-step graph; per rebuild 8 more (cell keys, 2 scan kernels,
    # scatter, cell sort, gather, lists with the copy back, done)
    builds = st1["nlist_builds"] - st0["nlist_builds"]
    launches = K * (2 + 1 + 4 * len(s.reactions)) + -(-K // 20) + 8 * builds

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": t_max * 1e3 / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": dict(workload_config(args, n), block_size=tune["block_size"], skin=tune["skin"],
                       list_block=tune.get("list_block") or 256, list_subcells=subcells),
        "autotune": {k: tune.get(k) for k in ("block_size", "skin", "list_block", "list_subcells", "cached", "key",
                                              "ms_per_step")},
        "gpu_launches": launches,
        "clocks": clk,
        "phases_ms_per_step": {k: round(v, 5) for k, v in ph.items()},
        "rebuild_ms_per_kernel": rebuild_ms,
        "bond_update_pairs_per_s": bond_pairs_per_s,
        "sweep_roofline": {"bound": "hbm", "algorithmic_bytes_per_sweep": sweep_bytes, "achieved": sweep_gbs,
                           "peak": measured_peaks()[0], "unit": "GB/s",
                           "frac": sweep_gbs / measured_peaks()[0] if sweep_gbs else None,
                           "sweep_ms": ph["sweep"], "note": "five kernels per sweep, each latency-bound"},
        "state_at_timing": {"equilibration_steps": E, "warmup_steps": W, "n_bonds": st0["n_bonds"],
                            "colloid_slot_occupancy": st0["n_bonds"] / (4.0 * args.n_c),
                            "graphs": "captured and uploaded for both buffer parities before the timed region"},
        "sweep": {"scanned_nlist_entries": st2["scanned"], "break_tested": st2["break_tested"],
                  "proposals": st2["proposals"], "formed": st2["formed"], "broken": st2["broken"],
                  "n_bonds": st2["n_bonds"], "mean_neighbours": nbar,
                  "nlist_builds_in_timed_region": st1["nlist_builds"] - st0["nlist_builds"]},
        "roofline": {"kernel": "k_step_md (mixed precision: pair + bond forces, Langevin update)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_kind, "traffic": traffic,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "launch_ms": md_ms},
    }
    if not args.no_fp64:
        sim.close()

        def fp64_leg():
            sim64 = make("fp64")
            try:
                sim64.set_state(state)
                sim64.step(W)
                sim64.prepare()
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
                pos64 = sim64.positions()
            finally:
                sim64.close()
            out["speedup_mixed_vs_fp64_plain"] = value / v64
            # the FP64 force + Langevin kernel is bound by the FP64 pipe, not HBM:
            # algorithmic FP64 FLOPs per particle, counted from the kernel's
            # operations (per list entry 14 for the separation and r^2, per pair
            # inside the cut 15 for the WCA force and its accumulation; per dynamic
            # bond end 24; 47 for the Langevin update and the relative coordinate),
            # against the FP64 rate of cuBLAS DGEMM on this GPU, measured here
            nb_dyn = 2.0 * st2["n_bonds"] / n
            frac_in = inside_cut_fraction(s, pos64, nbar)
            flop_pp = 14 * nbar + 15 * nbar * (frac_in or 0.0) + 24 * nb_dyn + 47
            md64_ms = ph64["md"]
            achieved = flop_pp * n / (md64_ms / 1e3) / 1e12
            peak64 = fp64_dgemm_tflops(torch)
            return {"value": v64, "ms_per_step": t64 * 1e3 / K64, "steps": K64,
                    "phases_ms_per_step": {k: round(v, 5) for k, v in ph64.items()},
                    "roofline": {"kernel": "k_step_md_fp64", "bound": "fp64", "achieved": achieved,
                                 "peak": peak64, "unit": "TFLOP/s",
                                 "frac": achieved / peak64 if peak64 else None,
                                 "flop_per_particle": flop_pp, "inside_cut_fraction": frac_in,
                                 "peak_source": "cuBLAS DGEMM 8192^3 on this GPU (torch.matmul, FP64), best of 3"}}

        run_leg(out, "fp64_plain", world, fp64_leg)
        sim = make("mixed")
        sim.set_state(state)
    if batch is not None:
        sim.close()
        run_leg(out, "batched", world,
                lambda: _run_batched(args, torch, snap, batch, barrier, max_all, sum_all, stream))
        sim = make("mixed")
        sim.set_state(state)
    if args.small_legs:
        sim.close()
        run_leg(out, "assoc_ab", world, lambda: _run_assoc_ab(args, torch, snap, max_all, sum_all, stream))
        run_leg(out, "telechelic", world, lambda: _run_telechelic(args, torch, snap, max_all, sum_all, stream))
        sim = make("mixed")
        sim.set_state(state)
    if args.competing_n > 0:
        sim.close()
        run_leg(out, "competing", world,
                lambda: _run_competing(args, torch, snap, barrier, max_all, sum_all, stream))
        sim = make("mixed")
        sim.set_state(state)
    if args.learned_events > 0:
        sim.close()
        run_leg(out, "learned", world, lambda: _run_learned(args, torch, snap, rank, stream))
        sim = make("mixed")
        sim.set_state(state)
    if not args.no_e2e:
        # end to end through the C ABI with host buffers in pinned memory: every
        # step uploads positions + velocities, runs one step and reads the
        # positions back
        pin = lambda: torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
        pos, vel = pin(), pin()
        sim.positions(out=pos)
        sim.velocities(out=vel)
        n_e2e = args.e2e_steps
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            sim.set_positions(pos, vel)
            sim.step(1)
            sim.positions(out=pos)
        torch.cuda.synchronize()
        te = max_all(time.perf_counter() - t0)
        out["e2e"] = {"value": n_all * n_e2e / te, "unit": UNIT, "h2d_bytes_per_step": 48 * n,
                      "d2h_bytes_per_step": 24 * n, "steps": n_e2e,
                      "what": "per step from pinned host buffers: snap_set_positions (positions + "
                              "velocities), snap_step(1) (the new positions force a list rebuild), "
                              "snap_get_positions (to host)"}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        o = oracle.OracleSystem(s)
        # the oracle at the GPU's equilibrated state: its forces against the GPU's in both
        # precisions, and one sweep against the GPU's sweep there (untimed)
        o.set_positions(eq_check["pos"])
        o.set_velocities(eq_check["vel"])
        o.set_bonds(eq_check["bonds"])
        o.step = int(eq_check["step"])
        f_o, e_o = o.forces()
        errs = {}
        for prec in ("mixed", "fp64"):
            d = np.linalg.norm(eq_check["f_" + prec] - f_o, axis=1)
            sc = e_o["fscale"]
            errs[prec] = {"normwise": float(np.linalg.norm(d) / np.linalg.norm(f_o)),
                          "max_per_particle_vs_sensitivity_scale": float(np.max(d[sc > 0] / sc[sc > 0]))}
        st_o = o.sweep(step=o.step)
        gs = eq_check["sweep_stats"]
        out["oracle_check"] = {
            "state": f"the equilibrated gel after {E} steps ({int(eq_check['bonds'].shape[0])} bonds)",
            "forces": errs, "force_tolerance": {"mixed": 1e-5, "fp64": 1e-12},
            "sweep_bit_exact": bool(np.array_equal(eq_check["bonds_after_sweep"], o.bonds()) and
                                    all(gs[k] == st_o[k] for k in ("in_window", "proposals", "edges", "survivors",
                                                                   "formed", "break_tested", "broken"))),
            "sweep_counters": {k: int(st_o[k]) for k in ("proposals", "formed", "broken")}}
        t0 = time.perf_counter()
        o.run(args.cpu_steps)
        tc = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": n * args.cpu_steps / tc, "unit": UNIT, "cores": 1,
                               "kind": "oracle",
                               "sample": f"{args.cpu_steps} full MD steps (sweep, forces, Langevin) "
                                         f"of the same {n}-particle gel from its equilibrated state, "
                                         "single thread, FP64"}
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
