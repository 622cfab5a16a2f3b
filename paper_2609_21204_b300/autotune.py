"""Autotuner for the launch shapes and neighbour-list skin of a context.

Candidates (threads per block for the particle kernels x neighbour-list skin,
then the list build's threads per block and its sub-cells along x per cell
at the best of those) are timed on
the caller's own system with CUDA events over a short run after a
warm-up; the fastest is returned and cached in a JSON file keyed by the GPU
name, the precision mode, the particle count (rounded to a power of two), the
number density (rounded to 0.05) and the number of replicas.  Block size does
not change results (every kernel is deterministic in its launch shape); the
skin changes when the neighbour list is rebuilt and therefore the rounding of
a trajectory, not its physics.
"""
from __future__ import annotations

import json
import math
import os
from pathlib import Path

DEFAULT_CACHE = Path(os.environ.get("SNAP_AUTOTUNE_CACHE",
                                    Path.home() / ".cache" / "snap_b300" / "autotune.json"))
BLOCKS = (64, 128, 256)
SKINS = (0.25, 0.3, 0.4)
LIST_BLOCKS = (128, 256, 64)   # the list build's block size, searched at the best (block, skin)
LIST_SUBCELLS = (0, 8, 2)      # its sub-cells along x per cell (0: the library's choice), searched after it


def cache_key(gpu_name: str, precision: str, n: int, density: float, n_replicas: int) -> str:
    nb = 1 << max(0, int(round(math.log2(max(n, 1)))))
    rho = round(round(density / 0.05) * 0.05, 2)
    return f"{gpu_name}|{precision}|N~{nb}|rho~{rho}|rep{n_replicas}"


def load_cache(path: Path = DEFAULT_CACHE) -> dict:
    try:
        return json.loads(Path(path).read_text())
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: Path = DEFAULT_CACHE) -> None:
    p = Path(path)
    p.parent.mkdir(parents=True, exist_ok=True)
    tmp = p.with_suffix(f".{os.getpid()}.tmp")
    tmp.write_text(json.dumps(cache, indent=1, sort_keys=True))
    os.replace(tmp, p)


def choose(trials):
    """trials: list of (config dict, ms per step); the fastest config, ties to
    the earlier trial."""
    best = None
    for cfg, ms in trials:
        if ms is None or not math.isfinite(ms):
            continue
        if best is None or ms < best[1]:
            best = (cfg, ms)
    if best is None:
        raise RuntimeError("no autotune trial succeeded")
    return dict(best[0], ms_per_step=best[1])


def autotune(systems, precision="mixed", blocks=BLOCKS, skins=SKINS, steps=60, warmup=30,
             cache_path: Path = DEFAULT_CACHE, use_cache=True, timer=None, state=None, list_blocks=LIST_BLOCKS,
             list_subcells=LIST_SUBCELLS):
    """Pick (block_size, skin, list_block, list_subcells) for these systems.  `systems` is one synth
    System or a list of them (a batched context).  `state` (bytes from
    Snap.get_state of a context over the same systems) starts every trial from
    that state instead of the systems' own coordinates, so that the choice is
    made in the regime that will be run (e.g. an equilibrated gel rather than
    its bond-free start).  `timer(cfg) -> ms/step` may replace the GPU timing
    (used by the host-side tests)."""
    systems = systems if isinstance(systems, (list, tuple)) else [systems]
    n = sum(s.n for s in systems)
    vol = sum(float(s.box[0] * s.box[1] * s.box[2]) for s in systems)
    gpu = "cpu"
    if timer is None:
        import torch
        gpu = torch.cuda.get_device_name()
    key = cache_key(gpu, precision, n, n / vol, len(systems))
    cache = load_cache(cache_path) if use_cache else {}
    if use_cache and key in cache:
        return dict(cache[key], cached=True, key=key)
    if timer is None:
        timer = _gpu_timer(systems, precision, steps, warmup, state)
    def timed(cfg):
        try:
            return timer(cfg)
        except Exception:
            return None

    lb0 = int(list_blocks[0]) if list_blocks else 256
    ls0 = int(list_subcells[0]) if list_subcells else 0
    trials = []
    for skin in skins:
        for block in blocks:
            cfg = dict(block_size=int(block), skin=float(skin), list_block=lb0, list_subcells=ls0)
            trials.append((cfg, timed(cfg)))
    best = choose(trials)
    # the list build's block size, then its sub-cells, at the best (block, skin)
    for lb in list(list_blocks)[1:]:
        cfg = dict(block_size=best["block_size"], skin=best["skin"], list_block=int(lb), list_subcells=ls0)
        trials.append((cfg, timed(cfg)))
    best = choose(trials)
    for ls in list(list_subcells)[1:]:
        cfg = dict(block_size=best["block_size"], skin=best["skin"], list_block=best["list_block"],
                   list_subcells=int(ls))
        trials.append((cfg, timed(cfg)))
    best = choose(trials)
    best["trials"] = [dict(c, ms_per_step=m) for c, m in trials]
    if use_cache:
        cache[key] = best
        save_cache(cache, cache_path)
    return dict(best, cached=False, key=key)


def _gpu_timer(systems, precision, steps, warmup, state=None):
    import torch
    from . import from_system

    def run(cfg):
        sim = from_system(systems if len(systems) > 1 else systems[0], precision=precision,
                          block_size=cfg["block_size"], skin=cfg["skin"], list_block=cfg.get("list_block"),
                          list_subcells=cfg.get("list_subcells"))
        try:
            if state is not None:
                sim.set_state(state)
            sim.step(warmup)
            sim.prepare()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            stream = torch.cuda.current_stream()
            torch.cuda.synchronize()
            e0.record(stream)
            sim.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / steps
        finally:
            sim.close()
    return run
