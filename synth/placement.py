"""Seeded geometric placement of particles in a periodic orthorhombic box.

This module only builds input coordinates (random sequential addition with a
cell grid, random-walk chains).  It contains none of the dynamic-bonding
arithmetic; both the CPU oracle and the CUDA path receive its output as input.
"""
from __future__ import annotations

import numpy as np


def _cell_ids(pos: np.ndarray, box: np.ndarray, ncell: np.ndarray) -> np.ndarray:
    c = np.floor(pos / box * ncell).astype(np.int64)
    c %= ncell
    return (c[:, 2] * ncell[1] + c[:, 1]) * ncell[0] + c[:, 0]


class _Grid:
    """Placed points sorted by cell id, queried for all points in the 27 cells
    around a set of probe points (vectorised, variable-length ranges)."""

    def __init__(self, box, cell_size):
        self.box = np.asarray(box, dtype=np.float64)
        self.ncell = np.maximum(np.floor(self.box / cell_size).astype(np.int64), 1)
        self.pos = np.zeros((0, 3))
        self.rad = np.zeros(0)
        self._sorted_ids = np.zeros(0, dtype=np.int64)
        self._order = np.zeros(0, dtype=np.int64)
        offs = np.array([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1)
                         for dx in (-1, 0, 1)], dtype=np.int64)
        # with fewer than 3 cells along an axis the 27 offsets alias; dedupe per axis
        self._offsets = offs

    def insert(self, pos, rad):
        self.pos = np.concatenate([self.pos, pos])
        self.rad = np.concatenate([self.rad, rad])
        ids = _cell_ids(self.pos, self.box, self.ncell)
        self._order = np.argsort(ids, kind="stable")
        self._sorted_ids = ids[self._order]

    def conflicts(self, pos, rad, factor):
        """Boolean per probe: True if any placed point lies closer than
        factor * (rad_probe + rad_placed)."""
        m = pos.shape[0]
        bad = np.zeros(m, dtype=bool)
        if self.pos.shape[0] == 0 or m == 0:
            return bad
        nc = self.ncell
        c = np.floor(pos / self.box * nc).astype(np.int64) % nc
        seen = set()
        for off in self._offsets:
            key = tuple(int(o) % int(n) if n < 3 else int(o) for o, n in zip(off, nc))
            if key in seen:
                continue
            seen.add(key)
            cc = (c + off) % nc
            cid = (cc[:, 2] * nc[1] + cc[:, 1]) * nc[0] + cc[:, 0]
            lo = np.searchsorted(self._sorted_ids, cid, side="left")
            hi = np.searchsorted(self._sorted_ids, cid, side="right")
            cnt = hi - lo
            tot = int(cnt.sum())
            if tot == 0:
                continue
            probe = np.repeat(np.arange(m), cnt)
            start = np.repeat(lo - np.concatenate([[0], np.cumsum(cnt)[:-1]]), cnt)
            idx = self._order[start + np.arange(tot)]
            d = self.pos[idx] - pos[probe]
            d -= self.box * np.rint(d / self.box)
            r2 = np.einsum("ij,ij->i", d, d)
            lim = factor * (rad[probe] + self.rad[idx])
            hit = r2 < lim * lim
            if hit.any():
                bad[np.unique(probe[hit])] = True
        return bad


def rsa(rng: np.random.Generator, box, radii: np.ndarray, factor: float = 1.0,
        grid: _Grid | None = None, batch: int = 65536, max_rounds: int = 10000):
    """Random sequential addition of spheres with the given radii (placed in the
    given order) so that no two centres are closer than factor*(r_i + r_j).
    Returns (positions, grid)."""
    box = np.asarray(box, dtype=np.float64)
    radii = np.asarray(radii, dtype=np.float64)
    cell = 2.0 * factor * max(float(radii.max()) if radii.size else 0.5,
                              float(grid.rad.max()) if grid is not None and grid.rad.size else 0.0)
    if grid is None:
        grid = _Grid(box, max(cell, 1e-3))
    out = np.empty((radii.size, 3))
    todo = np.arange(radii.size)
    rounds = 0
    while todo.size:
        rounds += 1
        if rounds > max_rounds:
            raise RuntimeError("random sequential addition did not converge")
        take = todo[:batch]
        cand = rng.random((take.size, 3)) * box
        ok = ~grid.conflicts(cand, radii[take], factor)
        # resolve conflicts inside the batch: a candidate loses to any lower-index survivor
        sub = np.nonzero(ok)[0]
        if sub.size > 1:
            # pairwise check within the batch through a grid of the batch survivors
            g2 = _Grid(box, max(cell, 1e-3))
            g2.insert(cand[sub], radii[take[sub]])
            ok[sub[_later_conflicts(g2, cand[sub], radii[take[sub]], factor)]] = False
        acc = np.nonzero(ok)[0]
        out[take[acc]] = cand[acc]
        grid.insert(cand[acc], radii[take[acc]])
        todo = np.concatenate([take[~ok], todo[batch:]])
    return out, grid


def _later_conflicts(g: _Grid, pos, rad, factor):
    """For points already inserted in g (in insertion order), flag every point
    that conflicts with some point of lower insertion index."""
    m = pos.shape[0]
    bad = np.zeros(m, dtype=bool)
    nc = g.ncell
    c = np.floor(pos / g.box * nc).astype(np.int64) % nc
    seen = set()
    for off in g._offsets:
        key = tuple(int(o) % int(n) if n < 3 else int(o) for o, n in zip(off, nc))
        if key in seen:
            continue
        seen.add(key)
        cc = (c + off) % nc
        cid = (cc[:, 2] * nc[1] + cc[:, 1]) * nc[0] + cc[:, 0]
        lo = np.searchsorted(g._sorted_ids, cid, side="left")
        hi = np.searchsorted(g._sorted_ids, cid, side="right")
        cnt = hi - lo
        tot = int(cnt.sum())
        if tot == 0:
            continue
        probe = np.repeat(np.arange(m), cnt)
        start = np.repeat(lo - np.concatenate([[0], np.cumsum(cnt)[:-1]]), cnt)
        idx = g._order[start + np.arange(tot)]
        sel = idx < probe
        probe, idx = probe[sel], idx[sel]
        d = g.pos[idx] - pos[probe]
        d -= g.box * np.rint(d / g.box)
        r2 = np.einsum("ij,ij->i", d, d)
        lim = factor * (rad[probe] + g.rad[idx])
        hit = r2 < lim * lim
        if hit.any():
            bad[np.unique(probe[hit])] = True
    return bad


def random_walk_chains(rng: np.random.Generator, box, n_chains: int, beads: int,
                       bond: float = 0.97, min_dist: float = 0.8, grid: _Grid | None = None,
                       bead_radius: float = 0.5):
    """Grow n_chains linear chains bead by bead as random walks with fixed bond
    length, rejecting steps closer than min_dist to any non-adjacent bead.
    Returns positions (n_chains*beads, 3) with chain c occupying rows
    [c*beads, (c+1)*beads), and the grid of placed beads (radius bead_radius)."""
    box = np.asarray(box, dtype=np.float64)
    factor = min_dist / (2.0 * bead_radius)
    if grid is None:
        grid = _Grid(box, max(min_dist, 1e-3))
    pos = np.empty((n_chains, beads, 3))
    rad = np.full(n_chains, bead_radius)
    # first beads: plain random sequential addition
    first, _ = rsa(rng, box, rad, factor=factor, grid=grid)
    pos[:, 0] = first
    for b in range(1, beads):
        todo = np.arange(n_chains)
        tries = 0
        while todo.size:
            tries += 1
            if tries > 3000:
                raise RuntimeError("chain growth stuck")
            # a chain end boxed in by its neighbours gets a slightly relaxed
            # excluded-volume distance (down to 0.9 of min_dist, still WCA-stable
            # at dt = 0.005) instead of stalling
            f_eff = factor * max(0.9, 0.97 ** max(0, (tries - 200) // 100))
            v = rng.normal(size=(todo.size, 3))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            cand = (pos[todo, b - 1] + bond * v) % box
            # the previous bead of the same chain sits at exactly `bond`; it is
            # closer than min_dist only if bond < min_dist, which is not used here
            ok = ~grid.conflicts(cand, rad[todo], f_eff)
            sub = np.nonzero(ok)[0]
            if sub.size > 1:
                g2 = _Grid(box, max(min_dist, 1e-3))
                g2.insert(cand[sub], rad[todo[sub]])
                ok[sub[_later_conflicts(g2, cand[sub], rad[todo[sub]], f_eff)]] = False
            acc = np.nonzero(ok)[0]
            pos[todo[acc], b] = cand[acc]
            grid.insert(cand[acc], rad[todo[acc]])
            todo = todo[~ok]
    return pos.reshape(-1, 3), grid
