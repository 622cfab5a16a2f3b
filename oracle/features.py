"""Pair features of the learned proposal, and the bond-formation events a plain
sweep yields for training it — TEST INFRASTRUCTURE (plain NumPy, brute force
over all particles; only the tests and the entry point's smoke check use it).

The learned proposal is an extension beyond the paper (the paper's sweep,
Sec. II.C, proposes the partner closest to the bond rest length).  For a site
i of reaction a = (type_a, type_b, r_min, r_max) and a candidate j the twelve
features are

  0  r_ij                       6  occ_i / max(v_i, 1)
  1  (r_ij - r0) / r_max         7  occ_j / max(v_j, 1)
  2  [type_i == type_a]          8  [occ_i < v_i]
  3  [type_i == type_b]          9  [occ_j < v_j]
  4  [type_j == type_a]         10  coord_i / 8
  5  [type_j == type_b]         11  coord_j / 8

with coord_x the number of particles of x's partner type inside x's
formation window r_min <= r <= r_max.  Candidates of i are the particles of
the compatible type that are free (occ < valence), not bonded to i and inside
the window (squared distance in FP64 with the minimum image, as in the sweep),
in ascending tag order.  Values are rounded to float32 at the end, each from
its FP64 (or exact integer) value.
"""
from __future__ import annotations

import numpy as np

NF = 12
MAX_CAND = 16


def dist2_from(pos, box, i):
    """Squared minimum-image distances from particle i to every particle:
    d = x_j - x_i; d -= L rint(d / L) (with 1/L precomputed);
    r^2 = (dx^2 + dy^2) + dz^2, each operation rounded once in FP64."""
    d = pos - pos[i]
    inv = 1.0 / np.asarray(box, dtype=np.float64)
    d = d - np.asarray(box) * np.rint(d * inv)
    return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]


class FeatureState:
    """Positions, types and the bond table (partners by tag) at one instant."""

    def __init__(self, pos, box, types, valence, partners, reaction, r0):
        self.pos = np.asarray(pos, dtype=np.float64)
        self.box = np.asarray(box, dtype=np.float64)
        self.types = np.asarray(types)
        self.valence = np.asarray(valence)
        self.partners = [set(int(p) for p in row if p >= 0) for row in partners]
        self.occ = np.array([len(p) for p in self.partners])
        self.ta, self.tb = reaction.type_a, reaction.type_b
        self.rmin2 = reaction.r_min * reaction.r_min
        self.rmax2 = reaction.r_max * reaction.r_max
        self.r0 = r0

    def partner_type(self, t):
        return self.tb if t == self.ta else self.ta

    def in_window(self, r2):
        return (r2 >= self.rmin2) & (r2 <= self.rmax2)

    def coord(self, x):
        r2 = dist2_from(self.pos, self.box, x)
        m = (self.types == self.partner_type(self.types[x])) & self.in_window(r2)
        m[x] = False
        return int(m.sum())

    def candidates(self, i):
        """(tags ascending, separations r) of i's candidates."""
        ti = self.types[i]
        r2 = dist2_from(self.pos, self.box, i)
        compat = ((ti == self.ta) & (self.types == self.tb)) | ((ti == self.tb) & (self.types == self.ta))
        free = self.occ < self.valence[self.types]
        m = compat & free & self.in_window(r2)
        m[i] = False
        for p in self.partners[i]:
            m[p] = False
        idx = np.nonzero(m)[0]
        return idx, np.sqrt(r2[idx])

    def features(self, i, j, r, coord_i, coord_j):
        ti, tj = self.types[i], self.types[j]
        vi, vj = max(int(self.valence[ti]), 1), max(int(self.valence[tj]), 1)
        rmax = np.sqrt(self.rmax2)
        f = np.zeros(NF, dtype=np.float32)
        f[0] = np.float32(r)
        f[1] = np.float32((r - self.r0) / rmax)
        f[2] = ti == self.ta
        f[3] = ti == self.tb
        f[4] = tj == self.ta
        f[5] = tj == self.tb
        f[6] = np.float32(self.occ[i]) / np.float32(vi)
        f[7] = np.float32(self.occ[j]) / np.float32(vj)
        f[8] = self.occ[i] < self.valence[ti]
        f[9] = self.occ[j] < self.valence[tj]
        f[10] = np.float32(coord_i) * np.float32(0.125)
        f[11] = np.float32(coord_j) * np.float32(0.125)
        return f

    def event(self, i, j):
        """Feature rows of all of i's candidates and the index of j among
        them, or None when i has no candidate, more than 16, or j is not one."""
        idx, r = self.candidates(i)
        if len(idx) == 0 or len(idx) > MAX_CAND or j not in idx:
            return None
        ci = self.coord(i)
        rows = np.stack([self.features(i, int(q), float(rq), ci, self.coord(int(q))) for q, rq in zip(idx, r)])
        return rows, int(np.nonzero(idx == j)[0][0])


def sweep_events(state: FeatureState, prop, matched, formed):
    """Events of one plain sweep from its trace: every site whose own
    proposal became a bond (prop[i] = matched[i], formed[i]) contributes the
    features of its candidates in the state before the sweep."""
    out = []
    for i in range(len(prop)):
        j = int(prop[i])
        if j < 0 or not formed[i] or int(matched[i]) != j:
            continue
        ev = state.event(i, j)
        if ev is not None:
            out.append(ev)
    return out
