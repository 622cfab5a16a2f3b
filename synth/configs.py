"""Seeded synthetic workloads for the dynamic-bonding MD hot path.

Each builder returns a `System`: plain parameter values (σ per type, valence per
type, bond stiffness/rest length, reaction cut-offs and the bond free energy ε
in units of kT) and the initial coordinates, velocities, types and static bonds.
Converting ε into per-sweep probabilities, and everything else the method
computes, is left to the consumer (the CUDA path or the oracle).

Units are reduced: σ = 1 for the reference species, m = 1 for every particle.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

from .placement import rsa, random_walk_chains

HARMONIC = 0
FENE = 1
FENEWCA = 2
TETHER = 3


@dataclass
class Reaction:
    type_a: int
    type_b: int
    bond_type: int
    r_min: float
    r_max: float
    eps: float            # bond free energy in kT (the paper's ε = ln K)
    self_avoid: int = 0
    slip_a: float = 0.0   # slip-bond parameter a of Eq. (slip); 0: constant P_off
    melt: tuple | None = None   # melting switch, Eqs. (gT)-(kT): (lambda, T_melt, k_on^init,
                                # k_off^init, k_on^melt, k_off^melt); rates replace eps


@dataclass
class BondType:
    kind: int             # HARMONIC, FENE, FENEWCA or TETHER
    k: float              # k (k_b for TETHER)
    r0: float             # rest length (harmonic), maximum extension R0 (FENE, FENEWCA), l_min (TETHER)
    extra: tuple = ()     # FENEWCA: (eps, sigma, delta); TETHER: (l_c1, l_c0, l_max)


@dataclass
class System:
    name: str
    box: np.ndarray                  # (3,) float64
    type_names: list
    sigma: np.ndarray                # (ntypes,) float64
    valence: np.ndarray              # (ntypes,) int32
    eps_pair: np.ndarray             # (ntypes, ntypes) float64
    rcut: np.ndarray | None          # (ntypes, ntypes) or None = WCA
    bond_types: list
    reactions: list
    pos: np.ndarray                  # (n, 3) float64, wrapped into [0, L)
    vel: np.ndarray                  # (n, 3) float64
    types: np.ndarray                # (n,) int32
    static_bonds: np.ndarray         # (nb, 2) int32 tags
    static_bond_types: np.ndarray    # (nb,) int32
    kT: float = 1.0
    gamma: float = 1.0
    dt: float = 0.005
    seed: int = 20260921
    bond_period: int = 1
    kinetic_T: int = 0      # 1: the sweep uses the instantaneous kinetic temperature (Sec. II.B)
    skin: float = 0.3
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _velocities(rng, n, kT):
    v = rng.normal(scale=math.sqrt(kT), size=(n, 3))
    v -= v.mean(axis=0, keepdims=True)
    return v


def assoc_ab(seed: int = 20260921, n_a: int = 500, n_b: int = 500, rho: float = 0.1,
             eps: float = 5.0, k: float = 100.0, r0: float = 1.1, r_max: float = 1.3,
             kT: float = 1.0) -> System:
    """A + B association: monovalent A and B (σ = 1) placed at random without
    overlap in a periodic cube at number density rho; dynamic harmonic A–B bonds."""
    rng = np.random.default_rng(seed)
    n = n_a + n_b
    L = (n / rho) ** (1.0 / 3.0)
    box = np.array([L, L, L])
    pos, _ = rsa(rng, box, np.full(n, 0.5), factor=1.0)
    types = np.concatenate([np.zeros(n_a, np.int32), np.ones(n_b, np.int32)])
    return System(
        name="assoc_ab", box=box, type_names=["A", "B"],
        sigma=np.array([1.0, 1.0]), valence=np.array([1, 1], np.int32),
        eps_pair=np.ones((2, 2)), rcut=None,
        bond_types=[BondType(HARMONIC, k, r0)],
        reactions=[Reaction(0, 1, 0, 0.0, r_max, eps)],
        pos=pos, vel=_velocities(rng, n, kT), types=types,
        static_bonds=np.zeros((0, 2), np.int32), static_bond_types=np.zeros(0, np.int32),
        kT=kT, seed=seed, meta=dict(rho=rho, n_a=n_a, n_b=n_b))


def telechelic(seed: int = 20260921, n_chains: int = 2000, beads: int = 12,
               n_x: int = 4000, rho: float = 0.3, eps: float = 8.0, k: float = 100.0,
               r0: float = 1.0, r_max: float = 1.25, kT: float = 1.0,
               fene_k: float = 30.0, fene_r0: float = 1.5) -> System:
    """Telechelic network: linear FENE+WCA chains whose end beads (type S,
    valence 1) bond to crosslinkers X (valence 3).  Types: 0 = M (middle bead),
    1 = S (chain end), 2 = X."""
    rng = np.random.default_rng(seed)
    n = n_chains * beads + n_x
    L = (n / rho) ** (1.0 / 3.0)
    box = np.array([L, L, L])
    chain_pos, grid = random_walk_chains(rng, box, n_chains, beads, bond=0.97, min_dist=0.8)
    x_pos, _ = rsa(rng, box, np.full(n_x, 0.5), factor=0.8, grid=grid)
    pos = np.concatenate([chain_pos, x_pos])
    types = np.zeros(n, np.int32)
    ch = np.arange(n_chains) * beads
    types[ch] = 1
    types[ch + beads - 1] = 1
    types[n_chains * beads:] = 2
    a = (ch[:, None] + np.arange(beads - 1)[None, :]).reshape(-1)
    sb = np.stack([a, a + 1], axis=1).astype(np.int32)
    return System(
        name="telechelic", box=box, type_names=["M", "S", "X"],
        sigma=np.array([1.0, 1.0, 1.0]), valence=np.array([0, 1, 3], np.int32),
        eps_pair=np.ones((3, 3)), rcut=None,
        bond_types=[BondType(FENE, fene_k, fene_r0), BondType(HARMONIC, k, r0)],
        reactions=[Reaction(1, 2, 1, 0.0, r_max, eps)],
        pos=pos, vel=_velocities(rng, n, kT), types=types,
        static_bonds=sb, static_bond_types=np.zeros(sb.shape[0], np.int32),
        kT=kT, seed=seed, meta=dict(rho=rho, n_chains=n_chains, beads=beads, n_x=n_x))


def colloid_linker(seed: int = 20260921, n_c: int = 200_000, n_l: int = 800_000,
                   eta: float | None = 0.25, rho: float | None = None, eps: float = 6.0,
                   k: float = 100.0, r0: float = 0.9, r_max: float = 1.2,
                   kT: float = 1.0) -> System:
    """Colloid–linker gel: type C (σ = 1, valence 4) and type L (σ = 0.5,
    valence 2) with C–L dynamic harmonic bonds only.  The box is set either by
    the packing fraction eta or by the number density rho.  Placement is random
    sequential addition with no overlap at σ_ij = (σ_i + σ_j)/2."""
    rng = np.random.default_rng(seed)
    n = n_c + n_l
    vol_particles = n_c * math.pi / 6.0 * 1.0 ** 3 + n_l * math.pi / 6.0 * 0.5 ** 3
    if rho is not None:
        V = n / rho
    else:
        V = vol_particles / eta
    L = V ** (1.0 / 3.0)
    box = np.array([L, L, L])
    # large spheres first (all of them), then the small ones into the remaining space
    pos_c, grid = rsa(rng, box, np.full(n_c, 0.5), factor=1.0, batch=131072)
    pos_l, _ = rsa(rng, box, np.full(n_l, 0.25), factor=1.0, grid=grid, batch=131072)
    pos = np.concatenate([pos_c, pos_l])
    types = np.concatenate([np.zeros(n_c, np.int32), np.ones(n_l, np.int32)])
    return System(
        name="colloid_linker", box=box, type_names=["C", "L"],
        sigma=np.array([1.0, 0.5]), valence=np.array([4, 2], np.int32),
        eps_pair=np.ones((2, 2)), rcut=None,
        bond_types=[BondType(HARMONIC, k, r0)],
        reactions=[Reaction(0, 1, 0, 0.0, r_max, eps)],
        pos=pos, vel=_velocities(rng, n, kT), types=types,
        static_bonds=np.zeros((0, 2), np.int32), static_bond_types=np.zeros(0, np.int32),
        kT=kT, seed=seed, meta=dict(eta=eta, rho=n / V, n_c=n_c, n_l=n_l))


def telechelic_sweep_specs(seed: int = 20260921, n_replicas: int = 256, n_lo: int = 2000,
                           n_hi: int = 50000, rho: float = 0.3):
    """Keyword arguments of `telechelic` for each replica of the batched sweep:
    total bead count log-uniform in [n_lo, n_hi], ε uniform in [2, 10] kT, kT
    uniform in [0.8, 1.2]; chain:crosslinker ratio of the 2000 × 12 + 4000
    system; replica r seeded seed + r."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=n_replicas))
    epss = rng.uniform(2.0, 10.0, size=n_replicas)
    kts = rng.uniform(0.8, 1.2, size=n_replicas)
    out = []
    for r in range(n_replicas):
        n = int(round(ns[r]))
        n_chains = max(1, int(round(n * 2000 / 28000)))
        n_x = max(1, n - 12 * n_chains)
        out.append(dict(seed=seed + r, n_chains=n_chains, n_x=n_x, rho=rho,
                        eps=float(epss[r]), kT=float(kts[r])))
    return out


def _telechelic_kw(kw):
    return telechelic(**kw)


def telechelic_sweep(seed: int = 20260921, n_replicas: int = 256, n_lo: int = 2000,
                     n_hi: int = 50000, rho: float = 0.3, processes: int = 1):
    """Batched parameter sweep of telechelic replicas (see telechelic_sweep_specs).
    With processes > 1 the replicas are generated in a spawned process pool."""
    specs = telechelic_sweep_specs(seed, n_replicas, n_lo, n_hi, rho)
    if processes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            return pool.map(_telechelic_kw, specs)
    return [telechelic(**kw) for kw in specs]


def frozen_pairs(seed: int = 1, n_pairs: int = 200, r: float = 1.1, spacing: float = 4.0,
                 eps: float = 5.0, k: float = 100.0, r0: float = 1.1, r_max: float = 1.3,
                 kT: float = 1.0) -> System:
    """Isolated A–B pairs held at separation r, far apart from each other on a
    cubic lattice of the given spacing (no pair is within reach of another)."""
    rng = np.random.default_rng(seed)
    m = int(math.ceil(n_pairs ** (1.0 / 3.0)))
    L = m * spacing
    g = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"),
                 axis=-1).reshape(-1, 3)[:n_pairs] * spacing + 0.5
    d = rng.normal(size=(n_pairs, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pa = g
    pb = g + r * d
    pos = np.empty((2 * n_pairs, 3))
    pos[0::2] = pa
    pos[1::2] = pb
    pos %= L
    types = np.tile(np.array([0, 1], np.int32), n_pairs)
    return System(
        name="frozen_pairs", box=np.array([L, L, L]), type_names=["A", "B"],
        sigma=np.array([1.0, 1.0]), valence=np.array([1, 1], np.int32),
        eps_pair=np.ones((2, 2)), rcut=None,
        bond_types=[BondType(HARMONIC, k, r0)],
        reactions=[Reaction(0, 1, 0, 0.0, r_max, eps)],
        pos=pos, vel=np.zeros_like(pos), types=types,
        static_bonds=np.zeros((0, 2), np.int32), static_bond_types=np.zeros(0, np.int32),
        kT=kT, seed=seed)


def random_frozen(seed: int, n: int, box: float, type_fracs=(0.5, 0.5), sigma=(1.0, 1.0),
                  valence=(1, 1), eps: float = 5.0, k: float = 100.0, r0: float = 1.1,
                  r_max: float = 1.3, r_min: float = 0.0, overlap_factor: float = 0.7,
                  kT: float = 1.0) -> System:
    """Random configuration (random sequential addition with a reduced overlap
    factor so that many candidate partners compete) for single-sweep parity."""
    rng = np.random.default_rng(seed)
    nt = len(type_fracs)
    counts = np.floor(np.asarray(type_fracs) * n).astype(int)
    counts[-1] = n - counts[:-1].sum()
    types = np.concatenate([np.full(c, t, np.int32) for t, c in enumerate(counts)])
    perm = rng.permutation(n)
    types = types[perm]
    radii = 0.5 * np.asarray(sigma)[types]
    b = np.array([box, box, box], dtype=np.float64)
    pos, _ = rsa(rng, b, radii, factor=overlap_factor)
    return System(
        name="random_frozen", box=b, type_names=[chr(65 + t) for t in range(nt)],
        sigma=np.asarray(sigma, np.float64), valence=np.asarray(valence, np.int32),
        eps_pair=np.ones((nt, nt)), rcut=None,
        bond_types=[BondType(HARMONIC, k, r0)],
        reactions=[Reaction(0, 1 if nt > 1 else 0, 0, r_min, r_max, eps)],
        pos=pos, vel=_velocities(rng, n, kT), types=types,
        static_bonds=np.zeros((0, 2), np.int32), static_bond_types=np.zeros(0, np.int32),
        kT=kT, seed=seed)


def frozen_squares(seed: int = 1, n_squares: int = 216, eps=(0.5, 1.5, 1.0, 2.0), spacing: float = 5.0,
                   k: float = 100.0, r0: float = 1.1, r_max: float = 1.3, kT: float = 1.0) -> System:
    """Four reactions competing for shared binders (App. A, Eq. Z): isolated
    squares with corners A, B, D, C in that order (types 0, 1, 3, 2; valence 1
    each), side r0, randomly rotated, on a cubic lattice of the given spacing.
    The four reactions A-B, A-C, D-B and D-C, one bond type each, join the
    four edges, all held at the rest length (U_b = 0); the diagonals A-D and
    B-C do not react.  eps: the four bond free energies in that order."""
    rng = np.random.default_rng(seed)
    m = int(math.ceil(n_squares ** (1.0 / 3.0)))
    L = m * spacing
    g = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"),
                 axis=-1).reshape(-1, 3)[:n_squares] * spacing + 0.5 * spacing
    corners = np.array([[0.0, 0.0, 0.0], [r0, 0.0, 0.0], [r0, r0, 0.0], [0.0, r0, 0.0]])
    corners -= corners.mean(axis=0)
    pos = np.empty((4 * n_squares, 3))
    for q in range(n_squares):
        rot, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        pos[4 * q:4 * q + 4] = g[q] + corners @ rot.T
    pos %= L
    types = np.tile(np.array([0, 1, 3, 2], np.int32), n_squares)
    ea, eb, ec, ed = (float(e) for e in eps)
    return System(
        name="frozen_squares", box=np.array([L, L, L]), type_names=["A", "B", "C", "D"],
        sigma=np.ones(4), valence=np.ones(4, np.int32),
        eps_pair=np.ones((4, 4)), rcut=None,
        bond_types=[BondType(HARMONIC, k, r0) for _ in range(4)],
        reactions=[Reaction(0, 1, 0, 0.0, r_max, ea), Reaction(0, 2, 1, 0.0, r_max, eb),
                   Reaction(3, 1, 2, 0.0, r_max, ec), Reaction(3, 2, 3, 0.0, r_max, ed)],
        pos=pos, vel=np.zeros_like(pos), types=types,
        static_bonds=np.zeros((0, 2), np.int32), static_bond_types=np.zeros(0, np.int32),
        kT=kT, seed=seed)


def four_reaction_soup(seed: int = 1, n: int = 2000, rho: float = 0.3, eps=(0.5, 1.5, 1.0, 2.0),
                       k: float = 100.0, r0: float = 1.1, r_max: float = 1.3, overlap_factor: float = 1.0,
                       kT: float = 1.0) -> System:
    """The four reactions of `frozen_squares` (A-B, A-C, D-B, D-C, valence 1,
    one bond type each) in a mobile WCA soup of equal numbers of A, B, C and D
    at number density rho (App. A, the dynamic version of the Eq. Z test).
    overlap_factor < 1 packs contested frozen configurations for sweep parity."""
    box = (n / rho) ** (1.0 / 3.0)
    s = random_frozen(seed=seed, n=n, box=box, type_fracs=(0.25, 0.25, 0.25, 0.25), sigma=(1.0,) * 4,
                      valence=(1, 1, 1, 1), k=k, r0=r0, r_max=r_max, overlap_factor=overlap_factor, kT=kT)
    ea, eb, ec, ed = (float(e) for e in eps)
    s.name = "four_reaction_soup"
    s.type_names = ["A", "B", "C", "D"]
    s.bond_types = [BondType(HARMONIC, k, r0) for _ in range(4)]
    s.reactions = [Reaction(0, 1, 0, 0.0, r_max, ea), Reaction(0, 2, 1, 0.0, r_max, eb),
                   Reaction(3, 1, 2, 0.0, r_max, ec), Reaction(3, 2, 3, 0.0, r_max, ed)]
    return s


def frozen_loops(seed: int = 1, n_units: int = 125, self_avoid: int = 1, eps: float = 1.0, d: float = 1.1,
                 spacing: float = 5.0, k: float = 100.0, r0: float = 1.1, r_max: float = 1.3,
                 kT: float = 1.0) -> System:
    """Intramolecular exclusion, both ways (Sec. II.D, App. A): every unit holds
    one molecule P-M-Q (P type 0 and Q type 1, valence 1, joined through a
    non-reactive bead M of type 2 by two static FENE bonds) whose two sites sit
    at distance d, and a control pair: a lone P and a lone Q, also at distance
    d, that belong to different molecules.  Units are randomly rotated on a
    cubic lattice of the given spacing; the reaction P-Q carries self_avoid."""
    rng = np.random.default_rng(seed)
    m = int(math.ceil(n_units ** (1.0 / 3.0)))
    L = m * spacing
    g = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"),
                 axis=-1).reshape(-1, 3)[:n_units] * spacing + 0.5 * spacing
    # molecule P, M, Q; control P', Q' two units of length away along z
    local = np.array([[0.0, 0.0, 0.0], [0.5 * d, 0.9, 0.0], [d, 0.0, 0.0],
                      [0.0, 0.0, 2.0], [d, 0.0, 2.0]])
    local -= local.mean(axis=0)
    pos = np.empty((5 * n_units, 3))
    for q in range(n_units):
        rot, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        pos[5 * q:5 * q + 5] = g[q] + local @ rot.T
    pos %= L
    types = np.tile(np.array([0, 2, 1, 0, 1], np.int32), n_units)
    base = 5 * np.arange(n_units, dtype=np.int32)
    sb = np.concatenate([np.stack([base, base + 1], axis=1), np.stack([base + 1, base + 2], axis=1)])
    return System(
        name="frozen_loops", box=np.array([L, L, L]), type_names=["P", "Q", "M"],
        sigma=np.ones(3), valence=np.array([1, 1, 0], np.int32),
        eps_pair=np.ones((3, 3)), rcut=None,
        bond_types=[BondType(FENE, 30.0, 1.5), BondType(HARMONIC, k, r0)],
        reactions=[Reaction(0, 1, 1, 0.0, r_max, eps, self_avoid)],
        pos=pos, vel=np.zeros_like(pos), types=types,
        static_bonds=sb.astype(np.int32), static_bond_types=np.zeros(sb.shape[0], np.int32),
        kT=kT, seed=seed)


def telechelic_rings(seed: int = 1, n_chains: int = 300, beads: int = 3, rho: float = 0.3,
                     self_avoid: int = 1, eps: float = 3.0, r_max: float = 1.25, kT: float = 1.0) -> System:
    """Short telechelic chains whose end beads (type S, valence 1) react with
    each other, S-S, with no crosslinkers: with self_avoid = 0 the two ends of
    one chain may close it into a ring (a self-loop of the molecule), with
    self_avoid = 1 they may not (Sec. II.D)."""
    s = telechelic(seed=seed, n_chains=n_chains, beads=beads, n_x=0, rho=rho, eps=eps, r_max=r_max, kT=kT)
    s.name = "telechelic_rings"
    s.valence = np.array([0, 1, 0], np.int32)
    s.reactions = [Reaction(1, 1, 1, 0.0, r_max, eps, self_avoid)]
    return s


def frozen_stars(seed: int = 1, n_stars: int = 125, arms: int = 4, r_lo: float = 1.0, r_hi: float = 1.25,
                 spacing: float = 5.0, eps: float = 1.0, k: float = 20.0, r0: float = 1.1,
                 r_max: float = 1.3, kT: float = 1.0, min_sep: float = 0.8) -> System:
    """Isolated stars: one A (valence 1) with `arms` B particles (valence 1)
    at distinct separations spread over [r_lo, r_hi] in random directions,
    stars on a cubic lattice of the given spacing so that no star reaches
    another.  Every B of a star competes for the same A.  Arms of a star are
    at least min_sep apart."""
    rng = np.random.default_rng(seed)
    m = int(math.ceil(n_stars ** (1.0 / 3.0)))
    L = m * spacing
    g = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"),
                 axis=-1).reshape(-1, 3)[:n_stars] * spacing + 0.5 * spacing
    per = arms + 1
    pos = np.empty((n_stars * per, 3))
    types = np.tile(np.array([0] + [1] * arms, np.int32), n_stars)
    for s in range(n_stars):
        pos[s * per] = g[s]
        radii = rng.permutation(np.linspace(r_lo, r_hi, arms))
        for a in range(arms):
            while True:
                d = rng.normal(size=3)
                d /= np.linalg.norm(d)
                p = g[s] + radii[a] * d
                if all(np.linalg.norm(p - pos[s * per + 1 + b]) > min_sep for b in range(a)):
                    break
            pos[s * per + 1 + a] = p
    pos %= L
    return System(
        name="frozen_stars", box=np.array([L, L, L]), type_names=["A", "B"],
        sigma=np.array([1.0, 1.0]), valence=np.array([1, 1], np.int32),
        eps_pair=np.ones((2, 2)), rcut=None,
        bond_types=[BondType(HARMONIC, k, r0)],
        reactions=[Reaction(0, 1, 0, 0.0, r_max, eps)],
        pos=pos, vel=np.zeros_like(pos), types=types,
        static_bonds=np.zeros((0, 2), np.int32), static_bond_types=np.zeros(0, np.int32),
        kT=kT, seed=seed, meta=dict(arms=arms))
