"""FP64 CPU oracle for the dynamic-bonding MD hot path — TEST INFRASTRUCTURE.

Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline /
reference legs may import this package.  The product path never does.

The arithmetic lives in `snap_oracle.c` (plain C, -ffp-contract=off); this
module compiles it on first use and wraps it with ctypes.  It shares no code
with the CUDA path: the only common input is the seeded `synth` workloads.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_LIB_PATH = _HERE / "liboracle.so"
_SRC = _HERE / "snap_oracle.c"

MAX_TYPES = 8
MAX_BTYPES = 8
MAX_RX = 8
VMAX = 4
SMAX = 4
HARMONIC, FENE, FENEWCA, TETHER = 0, 1, 2, 3
FORM, BREAK, MATCH, ORDER, LANGEVIN = 1, 2, 3, 4, 5


def build(force: bool = False) -> Path:
    """Compile liboracle.so next to its source (plain gcc, no GPU code)."""
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < max(
            _SRC.stat().st_mtime, (_HERE / "snap_oracle.h").stat().st_mtime):
        tmp = _LIB_PATH.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", str(tmp), str(_SRC), "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Reaction(C.Structure):
    _fields_ = [("type_a", C.c_int32), ("type_b", C.c_int32), ("bond_type", C.c_int32),
                ("r_min", C.c_double), ("r_max", C.c_double),
                ("p_on0", C.c_double), ("p_off", C.c_double), ("self_avoid", C.c_int32),
                ("slip_a", C.c_double), ("melt", C.c_int32), ("melt_lambda", C.c_double),
                ("melt_t", C.c_double), ("kon_init", C.c_double), ("koff_init", C.c_double),
                ("kon_melt", C.c_double), ("koff_melt", C.c_double)]


class Params(C.Structure):
    _fields_ = [("n", C.c_int64), ("box", C.c_double * 3), ("dt", C.c_double),
                ("kT", C.c_double), ("gamma", C.c_double), ("seed", C.c_uint64),
                ("ntypes", C.c_int32), ("sigma", C.c_double * MAX_TYPES),
                ("eps", C.c_double * (MAX_TYPES * MAX_TYPES)),
                ("rcut", C.c_double * (MAX_TYPES * MAX_TYPES)),
                ("valence", C.c_int32 * MAX_TYPES), ("nbtypes", C.c_int32),
                ("bkind", C.c_int32 * MAX_BTYPES), ("bk", C.c_double * MAX_BTYPES),
                ("br0", C.c_double * MAX_BTYPES), ("bx", (C.c_double * 3) * MAX_BTYPES),
                ("nrx", C.c_int32),
                ("rx", Reaction * MAX_RX), ("bond_period", C.c_int32), ("kinetic_T", C.c_int32)]


class State(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("vx", C.c_void_p), ("vy", C.c_void_p), ("vz", C.c_void_p),
                ("img", C.c_void_p), ("type", C.c_void_p), ("sp", C.c_void_p),
                ("sbt", C.c_void_p), ("dp", C.c_void_p), ("drx", C.c_void_p),
                ("dbirth", C.c_void_p), ("occ", C.c_void_p),
                ("fx", C.c_void_p), ("fy", C.c_void_p), ("fz", C.c_void_p),
                ("pe", C.c_void_p), ("life_hist", C.c_void_p), ("nhist", C.c_int32),
                ("step", C.c_int64), ("mol", C.c_void_p), ("fscale", C.c_void_p),
                ("vabs", C.c_double)]


class SweepStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("scanned", "in_window", "proposals", "edges",
                                         "survivors", "formed", "break_tested", "broken")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class MHStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("form_attempts", "form_accepts", "break_attempts",
                                         "break_accepts")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Trace(C.Structure):
    _fields_ = [("prop", C.c_void_p), ("prop_r", C.c_void_p), ("matched", C.c_void_p),
                ("formed", C.c_void_p), ("order", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(str(build()))
        _lib.orc_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.orc_u53.argtypes = [C.c_uint32, C.c_uint32]
        _lib.orc_u53.restype = C.c_double
        _lib.orc_exp.argtypes = [C.c_double]
        _lib.orc_exp.restype = C.c_double
        _lib.orc_log.argtypes = [C.c_double]
        _lib.orc_log.restype = C.c_double
        _lib.orc_bond_energy.argtypes = [C.POINTER(Params), C.c_int32, C.c_double]
        _lib.orc_bond_energy.restype = C.c_double
        _lib.orc_aim_separation.argtypes = [C.POINTER(Params), C.c_int32]
        _lib.orc_aim_separation.restype = C.c_double
        _lib.orc_sweep.argtypes = [C.POINTER(Params), C.POINTER(State), C.c_int64,
                                   C.POINTER(SweepStats), C.c_void_p]
        _lib.orc_forces.argtypes = [C.POINTER(Params), C.POINTER(State), C.c_void_p,
                                    C.c_void_p, C.c_void_p]
        _lib.orc_run.argtypes = [C.POINTER(Params), C.POINTER(State), C.c_int64, C.c_void_p]
        _lib.orc_pairs_within.argtypes = [C.POINTER(Params), C.POINTER(State), C.c_double,
                                          C.c_int, C.c_void_p, C.c_int64]
        _lib.orc_pairs_within.restype = C.c_int64
        _lib.orc_candidates.argtypes = [C.POINTER(Params), C.POINTER(State), C.c_int32,
                                        C.c_int64, C.c_void_p, C.c_int32]
        _lib.orc_candidates.restype = C.c_int32
        _lib.orc_mh_sweep.argtypes = [C.POINTER(Params), C.POINTER(State), C.c_int64, C.POINTER(MHStats)]
        _lib.orc_rdf.argtypes = [C.POINTER(Params), C.POINTER(State), C.c_int32, C.c_int32, C.c_double,
                                 C.c_int32, C.c_void_p]
        _lib.orc_kinetic_T.argtypes = [C.POINTER(Params), C.POINTER(State)]
        _lib.orc_kinetic_T.restype = C.c_double
        _lib.orc_tanh.argtypes = [C.c_double]
        _lib.orc_tanh.restype = C.c_double
    return _lib


def _ptr(a):
    return a.ctypes.data if a is not None else None


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u53(w0, w1):
    return lib().orc_u53(int(w0), int(w1))


def exp(x: float) -> float:
    return lib().orc_exp(float(x))


def tanh(x: float) -> float:
    return lib().orc_tanh(float(x))


def log(x: float) -> float:
    return lib().orc_log(float(x))


def rates_from_eps(eps: float, p_on0: float = 1.0):
    """Closure of Eqs. (1)-(2): with P_on^0 fixed, K = e^eps fixes
    P_off = P_on^0 / K (the ratio k_on/k_off equals P_on^0/P_off)."""
    return p_on0, p_on0 * math.exp(-eps)


def melting_rates(T, lam, t_melt, kon_init, koff_init, kon_melt, koff_melt, n, dt):
    """Melting switch, Eqs. (gT)-(kT), and per-sweep probabilities, Eq. (2):
    g = (tanh(lam (T - T_melt)) + 1) / 2, k(T) = k_init (1 - g) + k_melt g,
    P = k n dt.  Returns (P_on^0, P_off)."""
    g = 0.5 * (math.tanh(lam * (T - t_melt)) + 1.0)
    kon = kon_init * (1.0 - g) + kon_melt * g
    koff = koff_init * (1.0 - g) + koff_melt * g
    return kon * n * dt, koff * n * dt


def rdf_normalise(counts, n_a, n_b, same, volume, r_max):
    """g(r) from pair counts: counts over the pair count an ideal gas of the
    same composition would put in each spherical shell (N_a N_b / V, or
    N_a (N_a - 1) / 2 / V for one type, times the shell volume)."""
    nb = len(counts)
    edges = np.linspace(0.0, r_max, nb + 1)
    shell = 4.0 / 3.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    pairs = n_a * (n_a - 1) / 2.0 if same else float(n_a) * n_b
    return np.asarray(counts, dtype=np.float64) / (pairs / volume * shell)


def molecules(n, static_bonds):
    """Molecule id of every particle (Sec. II.D): the connected components of
    the graph whose edges are the static bonds, labelled by scipy's
    connected-components routine; a particle without static bonds is a
    molecule of its own."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    b = np.asarray(static_bonds, dtype=np.int64).reshape(-1, 2)
    g = coo_matrix((np.ones(b.shape[0]), (b[:, 0], b[:, 1])), shape=(n, n))
    _, labels = connected_components(g, directed=False)
    return labels.astype(np.int32)


class OracleSystem:
    """One system held in tag order with numpy arrays the C code reads and writes."""

    def __init__(self, sysdef, nhist: int = 256, p_on0: float = 1.0):
        s = sysdef
        n = s.n
        P = Params()
        P.n = n
        for d in range(3):
            P.box[d] = float(s.box[d])
        P.dt, P.kT, P.gamma, P.seed = float(s.dt), float(s.kT), float(s.gamma), int(s.seed)
        nt = len(s.sigma)
        P.ntypes = nt
        for a in range(nt):
            P.sigma[a] = float(s.sigma[a])
            P.valence[a] = int(s.valence[a])
            for b in range(nt):
                P.eps[a * MAX_TYPES + b] = float(s.eps_pair[a, b])
                P.rcut[a * MAX_TYPES + b] = float(s.rcut[a, b]) if s.rcut is not None else 0.0
        P.nbtypes = len(s.bond_types)
        for i, bt in enumerate(s.bond_types):
            P.bkind[i], P.bk[i], P.br0[i] = int(bt.kind), float(bt.k), float(bt.r0)
            for q, v in enumerate(getattr(bt, "extra", ()) or ()):
                P.bx[i][q] = float(v)
        P.nrx = len(s.reactions)
        for i, r in enumerate(s.reactions):
            if getattr(r, "melt", None) is not None:
                pon, poff = melting_rates(float(s.kT), *r.melt, int(s.bond_period), float(s.dt))
            else:
                pon, poff = rates_from_eps(r.eps, p_on0)
            melt = getattr(r, "melt", None)
            P.rx[i] = Reaction(r.type_a, r.type_b, r.bond_type, r.r_min, r.r_max, pon, poff,
                               r.self_avoid, float(getattr(r, "slip_a", 0.0)),
                               1 if melt is not None else 0, *(map(float, melt) if melt is not None else [0.0] * 6))
        P.bond_period = int(s.bond_period)
        P.kinetic_T = int(getattr(s, "kinetic_T", 0))
        self.params = P
        self.n = n
        self.x = np.ascontiguousarray(s.pos[:, 0], dtype=np.float64).copy()
        self.y = np.ascontiguousarray(s.pos[:, 1], dtype=np.float64).copy()
        self.z = np.ascontiguousarray(s.pos[:, 2], dtype=np.float64).copy()
        self.vx = np.ascontiguousarray(s.vel[:, 0], dtype=np.float64).copy()
        self.vy = np.ascontiguousarray(s.vel[:, 1], dtype=np.float64).copy()
        self.vz = np.ascontiguousarray(s.vel[:, 2], dtype=np.float64).copy()
        self.img = np.zeros(3 * n, dtype=np.int32)
        self.type = np.ascontiguousarray(s.types, dtype=np.int32).copy()
        self.sp = np.full(n * SMAX, -1, dtype=np.int32)
        self.sbt = np.zeros(n * SMAX, dtype=np.int32)
        cnt = np.zeros(n, dtype=np.int64)
        for (a, b), t in zip(s.static_bonds, s.static_bond_types):
            for u, v in ((a, b), (b, a)):
                if cnt[u] >= SMAX:
                    raise ValueError("too many static bonds on one particle")
                self.sp[u * SMAX + cnt[u]] = v
                self.sbt[u * SMAX + cnt[u]] = t
                cnt[u] += 1
        self.dp = np.full(n * VMAX, -1, dtype=np.int32)
        self.drx = np.full(n * VMAX, -1, dtype=np.int32)
        self.dbirth = np.zeros(n * VMAX, dtype=np.int64)
        self.occ = np.zeros(n, dtype=np.int32)
        self.fx = np.zeros(n)
        self.fy = np.zeros(n)
        self.fz = np.zeros(n)
        self.pe = np.zeros(n)
        self.fscale = np.zeros(n)
        self.life_hist = np.zeros(nhist, dtype=np.int64)
        self.mol = molecules(n, s.static_bonds)
        self.step = 0
        self._state = State()
        self._sync_ptrs()

    def _sync_ptrs(self):
        S = self._state
        for f in ("x", "y", "z", "vx", "vy", "vz", "img", "type", "sp", "sbt", "dp", "drx",
                  "dbirth", "occ", "fx", "fy", "fz", "pe", "life_hist", "mol", "fscale"):
            setattr(S, f, _ptr(getattr(self, f)))
        S.nhist = self.life_hist.size
        S.step = self.step

    # -- positions ---------------------------------------------------------
    @property
    def pos(self):
        return np.stack([self.x, self.y, self.z], axis=1)

    def set_positions(self, pos):
        self.x[:] = pos[:, 0]
        self.y[:] = pos[:, 1]
        self.z[:] = pos[:, 2]

    # -- bonds -------------------------------------------------------------
    def bonds(self):
        """Dynamic bonds as an (m, 3) int array of (min tag, max tag, reaction),
        ascending by (min tag, max tag)."""
        dp = self.dp.reshape(self.n, VMAX)
        drx = self.drx.reshape(self.n, VMAX)
        i, s = np.nonzero(dp >= 0)
        j = dp[i, s]
        keep = j > i
        out = np.stack([i[keep], j[keep], drx[i, s][keep]], axis=1).astype(np.int64)
        order = np.lexsort((out[:, 1], out[:, 0]))
        return out[order]

    def set_bonds(self, bonds, birth=0):
        """Replace the dynamic-bond set with rows (a, b, reaction)."""
        self.dp[:] = -1
        self.drx[:] = -1
        self.dbirth[:] = 0
        self.occ[:] = 0
        per = {}
        for a, b, r in bonds:
            per.setdefault(int(a), []).append((int(b), int(r)))
            per.setdefault(int(b), []).append((int(a), int(r)))
        for i, lst in per.items():
            lst.sort()
            if len(lst) > VMAX:
                raise ValueError("more than VMAX dynamic bonds on a particle")
            for s, (j, r) in enumerate(lst):
                self.dp[i * VMAX + s] = j
                self.drx[i * VMAX + s] = r
                self.dbirth[i * VMAX + s] = birth
            self.occ[i] = len(lst)

    # -- calls -------------------------------------------------------------
    def sweep(self, step=None, trace=False):
        if step is None:
            step = self.step
        self._sync_ptrs()
        st = SweepStats()
        tr = None
        tarr = None
        if trace:
            tarr = dict(prop=np.full(self.n, -1, np.int32), prop_r=np.zeros(self.n),
                        matched=np.full(self.n, -1, np.int32), formed=np.zeros(self.n, np.uint8),
                        order=np.zeros(MAX_RX, np.int32))
            tr = Trace(*[_ptr(tarr[k]) for k in ("prop", "prop_r", "matched", "formed", "order")])
        rc = lib().orc_sweep(C.byref(self.params), C.byref(self._state), int(step),
                             C.byref(st), C.byref(tr) if tr is not None else None)
        if rc != 0:
            raise RuntimeError(f"orc_sweep failed: {rc}")
        return (st.as_dict(), tarr) if trace else st.as_dict()

    def mh_sweep(self, step=None):
        """One Metropolis–Hastings sweep with the uniform proposal."""
        if step is None:
            step = self.step
        self._sync_ptrs()
        st = MHStats()
        rc = lib().orc_mh_sweep(C.byref(self.params), C.byref(self._state), int(step), C.byref(st))
        if rc != 0:
            raise RuntimeError(f"orc_mh_sweep failed: {rc}")
        return st.as_dict()

    def rdf_counts(self, type_a, type_b, r_max, nbins):
        """Pair counts per distance bin behind g(r) (see orc_rdf)."""
        self._sync_ptrs()
        h = np.zeros(int(nbins), dtype=np.int64)
        rc = lib().orc_rdf(C.byref(self.params), C.byref(self._state), int(type_a), int(type_b),
                           float(r_max), int(nbins), _ptr(h))
        if rc != 0:
            raise RuntimeError("orc_rdf failed")
        return h

    def kinetic_T(self):
        """The instantaneous kinetic temperature a sweep would use now."""
        self._sync_ptrs()
        return lib().orc_kinetic_T(C.byref(self.params), C.byref(self._state))

    def set_velocities(self, vel):
        self.vx[:] = vel[:, 0]
        self.vy[:] = vel[:, 1]
        self.vz[:] = vel[:, 2]

    def forces(self):
        self._sync_ptrs()
        e = np.zeros(3)
        rc = lib().orc_forces(C.byref(self.params), C.byref(self._state), _ptr(e[0:1]),
                              _ptr(e[1:2]), _ptr(e[2:3]))
        f = np.stack([self.fx, self.fy, self.fz], axis=1).copy()
        return f, dict(e_pair=e[0], e_bond=e[1], virial=e[2], status=rc,
                       fscale=self.fscale.copy(), virial_scale=float(self._state.vabs))

    def run(self, nsteps):
        self._sync_ptrs()
        ke = np.zeros(1)
        rc = lib().orc_run(C.byref(self.params), C.byref(self._state), int(nsteps), _ptr(ke))
        self.step = int(self._state.step)
        return dict(ke=float(ke[0]), status=rc)

    def pairs_within(self, extra=0.0, reactive=True):
        self._sync_ptrs()
        cap = max(16, self.n * 64)
        out = np.zeros(2 * cap, dtype=np.int32)
        m = lib().orc_pairs_within(C.byref(self.params), C.byref(self._state), float(extra),
                                   int(reactive), _ptr(out), cap)
        if m < 0:
            raise RuntimeError("orc_pairs_within failed")
        if m > cap:
            raise RuntimeError("pair buffer too small")
        return out[: 2 * m].reshape(m, 2).copy()

    def candidates(self, i, rx=0, cap=512):
        self._sync_ptrs()
        out = np.zeros(cap, dtype=np.int32)
        m = lib().orc_candidates(C.byref(self.params), C.byref(self._state), int(rx), int(i),
                                 _ptr(out), cap)
        return np.sort(out[:min(m, cap)])

    def bond_energy(self, bond_type, r):
        return lib().orc_bond_energy(C.byref(self.params), int(bond_type), float(r))

    def aim_separation(self, bond_type):
        return lib().orc_aim_separation(C.byref(self.params), int(bond_type))
