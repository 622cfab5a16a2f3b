"""B300-native dynamic-bonding molecular dynamics (DyBond-v2 hot path).

Thin Python binding over the C ABI of include/snap.h: every step of the MD
step and of the bond sweep runs in the CUDA kernels of libsnap_b300.so; this
module only marshals arguments.  PyTorch, when present, supplies the device
allocator and the stream.  There is no CPU fallback: if the library is missing
the constructor raises.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import _abi
from ._abi import SNAP_FP64, SNAP_MIXED, SNAP_HARMONIC, SNAP_FENE

__all__ = ["Snap", "Mlp", "mlp_init_weights", "SnapError", "closure", "rates_from_eps", "from_system", "pair_energy_noalloc",
           "SNAP_FP64",
           "SNAP_MIXED", "SNAP_HARMONIC", "SNAP_FENE"]


class SnapError(RuntimeError):
    def __init__(self, code: int, msg: str):
        self.code = code
        self.name = _abi.STATUS_NAMES.get(code, str(code))
        super().__init__(f"{self.name}: {msg}")


def closure(dt: float, period: int = 1, k_on=None, k_off=None, eps=None, p_on0=None, p_off=None):
    """Complete the rate parameters of one reaction from any sufficient subset
    (Eqs. 1-2 of the DyBond-v2 paper: P_on^0 = k_on n dt, P_off = k_off n dt,
    eps = ln(k_on / k_off)).  Over-specified inputs are checked for consistency."""
    ndt = period * dt
    known = {k: v for k, v in dict(k_on=k_on, k_off=k_off, eps=eps, p_on0=p_on0,
                                   p_off=p_off).items() if v is not None}
    kon = k_on if k_on is not None else (p_on0 / ndt if p_on0 is not None else None)
    koff = k_off if k_off is not None else (p_off / ndt if p_off is not None else None)
    if kon is None and koff is not None and eps is not None:
        kon = koff * math.exp(eps)
    if koff is None and kon is not None and eps is not None:
        koff = kon * math.exp(-eps)
    if kon is None or koff is None:
        raise ValueError(f"under-specified rates: {sorted(known)}")
    out = dict(k_on=kon, k_off=koff, eps=math.log(kon / koff) if koff > 0 else math.inf,
               p_on0=kon * ndt, p_off=koff * ndt)
    for k, v in known.items():
        if not math.isclose(out[k], v, rel_tol=1e-9, abs_tol=1e-15):
            raise ValueError(f"inconsistent rate parameters: {k}={v} but the others give {out[k]}")
    if out["p_on0"] > 1.0 or out["p_off"] > 1.0:
        raise ValueError("per-sweep probabilities exceed 1: k_max = 1/(n dt) (Eq. 2)")
    return out


def rates_from_eps(eps: float, p_on0: float = 1.0, dt: float = 0.005, period: int = 1):
    """(P_on^0, P_off) for a bond free energy eps (in kT) at a given P_on^0:
    K = P_on^0 / P_off = e^eps (Eqs. 1-2), checked against the full closure."""
    p_off = p_on0 * math.exp(-eps)
    closure(dt, period, eps=eps, p_on0=p_on0, p_off=p_off)
    return p_on0, p_off


def _c_array(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


class Snap:
    """One simulation context (one system, or a batch of independent replicas)."""

    def __init__(self, n, box, dt=0.005, kT=1.0, gamma=1.0, seed=20260921, precision="mixed",
                 bond_period=1, skin=0.3, replicas=None, stream=None, torch_allocator=True,
                 block_size=0, nlist_capacity=0, lifetime_bins=256, lib=None):
        self._lib = _abi.load(lib)
        self._ctx = C.c_void_p()
        self._keep = []
        cfg = _abi.Config()
        cfg.n = int(n)
        for d in range(3):
            cfg.box[d] = float(box[d])
        cfg.dt, cfg.kT, cfg.gamma, cfg.seed = float(dt), float(kT), float(gamma), int(seed)
        prec = {"mixed": SNAP_MIXED, "fp64": SNAP_FP64, SNAP_MIXED: SNAP_MIXED,
                SNAP_FP64: SNAP_FP64}[precision]
        cfg.precision = prec
        self.precision = "fp64" if prec == SNAP_FP64 else "mixed"
        cfg.bond_period, cfg.skin = int(bond_period), float(skin)
        cfg.block_size, cfg.nlist_capacity, cfg.lifetime_bins = int(block_size), int(nlist_capacity), int(lifetime_bins)
        if replicas:
            rn = np.ascontiguousarray([r["n"] for r in replicas], dtype=np.int64)
            rb = np.ascontiguousarray([r["box"] for r in replicas], dtype=np.float64).reshape(-1)
            rk = np.ascontiguousarray([r.get("kT", kT) for r in replicas], dtype=np.float64)
            rs = np.ascontiguousarray([r.get("seed", seed + i) for i, r in enumerate(replicas)],
                                      dtype=np.uint64)
            self._keep += [rn, rb, rk, rs]
            cfg.n_replicas = len(replicas)
            cfg.replica_n = _c_array(rn, C.c_int64)
            cfg.replica_box = _c_array(rb, C.c_double)
            cfg.replica_kT = _c_array(rk, C.c_double)
            cfg.replica_seed = _c_array(rs, C.c_uint64)
            self.n_replicas = len(replicas)
        else:
            self.n_replicas = 1
        self._torch = None
        if torch_allocator or stream is not None:
            try:
                import torch
                if torch.cuda.is_available():
                    self._torch = torch
            except ImportError:
                self._torch = None
        if self._torch is not None:
            torch = self._torch
            dev = torch.cuda.current_device()
            s = stream if stream is not None else torch.cuda.current_stream()
            self._stream = s
            cfg.stream = C.c_void_p(s.cuda_stream)
            if torch_allocator:
                def _alloc(nbytes, user, _t=torch, _d=dev, _s=s):
                    try:
                        return _t.cuda.caching_allocator_alloc(int(nbytes), _d, _s)
                    except Exception:
                        return None

                def _free(ptr, user, _t=torch):
                    _t.cuda.caching_allocator_delete(ptr)

                fa, ff = _abi.ALLOC_FN(_alloc), _abi.FREE_FN(_free)
                self._keep += [fa, ff]
                cfg.alloc, cfg.free = fa, ff
        self.n = int(n)
        self._check(self._lib.snap_init(C.byref(self._ctx), C.byref(cfg)), init=True)
        self.reactions = 0

    # -- plumbing ------------------------------------------------------------
    def _check(self, code, init=False):
        if code != 0:
            msg = "" if init else (self._lib.snap_last_error(self._ctx) or b"").decode()
            raise SnapError(code, msg)

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self._lib.snap_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- model ---------------------------------------------------------------
    def set_types(self, sigma, eps_pair, rcut=None):
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        e = np.ascontiguousarray(eps_pair, dtype=np.float64)
        rc = None if rcut is None else np.ascontiguousarray(rcut, dtype=np.float64)
        self._check(self._lib.snap_set_types(self._ctx, sigma.size, sigma.ctypes.data, e.ctypes.data,
                                             rc.ctypes.data if rc is not None else None))

    def set_valence(self, valence):
        v = np.ascontiguousarray(valence, dtype=np.int32)
        self._check(self._lib.snap_set_valence(self._ctx, v.ctypes.data))

    def set_bond_params(self, bt, kind, k, r0, extra=()):
        """Bond type bt: harmonic (k, r0), FENE (k, R0), FENEWCA (k, R0, extra =
        (eps, sigma, delta)) or Tether (k_b, l_min, extra = (l_c1, l_c0, l_max))."""
        p = np.array([k, r0, *extra], dtype=np.float64)
        self._check(self._lib.snap_set_bond_params_ex(self._ctx, int(bt), int(kind), p.ctypes.data, p.size))

    def add_static_bonds(self, pairs, bt):
        p = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        self._check(self._lib.snap_add_static_bonds(self._ctx, p.shape[0], p.ctypes.data, int(bt)))

    def add_reaction(self, type_a, type_b, bt, r_min, r_max, p_on0, p_off, self_avoid=0):
        idx = C.c_int32(-1)
        self._check(self._lib.snap_add_reaction(self._ctx, int(type_a), int(type_b), int(bt),
                                                float(r_min), float(r_max), float(p_on0),
                                                float(p_off), int(self_avoid), C.byref(idx)))
        self.reactions += 1
        return idx.value

    def set_reaction_rates(self, reaction, replica, p_on0, p_off):
        self._check(self._lib.snap_set_reaction_rates(self._ctx, int(reaction), int(replica),
                                                      float(p_on0), float(p_off)))

    def set_slip(self, reaction, a):
        """Slip-bond modifier of one reaction (Eq. slip); a = 0 switches it off."""
        self._check(self._lib.snap_set_slip(self._ctx, int(reaction), float(a)))

    def set_melting(self, reaction, lam, t_melt, kon_init, koff_init, kon_melt, koff_melt):
        """Melting switch of one reaction (Eqs. gT-kT) at every replica's kT."""
        self._check(self._lib.snap_set_melting(self._ctx, int(reaction), float(lam), float(t_melt),
                                               float(kon_init), float(koff_init), float(kon_melt),
                                               float(koff_melt)))

    # -- state ---------------------------------------------------------------
    def set_particles(self, pos, vel, types):
        p = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        v = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3)
        t = np.ascontiguousarray(types, dtype=np.int32)
        self._check(self._lib.snap_set_particles(self._ctx, p.ctypes.data,
                                                 v.ctypes.data if v is not None else None,
                                                 t.ctypes.data))

    def set_positions(self, pos, vel=None):
        p = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        v = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3)
        self._check(self._lib.snap_set_positions(self._ctx, p.ctypes.data,
                                                 v.ctypes.data if v is not None else None))

    def set_bonds(self, pairs, reaction=None):
        p = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        r = None if reaction is None else np.ascontiguousarray(reaction, dtype=np.int32)
        self._check(self._lib.snap_set_bonds(self._ctx, p.shape[0], p.ctypes.data,
                                             r.ctypes.data if r is not None else None))

    def step(self, nsteps=1):
        self._check(self._lib.snap_step(self._ctx, int(nsteps)))

    def set_kinetic_temperature(self, on=True):
        """Use the instantaneous kinetic temperature (deterministic fixed-point
        sum over the half-step velocities) in every sweep instead of the
        set-point kT (Sec. II.B)."""
        self._check(self._lib.snap_set_kinetic_temperature(self._ctx, 1 if on else 0))

    def set_retry_limit(self, limit):
        """Retry limit of the push-mode compare-and-swap loop (default 65536);
        reaching it makes the step return SNAP_ERR_TIMEOUT without taking it."""
        self._check(self._lib.snap_set_retry_limit(self._ctx, int(limit)))

    def set_list_block(self, threads):
        """Threads per block of the neighbour-list build: 64, 128 or 256 (a
        launch shape; results do not depend on it)."""
        self._check(self._lib.snap_set_list_block(self._ctx, int(threads)))

    def set_list_subcells(self, k):
        """Sub-cells along x per neighbour cell for the list build: 1, 2, 4 or
        8, or 0 for automatic; only before the particles are set (the lists
        hold the same pairs for every k)."""
        self._check(self._lib.snap_set_list_subcells(self._ctx, int(k)))

    def list_subcells(self):
        """Sub-cells along x per cell in use."""
        k = C.c_int32()
        self._check(self._lib.snap_get_list_subcells(self._ctx, C.byref(k)))
        return int(k.value)

    def prepare(self):
        """Capture and upload the step graphs of both buffer parities now (no
        step runs), so that no later step() pays for a capture."""
        self._check(self._lib.snap_prepare(self._ctx))

    def step_profiled(self, nsteps):
        """Run nsteps without graphs, timing each phase with CUDA events; returns
        average ms per step of (rebuild, sweep, md = the fused force + Langevin
        kernel, step_end)."""
        ms = np.zeros(4)
        self._check(self._lib.snap_step_profiled(self._ctx, int(nsteps), ms.ctypes.data))
        return dict(rebuild=ms[0], sweep=ms[1], md=ms[2], step_end=ms[3])

    REBUILD_PHASES = ("cell_key", "scan", "scatter", "cell_sort", "gather", "copyback", "nlist", "done")

    def rebuild_profiled(self):
        """Force one neighbour-list rebuild and time each of its kernels (ms)."""
        ms = np.zeros(len(self.REBUILD_PHASES))
        self._check(self._lib.snap_rebuild_profiled(self._ctx, ms.ctypes.data))
        return dict(zip(self.REBUILD_PHASES, ms.tolist()))

    def bond_update(self):
        self._check(self._lib.snap_bond_update(self._ctx))

    def forces(self):
        f = np.zeros((self.n, 3))
        self._check(self._lib.snap_get_forces(self._ctx, f.ctypes.data))
        return f

    def bonds(self):
        """(m, 3) int64 array of (min tag, max tag, reaction), ascending."""
        n_out = C.c_int64(0)
        cap = max(16, self.n * 2)
        pairs = np.zeros(2 * cap, dtype=np.int32)
        rx = np.zeros(cap, dtype=np.int32)
        self._check(self._lib.snap_get_bonds(self._ctx, pairs.ctypes.data, rx.ctypes.data, cap,
                                             C.byref(n_out)))
        m = n_out.value
        return np.stack([pairs[0:2 * m:2], pairs[1:2 * m:2], rx[:m]], axis=1).astype(np.int64)

    @staticmethod
    def _out3(n, out):
        if out is None:
            return np.empty((n, 3))
        if out.dtype != np.float64 or out.shape != (n, 3) or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous float64 array of shape (n, 3)")
        return out

    def positions(self, out=None):
        """Wrapped positions in tag order; `out` (e.g. a pinned array) is filled in place."""
        p = self._out3(self.n, out)
        self._check(self._lib.snap_get_positions(self._ctx, p.ctypes.data))
        return p

    def velocities(self, out=None):
        v = self._out3(self.n, out)
        self._check(self._lib.snap_get_velocities(self._ctx, v.ctypes.data))
        return v

    def images(self):
        im = np.zeros((self.n, 3), dtype=np.int32)
        self._check(self._lib.snap_get_images(self._ctx, im.ctypes.data))
        return im

    def neighbors(self):
        n_out = C.c_int64(0)
        cap = max(64, self.n * 64)
        while True:
            pairs = np.zeros(2 * cap, dtype=np.int32)
            code = self._lib.snap_get_neighbors(self._ctx, pairs.ctypes.data, cap, C.byref(n_out))
            if code == 1 and n_out.value > cap:
                cap = n_out.value
                continue
            self._check(code)
            m = n_out.value
            return pairs[: 2 * m].reshape(m, 2).copy()

    def stats(self):
        s = _abi.Stats()
        self._check(self._lib.snap_get_stats(self._ctx, C.byref(s)))
        return s.as_dict()

    def energy(self):
        e = _abi.Energy()
        self._check(self._lib.snap_get_energy(self._ctx, C.byref(e)))
        return dict(e_pair=e.e_pair, e_bond=e.e_bond, kinetic=e.kinetic, virial=e.virial)

    def rdf_counts(self, type_a, type_b, r_max, nbins, replica=0):
        """Pair counts per distance bin behind g(r) (snap_get_rdf)."""
        h = np.zeros(int(nbins), dtype=np.int64)
        self._check(self._lib.snap_get_rdf(self._ctx, int(replica), int(type_a), int(type_b), float(r_max),
                                           int(nbins), h.ctypes.data))
        return h

    def lifetime_hist(self, nbins=256):
        h = np.zeros(nbins, dtype=np.int64)
        self._check(self._lib.snap_get_lifetime_hist(self._ctx, h.ctypes.data, int(nbins)))
        return h

    def get_state(self) -> bytes:
        n = C.c_size_t(0)
        self._check(self._lib.snap_get_state(self._ctx, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(self._lib.snap_get_state(self._ctx, buf, C.byref(n)))
        return buf.raw[: n.value]

    def set_state(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        self._check(self._lib.snap_set_state(self._ctx, buf, len(data)))

    def sync(self):
        self._check(self._lib.snap_sync(self._ctx))

    # -- Metropolis-Hastings moves and the event log -------------------------
    def set_mh(self, mode, mlp=None, eps_u=0.05):
        """mode 0: DyBond sweep; 1: MH, uniform proposal; 2: MH, learned proposal."""
        self._mlp = mlp  # the network must outlive its use by this context
        self._check(self._lib.snap_set_mh(self._ctx, int(mode), mlp._h if mlp is not None else None,
                                          float(eps_u)))

    def mh_sweep(self):
        self._check(self._lib.snap_mh_sweep(self._ctx))

    def set_step(self, step):
        self._check(self._lib.snap_set_step(self._ctx, int(step)))

    def log_events(self, capacity):
        self._check(self._lib.snap_log_events(self._ctx, int(capacity)))

    def get_events(self, clear=True):
        """Logged bond-formation events: (features[rows, 12] float32,
        offsets[events + 1] int32, labels[events] int32)."""
        ne, nr = C.c_int64(0), C.c_int64(0)
        code = self._lib.snap_get_events(self._ctx, None, None, None, 0, 0, C.byref(ne), C.byref(nr), 0)
        if code not in (0, 1):
            self._check(code)
        feat = np.zeros((max(nr.value, 1), 12), dtype=np.float32)
        off = np.zeros(ne.value + 1, dtype=np.int32)
        lab = np.zeros(max(ne.value, 1), dtype=np.int32)
        self._check(self._lib.snap_get_events(self._ctx, feat.ctypes.data, off.ctypes.data, lab.ctypes.data,
                                              ne.value, nr.value, C.byref(ne), C.byref(nr), int(clear)))
        return feat[: nr.value], off[: ne.value + 1], lab[: ne.value]


def mlp_init_weights(seed=0):
    """Initial FP32 parameters of the proposal network in the packed layout
    W1[16][64] (rows 12..15 zero), b1[64], W2[64][64], b2[64], w3[64], b3:
    zero biases and normal weights with variance 2 / fan-in (1 / fan-in for
    the linear output layer)."""
    rng = np.random.default_rng(seed)
    w1 = np.zeros((16, 64))
    w1[:12] = rng.normal(0.0, math.sqrt(2.0 / 12), (12, 64))
    w2 = rng.normal(0.0, math.sqrt(2.0 / 64), (64, 64))
    w3 = rng.normal(0.0, math.sqrt(1.0 / 64), 64)
    z = np.zeros(64)
    return np.concatenate([w1.ravel(), z, w2.ravel(), z, w3, [0.0]]).astype(np.float32)


class Mlp:
    """The 12 -> 64 -> 64 -> 1 proposal network on the tensor cores.  Device
    arrays are passed as integer pointers (e.g. torch tensor.data_ptr())."""

    NPARAM = 5313

    def __init__(self, weights=None, stream=None):
        self._lib = _abi.load()
        self._h = C.c_void_p()
        s = stream if stream is not None else 0
        code = self._lib.snap_mlp_create(C.byref(self._h), C.c_void_p(s))
        if code != 0:
            raise SnapError(code, "snap_mlp_create")
        if weights is not None:
            self.set_weights(weights)

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == self.NPARAM
        code = self._lib.snap_mlp_set_weights(self._h, w.ctypes.data)
        if code != 0:
            raise SnapError(code, "snap_mlp_set_weights")

    def weights(self):
        w = np.zeros(self.NPARAM, dtype=np.float32)
        code = self._lib.snap_mlp_get_weights(self._h, w.ctypes.data)
        if code != 0:
            raise SnapError(code, "snap_mlp_get_weights")
        return w

    def forward(self, d_feat, rows, d_logits):
        code = self._lib.snap_mlp_forward(self._h, d_feat, int(rows), d_logits)
        if code != 0:
            raise SnapError(code, "snap_mlp_forward")

    def loss_grad(self, d_feat, rows, d_offsets, d_labels, events):
        loss = C.c_double(0.0)
        g = np.zeros(self.NPARAM, dtype=np.float32)
        code = self._lib.snap_mlp_loss_grad(self._h, d_feat, int(rows), d_offsets, d_labels, int(events),
                                            C.byref(loss), g.ctypes.data)
        if code != 0:
            raise SnapError(code, "snap_mlp_loss_grad")
        return loss.value, g

    def train(self, d_feat, rows, d_offsets, d_labels, events, epochs=10, batch_events=4096, lr=1e-3,
              seed=0):
        losses = np.zeros(int(epochs))
        code = self._lib.snap_mlp_train(self._h, d_feat, int(rows), d_offsets, d_labels, int(events),
                                        int(epochs), int(batch_events), float(lr), int(seed),
                                        losses.ctypes.data)
        if code != 0:
            raise SnapError(code, "snap_mlp_train")
        return losses

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.snap_mlp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pair_energy_noalloc(n, d_pos3, d_type, box, sigma, eps_pair, rcut=None, d_out=None, stream=None):
    """Pair energy and virial of n particles whose positions (n*3 doubles) and
    types (n int32) are already on the device, written to d_out (2 doubles on
    the device).  Device pointers are integers (e.g. tensor.data_ptr()).  The
    library allocates nothing for this call (see snap_pair_energy_noalloc)."""
    lib = _abi.load()
    b = np.ascontiguousarray(box, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    ep = np.ascontiguousarray(eps_pair, dtype=np.float64)
    rc = None if rcut is None else np.ascontiguousarray(rcut, dtype=np.float64)
    code = lib.snap_pair_energy_noalloc(int(n), d_pos3, d_type, b.ctypes.data, sg.size,
                                        sg.ctypes.data, ep.ctypes.data,
                                        rc.ctypes.data if rc is not None else None, d_out, stream)
    if code != 0:
        raise SnapError(code, "snap_pair_energy_noalloc")


def from_system(sysdef, precision="mixed", p_on0=1.0, skin=None, list_block=None, list_subcells=None,
                **kw) -> Snap:
    """Build a context from a `synth.System` (or any object with the same fields).
    A list of systems becomes one batched context of independent replicas.
    `skin` overrides the systems' neighbour-list skin; `list_block` sets the
    list build's threads per block and `list_subcells` its sub-cells along x
    per cell."""
    systems = sysdef if isinstance(sysdef, (list, tuple)) else [sysdef]
    s0 = systems[0]
    n = sum(s.n for s in systems)
    reps = None
    if len(systems) > 1:
        reps = [dict(n=s.n, box=list(map(float, s.box)), kT=float(s.kT), seed=int(s.seed))
                for s in systems]
    sim = Snap(n, s0.box, dt=s0.dt, kT=s0.kT, gamma=s0.gamma, seed=s0.seed, precision=precision,
               bond_period=s0.bond_period, skin=s0.skin if skin is None else skin, replicas=reps, **kw)
    sim.set_types(s0.sigma, s0.eps_pair, s0.rcut)
    if list_block:
        sim.set_list_block(list_block)
    if list_subcells:
        sim.set_list_subcells(list_subcells)
    sim.set_valence(s0.valence)
    for i, bt in enumerate(s0.bond_types):
        sim.set_bond_params(i, bt.kind, bt.k, bt.r0, getattr(bt, "extra", ()) or ())
    off = 0
    for s in systems:
        if s.static_bonds.shape[0]:
            for t in np.unique(s.static_bond_types):
                sel = s.static_bond_types == t
                sim.add_static_bonds(s.static_bonds[sel] + off, int(t))
        off += s.n
    for r in s0.reactions:
        pon, poff = rates_from_eps(r.eps, p_on0, s0.dt, s0.bond_period)
        sim.add_reaction(r.type_a, r.type_b, r.bond_type, r.r_min, r.r_max, pon, poff, r.self_avoid)
    if len(systems) > 1:
        for ri, s in enumerate(systems):
            for a, r in enumerate(s.reactions):
                pon, poff = rates_from_eps(r.eps, p_on0, s.dt, s.bond_period)
                sim.set_reaction_rates(a, ri, pon, poff)
    for a, r in enumerate(s0.reactions):
        if getattr(r, "slip_a", 0.0):
            sim.set_slip(a, r.slip_a)
        if getattr(r, "melt", None) is not None:
            sim.set_melting(a, *r.melt)
    if getattr(s0, "kinetic_T", 0):
        sim.set_kinetic_temperature(True)
    pos = np.concatenate([s.pos for s in systems])
    vel = np.concatenate([s.vel for s in systems])
    types = np.concatenate([s.types for s in systems])
    sim.set_particles(pos, vel, types)
    return sim
