"""ctypes declarations of the C ABI in include/snap.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
from pathlib import Path

LIB_PATH = Path(__file__).resolve().parent / "libsnap_b300.so"

SNAP_OK = 0
STATUS_NAMES = {0: "SNAP_OK", 1: "SNAP_ERR_ARG", 2: "SNAP_ERR_STATE", 3: "SNAP_ERR_CUDA",
                4: "SNAP_ERR_OOM", 5: "SNAP_ERR_NLIST_OVERFLOW", 6: "SNAP_ERR_FENE_OVERSTRETCH",
                7: "SNAP_ERR_NONFINITE", 8: "SNAP_ERR_TIMEOUT"}
SNAP_FP64, SNAP_MIXED = 0, 1
SNAP_HARMONIC, SNAP_FENE = 0, 1

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Config(C.Structure):
    _fields_ = [("n", C.c_int64), ("box", C.c_double * 3), ("dt", C.c_double),
                ("kT", C.c_double), ("gamma", C.c_double), ("seed", C.c_uint64),
                ("precision", C.c_int32), ("bond_period", C.c_int32), ("skin", C.c_double),
                ("n_replicas", C.c_int32), ("replica_n", C.POINTER(C.c_int64)),
                ("replica_box", C.POINTER(C.c_double)), ("replica_kT", C.POINTER(C.c_double)),
                ("replica_seed", C.POINTER(C.c_uint64)), ("stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
                ("block_size", C.c_int32), ("nlist_capacity", C.c_int32),
                ("lifetime_bins", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in (
        "step", "n_bonds", "sweeps", "formed_total", "broken_total", "scanned", "in_window",
        "proposals", "edges", "survivors", "formed", "break_tested", "broken",
        "nlist_builds", "nlist_entries", "mh_form_attempts", "mh_form_accepts", "mh_break_attempts",
        "mh_break_accepts", "events_logged", "rnlist_entries", "rebuild_launches")] + [("nlist_capacity", C.c_int32), ("status", C.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Energy(C.Structure):
    _fields_ = [("e_pair", C.c_double), ("e_bond", C.c_double), ("kinetic", C.c_double),
                ("virial", C.c_double)]


_P = C.c_void_p
# name -> (restype, argtypes)
SIGNATURES = {
    "snap_init": (C.c_int, [C.POINTER(_P), C.POINTER(Config)]),
    "snap_set_types": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "snap_set_valence": (C.c_int, [_P, _P]),
    "snap_set_bond_params": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_double, C.c_double]),
    "snap_set_bond_params_ex": (C.c_int, [_P, C.c_int32, C.c_int32, _P, C.c_int32]),
    "snap_add_static_bonds": (C.c_int, [_P, C.c_int64, _P, C.c_int32]),
    "snap_add_reaction": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double,
                                    C.c_double, C.c_double, C.c_int32, C.POINTER(C.c_int32)]),
    "snap_set_reaction_rates": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_double, C.c_double]),
    "snap_set_slip": (C.c_int, [_P, C.c_int32, C.c_double]),
    "snap_set_melting": (C.c_int, [_P, C.c_int32] + [C.c_double] * 6),
    "snap_set_particles": (C.c_int, [_P, _P, _P, _P]),
    "snap_set_positions": (C.c_int, [_P, _P, _P]),
    "snap_set_bonds": (C.c_int, [_P, C.c_int64, _P, _P]),
    "snap_step": (C.c_int, [_P, C.c_int64]),
    "snap_prepare": (C.c_int, [_P]),
    "snap_set_retry_limit": (C.c_int, [_P, C.c_int32]),
    "snap_set_list_block": (C.c_int, [_P, C.c_int32]),
    "snap_set_list_subcells": (C.c_int, [_P, C.c_int32]),
    "snap_get_list_subcells": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "snap_set_kinetic_temperature": (C.c_int, [_P, C.c_int32]),
    "snap_step_profiled": (C.c_int, [_P, C.c_int64, _P]),
    "snap_bond_update": (C.c_int, [_P]),
    "snap_get_forces": (C.c_int, [_P, _P]),
    "snap_get_bonds": (C.c_int, [_P, _P, _P, C.c_int64, C.POINTER(C.c_int64)]),
    "snap_get_positions": (C.c_int, [_P, _P]),
    "snap_get_velocities": (C.c_int, [_P, _P]),
    "snap_get_images": (C.c_int, [_P, _P]),
    "snap_get_neighbors": (C.c_int, [_P, _P, C.c_int64, C.POINTER(C.c_int64)]),
    "snap_get_stats": (C.c_int, [_P, C.POINTER(Stats)]),
    "snap_get_rdf": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_int32, _P]),
    "snap_get_energy": (C.c_int, [_P, C.POINTER(Energy)]),
    "snap_get_lifetime_hist": (C.c_int, [_P, _P, C.c_int32]),
    "snap_get_state": (C.c_int, [_P, _P, C.POINTER(C.c_size_t)]),
    "snap_set_state": (C.c_int, [_P, _P, C.c_size_t]),
    "snap_set_mh": (C.c_int, [_P, C.c_int32, _P, C.c_double]),
    "snap_mh_sweep": (C.c_int, [_P]),
    "snap_set_step": (C.c_int, [_P, C.c_int64]),
    "snap_rebuild_profiled": (C.c_int, [_P, _P]),
    "snap_log_events": (C.c_int, [_P, C.c_int64]),
    "snap_get_events": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_int64, C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64), C.c_int32]),
    "snap_mlp_create": (C.c_int, [C.POINTER(_P), _P]),
    "snap_mlp_set_weights": (C.c_int, [_P, _P]),
    "snap_mlp_get_weights": (C.c_int, [_P, _P]),
    "snap_mlp_forward": (C.c_int, [_P, _P, C.c_int64, _P]),
    "snap_mlp_loss_grad": (C.c_int, [_P, _P, C.c_int64, _P, _P, C.c_int64, C.POINTER(C.c_double), _P]),
    "snap_mlp_train": (C.c_int, [_P, _P, C.c_int64, _P, _P, C.c_int64, C.c_int32, C.c_int64, C.c_float,
                                 C.c_uint64, _P]),
    "snap_mlp_destroy": (None, [_P]),
    "snap_pair_energy_noalloc": (C.c_int, [C.c_int64, _P, _P, _P, C.c_int32, _P, _P, _P, _P, _P]),
    "snap_sync": (C.c_int, [_P]),
    "snap_last_error": (C.c_char_p, [_P]),
    "snap_destroy": (None, [_P]),
}

_lib = None


def load(path: Path | None = None):
    """Load the CUDA library; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise RuntimeError(f"{p} is missing: build the CUDA extension first "
                           "(python -m paper_2609_21204_b300.build)")
    lib = C.CDLL(str(p))
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
