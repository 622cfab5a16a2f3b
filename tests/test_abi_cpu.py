"""Host-side checks that need no GPU: the C-ABI library loads, exports every
symbol include/snap.h declares, rejects bad configurations before touching
the device, and the rate closure (Eqs. 1-2) is consistent."""
import ctypes as C
import math
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    from paper_2609_21204_b300 import build, _abi
    build.build()
    return _abi.load()


def _declared_symbols():
    txt = (ROOT / "include" / "snap.h").read_text()
    return sorted(set(re.findall(r"\b(snap_[a-z_]+)\s*\(", txt)))


def test_header_declares_expected_entry_points():
    syms = _declared_symbols()
    for name in ("snap_init", "snap_set_types", "snap_set_valence", "snap_set_bond_params",
                 "snap_step", "snap_get_bonds", "snap_get_forces", "snap_bond_update",
                 "snap_add_reaction", "snap_destroy"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_2609_21204_b300 import _abi
    assert set(_declared_symbols()) == set(_abi.SIGNATURES)


def test_init_rejects_bad_config_without_device(lib):
    from paper_2609_21204_b300 import _abi
    ctx = C.c_void_p()
    good = dict(n=10, dt=0.005, kT=1.0, gamma=1.0, skin=0.3, bond_period=1, precision=1)
    bad_cases = [dict(dt=0.0), dict(kT=-1.0), dict(skin=0.0), dict(bond_period=0),
                 dict(precision=7), dict(n=-1), dict(block_size=33), dict(block_size=512)]
    for bad in bad_cases:
        cfg = _abi.Config()
        for k, v in {**good, **bad}.items():
            setattr(cfg, k, v)
        for d in range(3):
            cfg.box[d] = 10.0
        assert lib.snap_init(C.byref(ctx), C.byref(cfg)) == 1, bad
        assert not ctx.value
    assert lib.snap_init(None, None) == 1


def test_rate_closure():
    from paper_2609_21204_b300 import closure, rates_from_eps
    r = closure(0.005, 1, eps=5.0, p_on0=1.0)
    assert r["k_on"] == pytest.approx(200.0)
    assert r["p_off"] == pytest.approx(math.exp(-5.0))
    assert r["eps"] == pytest.approx(5.0)
    r2 = closure(0.005, 10, k_on=2.0, k_off=0.5)
    assert r2["p_on0"] == pytest.approx(0.1) and r2["eps"] == pytest.approx(math.log(4))
    with pytest.raises(ValueError):
        closure(0.005, 1, eps=5.0, p_on0=1.0, p_off=0.5)       # over-specified, inconsistent
    with pytest.raises(ValueError):
        closure(0.005, 1, k_on=1000.0, eps=1.0)                 # P_on^0 > 1
    with pytest.raises(ValueError):
        closure(0.005, 1, eps=1.0)                              # under-specified
    assert rates_from_eps(6.0) == (1.0, math.exp(-6.0))
