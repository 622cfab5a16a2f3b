"""Pins of the oracle's pair features and event extraction (learned-proposal
extension): a hand-worked three-particle example across the periodic
boundary, with and without an existing bond, and the event conditions."""
import numpy as np

from oracle.features import FeatureState, sweep_events
from synth import Reaction


def _state(partners):
    box = [10.0, 10.0, 10.0]
    # A at the corner; B1 at distance 1.0 through the x boundary, B2 at 1.2 along y
    pos = [[0.05, 5.0, 5.0], [9.05, 5.0, 5.0], [0.05, 6.2, 5.0]]
    rx = Reaction(type_a=0, type_b=1, bond_type=0, r_min=0.0, r_max=1.3, eps=1.0)
    return FeatureState(pos, box, [0, 1, 1], [2, 1], partners, rx, r0=1.1)


def test_features_worked_example():
    s = _state([[-1] * 4, [-1] * 4, [-1] * 4])
    idx, r = s.candidates(0)
    assert list(idx) == [1, 2]
    np.testing.assert_allclose(r, [1.0, 1.2], rtol=1e-12)
    rows, lab = s.event(0, 2)
    assert lab == 1
    e1 = [1.0, (1.0 - 1.1) / 1.3, 1, 0, 0, 1, 0.0, 0.0, 1, 1, 2 / 8, 1 / 8]
    e2 = [1.2, (1.2 - 1.1) / 1.3, 1, 0, 0, 1, 0.0, 0.0, 1, 1, 2 / 8, 1 / 8]
    np.testing.assert_allclose(rows, np.array([e1, e2], np.float32), rtol=1e-6, atol=1e-7)
    # B2 sees only A (B-B is not a reaction pair)
    assert s.coord(2) == 1 and list(s.candidates(2)[0]) == [0]


def test_features_with_existing_bond():
    s = _state([[2, -1, -1, -1], [-1] * 4, [0, -1, -1, -1]])
    idx, _ = s.candidates(0)
    assert list(idx) == [1]            # bonded partner excluded
    rows, lab = s.event(0, 1)
    assert lab == 0 and rows.shape == (1, 12)
    assert rows[0, 6] == np.float32(0.5) and rows[0, 8] == 1.0   # occ_A = 1 of 2, still free
    assert s.event(0, 2) is None       # not a candidate
    assert list(s.candidates(1)[0]) == [0]
    assert len(s.candidates(2)[0]) == 0   # B2 is full


def test_sweep_events_selects_own_formed_proposals():
    s = _state([[-1] * 4, [-1] * 4, [-1] * 4])
    prop = np.array([1, 0, 0])
    matched = np.array([1, 0, -1])
    formed = np.array([1, 1, 0], np.uint8)
    ev = sweep_events(s, prop, matched, formed)
    # site 0 proposed 1 and formed with it; site 1 proposed 0 and formed with it
    assert len(ev) == 2 and ev[0][1] == 0 and ev[1][1] == 0 and ev[1][0].shape == (1, 12)
