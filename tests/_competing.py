"""Helpers of the four-reaction tests (App. A, Eq. Z): exact state
probabilities of a frozen square and the state mask of every square."""
import math

import numpy as np

# bond bit of each reaction in a square's state mask (reactions in the order
# A-B, A-C, D-B, D-C)
AB, AC, DB, DC = 1, 2, 4, 8


def eq_z_states(eps):
    """Exact probabilities of the seven states of Eq. Z, keyed by bond mask."""
    kab, kac, kdb, kdc = (math.exp(e) for e in eps)
    w = {0: 1.0, AB: kab, AC: kac, DB: kdb, DC: kdc, AB | DC: kab * kdc, AC | DB: kac * kdb}
    z = sum(w.values())
    return {m: v / z for m, v in w.items()}


def square_masks(bonds, n_squares):
    """Bond mask of every square from (min tag, max tag, reaction) rows; a
    square's four particles have tags 4q .. 4q+3."""
    assert np.all(bonds[:, 0] // 4 == bonds[:, 1] // 4)   # no bond across squares
    mask = np.zeros(n_squares, np.int64)
    np.add.at(mask, bonds[:, 0] // 4, 1 << bonds[:, 2])
    return mask
