"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

Holds geometry and parameter values only; no dynamic-bonding arithmetic."""
from .configs import (System, Reaction, BondType, HARMONIC, FENE, FENEWCA, TETHER, assoc_ab, telechelic,
                      colloid_linker, telechelic_sweep, telechelic_sweep_specs, frozen_pairs,
                      random_frozen, frozen_stars, frozen_squares, four_reaction_soup,
                      frozen_loops, telechelic_rings)

__all__ = ["System", "Reaction", "BondType", "HARMONIC", "FENE", "FENEWCA", "TETHER", "assoc_ab", "telechelic",
           "colloid_linker", "telechelic_sweep", "telechelic_sweep_specs", "frozen_pairs",
           "random_frozen", "frozen_stars", "frozen_squares", "four_reaction_soup",
           "frozen_loops", "telechelic_rings"]
