"""Seeded synthetic input generators shared by the oracle, the tests and the benchmark."""
from .tightbinding import (Pencil, make_pair, perfect_diamond_pencil, sband_cubic_pencil,
                           diagonal_pencil, workload, neighbour_pairs, diamond_sites)

__all__ = ["Pencil", "make_pair", "perfect_diamond_pencil", "sband_cubic_pencil",
           "diagonal_pencil", "workload", "neighbour_pairs", "diamond_sites"]
