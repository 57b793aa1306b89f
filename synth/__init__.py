"""Seeded synthetic protein and nucleotide families and model parameters.

This module is the only code shared by the CUDA path's tests/benchmarks and the
oracle's tests.  It produces *inputs*: residue strings, family layouts, arrival
schedules and the numeric model parameters.  It contains none of the posterior
method's arithmetic (no DP, no posterior, no MEA, no distance).
"""
from .families import (ALPHABET, NUCLEOTIDES, Family, background, nucleotide_background, evolve, make_family,
                       star_family, tree_family, domain_family, pair_index, make_serving_trace,
                       family_from_strings, random_guide_tree, CONFIGS)
from .params import ModelParams, default_params, gtr_joint, nucleotide_params

__all__ = [
    "ALPHABET", "NUCLEOTIDES", "Family", "background", "nucleotide_background", "evolve", "make_family", "star_family", "tree_family", "domain_family", "pair_index",
    "make_serving_trace", "family_from_strings", "random_guide_tree", "CONFIGS",
    "ModelParams", "default_params", "gtr_joint", "nucleotide_params",
]
