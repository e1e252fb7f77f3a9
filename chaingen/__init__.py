"""Seeded synthetic Markov chains shaped like the test problems of Section 7.

This package only builds inputs: column-stochastic transition matrices ``A``
(``a_ij`` = probability of the move j -> i, Section 2) in CSR form, with the
grid shape where the chain has one.  It holds none of the multigrid method's
arithmetic, so both the CPU oracle and the CUDA library may consume it.
"""
from .chains import (Chain, lattice2d, uniform2d, tandem, birth_death,
                     delaunay_walk, chain_mix, training_mix, to_dense)

__all__ = ["Chain", "lattice2d", "uniform2d", "tandem", "birth_death",
           "delaunay_walk", "chain_mix", "training_mix", "to_dense"]
