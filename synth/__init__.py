"""Seeded synthetic inputs of the shape the paper's experiments use (§4.2, Synthetic Data).

This module produces INPUTS only: ground-truth weights and factors, and the stored dense tensor
X = X_true + eta (||X_true|| / ||N||) N.  It holds none of CPRAND's arithmetic (no sampling, no
least squares, no mixing, no fit estimate).  Both the CUDA path and the CPU oracle consume what
it produces; neither imports the other.

Factor matrices with collinearity C (any two columns of a factor have cosine exactly C): the
paper defers to Tomasi & Bro (2006) for the construction; the reading taken here is
A = Q L^T, with Q the orthonormal basis of an I x R Gaussian matrix and L the Cholesky factor of
(1 - C) I + C 1 1^T, which gives unit columns with pairwise inner product C (needs I >= R).

Storage is column-major (i_1 fastest, the order of the §2.1 unfolding): a tensor is returned as a
flat 1-D torch tensor plus its dims.
"""
from .generate import (Problem, collinear_factor, make_problem, to_oracle_array,
                       batch_problem_specs)

__all__ = ["Problem", "collinear_factor", "make_problem", "to_oracle_array",
           "batch_problem_specs"]
