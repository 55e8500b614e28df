"""The score metric of the experiments (§4.2, eq. (score)): how well a CP decomposition recovers known
factors.

TEST INFRASTRUCTURE ONLY (CPU oracle, FP64).  Shares no code with the library or bench.py.

For two rank-one tensors the score is the product over the modes of the cosines between their factor
vectors (the weights are ignored).  For R > 1 the pair scores are averaged over the true components,
maximized over all ways of matching them to distinct estimated components (every permutation; with
more estimated than true components, every injective matching).
"""
import itertools

import numpy as np


def pair_scores(true_factors, est_factors):
    """Matrix S[k, r] = prod_n cos(a_k^(n), b_r^(n)) for true component k and estimated component r."""
    S = None
    for A, B in zip(true_factors, est_factors):
        An = A / np.linalg.norm(A, axis=0, keepdims=True)
        Bn = B / np.linalg.norm(B, axis=0, keepdims=True)
        C = An.T @ Bn
        S = C if S is None else S * C
    return S


def score(true_factors, est_factors):
    """Max over injective matchings of true components to estimated ones of the mean pair score
    (brute force over all matchings)."""
    S = pair_scores(true_factors, est_factors)
    Rt, Re = S.shape
    best = -np.inf
    for perm in itertools.permutations(range(Re), Rt):
        best = max(best, float(np.mean(S[np.arange(Rt), list(perm)])))
    return best
