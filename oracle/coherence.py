"""Leverage scores and coherence (§2.2 definitions, §3.2.2 lemmas).

TEST INFRASTRUCTURE ONLY (CPU oracle).
"""
import numpy as np


def leverage_scores(A):
    """l_i = ||U(i, :)||_2^2 with U the left singular vectors of A (n x d, full column rank),
    §2.2 definition.  A thin QR spans the same column space, so its Q rows give the same scores."""
    Q, _ = np.linalg.qr(A, mode="reduced")
    return np.sum(Q * Q, axis=1)


def coherence(A):
    """mu(A) = max_i l_i  (§2.2); d / n <= mu <= 1."""
    return float(np.max(leverage_scores(A)))


def kron(A, B):
    return np.kron(A, B)
