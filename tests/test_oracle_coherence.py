"""Pins for leverage scores and the coherence lemmas of §3.2.2 (CPU only)."""
import json
import os

import numpy as np

from oracle import coherence, cp

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_leverage_scores_match_svd_definition():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((30, 4))
    U = np.linalg.svd(A, full_matrices=False)[0]
    np.testing.assert_allclose(coherence.leverage_scores(A), np.sum(U * U, axis=1), atol=1e-13)


def test_coherence_range():
    rng = np.random.default_rng(1)
    for n, d in [(10, 3), (50, 5), (7, 7)]:
        mu = coherence.coherence(rng.standard_normal((n, d)))
        assert d / n - 1e-12 <= mu <= 1 + 1e-12
    # a row holding the only nonzero of a column has leverage 1
    A = np.vstack([np.eye(2), np.zeros((3, 2))])
    A[2:, 0] = 1.0
    assert abs(coherence.coherence(A) - 1.0) < 1e-12


def test_lemma_kronecker_coherence_is_product():
    rng = np.random.default_rng(2)
    for _ in range(5):
        A, B = rng.standard_normal((6, 2)), rng.standard_normal((5, 3))
        assert abs(coherence.coherence(np.kron(A, B))
                   - coherence.coherence(A) * coherence.coherence(B)) < 1e-12


def test_lemma_khatri_rao_coherence_bound():
    rng = np.random.default_rng(3)
    for _ in range(20):
        A = rng.standard_normal((8, 3)) ** 3
        B = rng.standard_normal((9, 3)) ** 3
        assert coherence.coherence(cp.khatri_rao([A, B])) <= \
            coherence.coherence(A) * coherence.coherence(B) + 1e-12


def test_lemma_khatri_rao_bound_is_tight_on_paper_example():
    ex = GOLDEN["coherence_tight_example"]
    A, B = np.array(ex["A"]), np.array(ex["B"])
    muA, muB = coherence.coherence(A), coherence.coherence(B)
    assert abs(muA - 0.5) < 1e-15 and abs(muB - 0.5) < 1e-15
    assert abs(coherence.coherence(cp.khatri_rao([A, B])) - muA * muB) < 1e-15
