"""Pins of the score oracle (eq. (score)): perfect recovery scores 1 whatever the order, scaling and
paired sign flips of the components; a hand-computed two-component case; an extra estimated component
is ignored when it helps no match; the brute force equals an exhaustive check of a tiny case."""
import numpy as np

from oracle import score


def test_exact_recovery_scores_one_under_permutation_scaling_and_sign_pairs():
    rng = np.random.default_rng(1)
    A = [rng.standard_normal((I, 4)) for I in (9, 8, 7)]
    perm = [2, 0, 3, 1]
    B = [A[0][:, perm] * np.array([2.0, 0.5, 3.0, 1.0]), -A[1][:, perm], -A[2][:, perm] * 7.0]
    assert abs(score.score(A, B) - 1.0) < 1e-12


def test_two_component_closed_form():
    # orthonormal true components; the estimate's first component is rotated by theta in mode 1 only
    e = np.eye(3)
    A = [e[:, :2], e[:, :2], e[:, :2]]
    th = 0.3
    b0 = np.cos(th) * e[:, 0] + np.sin(th) * e[:, 2]
    B = [np.stack([b0, e[:, 1]], axis=1), e[:, :2], e[:, :2]]
    assert abs(score.score(A, B) - (np.cos(th) + 1.0) / 2.0) < 1e-12


def test_extra_estimated_component():
    rng = np.random.default_rng(2)
    A = [rng.standard_normal((I, 3)) for I in (6, 5, 4)]
    junk = [rng.standard_normal((I, 1)) for I in (6, 5, 4)]
    B = [np.concatenate([j, a[:, ::-1]], axis=1) for a, j in zip(A, junk)]
    assert abs(score.score(A, B) - 1.0) < 1e-12


def test_matches_exhaustive_pair_enumeration():
    rng = np.random.default_rng(3)
    A = [rng.standard_normal((I, 2)) for I in (4, 4, 4)]
    B = [rng.standard_normal((I, 3)) for I in (4, 4, 4)]
    S = np.ones((2, 3))
    for a, b in zip(A, B):
        for k in range(2):
            for r in range(3):
                S[k, r] *= a[:, k] @ b[:, r] / np.linalg.norm(a[:, k]) / np.linalg.norm(b[:, r])
    best = max((S[0, r0] + S[1, r1]) / 2 for r0 in range(3) for r1 in range(3) if r0 != r1)
    assert abs(score.score(A, B) - best) < 1e-12


def test_benchmark_score_by_assignment_equals_the_brute_force():
    # bench.py scores the recovery study by linear assignment on the pair-score matrix; the oracle
    # enumerates every matching
    import bench
    rng = np.random.default_rng(4)
    for Rt, Re in ((5, 5), (5, 6), (3, 4)):
        A = [rng.standard_normal((I, Rt)) for I in (7, 6, 5)]
        B = [a[:, rng.permutation(Rt)] @ np.eye(Rt, Re) + 0.3 * rng.standard_normal((a.shape[0], Re)) for a in A]
        assert abs(bench.score_assignment(A, B) - score.score(A, B)) < 1e-12
