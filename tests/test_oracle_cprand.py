"""Pins for the oracle's CP-ALS, CPRAND, stopping rules and sampled fit (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import cp, streams
from synth import make_problem, to_oracle_array

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _noiseless(dims, R, seed=0, C=0.0):
    prob = make_problem(dims, R, C=C, eta=0.0, seed=seed, dtype=__import__("torch").float64)
    return to_oracle_array(prob.X, dims), prob


def test_sample_size_rule_matches_paper():
    for R, S in GOLDEN["sample_size"]["R_to_S"].items():
        assert cp.sample_size(int(R)) == S


def test_chernoff_gamma_value():
    g = GOLDEN["chernoff_gamma"]
    assert abs((g["sqrt_one_plus_gamma"] ** 2 - 1.0) - g["gamma"]) < 1e-12


def test_full_row_sample_reduces_to_cp_als_update():
    # With every row of Z^(n) taken exactly once, Alg. 3's LS problem is Alg. 1's.
    dims = (5, 4, 6)
    rng = np.random.default_rng(0)
    T = rng.standard_normal(dims)
    factors = [rng.standard_normal((d, 3)) for d in dims]
    for n in range(3):
        others = [m for m in range(3) if m != n]
        grid = np.array(np.meshgrid(*[np.arange(dims[m]) for m in others], indexing="ij"))
        idx = np.zeros((int(np.prod([dims[m] for m in others])), 3), dtype=np.int64)
        for k, m in enumerate(others):
            idx[:, m] = grid[k].ravel()
        A1, l1 = cp.cprand_update(T, factors, n, idx)
        A2, l2 = cp.cp_als_update(T, factors, n)
        np.testing.assert_allclose(A1, A2, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(l1, l2, rtol=1e-10)


def test_true_factors_are_a_fixed_point_of_sampled_update():
    # noiseless rank-R data: the sampled system is consistent, so the truth solves it exactly
    dims = (20, 15, 12)
    T, prob = _noiseless(dims, 4, seed=3, C=0.5)
    for n in range(3):
        idx = streams.ls_sample_indices(5, 0, 0, n, 40, dims)
        A, lam = cp.cprand_update(T, [f.copy() for f in prob.factors], n, idx)
        np.testing.assert_allclose(A, prob.factors[n], rtol=0, atol=1e-10)
        np.testing.assert_allclose(lam, prob.lam, rtol=1e-10)


def test_cp_als_recovers_noiseless_tensor():
    dims = (12, 10, 9)
    T, prob = _noiseless(dims, 3, seed=1, C=0.3)
    f0 = [streams.init_factor(4, 0, n, d, 3) for n, d in enumerate(dims)]
    lam, factors, iters, fits = cp.cp_als(T, 3, f0, max_iters=500, tol=1e-12)
    assert fits[-1] > 1 - 1e-6
    # monotone (up to rounding) for exact ALS
    assert np.all(np.diff(fits) > -1e-10)


def test_cprand_recovers_noiseless_tensor():
    dims = (30, 25, 20)
    T, prob = _noiseless(dims, 4, seed=2, C=0.5)
    S = cp.sample_size(4) + 20
    out = cp.cprand(T, 4, S, seed=17, rule=cp.StopRule(max_iters=300, tol=0, stall_iters=0))
    assert cp.exact_fit(T, out["lam"], out["factors"]) > 1 - 1e-6


def test_stop_rules():
    r = cp.StopRule(max_iters=5, tol=1e-4)
    assert [r.update(f) for f in [0.1, 0.5, 0.6, 0.7, 0.8]] == [False, False, False, False, True]
    r = cp.StopRule(max_iters=200, tol=1e-4)
    assert [r.update(f) for f in [0.5, 0.50005]] == [False, True]
    r = cp.StopRule(max_iters=200, tol=1e-4, eta=0.01)
    assert [r.update(f) for f in [0.5, 0.98, 0.9881]] == [False, False, True]
    r = cp.StopRule(max_iters=200, tol=-1.0, stall_iters=2)
    assert [r.update(f) for f in [0.5, 0.6, 0.55, 0.58]] == [False, False, False, True]
    r = cp.StopRule(fixed_iters=3, tol=1.0, eta=0.5)
    assert [r.update(f) for f in [0.9, 0.9, 0.9]] == [False, False, True]


def test_sampled_fit_with_every_entry_is_exact_fit():
    dims = (6, 5, 4)
    rng = np.random.default_rng(3)
    T = rng.standard_normal(dims)
    lam = rng.uniform(0.2, 0.8, 3)
    factors = [rng.standard_normal((d, 3)) for d in dims]
    idx = np.array(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij")).reshape(3, -1).T
    x = T[tuple(idx[:, m] for m in range(3))]
    P = T.size
    f = cp.sampled_fit(x, lam, factors, idx, np.linalg.norm(T), P)
    assert abs(f - cp.exact_fit(T, lam, factors)) < 1e-12


def test_sampled_error_is_unbiased():
    # E[P * mean_i e_i^2] = ||E||^2 for i.i.d. uniform entries (§3.4)
    dims = (8, 9, 10)
    rng = np.random.default_rng(4)
    E = rng.standard_normal(dims) ** 3           # heavy-ish tails
    P = E.size
    est = []
    for s in range(4000):
        idx = streams.fit_sample_indices(1000 + s, 0, 64, dims)
        e = E[tuple(idx[:, m] for m in range(3))]
        est.append(P * np.mean(e * e))
    est = np.array(est)
    truth = np.sum(E * E)
    assert abs(est.mean() - truth) < 4 * est.std() / np.sqrt(est.size)


def test_sampled_fit_accuracy_at_95_percent():
    # §4.1: P_hat = 2^14, fit 95% -> largest relative error of the estimate below 1e-3
    g = GOLDEN["sampled_fit_accuracy"]
    dims = (60, 50, 40)
    prob = make_problem(dims, 5, C=0.5, eta=1.0 - g["fit"], seed=8,
                        dtype=__import__("torch").float64)
    T = to_oracle_array(prob.X, dims)
    lam, factors = prob.lam, prob.factors
    F = cp.exact_fit(T, lam, factors)
    assert abs(F - g["fit"]) < 2e-3
    worst = 0.0
    for s in range(20):
        idx = streams.fit_sample_indices(300 + s, 0, g["P_hat"], dims)
        x = T[tuple(idx[:, m] for m in range(3))]
        Fh = cp.sampled_fit(x, lam, factors, idx, np.linalg.norm(T), T.size)
        worst = max(worst, abs(Fh - F) / F)
    assert worst < g["max_rel_error"]
