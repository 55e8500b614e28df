"""Checks of the shared input generator (not the method): congruence, noise level, layout."""
import numpy as np
import torch

from oracle import cp
from synth import collinear_factor, make_problem, to_oracle_array, batch_problem_specs


def test_collinear_factor_has_exact_congruence():
    rng = np.random.default_rng(0)
    for C in [0.0, 0.5, 0.9]:
        A = collinear_factor(rng, 40, 6, C)
        G = A.T @ A
        np.testing.assert_allclose(np.diag(G), 1.0, atol=1e-12)
        off = G[~np.eye(6, dtype=bool)]
        np.testing.assert_allclose(off, C, atol=1e-12)


def test_noiseless_problem_is_cp_model_in_column_major_order():
    dims = (5, 6, 7)
    prob = make_problem(dims, 3, C=0.5, eta=0.0, seed=1, dtype=torch.float64)
    T = to_oracle_array(prob.X, dims)
    np.testing.assert_allclose(T, cp.full_tensor(prob.lam, prob.factors), atol=1e-13)
    assert np.all((prob.lam >= 0.2) & (prob.lam <= 0.8))


def test_noise_level_is_eta():
    dims = (20, 21, 22)
    clean = make_problem(dims, 3, C=0.2, eta=0.0, seed=2, dtype=torch.float64)
    noisy = make_problem(dims, 3, C=0.2, eta=0.05, seed=2, dtype=torch.float64)
    N = (noisy.X - clean.X).norm().item()
    assert abs(N / clean.X.norm().item() - 0.05) < 1e-12


def test_gaussian_factors_and_dtypes():
    p = make_problem((10, 11, 12), 5, eta=0.01, seed=3, gaussian_factors=True, dtype=torch.float64)
    assert np.all(p.lam == 1.0)
    q = make_problem((10, 11, 12), 5, eta=0.01, seed=3, gaussian_factors=True,
                     dtype=torch.bfloat16)
    assert q.X.dtype == torch.bfloat16 and q.X.numel() == 1320


def test_batch_specs_ranges():
    specs = batch_problem_specs(4, B=64)
    assert len(specs) == 64
    for s in specs:
        assert all(64 <= d <= 512 for d in s["dims"]) and 4 <= s["R"] <= 32
        assert 0.0 <= s["C"] <= 0.9
