"""Pins for the oracle's mixing preprocess and CPRAND-MIX (Alg. 5), CPU only."""
import numpy as np
import pytest
import scipy.fft

from oracle import cp, mixing
from synth import make_problem, to_oracle_array


@pytest.mark.parametrize("I", [1, 2, 7, 64, 400])
def test_dct_matrix_matches_library_and_is_orthogonal(I):
    F = mixing.dct2_matrix(I)
    ref = scipy.fft.dct(np.eye(I), type=2, norm="ortho", axis=0)   # column i = DCT of e_i
    np.testing.assert_allclose(F, ref, rtol=0, atol=1e-13)
    np.testing.assert_allclose(F @ F.T, np.eye(I), rtol=0, atol=1e-13)


def test_mixing_preserves_norm_and_unmixes():
    dims = (6, 7, 5)
    rng = np.random.default_rng(0)
    T = rng.standard_normal(dims)
    ops = mixing.mixing_operators(12, 0, dims)
    Th = mixing.mix_tensor(T, ops)
    assert abs(np.linalg.norm(Th) - np.linalg.norm(T)) < 1e-12 * np.linalg.norm(T)
    back = T
    Y = Th
    for n, U in enumerate(ops):
        Y = cp.mode_product(Y, U.T, n)
    np.testing.assert_allclose(Y, T, rtol=0, atol=1e-12)
    factors = [rng.standard_normal((d, 3)) for d in dims]
    np.testing.assert_allclose(mixing.unmix_factors(mixing.mix_factors(factors, ops), ops)[1],
                               factors[1], atol=1e-12)


def test_mixed_cp_model_is_model_of_mixed_factors():
    # eq. (ttensor) with eq. (krdist): mixing a CP tensor mixes each factor
    dims = (5, 4, 6)
    rng = np.random.default_rng(1)
    lam = rng.uniform(0.2, 0.8, 3)
    factors = [rng.standard_normal((d, 3)) for d in dims]
    ops = mixing.mixing_operators(3, 0, dims)
    lhs = mixing.mix_tensor(cp.full_tensor(lam, factors), ops)
    rhs = cp.full_tensor(lam, mixing.mix_factors(factors, ops))
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12)
    # column norms (so lambda) are invariant under the orthogonal mixing
    for A, Ah in zip(factors, mixing.mix_factors(factors, ops)):
        np.testing.assert_allclose(np.linalg.norm(A, axis=0), np.linalg.norm(Ah, axis=0),
                                   rtol=1e-12)


def test_identity_mixing_reduces_to_cprand():
    dims = (14, 12, 10)
    import torch
    prob = make_problem(dims, 3, C=0.5, eta=0.01, seed=5, dtype=torch.float64)
    T = to_oracle_array(prob.X, dims)
    a = mixing.cprand_mix(T, 3, 40, seed=9, identity=True,
                          rule=cp.StopRule(fixed_iters=4))
    b = cp.cprand(T, 3, 40, seed=9, rule=cp.StopRule(fixed_iters=4))
    for x, y in zip(a["factors"], b["factors"]):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a["lam"], b["lam"])


def test_premix_solution_fits_original_tensor_as_mixed_fits_mixed():
    # Alg. 5: CPRAND in the mixed basis, then unmix; orthogonality makes the two fits equal
    dims = (16, 12, 14)
    import torch
    prob = make_problem(dims, 3, C=0.5, eta=0.01, seed=6, dtype=torch.float64)
    T = to_oracle_array(prob.X, dims)
    out = mixing.cprand_mix(T, 3, 60, seed=10, rule=cp.StopRule(fixed_iters=15))
    f_orig = cp.exact_fit(T, out["lam"], out["factors"])
    f_mix = cp.exact_fit(out["T_mixed"], out["lam"], out["factors_mixed"])
    assert abs(f_orig - f_mix) < 1e-12
    assert f_orig > 0.98
