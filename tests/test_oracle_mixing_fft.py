"""Pins of the complex-transform CPRAND-MIX oracle (Alg. 4): the DFT against NumPy's FFT, the mixed
tensor against an N-dimensional FFT, the reduction to CPRAND without mixing, the exact ALS update
when every fiber is sampled (the unitary mixing leaves the least-squares solution unchanged), the
real least squares on an exactly solvable problem, and exact recovery of a noiseless CP tensor."""
import itertools

import numpy as np

from oracle import cp, mixing_fft, streams


def test_dft_matrix_is_numpy_fft_and_unitary():
    for I in (1, 2, 7, 16, 45):
        F = mixing_fft.dft_matrix(I)
        np.testing.assert_allclose(F, np.fft.fft(np.eye(I), axis=0) / np.sqrt(I), atol=1e-13)
        np.testing.assert_allclose(F @ F.conj().T, np.eye(I), atol=1e-13)


def test_mixed_tensor_is_an_n_dimensional_fft_of_the_sign_flipped_tensor():
    dims = (6, 5, 4)
    rng = np.random.default_rng(1)
    T = rng.standard_normal(dims)
    ops = mixing_fft.dft_operators(11, 2, dims)
    D = np.ones(dims)
    for n, I in enumerate(dims):
        d = streams.sign_vector(11, 2, n, I)
        D = D * d.reshape([I if m == n else 1 for m in range(len(dims))])
    ref = np.fft.fftn(T * D, norm="ortho")
    Th = mixing_fft.mix_tensor(T, ops)
    np.testing.assert_allclose(Th, ref, atol=1e-12)
    assert abs(np.linalg.norm(Th) - np.linalg.norm(T)) < 1e-12 * np.linalg.norm(T)


def test_mixed_cp_model_is_model_of_mixed_factors():
    dims, R = (5, 4, 6), 3
    rng = np.random.default_rng(2)
    lam = rng.random(R)
    A = [rng.standard_normal((I, R)) for I in dims]
    ops = mixing_fft.dft_operators(3, 0, dims)
    lhs = mixing_fft.mix_tensor(cp.full_tensor(lam, A), ops)
    N = len(dims)
    rhs = np.einsum("r,ir,jr,kr->ijk", lam, *[ops[m] @ A[m] for m in range(N)])
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


def test_real_ls_recovers_an_exact_real_solution():
    rng = np.random.default_rng(3)
    S, R, I = 30, 4, 7
    Z = rng.standard_normal((S, R)) + 1j * rng.standard_normal((S, R))
    A0 = rng.standard_normal((I, R))
    X = A0 @ Z.T                                  # I x S, complex
    np.testing.assert_allclose(mixing_fft.real_ls(Z, X), A0, atol=1e-12)


def test_identity_mixing_reduces_to_cprand():
    dims = (12, 10, 9)
    rng = np.random.default_rng(4)
    T = rng.standard_normal(dims)
    rule = lambda: cp.StopRule(fixed_iters=4)
    a = mixing_fft.cprand_mix_fft(T, 3, 25, seed=5, rule=rule(), identity=True)
    b = cp.cprand(T, 3, 25, seed=5, rule=rule())
    np.testing.assert_allclose(a["fits"], b["fits"], atol=1e-10)
    for A, B in zip(a["factors"], b["factors"]):
        np.testing.assert_allclose(A, B, atol=1e-9)


def test_full_sampling_gives_the_exact_als_update():
    # every fiber sampled once: D_n F_n^* X^_(n) = X_(n) K^T with K unitary, so the stacked real
    # problem has the normal equations of the exact update (Alg. 1)
    dims, R = (5, 4, 3), 2
    rng = np.random.default_rng(5)
    T = rng.standard_normal(dims)
    ops = mixing_fft.dft_operators(7, 0, dims)
    Th = mixing_fft.mix_tensor(T, ops)
    factors = [rng.standard_normal((I, R)) for I in dims]
    mixed = [ops[m] @ factors[m] for m in range(3)]
    for n in range(3):
        others = [range(I) if m != n else [0] for m, I in enumerate(dims)]
        idx = np.array(list(itertools.product(*others)), dtype=np.int64)
        A, lam, Ah = mixing_fft.update(Th, ops, mixed, n, idx)
        A_ref, lam_ref = cp.cp_als_update(T, factors, n)
        np.testing.assert_allclose(A, A_ref, atol=1e-10)
        np.testing.assert_allclose(lam, lam_ref, atol=1e-10)
        np.testing.assert_allclose(Ah, ops[n] @ A, atol=1e-12)


def test_noiseless_cp_tensor_is_recovered():
    dims, R = (14, 12, 10), 3
    rng = np.random.default_rng(6)
    A = [rng.standard_normal((I, R)) for I in dims]
    T = cp.full_tensor(np.ones(R), A)
    out = mixing_fft.cprand_mix_fft(T, R, 40, seed=9, rule=cp.StopRule(fixed_iters=30))
    assert cp.exact_fit(T, out["lam"], out["factors"]) > 1 - 1e-6
