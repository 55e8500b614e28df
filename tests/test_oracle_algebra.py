"""Pins for the oracle's §2.1 tensor algebra: brute-force loops and closed-form identities."""
import itertools

import numpy as np
import pytest

from oracle import cp


def _brute_unfold(T, n):
    """X_(n) by looping over every entry and applying the §2.1 index map term by term."""
    dims = T.shape
    N = len(dims)
    ncols = int(np.prod([dims[k] for k in range(N) if k != n]))
    U = np.zeros((dims[n], ncols))
    for idx in itertools.product(*[range(d) for d in dims]):
        j = 0
        for k in range(N):
            if k == n:
                continue
            Jk = 1
            for m in range(k):
                if m != n:
                    Jk *= dims[m]
            j += idx[k] * Jk
        U[idx[n], j] = T[idx]
    return U


def _brute_cp_tensor(lam, factors):
    dims = tuple(A.shape[0] for A in factors)
    T = np.zeros(dims)
    for idx in itertools.product(*[range(d) for d in dims]):
        s = 0.0
        for r in range(len(lam)):
            p = lam[r]
            for m, A in enumerate(factors):
                p *= A[idx[m], r]
            s += p
        T[idx] = s
    return T


@pytest.mark.parametrize("dims", [(2, 3, 4), (3, 1, 2, 2), (4, 5)])
def test_unfold_matches_index_map(dims):
    rng = np.random.default_rng(0)
    T = rng.standard_normal(dims)
    for n in range(len(dims)):
        np.testing.assert_array_equal(cp.unfold(T, n), _brute_unfold(T, n))


def test_unfold_column_matches_index_map():
    dims = (3, 4, 5, 2)
    rng = np.random.default_rng(1)
    T = rng.standard_normal(dims)
    idx = np.stack([rng.integers(0, d, 50) for d in dims], axis=1)
    for n in range(4):
        U = _brute_unfold(T, n)
        cols = cp.unfold_column(idx, dims, n)
        for s in range(50):
            full = list(idx[s])
            for i in range(dims[n]):
                full[n] = i
                assert U[i, cols[s]] == T[tuple(full)]


def test_khatri_rao_columns_are_kronecker_products():
    rng = np.random.default_rng(2)
    A, B, C = rng.standard_normal((3, 4)), rng.standard_normal((5, 4)), rng.standard_normal((2, 4))
    Z = cp.khatri_rao([A, B, C])
    for r in range(4):
        np.testing.assert_allclose(Z[:, r], np.kron(np.kron(A[:, r], B[:, r]), C[:, r]),
                                   rtol=0, atol=1e-14)


def test_khatri_rao_gram_identity():
    # eq. (KRGram): (A kr B)^T (A kr B) = A^T A * B^T B
    rng = np.random.default_rng(3)
    A, B = rng.standard_normal((7, 5)), rng.standard_normal((6, 5))
    Z = cp.khatri_rao([A, B])
    np.testing.assert_allclose(Z.T @ Z, (A.T @ A) * (B.T @ B), rtol=1e-12, atol=1e-12)


def test_khatri_rao_distributive_identity():
    # eq. (krdist): AB kr CD = (A kron C)(B kr D)
    rng = np.random.default_rng(4)
    A, B = rng.standard_normal((3, 4)), rng.standard_normal((4, 6))
    C, D = rng.standard_normal((5, 2)), rng.standard_normal((2, 6))
    np.testing.assert_allclose(cp.khatri_rao([A @ B, C @ D]),
                               np.kron(A, C) @ cp.khatri_rao([B, D]), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dims", [(3, 4, 5), (2, 3, 2, 3)])
def test_cp_unfolding_identity(dims):
    # eq. (Zn): X~_(n) = A^(n) diag(lam) Z^(n)^T, against a tensor built entry by entry
    rng = np.random.default_rng(5)
    R = 3
    lam = rng.uniform(0.2, 0.8, R)
    factors = [rng.standard_normal((d, R)) for d in dims]
    T = _brute_cp_tensor(lam, factors)
    np.testing.assert_allclose(cp.full_tensor(lam, factors), T, rtol=1e-12, atol=1e-12)
    for n in range(len(dims)):
        np.testing.assert_allclose(cp.unfold(T, n),
                                   (factors[n] * lam) @ cp.kr_of_others(factors, n).T,
                                   rtol=1e-12, atol=1e-12)


def test_mttkrp_brute_force():
    dims = (3, 4, 2)
    rng = np.random.default_rng(6)
    T = rng.standard_normal(dims)
    R = 2
    factors = [rng.standard_normal((d, R)) for d in dims]
    for n in range(3):
        W = np.zeros((dims[n], R))
        for idx in itertools.product(*[range(d) for d in dims]):
            for r in range(R):
                p = T[idx]
                for m in range(3):
                    if m != n:
                        p *= factors[m][idx[m], r]
                W[idx[n], r] += p
        np.testing.assert_allclose(cp.unfold(T, n) @ cp.kr_of_others(factors, n), W,
                                   rtol=1e-12, atol=1e-12)


def test_skr_and_fiber_gather_select_unfolding_rows_and_columns():
    dims = (4, 3, 5, 2)
    rng = np.random.default_rng(7)
    T = rng.standard_normal(dims)
    factors = [rng.standard_normal((d, 3)) for d in dims]
    idx = np.stack([rng.integers(0, d, 30) for d in dims], axis=1)
    for n in range(4):
        cols = cp.unfold_column(idx, dims, n)
        np.testing.assert_allclose(cp.skr(factors, idx, n), cp.kr_of_others(factors, n)[cols],
                                   rtol=1e-14, atol=0)
        Xs = cp.gather_fibers(T, idx, n)
        for s in range(30):
            full = list(idx[s])
            for i in range(dims[n]):
                full[n] = i
                assert Xs[i, s] == T[tuple(full)]


def test_mode_product_brute_force_and_ttensor_identity():
    dims = (3, 2, 4)
    rng = np.random.default_rng(8)
    T = rng.standard_normal(dims)
    Us = [rng.standard_normal((d, d)) for d in dims]
    for n in range(3):
        Y = cp.mode_product(T, Us[n], n)
        for idx in itertools.product(*[range(d) for d in dims]):
            s = 0.0
            for k in range(dims[n]):
                src = list(idx)
                src[n] = k
                s += Us[n][idx[n], k] * T[tuple(src)]
            assert abs(Y[idx] - s) < 1e-12
    # eq. (ttensor): Y_(n) = U_n X_(n) (U_N kron ... kron U_1 without n)^T
    Y = T
    for n in range(3):
        Y = cp.mode_product(Y, Us[n], n)
    for n in range(3):
        K = np.ones((1, 1))
        for m in reversed(range(3)):
            if m != n:
                K = np.kron(K, Us[m])
        np.testing.assert_allclose(cp.unfold(Y, n), Us[n] @ cp.unfold(T, n) @ K.T,
                                   rtol=1e-12, atol=1e-12)


def test_sampled_ls_matches_library_least_squares():
    rng = np.random.default_rng(9)
    for S, R, I in [(80, 5, 50), (230, 10, 7), (12, 12, 3)]:
        Z = rng.standard_normal((S, R))
        Xs = rng.standard_normal((I, S))
        ref = np.linalg.lstsq(Z, Xs.T, rcond=None)[0].T    # SVD-based LAPACK solver
        np.testing.assert_allclose(cp.sampled_ls(Z, Xs), ref, rtol=1e-10, atol=1e-12)


def test_normalize_columns():
    A = np.array([[3.0, 0.0, 1.0], [4.0, 0.0, -1.0]])
    An, lam = cp.normalize_columns(A)
    np.testing.assert_allclose(lam, [5.0, 0.0, np.sqrt(2.0)])
    np.testing.assert_allclose(An[:, 0], [0.6, 0.8])
    np.testing.assert_array_equal(An[:, 1], [0.0, 0.0])
    np.testing.assert_allclose(np.linalg.norm(An[:, 2]), 1.0)
