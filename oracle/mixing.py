"""Mixing preprocess and CPRAND-MIX in its real-transform form (Alg. 5, §3.3).

TEST INFRASTRUCTURE ONLY (CPU oracle, FP64).  Shares no code with the CUDA library.

The paper mixes every mode with F_n D_n: D_n a random sign flip, F_n a unitary fast transform
(FFT in the experiments; DCT and WHT named as equivalent choices, §2.2).  With a REAL orthogonal
F_n, CPRAND-MIX reduces to: mix the tensor once, run CPRAND on it, unmix the factors (Alg. 5).
Reading taken here: F_n is the orthonormal DCT-II,
    F_n[k, i] = c_k cos(pi (2 i + 1) k / (2 I_n)),  c_0 = sqrt(1 / I_n), c_k = sqrt(2 / I_n).
"""
import numpy as np

from . import cp, streams


def dct2_matrix(I):
    """Orthonormal DCT-II matrix, I x I, row k = frequency k."""
    k = np.arange(I, dtype=np.float64)[:, None]
    i = np.arange(I, dtype=np.float64)[None, :]
    F = np.cos(np.pi * (2.0 * i + 1.0) * k / (2.0 * I))
    F[0, :] *= np.sqrt(1.0 / I)
    F[1:, :] *= np.sqrt(2.0 / I)
    return F


def mixing_operators(seed, b, dims, identity=False):
    """The per-mode operators F_n D_n (Alg. 5, first step).  identity=True gives F_n = D_n = I,
    the special case in which CPRAND-MIX must reduce to CPRAND."""
    ops = []
    for n, I in enumerate(dims):
        if identity:
            ops.append(np.eye(I))
        else:
            d = streams.sign_vector(seed, b, n, I)
            ops.append(dct2_matrix(I) * d[None, :])
    return ops


def mix_tensor(T, ops):
    """X^ = X x_1 F_1 D_1 x_2 ... x_N F_N D_N  (Alg. 5 mixing step), mode 1 first."""
    Y = T
    for n, U in enumerate(ops):
        Y = cp.mode_product(Y, U, n)
    return Y


def unmix_factors(factors_hat, ops):
    """A^(n) = D_n F_n^T A^^(n)  (Alg. 5 unmixing step): the transpose of each orthogonal
    operator undoes the mixing of its mode."""
    return [U.T @ Ah for U, Ah in zip(ops, factors_hat)]


def mix_factors(factors, ops):
    """A^^(n) = F_n D_n A^(n)  (Alg. 4, factor mixing)."""
    return [U @ A for U, A in zip(ops, factors)]


def cprand_mix(T, R, S, seed, b=0, fit_samples=16384, rule=None, identity=False):
    """CPRAND-MIX, real-transform form (Alg. 5): mix, CPRAND in the mixed basis, unmix.
    The initial factors are drawn directly in the mixed basis (Alg. 5 hands the mixed tensor to
    CPRAND unchanged).  Returns the CPRAND result dict with factors unmixed and the mixed
    tensor under 'T_mixed'."""
    ops = mixing_operators(seed, b, T.shape, identity)
    Th = mix_tensor(T, ops)
    out = cp.cprand(Th, R, S, seed, b, fit_samples, rule)
    out["factors_mixed"] = out["factors"]
    out["factors"] = unmix_factors(out["factors"], ops)
    out["T_mixed"] = Th
    return out
