"""The error floor of the FP32 form on a given problem, for the parity tests of ill-conditioned
least-squares problems (test infrastructure; it calls the oracle's steps only)."""
import numpy as np

from oracle import cp, mixing, streams


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def fp32_product_floor(T, R, S, seed, iters, ref, ops=None):
    """Per factor, how far a plain FP32 form of the sampled update lands from the oracle after `iters`
    outer iterations: the oracle's own draws and skr / gather steps (Alg. 3), M = X_S Z_S as one FP32
    matrix product (NumPy's SGEMM), and an exact FP64 solve against the FP64 Gram.  The part of the
    error that the rounding of M alone causes, amplified by the conditioning of the sampled Gram.
    With ops (CPRAND-MIX: T is the mixed tensor), the factors are unmixed before the comparison."""
    N, dims = T.ndim, T.shape
    factors = [np.zeros((dims[0], R))] + [streams.init_factor(seed, 0, n, dims[n], R) for n in range(1, N)]
    for t in range(iters):
        for n in range(N):
            idx = streams.ls_sample_indices(seed, 0, t, n, S, dims)
            Z = cp.skr(factors, idx, n)
            M = (cp.gather_fibers(T, idx, n).astype(np.float32) @ Z.astype(np.float32)).astype(np.float64)
            factors[n], _ = cp.normalize_columns(np.linalg.solve(Z.T @ Z, M.T).T)
    if ops is not None:
        factors = mixing.unmix_factors(factors, ops)
    return [rel(A, Ar) for A, Ar in zip(factors, ref["factors"])]
