"""The error floor of the FP32 form on a given problem, for the parity tests of ill-conditioned
least-squares problems (test infrastructure; it calls the oracle's steps only)."""
import numpy as np

from oracle import cp, mixing, streams


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def fp32_product(XS, Z, variant):
    """M = X_S Z_S rounded the FP32 way: 0, one SGEMM; 1, the same with the samples in reverse order;
    2, FP32 partial products of 32 samples each, summed in FP32 (the order of a chunked kernel)."""
    X32, Z32 = XS.astype(np.float32), Z.astype(np.float32)
    if variant == 1:
        X32, Z32 = X32[:, ::-1].copy(), Z32[::-1].copy()
    if variant == 2:
        M = np.zeros((XS.shape[0], Z.shape[1]), dtype=np.float32)
        for j in range(0, Z.shape[0], 32):
            M += X32[:, j:j + 32] @ Z32[j:j + 32]
        return M.astype(np.float64)
    return (X32 @ Z32).astype(np.float64)


def fp32_product_run(T, R, S, seed, iters, fit_samples=16384, variant=0):
    """CPRAND (Alg. 3) as the oracle runs it -- its draws, skr and gather steps, its sampled fit (§3.4)
    -- except that M = X_S Z_S is rounded to FP32 (`fp32_product`), then solved exactly in FP64
    against the FP64 Gram.  Returns (factors, lam, fits)."""
    N, dims = T.ndim, T.shape
    factors = [np.zeros((dims[0], R))] + [streams.init_factor(seed, 0, n, dims[n], R) for n in range(1, N)]
    normT = np.linalg.norm(T.ravel())
    P = int(np.prod(dims))
    fit_idx = streams.fit_sample_indices(seed, 0, fit_samples, dims)
    fit_x = T[tuple(fit_idx[:, m] for m in range(N))]
    fits, lam = [], None
    for t in range(iters):
        for n in range(N):
            idx = streams.ls_sample_indices(seed, 0, t, n, S, dims)
            Z = cp.skr(factors, idx, n)
            M = fp32_product(cp.gather_fibers(T, idx, n), Z, variant)
            factors[n], lam = cp.normalize_columns(np.linalg.solve(Z.T @ Z, M.T).T)
        fits.append(cp.sampled_fit(fit_x, lam, factors, fit_idx, normT, P))
    return factors, lam, np.array(fits)


def fp32_product_floor(T, R, S, seed, iters, ref, ops=None):
    """Per factor, how far the plain FP32 forms above land from the oracle's run `ref` after `iters`
    outer iterations (the largest over the three roundings of M): the part of the error that the
    FP32 rounding of M alone causes, amplified by the conditioning of the sampled Gram.  With ops
    (CPRAND-MIX: T is the mixed tensor), the factors are unmixed before the comparison."""
    worst = None
    for variant in range(3):
        factors, _, _ = fp32_product_run(T, R, S, seed, iters, variant=variant)
        if ops is not None:
            factors = mixing.unmix_factors(factors, ops)
        errs = [rel(A, Ar) for A, Ar in zip(factors, ref["factors"])]
        worst = errs if worst is None else [max(a, b) for a, b in zip(worst, errs)]
    return worst


def fp32_trace_floor(T, R, S, seed, iters, ref_fits):
    """The largest per-iteration difference between a plain FP32 form's sampled-fit trace and the
    oracle's (ref_fits) over `iters` outer iterations, over the three roundings of M."""
    worst = 0.0
    for variant in range(3):
        _, _, fits = fp32_product_run(T, R, S, seed, iters, variant=variant)
        worst = max(worst, float(np.max(np.abs(fits - np.asarray(ref_fits)[:iters]))))
    return worst
