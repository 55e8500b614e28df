"""CPRAND-MIX with a complex unitary transform (Alg. 4, §3.3), the paper's experimental form.

TEST INFRASTRUCTURE ONLY (CPU oracle, FP64 / complex128).  Shares no code with the CUDA library.

The mixing operator of mode n is F_n D_n with D_n the random sign flip and F_n the unitary DFT,
    F_n[k, i] = exp(-2 pi i k i / I_n) / sqrt(I_n).
The mixed tensor is complex.  The factors stay real: Alg. 4 keeps A^(n) and its mixed copy
A^^(n) = F_n D_n A^(n); the sampled rows of the mixed Khatri-Rao product come from the mixed
factors, the sampled fibers of the mixed tensor are unmixed in mode n (D_n F_n^* applied to each),
and the least-squares problem is solved over real A by stacking real and imaginary parts (eq.
(rcLS)).  The stopping test is the sampled fit of §3.4 on the original tensor with the real
factors.
"""
import numpy as np

from . import cp, streams


def dft_matrix(I):
    """Unitary DFT matrix, I x I: F[k, i] = exp(-2 pi i k i / I) / sqrt(I)."""
    k = np.arange(I, dtype=np.float64)[:, None]
    i = np.arange(I, dtype=np.float64)[None, :]
    return np.exp(-2j * np.pi * ((k * i) % I) / I) / np.sqrt(I)


def dft_operators(seed, b, dims, identity=False):
    """The per-mode operators F_n D_n of Alg. 4 (the same sign stream as the real form);
    identity=True gives F_n = D_n = I, the case in which Alg. 4 reduces to CPRAND."""
    ops = []
    for n, I in enumerate(dims):
        if identity:
            ops.append(np.eye(I, dtype=np.complex128))
        else:
            d = streams.sign_vector(seed, b, n, I)
            ops.append(dft_matrix(I) * d[None, :])
    return ops


def mix_tensor(T, ops):
    """X^ = X x_1 F_1 D_1 ... x_N F_N D_N (complex), mode 1 first."""
    Y = np.asarray(T, dtype=np.complex128)
    for n, U in enumerate(ops):
        Y = cp.mode_product(Y, U, n)
    return Y


def real_ls(Z_S, X_S):
    """argmin over REAL A of || Z_S A^T - X_S^T ||_F for complex Z_S (S x R) and X_S (I_n x S):
    the stacked real problem of eq. (rcLS), [Re Z_S; Im Z_S] A^T = [Re X_S^T; Im X_S^T], by QR."""
    Zr = np.vstack([Z_S.real, Z_S.imag])
    Xr = np.hstack([X_S.real, X_S.imag])
    return cp.sampled_ls(Zr, Xr)


def update(Th, ops, mixed, n, idx):
    """One mode-n update of Alg. 4 for the sampled multi-indices idx (S x N): the rows of the mixed
    Khatri-Rao product, the sampled fibers of the mixed tensor unmixed in mode n, the real least
    squares, normalization.  Returns (A_new normalized, lam, its mixed copy)."""
    Z_S = cp.skr(mixed, idx, n)
    X_S = ops[n].conj().T @ cp.gather_fibers(Th, idx, n)       # D_n F_n^* per sampled fiber
    A, lam = cp.normalize_columns(real_ls(Z_S, X_S))
    return A, lam, ops[n] @ A


def cprand_mix_fft(T, R, S, seed, b=0, fit_samples=16384, rule=None, identity=False):
    """Alg. 4.  Initial factors for modes 2..N from the init stream (as CPRAND), mixed once; every
    outer iteration updates modes 1..N with fresh samples (the same sample stream as CPRAND) and
    then checks the sampled fit on X.  Returns lam, the real factors, iters, fits."""
    N = T.ndim
    dims = T.shape
    if rule is None:
        rule = cp.StopRule()
    ops = dft_operators(seed, b, dims, identity)
    Th = mix_tensor(T, ops)
    factors = [np.zeros((dims[0], R))] + [streams.init_factor(seed, b, n, dims[n], R) for n in range(1, N)]
    mixed = [ops[n] @ factors[n] for n in range(N)]
    lam = np.ones(R)
    normT = np.linalg.norm(np.asarray(T).ravel())
    P = int(np.prod(dims))
    fit_idx = streams.fit_sample_indices(seed, b, fit_samples, dims)
    fit_x = np.asarray(T)[tuple(fit_idx[:, m] for m in range(N))]
    t = 0
    while True:
        for n in range(N):
            idx = streams.ls_sample_indices(seed, b, t, n, S, dims)
            factors[n], lam, mixed[n] = update(Th, ops, mixed, n, idx)
        f = cp.sampled_fit(fit_x, lam, factors, fit_idx, normT, P)
        t += 1
        if rule.update(f):
            break
    return {"lam": lam, "factors": factors, "iters": len(rule.fits), "fits": np.array(rule.fits)}
