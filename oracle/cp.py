"""Plain FP64 CPU restatement of CP-ALS and CPRAND (Battaglino, Ballard, Kolda, §2-§3).

TEST INFRASTRUCTURE ONLY.  This is the oracle the CUDA library is checked against: slow,
unblocked, and written to be read next to the paper.  Only tests, the smoke check and the
benchmark's CPU-baseline leg may import it.  It shares no code with the CUDA library.

Conventions
  * A tensor is a NumPy array of shape (I_1, ..., I_N); its storage order is column-major
    (i_1 fastest), which is the order the mode-n unfolding of §2.1 assumes.
  * Modes are 0-based here (mode n of the code is mode n+1 of the paper).
  * Factor matrices are I_n x R arrays; lam is the length-R weight vector of eq. (cpform+lambda).
"""
import math

import numpy as np
import scipy.linalg

from . import streams


# --------------------------------------------------------------------------------------------
# §2.1 tensor algebra
# --------------------------------------------------------------------------------------------

def unfold(T, n):
    """Mode-n unfolding X_(n) (§2.1): entry (i_1..i_N) goes to row i_n and column
    j = sum_{k != n} i_k J_k with J_k = prod_{m < k, m != n} I_m (0-based)."""
    return np.reshape(np.moveaxis(T, n, 0), (T.shape[n], -1), order="F")


def unfold_column(idx, dims, n):
    """Column j of X_(n) that holds the fiber with multi-index idx (the mode-n slot is ignored);
    the index map of §2.1 written out.  idx: (S, N) integer array.  Returns (S,) int64."""
    col = np.zeros(idx.shape[0], dtype=np.int64)
    J = 1
    for k in range(len(dims)):
        if k == n:
            continue
        col += idx[:, k].astype(np.int64) * J
        J *= int(dims[k])
    return col


def khatri_rao(mats):
    """Khatri-Rao product M_1 (.) M_2 (.) ... (.) M_k (§2.1): column r is the Kronecker product
    of the r-th columns, so the row index of the LAST matrix varies fastest."""
    Z = mats[0]
    for M in mats[1:]:
        Z = np.einsum("ir,jr->ijr", Z, M).reshape(-1, Z.shape[1])
    return Z


def kr_of_others(factors, n):
    """Z^(n) = A^(N) (.) ... (.) A^(n+1) (.) A^(n-1) (.) ... (.) A^(1)  (eq. Zn)."""
    N = len(factors)
    return khatri_rao([factors[m] for m in reversed(range(N)) if m != n])


def mode_product(T, U, n):
    """Y = T x_n U, i.e. Y_(n) = U T_(n) (§2.1)."""
    return np.moveaxis(np.tensordot(U, T, axes=(1, n)), 0, n)


def full_tensor(lam, factors):
    """The CP model of eq. (cpform+lambda): sum_r lam_r a_r^(1) o ... o a_r^(N)."""
    N = len(factors)
    dims = tuple(A.shape[0] for A in factors)
    # X~_(1) = A^(1) diag(lam) Z^(1)^T  (eq. Zn)
    X1 = (factors[0] * lam[None, :]) @ kr_of_others(factors, 0).T
    return np.reshape(X1, dims, order="F") if N > 1 else X1.reshape(dims)


def normalize_columns(A):
    """Column 2-norms become the weights and the columns get unit length (Alg. 1 and Alg. 3,
    normalization step).  A zero column keeps weight 0 and stays as it is."""
    lam = np.sqrt(np.sum(A * A, axis=0))
    safe = np.where(lam > 0, lam, 1.0)
    return A / safe[None, :], lam


# --------------------------------------------------------------------------------------------
# §3.1 CP-ALS (Alg. 1)
# --------------------------------------------------------------------------------------------

def cp_als_update(T, factors, n):
    """One mode-n update of Alg. 1: V = Hadamard product of the other Gram matrices,
    W = X_(n) Z^(n) (MTTKRP), solve A V = W, normalize.  Returns (A_new, lam)."""
    R = factors[0].shape[1]
    V = np.ones((R, R))
    for m, A in enumerate(factors):
        if m != n:
            V *= A.T @ A
    W = unfold(T, n) @ kr_of_others(factors, n)
    A_new = scipy.linalg.solve(V, W.T, assume_a="sym").T
    return normalize_columns(A_new)


def exact_fit(T, lam, factors, normT=None):
    """F = 1 - ||X - X~|| / ||X||  (§4.2)."""
    if normT is None:
        normT = np.linalg.norm(T.ravel())
    return 1.0 - np.linalg.norm((T - full_tensor(lam, factors)).ravel()) / normT


def cp_als(T, R, factors0, max_iters=200, tol=1e-4, fixed_iters=0):
    """Alg. 1 with the change-in-fit rule of §4.2.  factors0[0] is not used (mode 1 is solved
    first).  Returns (lam, factors, iters, fits)."""
    factors = [np.array(A, dtype=np.float64) for A in factors0]
    lam = np.ones(R)
    normT = np.linalg.norm(T.ravel())
    fits = []
    iters = fixed_iters if fixed_iters > 0 else max_iters
    for it in range(iters):
        for n in range(T.ndim):
            factors[n], lam = cp_als_update(T, factors, n)
        fits.append(exact_fit(T, lam, factors, normT))
        if fixed_iters == 0 and it > 0 and abs(fits[-1] - fits[-2]) <= tol:
            break
    return lam, factors, len(fits), np.array(fits)


# --------------------------------------------------------------------------------------------
# §3.2 CPRAND (Alg. 2 and Alg. 3)
# --------------------------------------------------------------------------------------------

def skr(factors, idx, n):
    """Sampled Khatri-Rao product (Alg. 2): row j is the Hadamard product of the rows
    A^(m)(i_m^(j), :) over m != n.  idx: (S, N).  Returns Z_S, S x R."""
    S = idx.shape[0]
    R = factors[0].shape[1]
    Z = np.ones((S, R))
    for m, A in enumerate(factors):
        if m != n:
            Z = Z * A[idx[:, m], :]
    return Z


def gather_fibers(T, idx, n):
    """X_S = (S X_(n)^T)^T, the I_n x S matrix of sampled mode-n fibers (§3.2): the columns of
    the unfolding selected through the index map of §2.1."""
    return unfold(T, n)[:, unfold_column(idx, T.shape, n)]


def sampled_ls(Z_S, X_S):
    """argmin_A || Z_S A^T - X_S^T ||_F by Householder QR (Alg. 3 least-squares step, cost in
    §3.2.1).  Returns A, I_n x R."""
    Q, Rm = np.linalg.qr(Z_S, mode="reduced")
    return scipy.linalg.solve_triangular(Rm, Q.T @ X_S.T, lower=False).T


def cprand_update(T, factors, n, idx):
    """One mode-n update of Alg. 3 for given sampled multi-indices idx (S x N).
    Returns (A_new normalized, lam)."""
    Z_S = skr(factors, idx, n)
    X_S = gather_fibers(T, idx, n)
    return normalize_columns(sampled_ls(Z_S, X_S))


def sample_size(R):
    """S = 10 R log R (natural log, rounded to nearest), §3.2 and §4.2."""
    return int(math.floor(10.0 * R * math.log(R) + 0.5))


class StopRule:
    """Termination rules of §3.4 and §4.2, applied to one fit value per outer iteration:
    stop after max_iters iterations; when |F_t - F_{t-1}| <= tol (from the second iteration
    on); when F_t >= 1 - 1.2 eta (only if eta >= 0); or, if stall_iters > 0, when the best fit
    has not strictly improved for stall_iters iterations.  fixed_iters > 0 overrides all rules."""

    def __init__(self, max_iters=200, tol=1e-4, eta=-1.0, stall_iters=0, fixed_iters=0):
        self.max_iters, self.tol, self.eta = max_iters, tol, eta
        self.stall_iters, self.fixed_iters = stall_iters, fixed_iters
        self.fits = []
        self.best = -np.inf
        self.stall = 0

    def update(self, fit):
        """Record the fit of the iteration just finished; return True to stop."""
        self.fits.append(fit)
        t = len(self.fits)
        if self.fixed_iters > 0:
            return t >= self.fixed_iters
        if fit > self.best:
            self.best, self.stall = fit, 0
        else:
            self.stall += 1
        if t >= self.max_iters:
            return True
        if t >= 2 and abs(self.fits[-1] - self.fits[-2]) <= self.tol:
            return True
        if self.eta >= 0 and fit >= 1.0 - 1.2 * self.eta:
            return True
        if self.stall_iters > 0 and self.stall >= self.stall_iters:
            return True
        return False


def sampled_fit(T_flat_values, lam, factors, fit_idx, normT, P):
    """Sampled fit estimate of §3.4: 1 - sqrt(P * mean_i e_i^2) / ||X|| over the entries fit_idx,
    with x values T_flat_values (one per entry)."""
    model = np.zeros(fit_idx.shape[0])
    R = lam.shape[0]
    for r in range(R):
        term = np.full(fit_idx.shape[0], lam[r])
        for m, A in enumerate(factors):
            term = term * A[fit_idx[:, m], r]
        model += term
    e = T_flat_values - model
    return 1.0 - math.sqrt(P * np.mean(e * e)) / normT


def cprand(T, R, S, seed, b=0, fit_samples=16384, rule=None, factors0=None, t0=0):
    """Alg. 3 (CPRAND) with the sampled stopping test of §3.4.

    Random initial factors for modes 2..N come from the init stream (mode 1 is solved first);
    factors0 overrides them.  Returns a dict with lam, factors, iters, fits (sampled)."""
    N = T.ndim
    dims = T.shape
    if rule is None:
        rule = StopRule()
    if factors0 is None:
        factors = [np.zeros((dims[0], R))] + [streams.init_factor(seed, b, n, dims[n], R)
                                               for n in range(1, N)]
    else:
        factors = [np.array(A, dtype=np.float64) for A in factors0]
    lam = np.ones(R)
    normT = np.linalg.norm(T.ravel())
    P = int(np.prod(dims))
    fit_idx = streams.fit_sample_indices(seed, b, fit_samples, dims)
    fit_x = T[tuple(fit_idx[:, m] for m in range(N))]
    t = t0
    while True:
        for n in range(N):
            idx = streams.ls_sample_indices(seed, b, t, n, S, dims)
            factors[n], lam = cprand_update(T, factors, n, idx)
        f = sampled_fit(fit_x, lam, factors, fit_idx, normT, P)
        t += 1
        if rule.update(f):
            break
    return {"lam": lam, "factors": factors, "iters": len(rule.fits), "fits": np.array(rule.fits)}
