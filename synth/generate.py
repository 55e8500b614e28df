"""Synthetic CP problems (§4.2).  See the package docstring for the recipe."""
from dataclasses import dataclass, field

import numpy as np
import torch


@dataclass
class Problem:
    dims: tuple
    lam: np.ndarray                 # ground-truth weights (FP64)
    factors: list                   # ground-truth factors, I_n x R_true (FP64)
    X: torch.Tensor                 # stored tensor, flat column-major, requested dtype/device
    eta: float
    meta: dict = field(default_factory=dict)


def collinear_factor(rng, I, R, C):
    """I x R matrix with unit columns and pairwise cosine exactly C (reading of §4.2)."""
    if I < R:
        raise ValueError("collinear factors need I >= R")
    Q, _ = np.linalg.qr(rng.standard_normal((I, R)), mode="reduced")
    K = (1.0 - C) * np.eye(R) + C * np.ones((R, R))
    L = np.linalg.cholesky(K)
    return Q @ L.T


def _kr_rows_fast_first(mats):
    """Rows of the Khatri-Rao product with the FIRST matrix's row index varying fastest
    (the column order of the mode-1 unfolding); torch, on the matrices' device."""
    Z = mats[0]
    for M in mats[1:]:
        Z = (M[:, None, :] * Z[None, :, :]).reshape(-1, Z.shape[1])
    return Z


def make_problem(dims, R_true, C=0.0, eta=0.01, seed=0, dtype=torch.float32, device="cpu",
                 gaussian_factors=False, lam_range=(0.2, 0.8), noise_chunk=1 << 26):
    """Build X = X_true + eta * (||X_true|| / ||N||) * N in column-major storage.

    gaussian_factors=True draws N(0,1) factors with lam = 1 (the plain 50^3 FP64 workload);
    otherwise lam ~ U[lam_range] and collinear factors with cosine C.  The noise is drawn in
    chunks from torch generators seeded by (seed, chunk), so the device does not need a second
    full-size buffer; the returned tensor is what both the GPU path and the oracle consume.
    """
    dims = tuple(int(d) for d in dims)
    rng = np.random.default_rng(seed)
    if gaussian_factors:
        lam = np.ones(R_true)
        factors = [rng.standard_normal((I, R_true)) for I in dims]
    else:
        lam = rng.uniform(lam_range[0], lam_range[1], size=R_true)
        factors = [collinear_factor(rng, I, R_true, C) for I in dims]
    dev = torch.device(device)
    acc = torch.float64 if (dtype == torch.float64 or dev.type == "cpu") else torch.float32
    # X_(1)^T = Z^(1) (A^(1) diag(lam))^T, stored row-major, is the column-major tensor
    A = [torch.as_tensor(f, dtype=acc, device=dev) for f in factors]
    lam_t = torch.as_tensor(lam, dtype=acc, device=dev)
    P = int(np.prod(dims))
    if len(dims) == 1:
        Xt = (A[0] * lam_t).sum(dim=1)
    else:
        Z = _kr_rows_fast_first(A[1:])
        Xt = (Z @ (A[0] * lam_t).T).reshape(-1)
    assert Xt.numel() == P
    true_norm = torch.linalg.vector_norm(Xt, dtype=torch.float64).item()
    # noise: two passes over the same seeded chunks (norm first, then add)
    def chunk_noise(c, n):
        g = torch.Generator(device=dev)
        g.manual_seed((seed * 1000003 + c) & 0x7FFFFFFFFFFFFFFF)
        return torch.randn(n, generator=g, device=dev, dtype=acc)
    nn2 = 0.0
    starts = list(range(0, P, noise_chunk))
    if eta > 0:
        for c, s in enumerate(starts):
            n = min(noise_chunk, P - s)
            nn2 += float(torch.sum(chunk_noise(c, n).double() ** 2).item())
        scale = eta * true_norm / np.sqrt(nn2)
        for c, s in enumerate(starts):
            n = min(noise_chunk, P - s)
            Xt[s:s + n] += scale * chunk_noise(c, n)
    X = Xt.to(dtype)
    return Problem(dims=dims, lam=lam, factors=factors, X=X, eta=eta,
                   meta={"R_true": R_true, "C": C, "seed": seed, "true_norm": true_norm})


def to_oracle_array(X_flat, dims):
    """The stored tensor as the oracle sees it: FP64 NumPy array of shape dims (column-major)."""
    x = X_flat.detach().to("cpu")
    if x.dtype == torch.bfloat16:
        x = x.float()
    x = x.double().numpy()
    return np.reshape(x, tuple(dims), order="F")


def batch_problem_specs(seed, B=64, dim_range=(64, 512), rank_range=(4, 32), C_range=(0.0, 0.9)):
    """Shapes for a batch of independent 3-way problems: every dim uniform in dim_range, rank
    uniform in rank_range, collinearity uniform in C_range (the many-starts workload)."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(B):
        dims = tuple(int(v) for v in rng.integers(dim_range[0], dim_range[1] + 1, size=3))
        R = int(rng.integers(rank_range[0], rank_range[1] + 1))
        C = float(rng.uniform(C_range[0], C_range[1]))
        specs.append({"dims": dims, "R": R, "C": C})
    return specs
