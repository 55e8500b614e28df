"""The test hooks of cpr_opts, through the C ABI.

user_samples: when every multi-index of the other modes is sampled exactly once, the sampled
least-squares problem of Alg. 3 is the full one of Alg. 1, so one outer iteration of CPRAND must
equal one outer iteration of CP-ALS from the same start: the library's CPRAND against its own
cpr_cp_als and against the oracle's cp_als_update, in FP64, to 1e-10.
"""
import itertools

import numpy as np
import pytest
import torch

from oracle import cp

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def cb():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1701_06600_gb300 import binding
    return binding


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def every_row_samples(dims):
    """N x S x N table: for each mode n, every multi-index of the other modes once (S = P / I_n, the
    same for every mode of a cube)."""
    N = len(dims)
    S = int(np.prod(dims)) // dims[0]
    tab = np.zeros((N, S, N), dtype=np.uint32)
    for n in range(N):
        others = [range(dims[m]) for m in range(N) if m != n]
        for j, combo in enumerate(itertools.product(*others)):
            k = 0
            for m in range(N):
                if m != n:
                    tab[n, j, m] = combo[k]
                    k += 1
    return tab, S


@pytest.mark.parametrize("dims,R", [((5, 5, 5), 3), ((4, 4, 4, 4), 2)])
def test_every_row_sampled_equals_cp_als(cb, dims, R):
    rng = np.random.default_rng(11)
    T = rng.standard_normal(dims)
    X = torch.tensor(T.ravel(order="F"), device=DEV)
    init = [rng.random((d, R)) for d in dims]
    tab, S = every_row_samples(dims)
    samples = torch.tensor(tab.ravel().astype(np.int64), dtype=torch.int32, device=DEV)
    opts = cb.cpr_default_opts(fixed_iters=1, loop_path=cb.LOOP_GRAPH, user_samples=samples.data_ptr(), user_S=S)
    out = cb.cpr_cprand(X, dims, R, S, opts=opts, init=[torch.tensor(a, device=DEV) for a in init])
    assert out["status"] == cb.OK and out["iters"] == 1
    als = cb.cpr_cp_als(X, dims, R, opts=cb.cpr_default_opts(fixed_iters=1),
                        init=[torch.tensor(a, device=DEV) for a in init])
    factors = [np.array(a) for a in init]
    lam = None
    for n in range(len(dims)):
        factors[n], lam = cp.cp_als_update(T, factors, n)
    for A, B, C in zip(out["factors"], als["factors"], factors):
        assert rel(A.cpu().numpy(), C) < 1e-10
        assert rel(A.cpu().numpy(), B.cpu().numpy()) < 1e-10
    assert rel(out["lam"].cpu().numpy(), lam) < 1e-10


def test_user_samples_must_match_S(cb):
    dims = (5, 5, 5)
    X = torch.zeros(125, dtype=torch.float64, device=DEV)
    tab, S = every_row_samples(dims)
    samples = torch.tensor(tab.ravel().astype(np.int64), dtype=torch.int32, device=DEV)
    opts = cb.cpr_default_opts(fixed_iters=1, user_samples=samples.data_ptr(), user_S=S - 1)
    with pytest.raises(cb.CprError):
        cb.cpr_cprand(X, dims, 3, S, opts=opts)
