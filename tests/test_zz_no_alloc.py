"""The allocation-free sampled fit (cpr_fit_estimate_noalloc) against the workspace version.

Callers that cannot allocate device memory when they need a fit use this entry point; its scratch
is a fixed array inside the library.  Collected last (file name) so that a run stopping at the
first failure has already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from synth import make_problem

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def cb():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1701_06600_gb300 import binding
    return binding


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64, torch.bfloat16])
def test_noalloc_fit_matches_workspace_fit_on_two_calls(cb, dtype):
    dims = (61, 47, 39)
    prob = make_problem(dims, 5, C=0.4, eta=0.05, seed=12, dtype=dtype, device=DEV)
    rng = np.random.default_rng(3)
    lam = torch.tensor(rng.uniform(0.2, 0.8, 5), device=DEV)
    facs = [torch.tensor(f + 0.01 * rng.standard_normal(f.shape), device=DEV) for f in prob.factors]
    ref = cb.cpr_fit_estimate(prob.X, dims, lam, facs, 16384, seed=77, b=1)
    ref_given_norm = cb.cpr_fit_estimate(prob.X, dims, lam, facs, 16384, seed=77, b=1, norm_x=2.5)
    # two calls in a row through the C ABI: the second must not see the first call's leftovers
    for _ in range(2):
        got = cb.cpr_fit_estimate_noalloc(prob.X, dims, lam, facs, 16384, seed=77, b=1)
        assert abs(got - ref) < 1e-6, (got, ref)
        got_n = cb.cpr_fit_estimate_noalloc(prob.X, dims, lam, facs, 16384, seed=77, b=1, norm_x=2.5)
        assert abs(got_n - ref_given_norm) < 1e-6, (got_n, ref_given_norm)
    # a different fit set size right after (fewer blocks than the previous call)
    small = cb.cpr_fit_estimate(prob.X, dims, lam, facs, 1000, seed=5)
    assert abs(cb.cpr_fit_estimate_noalloc(prob.X, dims, lam, facs, 1000, seed=5) - small) < 1e-6


def test_noalloc_fit_rejects_fit_sets_beyond_its_scratch(cb):
    dims = (20, 21, 22)
    prob = make_problem(dims, 3, eta=0.01, seed=1, dtype=torch.float32, device=DEV)
    lam = torch.ones(3, dtype=torch.float64, device=DEV)
    facs = [torch.tensor(f, device=DEV) for f in prob.factors]
    d = cb.tensor_desc(prob.X, dims)
    k = cb.ktensor_desc(lam, facs)
    out = ctypes.c_double(-7.0)
    too_big = (1 << 20) + 1
    st = cb.lib().cpr_fit_estimate_noalloc(ctypes.byref(d), ctypes.byref(k), too_big, ctypes.c_uint64(0), 0, -1.0,
                                           ctypes.byref(out), None)
    assert st == cb.EINVAL and out.value == -7.0
