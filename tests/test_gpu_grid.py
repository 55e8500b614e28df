"""GPU parity of the whole-GPU iteration loop (loop_path 5: one cooperative launch of one CTA per SM,
grid-wide barriers between the phases of a mode update) against the CPU oracle, and its failure
paths: a singular Gram, a non-finite tensor, a barrier wait that runs out.

Bars: the sampled-fit trace within 1e-4 absolute and the factors within 1e-4 relative Frobenius
of the oracle's CPRAND (Alg. 3) run on the same stored tensor with the same Philox draws, after
three outer iterations (nine mode updates).
"""
import numpy as np
import pytest
import torch

from oracle import cp, mixing
from synth import make_problem, to_oracle_array
from fp32_floor import fp32_product_floor

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


# shapes: several 96-row tiles with a ragged last tile, modes shorter than a tile, 4-way, ranks that
# take each column-group width (R <= 16, 32, 48, 64), S not a multiple of the split
CASES = [
    ((260, 190, 150), 16, 300, torch.float32, False),
    ((1000, 40, 30), 8, 100, torch.float32, False),
    ((300, 200, 250), 50, 600, torch.float32, False),
    ((200, 150, 120), 40, 500, torch.bfloat16, False),
    ((40, 30, 20, 25), 10, 200, torch.float32, True),
    ((130, 97, 101), 24, 333, torch.bfloat16, True),
]


@pytest.fixture(params=["tc", "fma"])
def contract(cb, request):
    """Runs a test with each contraction engine of the whole-GPU loop (tensor cores, FP32 FMA)."""
    prev = cb.cpr_set_contract_engine(cb.CONTRACT_TC if request.param == "tc" else cb.CONTRACT_FMA)
    yield request.param
    cb.cpr_set_contract_engine(prev)


@pytest.mark.parametrize("dims,R,S,dtype,mix", CASES)
def test_grid_loop_matches_oracle(cb, contract, dims, R, S, dtype, mix):
    prob = make_problem(dims, min(R, 8), C=0.5, eta=0.01, seed=301, dtype=dtype, device=DEV)
    T = to_oracle_array(prob.X, dims)
    iters = 3
    trace = torch.zeros(iters, dtype=torch.float64, device=DEV)
    opts = cb.cpr_default_opts(seed=17, fixed_iters=iters, fit_trace_dev=trace.data_ptr(), loop_path=cb.LOOP_GRID)
    fn = cb.cpr_cprand_mix if mix else cb.cpr_cprand
    out = fn(prob.X, dims, R, S, opts=opts)
    assert out["status"] == cb.OK and out["iters"] == iters
    if mix:
        Th = to_oracle_array(cb.cpr_mix_tensor(prob.X, dims, seed=17), dims)
        ops = mixing.mixing_operators(17, 0, dims)
        ref = cp.cprand(Th, R, S, seed=17, rule=cp.StopRule(fixed_iters=iters))
        ref["factors"] = mixing.unmix_factors(ref["factors"], ops)
    else:
        ref = cp.cprand(T, R, S, seed=17, rule=cp.StopRule(fixed_iters=iters))
    np.testing.assert_allclose(trace.cpu().numpy(), ref["fits"], rtol=0, atol=1e-4)
    # 1e-4, or, where the problem's conditioning makes the FP32 rounding of M alone move the factors
    # further (R = 50 fitted to a rank-8 tensor: the extra components fit noise and the sampled Grams
    # lose conditioning), no worse than a plain FP32 product with an exact FP64 solve
    floor = fp32_product_floor(Th if mix else T, R, S, 17, iters, ref, ops=ops if mix else None)
    for A, Ar, f in zip(out["factors"], ref["factors"], floor):
        assert rel(A.cpu().numpy(), Ar) < max(1e-4, f)
    assert rel(out["lam"].cpu().numpy(), ref["lam"]) < max(1e-4, max(floor))


def test_grid_loop_rank_64_matches_oracle(cb, contract):
    # the widest column groups (R = 64): a tensor of true rank 64 with orthogonal factors and a start
    # near the truth, so that every sampled Gram is well conditioned and the 1e-4 bar measures the
    # kernel, not the amplification of FP32 rounding by an ill-conditioned least-squares problem
    dims, R, S = (160, 150, 140), 64, 900
    prob = make_problem(dims, R, C=0.0, eta=0.01, seed=302, dtype=torch.float32, device=DEV)
    T = to_oracle_array(prob.X, dims)
    rng = np.random.default_rng(4)
    init = [f * prob.lam[None, :] ** (1.0 / 3.0) + 0.05 * rng.standard_normal(f.shape) / np.sqrt(f.shape[0])
            for f in prob.factors]
    iters = 3
    trace = torch.zeros(iters, dtype=torch.float64, device=DEV)
    opts = cb.cpr_default_opts(seed=17, fixed_iters=iters, fit_trace_dev=trace.data_ptr(), loop_path=cb.LOOP_GRID)
    out = cb.cpr_cprand(prob.X, dims, R, S, opts=opts, init=[torch.tensor(a, device=DEV) for a in init])
    assert out["status"] == cb.OK and out["iters"] == iters
    ref = cp.cprand(T, R, S, seed=17, rule=cp.StopRule(fixed_iters=iters), factors0=init)
    np.testing.assert_allclose(trace.cpu().numpy(), ref["fits"], rtol=0, atol=1e-4)
    for A, Ar in zip(out["factors"], ref["factors"]):
        assert rel(A.cpu().numpy(), Ar) < 1e-4


def test_grid_loop_is_the_automatic_choice_and_reproducible(cb):
    # R = 50 does not fit the replicated-factor cluster: the automatic path is the whole GPU, and two
    # calls give bit-identical results (every reduction runs in a fixed order)
    dims = (300, 200, 250)
    prob = make_problem(dims, 8, C=0.5, eta=0.01, seed=5, dtype=torch.float32, device=DEV)
    outs = []
    for path in (cb.LOOP_AUTO, cb.LOOP_GRID, cb.LOOP_AUTO):
        trace = torch.zeros(4, dtype=torch.float64, device=DEV)
        opts = cb.cpr_default_opts(seed=9, fixed_iters=4, fit_trace_dev=trace.data_ptr(), loop_path=path)
        out = cb.cpr_cprand(prob.X, dims, 50, 600, opts=opts)
        outs.append((trace.cpu().numpy(), [A.cpu().numpy() for A in out["factors"]]))
    for tr, facs in outs[1:]:
        np.testing.assert_array_equal(tr, outs[0][0])
        for A, B in zip(facs, outs[0][1]):
            np.testing.assert_array_equal(A, B)


def test_grid_loop_reports_a_singular_gram(cb):
    dims = (200, 150, 120)
    prob = make_problem(dims, 4, C=0.5, eta=0.01, seed=8, dtype=torch.float32, device=DEV)
    rng = np.random.default_rng(3)
    init = [torch.tensor(rng.random((d, 20)), device=DEV) for d in dims]
    init[1][:, 7] = 0.0          # a zero column of A^(2): Z_S of the first update has a zero column
    opts = cb.cpr_default_opts(seed=2, fixed_iters=2, loop_path=cb.LOOP_GRID)
    out = cb.cpr_cprand(prob.X, dims, 20, 200, opts=opts, init=init)
    assert out["status"] == cb.ESINGULAR


@pytest.mark.parametrize("path", ["grid", "cluster", "graph"])
def test_non_finite_tensor_is_reported(cb, path):
    # a NaN entry makes ||X|| (and so every sampled fit) non-finite: the run reports CPR_ENONFINITE
    # before its first iteration
    dims = (200, 150, 120) if path == "grid" else (40, 30, 20)
    prob = make_problem(dims, 4, C=0.5, eta=0.01, seed=8, dtype=torch.float32, device="cpu")
    X = prob.X.clone()
    X[12345 % X.numel()] = float("nan")
    X = X.to(DEV)
    lp = {"grid": cb.LOOP_GRID, "cluster": cb.LOOP_CLUSTER, "graph": cb.LOOP_GRAPH}[path]
    out = cb.cpr_cprand(X, dims, 4, 60, opts=cb.cpr_default_opts(seed=1, max_iters=5, loop_path=lp))
    assert out["status"] == cb.ENONFINITE and out["iters"] == 0


def test_grid_barrier_wait_budget_runs_out(cb):
    # one poll per barrier wait: CTAs that arrive before the last one give up, every CTA leaves at its
    # next barrier, and the call returns CPR_ETIMEOUT; the context stays usable (the same call with the
    # default budget then succeeds on the same buffers)
    dims = (300, 200, 250)
    prob = make_problem(dims, 8, C=0.5, eta=0.01, seed=5, dtype=torch.float32, device=DEV)
    opts = cb.cpr_default_opts(seed=9, fixed_iters=2, loop_path=cb.LOOP_GRID, wait_budget=1)
    with pytest.raises(cb.CprError) as ei:
        cb.cpr_cprand(prob.X, dims, 50, 600, opts=opts)
    assert ei.value.status == cb.ETIMEOUT
    opts = cb.cpr_default_opts(seed=9, fixed_iters=2, loop_path=cb.LOOP_GRID)
    out = cb.cpr_cprand(prob.X, dims, 50, 600, opts=opts)
    assert out["status"] == cb.OK and out["iters"] == 2


def test_grid_path_rejects_unsupported_problems(cb):
    X = torch.zeros(40 * 30 * 20, dtype=torch.float64, device=DEV)
    with pytest.raises(cb.CprError):          # FP64 tensors do not take the whole-GPU loop
        cb.cpr_cprand(X, (40, 30, 20), 4, 60, opts=cb.cpr_default_opts(fixed_iters=1, loop_path=cb.LOOP_GRID))
