"""GPU parity of CPRAND-MIX in its complex form (Alg. 4) against the FP64 oracle (oracle/mixing_fft.py).

The library and the oracle draw the same samples, initial factors and fit entries (Philox streams), so
the runs agree update by update up to rounding (FP32 mixed tensor and FP32 unmixing on the GPU, FP64
in the oracle): the factors after one outer iteration to 1e-4 relative, the sampled-fit trace over
the first iterations to 1e-4, and the exact fit of whole runs to 1e-3.
"""
import numpy as np
import pytest
import torch

from oracle import cp, mixing_fft
from synth import make_problem, to_oracle_array

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


@pytest.mark.parametrize("dims,R,S", [((40, 36, 30), 4, 60), ((64, 48, 40), 5, 81), ((20, 15, 12, 10), 3, 40),
                                      ((100, 21, 14), 6, 108)])
def test_first_iterations_match_oracle(cb, dims, R, S):
    prob = make_problem(dims, R, C=0.5, eta=0.01, seed=61, dtype=torch.float32, device=DEV)
    T = to_oracle_array(prob.X, dims)
    trace = torch.zeros(3, dtype=torch.float64, device=DEV)
    out1 = cb.cpr_cprand_mix_fft(prob.X, dims, R, S, opts=cb.cpr_default_opts(seed=17, fixed_iters=1))
    ref1 = mixing_fft.cprand_mix_fft(T, R, S, seed=17, rule=cp.StopRule(fixed_iters=1))
    assert out1["status"] == cb.OK and out1["iters"] == 1
    for A, Ar in zip(out1["factors"], ref1["factors"]):
        assert rel(A.cpu().numpy(), Ar) < 1e-4
    assert rel(out1["lam"].cpu().numpy(), ref1["lam"]) < 1e-4
    out3 = cb.cpr_cprand_mix_fft(prob.X, dims, R, S,
                                 opts=cb.cpr_default_opts(seed=17, fixed_iters=3, fit_trace_dev=trace.data_ptr()))
    ref3 = mixing_fft.cprand_mix_fft(T, R, S, seed=17, rule=cp.StopRule(fixed_iters=3))
    np.testing.assert_allclose(trace.cpu().numpy(), ref3["fits"], rtol=0, atol=1e-4)


def test_whole_run_reaches_oracle_fit(cb):
    dims, R = (60, 50, 40), 5
    prob = make_problem(dims, R, C=0.5, eta=0.01, seed=23, dtype=torch.float32, device=DEV)
    T = to_oracle_array(prob.X, dims)
    S = cp.sample_size(R)
    out = cb.cpr_cprand_mix_fft(prob.X, dims, R, S, opts=cb.cpr_default_opts(seed=41, noise_eta=0.01))
    ref = mixing_fft.cprand_mix_fft(T, R, S, seed=41, rule=cp.StopRule(eta=0.01))
    assert out["status"] == cb.OK
    f_gpu = cp.exact_fit(T, out["lam"].cpu().numpy(), [A.cpu().numpy() for A in out["factors"]])
    f_ref = cp.exact_fit(T, ref["lam"], ref["factors"])
    assert abs(f_gpu - f_ref) < 1e-3, (f_gpu, f_ref, out["iters"], ref["iters"])


def test_rejects_unsupported_inputs(cb):
    X = torch.randn(37 * 29 * 41, device=DEV)          # 37, 29, 41: prime factors above 7
    with pytest.raises(cb.CprError):
        cb.cpr_cprand_mix_fft(X, (37, 29, 41), 3, 40)
    X = torch.randn(40 * 36 * 30, device=DEV, dtype=torch.float64)
    with pytest.raises(cb.CprError):
        cb.cpr_cprand_mix_fft(X, (40, 36, 30), 3, 40)   # FP32 only


def test_400_cubed_iteration_rate_is_reported(cb):
    # the 400^3 workload (rank 10, congruence 0.9), five outer iterations of the complex form: its
    # time per iteration next to the real form's, and its fit estimate tracking the exact fit
    dims = (400, 400, 400)
    prob = make_problem(dims, 10, C=0.9, eta=0.01, seed=1001, dtype=torch.float32, device=DEV)
    opts = cb.cpr_default_opts(seed=2001, fixed_iters=5)
    warm = cb.cpr_cprand_mix_fft(prob.X, dims, 10, 230, opts=cb.cpr_default_opts(seed=2001, fixed_iters=1))
    out = cb.cpr_cprand_mix_fft(prob.X, dims, 10, 230, opts=opts, ws=warm["ws"])
    cb.cpr_cprand_mix(prob.X, dims, 10, 230, opts=cb.cpr_default_opts(seed=2001, fixed_iters=1))
    real = cb.cpr_cprand_mix(prob.X, dims, 10, 230, opts=cb.cpr_default_opts(seed=2001, fixed_iters=5))
    assert out["status"] == cb.OK and out["iters"] == 5
    A = [f.double() for f in out["factors"]]
    lam = out["lam"].double()
    Xv = prob.X.double().view(400, 400, 400)            # Xv[i3, i2, i1]
    model = torch.einsum("r,ir,jr,kr->kji", lam, *A)
    f_true = 1.0 - (torch.linalg.vector_norm(Xv - model) / torch.linalg.vector_norm(Xv)).item()
    print("400^3 complex form: setup %.2f ms, %.1f us per outer iteration (real form %.1f us); fit estimate "
          "%.5f, exact %.5f" % (out["ms_setup"], 1e3 * out["ms_iterate"] / 5, 1e3 * real["ms_iterate"] / 5,
                                out["fit_est"], f_true))
    assert abs(out["fit_est"] - f_true) < 2e-3
