"""The autotuner on the GPU: it times the candidate schedules of a batch, records the fastest for the
batch's bucket, and every later automatic call in that bucket runs with it; a schedule saved to a
file, cleared and loaded back gives a bit-identical run (every reduction has a fixed order)."""
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


def run(cb, X, dims, R, S):
    trace = torch.zeros(3, dtype=torch.float64, device=DEV)
    out = cb.cpr_cprand_mix(X, dims, R, S, opts=cb.cpr_default_opts(seed=5, fixed_iters=3,
                                                                      fit_trace_dev=trace.data_ptr()))
    assert out["status"] == cb.OK
    return trace.cpu().numpy(), [a.cpu().numpy() for a in out["factors"]]


@pytest.mark.parametrize("dims,R,S", [((300, 200, 250), 50, 600), ((120, 110, 100), 12, 300)])
def test_tuned_schedule_is_recorded_reused_and_persisted(cb, tmp_path, dims, R, S):
    cb.cpr_tune_clear()
    prob = make_problem(dims, min(R, 8), C=0.5, eta=0.01, seed=12, dtype=torch.float32, device=DEV)
    best, _ = cb.cpr_autotune([prob.X], [dims], [R], [S], [cb.cpr_default_opts(seed=5)], mix=True)
    assert best["loop_path"] in (1, 2, 4, 5) and best["ms_per_iter"] > 0
    assert cb.cpr_tune_lookup([dims], [R], [S], mix=True) == best
    a = run(cb, prob.X, dims, R, S)
    path = tmp_path / "tune.txt"
    cb.cpr_tune_save(path)
    cb.cpr_tune_clear()
    assert cb.cpr_tune_lookup([dims], [R], [S], mix=True) is None
    cb.cpr_tune_load(path)
    assert cb.cpr_tune_lookup([dims], [R], [S], mix=True) == best
    b = run(cb, prob.X, dims, R, S)
    np.testing.assert_array_equal(a[0], b[0])
    for x, y in zip(a[1], b[1]):
        np.testing.assert_array_equal(x, y)
    cb.cpr_tune_clear()
