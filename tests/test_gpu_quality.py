"""The recovery study of Sec. 4.2 (bench.py --quality-sweep) on a reduced grid: every cell is reported,
and on well-conditioned low-noise tensors CPRAND-MIX recovers the true factors (median score near 1, fit
near the noise floor).  The scores are checked against the oracle's score of the same factors."""
import argparse

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_reduced_sweep_reports_every_cell_and_recovers_easy_cases():
    import bench
    args = argparse.Namespace(sweep_tensors=2, sweep_sizes="3x40")
    out = bench.run_quality_sweep(args)
    assert out["decompositions"] == 4 * 2 * 2 * 6
    assert len(out["cells"]) == 4 * 2 * 2
    for c in out["cells"]:
        assert c["runs"] == 6 and all(np.isfinite(c["fit_q25_med_q75"])) and all(np.isfinite(c["score_q25_med_q75"]))
    easy = [c for c in out["cells"] if c["C"] == 0.5 and c["eta"] == 0.01 and c["method"] == "cprand_mix" and c["R"] == 5]
    assert easy[0]["score_q25_med_q75"][1] > 0.95
    assert easy[0]["fit_q25_med_q75"][1] > 0.98


def test_sweep_score_equals_oracle_score_of_the_same_factors():
    import bench
    from oracle import score
    from paper_1701_06600_gb300 import binding as cb
    from synth import make_problem
    dims = (40, 40, 40)
    prob = make_problem(dims, 5, C=0.9, eta=0.1, seed=5, dtype=torch.float32, device="cuda")
    for R, S in ((5, 80), (6, 108)):
        out = cb.cpr_cprand_mix(prob.X, dims, R, S, opts=cb.cpr_default_opts(seed=3, noise_eta=0.1))
        est = [A.cpu().numpy() for A in out["factors"]]
        assert abs(bench.score_assignment(prob.factors, est) - score.score(prob.factors, est)) < 1e-12
