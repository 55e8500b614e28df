"""The schedule table of the autotuner, host side: a cache file's buckets are loaded, looked up by the
bucket of a batch (extents and sample counts rounded up to powers of two, ranks to multiples of 8),
written back unchanged, and cleared.  No GPU work."""
import pytest


@pytest.fixture(scope="module")
def cb():
    from paper_1701_06600_gb300 import build
    build.build()
    from paper_1701_06600_gb300 import binding
    return binding


def test_cache_file_round_trip_and_bucketing(cb, tmp_path):
    cb.cpr_tune_clear()
    assert cb.cpr_tune_lookup([(1500, 1500, 1500)], [50], [2000]) is None
    # the bucket of 1500^3 FP32, one problem, CPRAND-MIX, R = 50, S = 2000: extents -> 2^11, R -> 7
    # (multiples of 8), S -> 2^11
    key = "d1:N3:B0:m1:I11,11,11:R7:S11"
    f = tmp_path / "tune.txt"
    f.write_text("%s 5 2 32 0.125\nnot-a-line\n" % key)
    cb.cpr_tune_load(f)
    got = cb.cpr_tune_lookup([(1500, 1500, 1500)], [50], [2000], mix=True)
    assert got == {"loop_path": 5, "split_per_sm": 2, "grid_min_split": 32, "ms_per_iter": 0.125}
    # the same bucket: 1100 .. 2048 per mode, R 49 .. 56, S 1025 .. 2048
    assert cb.cpr_tune_lookup([(1100, 2048, 1025)], [56], [1025], mix=True) == got
    assert cb.cpr_tune_lookup([(1500, 1500, 1500)], [50], [2000], mix=False) is None
    assert cb.cpr_tune_lookup([(1500, 1500, 1500)], [57], [2000], mix=True) is None
    g = tmp_path / "out.txt"
    cb.cpr_tune_save(g)
    assert g.read_text().split() == [key, "5", "2", "32", "0.125"]
    cb.cpr_tune_clear()
    assert cb.cpr_tune_lookup([(1500, 1500, 1500)], [50], [2000], mix=True) is None
    with pytest.raises(cb.CprError):
        cb.cpr_tune_load(tmp_path / "missing.txt")
