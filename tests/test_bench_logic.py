"""Host logic of bench.py: time-to-cut against a reference value (reading
c10: the first step within 1e-6, and the last step must be within it too),
the oracle's reference values on file, and the CPU baseline's sample."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import gen  # noqa: E402


def test_time_to_cut_first_step_within_tolerance():
    track = [(110.0, 1.0), (100.5, 2.0), (100.001, 3.0), (100.0000001, 4.0), (100.0, 5.0)]
    r = bench.time_to_cut(track, 100.0)
    assert r["reached"] and r["step"] == 3 and r["ms"] == 10.0 and r["solve_ms"] == 15.0


def test_time_to_cut_requires_the_last_step():
    track = [(100.0, 1.0), (100.0, 1.0), (100.01, 1.0)]
    r = bench.time_to_cut(track, 100.0)
    assert not r["reached"] and r["ms"] is None and r["final_rel_err"] == pytest.approx(1e-4)


def test_time_to_cut_without_reference():
    assert bench.time_to_cut([(1.0, 1.0)], None)["reached"] is False


def test_oracle_reference_values_on_file():
    mu = bench.golden_mu_ref("grid2048")
    assert mu is not None and mu > 0
    assert bench.golden_mu_ref("no-such-workload") is None


def test_cpu_baseline_sample_counts_iterations_and_cores():
    g = gen.config_graph(1, scale=32)
    r = bench.cpu_oracle_sample(g, budget_s=0.05, threads=2)
    assert r["cores"] == 2 and r["iters"] > 0 and r["value"] > 0 and r["kind"] == "oracle"


def test_time_to_cut_with_one_sweep():
    # steps of 5 ms each, 1 ms of which is the sweep: reached at step 2
    track = [(110.0, 5.0), (101.0, 5.0), (100.0, 5.0), (100.0, 5.0)]
    r = bench.time_to_cut(track, 100.0, sweep_ms=1.0)
    assert r["step"] == 2 and r["ms"] == 15.0 and r["ms_one_sweep"] == 13.0


def test_sequence_reference_values_on_file():
    """Every evaluation problem of the default sequence (100-199) has the
    oracle's mu_ref; other sequences have none (the bench then falls back to
    the plain FP64 arm's final cut and says so)."""
    ref = bench.sequence_mu_ref(128, 200, 1e-3)
    assert sorted(ref) == list(range(100, 200))
    assert all(v > 0 for v in ref.values())
    assert bench.sequence_mu_ref(64, 200, 1e-3) == {}
    assert bench.sequence_mu_ref(128, 20, 1e-3) == {}
    assert bench.sequence_mu_ref(128, 200, 1e-10) == {}


def test_golden_reference_files_name_their_oracle_runs():
    """The stored reference values come from the committed oracle script:
    each file names the command that wrote it."""
    import json
    with open(bench.MU_REF_JSON) as f:
        d = json.load(f)
    assert set(d) >= {"grid64", "grid2048", "vol256"}
    for name, rec in d.items():
        assert rec["command"] == f"python tests/golden/make_mu_ref.py {name}"
        assert rec["steps"][-1]["sweep_value"] == rec["mu_ref"]
    with open(bench.MU_REF_SEQ_JSON) as f:
        seq = json.load(f)
    assert seq["command"] == "python tests/golden/make_mu_ref.py seq128"
