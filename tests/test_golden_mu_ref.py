"""The stored reference cut values against an independent route through the
oracle.

tests/golden/mu_ref.json is written by make_mu_ref.py with the oracle's
Jacobi-PCG to 1e-12 (the only route that fits the large workloads).  On the
64x64 grid the oracle's exact sparse-LU IRLS (Section 2.1: x^(0) with
W^(0) = C, then T = 50 reweighted solves) finishes in about a second; its
final sweep cut (Section 3.3) must give the same mu_ref, and the sweeps of
its iterates the same first step within 1e-6 for good."""
import json
import os

import gen
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def test_grid64_mu_ref_equals_the_exact_solve_route():
    with open(os.path.join(HERE, "golden", "mu_ref.json")) as f:
        rec = json.load(f)["grid64"]
    prob = O.Problem.from_graph(gen.config_graph(1))
    T = rec["T"]
    xs, _ = O.irls(prob, T, O.eps_schedule(T))
    values = [O.sweep_cut(prob, x)["value"] for x in xs]
    mu = values[-1]
    assert abs(mu - rec["mu_ref"]) <= 1e-12 * mu, (mu, rec["mu_ref"])
    first = next(l for l in range(T + 1) if all(abs(v - mu) <= 1e-6 * mu for v in values[l:]))
    assert first == rec["first_step_within_1e-6_for_good"]
    # the stored per-step sweep values follow the same trajectory
    for l, step in enumerate(rec["steps"]):
        assert abs(step["sweep_value"] - values[l]) <= 1e-9 * values[l], l


def _script():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_mu_ref", os.path.join(HERE, "golden", "make_mu_ref.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_sequence_script_ranges_merge_and_oracle_route(tmp_path):
    """The sequence mode of make_mu_ref.py on a small sequence (a 6^3 volume,
    6 problems, T = 4, PCG to 1e-3): the evaluation half written in one go
    equals two ranges written to part files and merged, and each problem's
    mu_ref equals the sweep cut (Section 3.3) of the oracle's IRLS of that
    problem through its Python Jacobi-PCG (Section 3.1)."""
    m = _script()
    base = gen.config_graph(3, scale=6)
    kw = dict(base=base, problems=6, T=4, tol=1e-3)
    whole, parts = str(tmp_path / "whole.json"), str(tmp_path / "parts.json")
    m.run_sequence(main=whole, **kw)
    m.run_sequence(lo=3, hi=5, main=parts, **kw)
    m.run_sequence(lo=5, hi=6, main=parts, **kw)
    with open(parts, "w") as f:
        json.dump({"mu_ref": {}}, f)
    m.merge_sequence_parts(main=parts)
    with open(whole) as f:
        a = json.load(f)["mu_ref"]
    with open(parts) as f:
        b = json.load(f)["mu_ref"]
    assert list(a) == ["3", "4", "5"] and a == b
    assert not list(tmp_path.glob("parts.part*.json"))
    for k, c in enumerate(gen.capacity_sequence(base, 6, seed=5, sigma=0.01)):
        if k < 3:
            continue
        prob = O.Problem.from_graph(gen.Graph(base.n, base.row_ptr, base.col, c, base.s, base.t))
        xs, _ = O.irls(prob, 4, O.eps_schedule(4), solver="pcg", tol=1e-3)
        v = O.sweep_cut(prob, xs[-1])["value"]
        assert abs(v - a[str(k)]["mu_ref"]) <= 1e-9 * v, k
