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
