"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins
of ``test_oracle_pins.py`` catch every one of them.

Each mutant replaces one oracle function with a subtly wrong variant (a dropped
term, a flipped sign, a wrong index, a transposed operand); the test runs the
pin functions against the mutated oracle and requires at least one to fail.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import oracle.pirmcut as OP
from tests import test_oracle_pins as pins


def _reweight_no_square(prob, x, eps, form=OP.WEIGHTED_L1):
    d = prob.B @ x
    if form == OP.PAPER:
        return prob.cap * prob.cap / np.sqrt(np.abs(prob.cap * d) + eps ** 2)
    return prob.cap / np.sqrt(np.abs(d) + eps ** 2)


def _reweight_paper_one_c(prob, x, eps, form=OP.WEIGHTED_L1):
    d = prob.B @ x
    if form == OP.PAPER:
        return prob.cap / np.sqrt((prob.cap * d) ** 2 + eps ** 2)
    return prob.cap / np.sqrt(d ** 2 + eps ** 2)


def _reduced_b_sign(prob, L):
    Lt = (prob.Z.T @ L @ prob.Z).tocsr()
    return Lt, prob.Z.T @ (L @ prob.e_s)


def _reduced_b_from_t(prob, L):
    Lt = (prob.Z.T @ L @ prob.Z).tocsr()
    e_t = np.zeros(prob.n)
    e_t[prob.t] = 1.0
    return Lt, -(prob.Z.T @ (L @ e_t))


def _laplacian_drop_terminal_diag(prob, g):
    L = (prob.B.T @ sp.diags(g) @ prob.B).tolil()
    for e in range(prob.m):
        u, v = prob.eu[e], prob.ev[e]
        if prob.t in (u, v) and prob.s not in (u, v):
            w = v if u == prob.t else u
            L[w, w] -= g[e]
    return L.tocsr()


def _initial_unweighted(prob):
    return prob.cap ** 2


def _full_x_swapped(self, v):
    e_t = np.zeros(self.n)
    e_t[self.t] = 1.0
    return self.Z @ v + e_t


def _candidates_split_ties(xs_sorted):
    return np.arange(xs_sorted.shape[0] + 1, dtype=np.int64)


def _sweep_order_ascending(prob, x):
    v = prob.nonterminals
    return v[np.lexsort((v, x[v]))]


def _cut_value_count_internal(prob, side):
    side = np.asarray(side, dtype=bool)
    crossing = side[prob.eu] != side[prob.ev]
    inside = side[prob.eu] & side[prob.ev]
    return float(np.sum(prob.cap[crossing]) + 0.5 * np.sum(prob.cap[inside]))


def _objective_no_eps(prob, x, eps, form=OP.WEIGHTED_L1):
    d = prob.B @ x
    if form == OP.PAPER:
        return float(np.sum(np.abs(prob.cap * d)))
    return float(np.sum(prob.cap * np.abs(d)))


MUTANTS = {
    "reweight drops the square": [("reweight", _reweight_no_square)],
    "paper reweight keeps one c": [("reweight", _reweight_paper_one_c)],
    "b has the wrong sign": [("reduced_system", _reduced_b_sign)],
    "b built from e_t": [("reduced_system", _reduced_b_from_t)],
    "terminal conductance dropped from the diagonal": [("laplacian", _laplacian_drop_terminal_diag)],
    "x0 weights c^2 (W0 = I)": [("initial_conductance", _initial_unweighted)],
    "x_t set to 1 instead of x_s": [("Problem.full_x", _full_x_swapped)],
    "sweep splits tied voltages": [("_candidates", _candidates_split_ties)],
    "sweep sorted ascending": [("_sweep_order", _sweep_order_ascending)],
    "cut counts internal edges": [("cut_value", _cut_value_count_internal)],
    "objective without eps": [("smoothed_objective", _objective_no_eps)],
}

PIN_TESTS = [
    lambda: [pins.test_x0_single_vertex_divider(a, b) for a, b in [(3.0, 1.0), (0.25, 2.0)]],
    pins.test_x0_series_chain_voltage_divider,
    lambda: [pins.test_one_irls_step_closed_form(f, 3.0, 1.0, 0.75, 0.1) for f in (OP.WEIGHTED_L1, OP.PAPER)],
    pins.test_reduced_system_hand_example,
    lambda: [pins.test_smoothed_objective_closed_form(v, e) for v, e in [(0.3, 0.1), (0.5, 0.0)]],
    lambda: [pins.test_laplacian_structure(f) for f in (OP.WEIGHTED_L1, OP.PAPER)],
    pins.test_maximum_principle_every_step,
    lambda: [pins.test_monotone_majorise_minimise(f) for f in (OP.WEIGHTED_L1, OP.PAPER)],
    lambda: [pins.test_exact_references_on_hand_examples(n) for n in sorted(pins.load_hand())],
    pins.test_sweep_cut_ties_and_candidates,
    pins.test_sweep_cut_order_hand_example,
    pins.test_irls_sweep_cut_finds_unique_min_cut,
    pins.test_cheeger_type_bounds,
]


def _apply(monkeypatch, patches):
    for name, fn in patches:
        if name.startswith("Problem."):
            monkeypatch.setattr(OP.Problem, name.split(".", 1)[1], fn)
            continue
        monkeypatch.setattr(OP, name, fn)
        if hasattr(oracle, name):
            monkeypatch.setattr(oracle, name, fn)


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_mutant(monkeypatch, mutant):
    _apply(monkeypatch, MUTANTS[mutant])
    caught = 0
    for pin in PIN_TESTS:
        try:
            with np.errstate(all="ignore"):
                pin()
        except Exception:  # an AssertionError, or the mutant crashing the pin
            caught += 1
    assert caught >= 1, f"no pin caught: {mutant}"


def test_unmutated_oracle_passes_every_pin():
    for pin in PIN_TESTS:
        pin()
