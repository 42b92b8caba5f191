"""Checks at full size: the benchmark's 2048x2048 segmentation grid
(4,194,304 non-terminals, DIA storage, one CUDA graph per IRLS step, as
bench.py times it) and the 256^3 volume (16.8M non-terminals).  The oracle's
exact solve does not finish at these sizes in test time, so the checks are
what it computes in seconds at any size: the
reduced system of every step (Eq. reduced-laplacian-system) from the oracle's
own reweighting, the true residual of the returned iterate in FP64, the
maximum principle, the cut value of the returned side by its definition, and
the sweep's value against cuts at sampled candidate thresholds."""
import numpy as np
import pytest

import gen
import oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the benchmark's pcg_tol
T = 4         # x^(0) and four reweighting steps (the benchmark runs 50 of the same)


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1501_03105_gb300 as pkg
    from paper_1501_03105_gb300 import binding, build
    import os
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return pkg


@pytest.fixture(scope="module")
def grid():
    g = gen.config_graph(2)
    return g, O.Problem.from_graph(g)


def run(P, g, precision):
    eps = O.eps_schedule(T)
    with P.Solver(g, pcg_tol=TOL, precision=precision) as s:
        assert s.problem_size()[2] == 1                     # DIA, as in the benchmark
        xs, infos = [], [s.initial()]
        xs.append(s.get_x())
        for l in range(1, T + 1):
            infos.append(s.irls_step(eps[l - 1]))
            xs.append(s.get_x())
        side, value, tau = s.cut()
    return xs, infos, side, value, tau


def true_residual(prob, g_cond, x):
    Lt, b = O.reduced_system(prob, O.laplacian(prob, g_cond))
    v = prob.Z.T @ x
    return float(np.linalg.norm(b - Lt @ v) / np.linalg.norm(b))


@pytest.mark.parametrize("precision", [0, 1])
def test_grid2048_steps_solve_the_reweighted_systems(P, grid, precision):
    g, prob = grid
    eps = O.eps_schedule(T)
    xs, infos, side, value, tau = run(P, g, precision)
    assert all(i.status == 0 for i in infos)
    # x^(0): W^(0) = C; then each step's system from the previous iterate
    assert true_residual(prob, O.initial_conductance(prob), xs[0]) <= 2 * TOL
    for l in range(1, T + 1):
        rel = true_residual(prob, O.reweight(prob, xs[l - 1], eps[l - 1]), xs[l])
        assert rel <= 2 * TOL, (l, rel)
        assert xs[l].min() >= -1e-12 and xs[l].max() <= 1 + 1e-12    # maximum principle
    # the returned side: s in, t out, the threshold rule, its value by definition
    sb = side.astype(bool)
    assert sb[prob.s] and not sb[prob.t]
    nt_mask = np.ones(g.n, dtype=bool)
    nt_mask[[prob.s, prob.t]] = False
    assert np.array_equal(sb[nt_mask], xs[-1][nt_mask] > tau)
    assert abs(O.cut_value(prob, sb) - value) <= 1e-12 * value
    # the sweep's minimum against 24 sampled candidate thresholds (positions
    # between strictly different x in the order x descending, index ascending)
    x = xs[-1]
    ids = np.flatnonzero(nt_mask)
    order = ids[np.lexsort((ids, -x[ids]))]
    xo = x[order]
    cand = np.flatnonzero(xo[:-1] > xo[1:]) + 1
    rng = np.random.default_rng(11)
    for k in rng.choice(cand, size=min(24, cand.size), replace=False):
        sk = np.zeros(g.n, dtype=bool)
        sk[prob.s] = True
        sk[order[:k]] = True
        assert O.cut_value(prob, sk) >= value * (1 - 1e-12), k


def test_grid2048_mixed_agrees_with_fp64(P, grid):
    g, prob = grid
    x64 = run(P, g, 0)
    xmx = run(P, g, 1)
    assert np.max(np.abs(x64[0][-1] - xmx[0][-1])) <= 1e-6
    assert abs(x64[3] - xmx[3]) <= 1e-9 * x64[3]


def test_vol256_steps_and_cut(P):
    """The 256^3 volume (16.8M non-terminals, DIA with three offsets, float32
    capacities): x^(0) and two IRLS steps, the same checks."""
    g = gen.config_graph(3)
    prob = O.Problem.from_graph(g)
    eps = O.eps_schedule(2)
    with P.Solver(g, pcg_tol=TOL) as s:
        assert s.problem_size()[2] == 1
        infos = [s.initial()]
        xs = [s.get_x()]
        for l in (1, 2):
            infos.append(s.irls_step(eps[l - 1]))
            xs.append(s.get_x())
        side, value, tau = s.cut()
    assert all(i.status == 0 for i in infos)
    assert true_residual(prob, O.initial_conductance(prob), xs[0]) <= 2 * TOL
    for l in (1, 2):
        assert true_residual(prob, O.reweight(prob, xs[l - 1], eps[l - 1]), xs[l]) <= 2 * TOL, l
        assert xs[l].min() >= -1e-12 and xs[l].max() <= 1 + 1e-12
    sb = side.astype(bool)
    assert sb[prob.s] and not sb[prob.t]
    assert abs(O.cut_value(prob, sb) - value) <= 1e-12 * value
    x = xs[-1]
    nt_mask = np.ones(g.n, dtype=bool)
    nt_mask[[prob.s, prob.t]] = False
    assert np.array_equal(sb[nt_mask], x[nt_mask] > tau)
    ids = np.flatnonzero(nt_mask)
    order = ids[np.lexsort((ids, -x[ids]))]
    xo = x[order]
    cand = np.flatnonzero(xo[:-1] > xo[1:]) + 1
    for k in np.random.default_rng(12).choice(cand, size=min(8, cand.size), replace=False):
        sk = np.zeros(g.n, dtype=bool)
        sk[prob.s] = True
        sk[order[:k]] = True
        assert O.cut_value(prob, sk) >= value * (1 - 1e-12), k
