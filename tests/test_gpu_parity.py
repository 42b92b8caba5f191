"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Bars (from the arithmetic and the method's tolerances):
* iterate x: max |x_gpu - x_oracle| <= 1e-9 (x lies in [0, 1], so this is the
  relative error in the max norm), per IRLS step, teacher-forced: both sides
  start step l from the oracle's x^(l-1); the GPU solves to 1e-13.
* cut value: |mu_gpu - mu_oracle| <= 1e-9 mu_oracle.
* cut side: identical on every vertex with |x_v - tau| >= 1e-6 whenever both
  sides chose the same threshold; otherwise (a tie of cut values between
  candidates) only the value is compared.
"""
import numpy as np
import pytest

import gen
import oracle as O

pytestmark = pytest.mark.gpu

XTOL = 1e-9
CUT_RTOL = 1e-9


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


def solver(P, g, **kw):
    kw.setdefault("pcg_tol", 1e-13)
    return P.Solver(g, **kw)


def check_cut(prob, x, side, value, tau):
    ref = O.sweep_cut(prob, x)
    assert abs(value - ref["value"]) <= CUT_RTOL * max(ref["value"], 1e-300), (value, ref["value"])
    assert abs(O.cut_value(prob, side.astype(bool)) - value) <= 1e-12 * max(value, 1e-300)
    if abs(tau - ref["tau"]) < 1e-12:
        far = np.abs(x - ref["tau"]) >= 1e-6
        far[[prob.s, prob.t]] = True
        assert np.array_equal(side.astype(bool)[far], ref["side"][far])
    return ref


GRAPHS = [
    ("grid16", lambda: gen.config_graph(1, scale=16)),
    ("grid37x41", lambda: gen.segmentation_grid(
        np.clip(gen.image_disks_2d(37, 41, [(18, 20, 9)]) + np.random.default_rng(7).normal(0, .05, (41, 37)), 0, 1))),
    ("vol9", lambda: gen.config_graph(3, scale=9)),
    ("vol8", lambda: gen.config_graph(3, scale=8)),          # n~ % 4 == 0: vectorised kernels
    ("grid12x20", lambda: gen.segmentation_grid(
        np.clip(gen.image_disks_2d(12, 20, [(6, 9, 4)]) + np.random.default_rng(8).normal(0, .05, (20, 12)), 0, 1))),
    ("random12", lambda: gen.random_graph(12, 0.3, 11, zero_frac=0.2, st_edge=True)),
    ("random40", lambda: gen.random_graph(40, 0.1, 12)),
    ("chunglu", lambda: gen.chung_lu_instance(3000, 5)),
]


@pytest.mark.parametrize("fmt", [0, 2])
@pytest.mark.parametrize("name,make", GRAPHS)
def test_x0_matches_oracle(P, name, make, fmt):
    """x^(0): the WLS with W^(0) = C (Section 2.1), cold-started PCG."""
    g = make()
    prob = O.Problem.from_graph(g)
    x0, _ = O.wls_step(prob, O.initial_conductance(prob))
    with solver(P, g, format=fmt) as s:
        info = s.initial()
        assert info.status == 0
        x = s.get_x()
    assert x[g.s] == 1.0 and x[g.t] == 0.0
    assert np.max(np.abs(x - x0)) <= XTOL


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("fmt", [0, 2])
def test_teacher_forced_steps_grid64(P, form, fmt):
    """Every IRLS step of the 64x64 workload, T = 50, each started from the
    oracle's previous iterate (Steps 1-2 of Section 2.1)."""
    g = gen.config_graph(1)
    prob = O.Problem.from_graph(g)
    T = 50
    eps = O.eps_schedule(T)
    xs, _ = O.irls(prob, T, eps, form=form)
    with solver(P, g, format=fmt, reweight_form=form) as s:
        for l in range(1, T + 1):
            s.set_x(xs[l - 1])
            info = s.irls_step(eps[l - 1])
            assert info.status == 0 and info.eps == eps[l - 1]
            x = s.get_x()
            assert np.max(np.abs(x - xs[l])) <= XTOL, l
            assert info.x_min >= -1e-12 and info.x_max <= 1 + 1e-12


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("fmt", [0, 2])
def test_step_objective_and_flow_value(P, fmt, form, precision):
    """options.step_stats: each step's record holds S_eps(x^(l)) and the flow
    value x^T L(g^(l)) x of the returned iterate, as the oracle computes them
    from that iterate (Eq. l1-min-smooth-version, Prop.
    wls-equal-electrical-flow); step 0 uses eps = 0 and g = c.  Off: NaN."""
    g = gen.config_graph(1)
    prob = O.Problem.from_graph(g)
    T = 10
    eps = O.eps_schedule(T)
    xs, _ = O.irls(prob, T, eps, form=form)
    with solver(P, g, format=fmt, reweight_form=form, precision=precision, step_stats=1) as s:
        info = s.initial()
        x = s.get_x()
        assert info.objective == pytest.approx(O.smoothed_objective(prob, x, 0.0, form), rel=1e-12)
        assert info.flow_value == pytest.approx(O.flow_value(prob, x, O.initial_conductance(prob)), rel=1e-12)
        for l in range(1, T + 1):
            s.set_x(xs[l - 1])
            info = s.irls_step(eps[l - 1])
            x = s.get_x()
            gl = O.reweight(prob, xs[l - 1], eps[l - 1], form)
            assert info.objective == pytest.approx(O.smoothed_objective(prob, x, eps[l - 1], form), rel=1e-12), l
            assert info.flow_value == pytest.approx(O.flow_value(prob, x, gl), rel=1e-11), l
            # the MM step: the objective does not rise along the step (reading c12)
            assert info.objective <= O.smoothed_objective(prob, xs[l - 1], eps[l - 1], form) * (1 + 1e-12)
    with solver(P, g, format=fmt) as s:
        info = s.initial()
        assert np.isnan(info.objective) and np.isnan(info.flow_value)


def objective_positive(prob, x, eps, form):
    """S_eps(x) over the edges of positive capacity: the form the library
    records.  The packed storage does not tell a listed edge of capacity 0
    from an absent one, so such an edge counts 0; in the paper's form the
    oracle's sum gives each of them sqrt((0 d)^2 + eps^2) = eps, which is
    taken out here (the weighted-l1 form gives them 0 already)."""
    m0 = int(np.count_nonzero(prob.cap == 0.0))
    s = O.smoothed_objective(prob, x, eps, form)
    return s - m0 * eps if form == O.PAPER else s


def flow_tolerance(prob, x, g):
    """Rounding bound of the oracle's flow value x^T (L x): the products
    cancel (L x vanishes at the non-terminals), so its error is a few units
    of FP64 rounding times |x|^T |L| |x| (row lengths up to the hub's)."""
    L = O.laplacian(prob, g)
    gross = float(np.abs(x) @ (abs(L) @ np.abs(x)))
    deg = int(np.diff(L.indptr).max())
    return 1e-12 * abs(float(x @ (L @ x))) + 2 * (deg + 2) * 2.0 ** -53 * gross


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("name,make", GRAPHS)
def test_step_objective_and_flow_value_graphs(P, name, make, form, precision):
    """The step statistics on every small graph: zero capacities
    (random12), a direct s-t edge (random12), CSR rows of every length and a
    hub row (chunglu), DIA grids and volumes; teacher-forced steps."""
    g = make()
    prob = O.Problem.from_graph(g)
    T = 8
    eps = O.eps_schedule(T)
    xs, _ = O.irls(prob, T, eps, form=form)
    with solver(P, g, reweight_form=form, precision=precision, step_stats=1) as s:
        info = s.initial()
        x = s.get_x()
        assert info.objective == pytest.approx(objective_positive(prob, x, 0.0, form), rel=1e-12)
        g0 = O.initial_conductance(prob)
        assert abs(info.flow_value - O.flow_value(prob, x, g0)) <= flow_tolerance(prob, x, g0)
        for l in range(1, T + 1):
            s.set_x(xs[l - 1])
            info = s.irls_step(eps[l - 1])
            x = s.get_x()
            gl = O.reweight(prob, xs[l - 1], eps[l - 1], form)
            assert info.objective == pytest.approx(objective_positive(prob, x, eps[l - 1], form), rel=1e-12), l
            assert abs(info.flow_value - O.flow_value(prob, x, gl)) <= flow_tolerance(prob, x, gl), l


@pytest.mark.parametrize("graph_launch", [1, 0])
def test_step_stats_after_update_weights_st_edge(P, graph_launch):
    """A sequence on one structure (Section 6) with a direct s-t edge whose
    capacity changes: after pirmcut_update_weights every step's objective and
    flow value use the new c(s,t) (the step graphs are rebuilt)."""
    g = gen.random_graph(30, 0.15, 21, st_edge=True)
    T = 4
    eps = O.eps_schedule(T)
    with solver(P, g, step_stats=1, graph_launch=graph_launch) as s:
        for k, scale in enumerate([1.0, 3.0, 0.25]):
            c = g.c.copy()
            rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
            st = ((rows == g.s) & (g.col == g.t)) | ((rows == g.t) & (g.col == g.s))
            assert st.sum() == 2
            c[st] *= scale
            prob = O.Problem(g.n, g.row_ptr, g.col, c, g.s, g.t)
            if k:
                s.update_weights(c)
            infos = s.solve(T, eps)
            xs, _ = O.irls(prob, T, eps)
            for l in range(T + 1):
                e = eps[l - 1] if l else 0.0
                gl = O.initial_conductance(prob) if l == 0 else O.reweight(prob, xs[l - 1], e)
                # free-running: the GPU and the oracle iterates agree to the solver tolerance
                assert infos[l].objective == pytest.approx(objective_positive(prob, xs[l], e, 0), rel=1e-9), (k, l)
                assert infos[l].flow_value == pytest.approx(O.flow_value(prob, xs[l], gl), rel=1e-9), (k, l)


@pytest.mark.parametrize("name,make", GRAPHS)
def test_teacher_forced_steps_small(P, name, make):
    g = make()
    prob = O.Problem.from_graph(g)
    T = 20
    eps = O.eps_schedule(T)
    xs, _ = O.irls(prob, T, eps)
    with solver(P, g) as s:
        for l in range(1, T + 1):
            s.set_x(xs[l - 1])
            s.irls_step(eps[l - 1])
            assert np.max(np.abs(s.get_x() - xs[l])) <= XTOL, l


def test_free_running_solve_grid64(P):
    """Algorithm 1 on the 64x64 workload with its own tolerance (1e-10):
    the final sweep cut matches the oracle's."""
    g = gen.config_graph(1)
    prob = O.Problem.from_graph(g)
    T = 50
    eps = O.eps_schedule(T)
    xs, _ = O.irls(prob, T, eps)
    with P.Solver(g, pcg_tol=1e-10) as s:
        infos = s.solve(T, eps)
        assert [i.step for i in infos] == list(range(T + 1))
        assert all(i.status == 0 for i in infos)
        assert all(i.rel_residual <= 1e-10 for i in infos)
        x = s.get_x()
        side, value, tau = s.cut()
    assert np.max(np.abs(x - xs[-1])) <= 1e-6      # free-running: reported, loose
    ref = check_cut(prob, xs[-1], side, value, tau)
    mu_star, _ = O.max_flow_min_cut(prob)
    assert value >= mu_star * (1 - 1e-12)           # a cut is never below the min cut
    assert abs(value - ref["value"]) <= CUT_RTOL * ref["value"]


@pytest.mark.parametrize("fmt", [0, 2])
def test_stopping_norm_is_the_true_residual(P, fmt):
    """The FP64 path sums ||r||^2 of its stopping test in FP32 (from r^ =
    D^-1/2 r and d^1/2): every step stops with the reported ||r|| / ||b|| at
    most pcg_tol, and the residual of the returned x, recomputed here in FP64
    from the oracle's system, agrees with it."""
    g = gen.config_graph(1)
    prob = O.Problem.from_graph(g)
    T = 20
    eps = O.eps_schedule(T)
    xs, _ = O.irls(prob, T, eps)
    tol = 1e-6
    with solver(P, g, format=fmt, pcg_tol=tol) as s:
        for l in range(1, T + 1):
            s.set_x(xs[l - 1])
            info = s.irls_step(eps[l - 1])
            assert info.status == 0 and info.rel_residual <= tol, l
            Lt, b = O.reduced_system(prob, O.laplacian(prob, O.reweight(prob, xs[l - 1], eps[l - 1])))
            v = prob.Z.T @ s.get_x()
            true = np.linalg.norm(b - Lt @ v) / np.linalg.norm(b)
            assert true <= 1.01 * tol and abs(true - info.rel_residual) <= 1e-2 * tol, (l, true, info.rel_residual)


@pytest.mark.parametrize("fmt", [0, 2])
def test_capacity_scaling_and_the_fp32_stopping_norm(P, fmt):
    """x is invariant under c -> lambda c (weighted-l1 form).  With lambda =
    2^20 every diagonal stays in the range where the stopping norm is summed
    in FP32 and every quantity scales by a power of two; lambda = 2^100 or
    2^-100 puts diagonals outside it, where the norm is summed in FP64."""
    g = gen.config_graph(1, scale=32)
    T = 8
    eps = O.eps_schedule(T)

    def run(lam):
        gg = gen.Graph(g.n, g.row_ptr, g.col, g.c * lam, g.s, g.t)
        with solver(P, gg, format=fmt, pcg_tol=1e-12) as s:
            infos = s.solve(T, eps)
            assert all(i.status == 0 and i.rel_residual <= 1e-12 for i in infos), lam
            return s.get_x(), [i.pcg_iters for i in infos]

    x1, it1 = run(1.0)
    x2, it2 = run(2.0 ** 20)
    assert all(abs(a - b) <= 1 for a, b in zip(it1, it2)) and np.max(np.abs(x2 - x1)) <= 1e-12
    for lam in (2.0 ** 100, 2.0 ** -100):
        x3, it3 = run(lam)
        assert np.max(np.abs(x3 - x1)) <= 1e-10, lam
        assert all(abs(a - b) <= 2 for a, b in zip(it1, it3)), (lam, it1, it3)


@pytest.mark.parametrize("name,make", GRAPHS)
@pytest.mark.parametrize("fmt", [0, 2])
def test_sweep_cut_on_given_x(P, name, make, fmt):
    """Sweep cut (Section 3.3) on a seeded x with ties, set through set_x."""
    g = make()
    prob = O.Problem.from_graph(g)
    rng = np.random.default_rng(3)
    x = np.round(rng.random(g.n) * 16) / 16          # heavy ties
    x[g.s], x[g.t] = 1.0, 0.0
    with solver(P, g, format=fmt) as s:
        s.set_x(x)
        side, value, tau = s.cut()
    ref = check_cut(prob, x, side, value, tau)
    assert abs(tau - ref["tau"]) < 1e-15


@pytest.mark.parametrize("nt", [1, 2, 3, 255, 256, 257, 2047, 2048, 2049, 4097])
def test_sweep_ragged_sizes(P, nt):
    """Sort tiles and scan tiles with ragged tails (chain graphs)."""
    rng = np.random.default_rng(nt)
    n = nt + 2
    s, t = nt, nt + 1
    u = list(range(nt - 1)) + list(range(nt)) + list(range(nt))
    v = list(range(1, nt)) + [s] * nt + [t] * nt
    c = list(rng.uniform(0.5, 1.5, len(u)))
    rp, col, cc = gen.csr_from_edges(n, u, v, c)
    g = gen.Graph(n, rp, col, cc, s, t)
    prob = O.Problem.from_graph(g)
    x = rng.random(n)
    x[:nt:3] = 0.5                                    # ties
    x[s], x[t] = 1.0, 0.0
    with solver(P, g) as s_:
        s_.set_x(x)
        side, value, tau = s_.cut()
        info = s_.initial()
        x0g = s_.get_x()
    check_cut(prob, x, side, value, tau)
    x0, _ = O.wls_step(prob, O.initial_conductance(prob))
    assert np.max(np.abs(x0g - x0)) <= XTOL


def test_terminals_anywhere_and_duplicates(P):
    """s and t in the middle of the numbering, parallel entries, unsorted rows."""
    g = gen.random_graph(15, 0.3, 21, st_edge=True)
    perm = np.random.default_rng(1).permutation(g.n)
    gp = gen.permute_graph(g, perm)
    # split every edge capacity into two parallel entries and reverse row order
    rows = np.repeat(np.arange(gp.n), np.diff(gp.row_ptr))
    m = rows < gp.col
    u, v, c = rows[m], gp.col[m].astype(np.int64), gp.c[m]
    rp, col, cc = gen.csr_from_edges(gp.n, np.r_[u, u], np.r_[v, v], np.r_[0.25 * c, 0.75 * c])
    for r in range(gp.n):
        col[rp[r]:rp[r + 1]] = col[rp[r]:rp[r + 1]][::-1].copy()
        cc[rp[r]:rp[r + 1]] = cc[rp[r]:rp[r + 1]][::-1].copy()
    gd = gen.Graph(gp.n, rp, col, cc, gp.s, gp.t)
    prob = O.Problem.from_graph(gd)
    xs, _ = O.irls(prob, 10)
    with solver(P, gd) as s:
        s.solve(10, O.eps_schedule(10))
        x = s.get_x()
        side, value, tau = s.cut()
    assert np.max(np.abs(x - xs[-1])) <= XTOL
    check_cut(prob, xs[-1], side, value, tau)


def test_host_reduction_paths_give_identical_solves(P):
    """The input reduction on a grid large enough to run in parallel: rows that
    are already sorted (copied as they are) and rows with split, reversed
    entries (sorted and merged), a terminal row in order and one reversed --
    the same reduced problem, so bit-identical solves."""
    g = gen.config_graph(1, scale=512)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    new_rp, new_col, new_c = [0], [], []
    for r in range(g.n):
        a, b = g.row_ptr[r], g.row_ptr[r + 1]
        cols, caps = g.col[a:b], g.c[a:b]
        if r % 3 == 0 or r == g.s:
            # c/2 + c/2 is exact: the merged capacity equals the original
            cols = np.repeat(cols, 2)[::-1]
            caps = np.repeat(caps / 2, 2)[::-1]
        new_col.append(cols)
        new_c.append(caps)
        new_rp.append(new_rp[-1] + len(cols))
    gd = gen.Graph(g.n, np.array(new_rp, dtype=np.int64), np.concatenate(new_col).astype(np.int32),
                   np.concatenate(new_c), g.s, g.t)
    eps = O.eps_schedule(3)
    out = []
    for gg in (g, gd):
        with solver(P, gg) as s:
            s.solve(3, eps)
            out.append((s.get_x(), s.cut()[1], s.problem_size()))
    assert out[0][2] == out[1][2]
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


@pytest.mark.parametrize("precision", [0, 1])
def test_live_spmv_timing_counts_every_working_launch(P, precision):
    """time_spmv with host launches: one timed SpMV per PCG iteration (FP32
    inner iterations for mixed), none for launches after the stop test; the
    same x as the graph-launched solve."""
    g = gen.config_graph(1)
    T = 8
    eps = O.eps_schedule(T)
    with solver(P, g, precision=precision) as a, \
            solver(P, g, precision=precision, graph_launch=0, time_spmv=1) as b:
        ia = a.solve(T, eps)
        ib = b.solve(T, eps)
        ms, n = b.spmv_timing()
        assert n == sum(i.pcg_iters for i in ib) and n > 0
        assert ms > 0
        assert b.spmv_timing() == (0.0, 0)       # reset by the first read
        assert np.array_equal(a.get_x(), b.get_x())
        assert [i.pcg_iters for i in ia] == [i.pcg_iters for i in ib]
        assert a.spmv_timing() == (0.0, 0)       # graph launches are not timed


def _hub_graph(n_nt=2800, seed=31):
    """A sparse random graph plus one hub joined to every other non-terminal
    (a row far longer than the rest, as in power-law FlowImprove graphs)."""
    g = gen.random_graph(n_nt, 4.0 / n_nt, seed)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    m = rows < g.col
    u, v, c = rows[m], g.col[m].astype(np.int64), g.c[m]
    hub = 0
    others = np.setdiff1d(np.arange(n_nt), np.r_[hub, v[u == hub], u[v == hub]])
    u = np.r_[u, np.full(others.shape, hub)]
    v = np.r_[v, others]
    c = np.r_[c, np.random.default_rng(seed).uniform(0.01, 0.05, others.shape[0])]
    rp, col, cc = gen.csr_from_edges(g.n, u, v, c)
    return gen.Graph(g.n, rp, col, cc, g.s, g.t)


def test_sweep_with_a_hub_row(P):
    """Rows far longer than the mean are swept by a block each."""
    g = _hub_graph()
    prob = O.Problem.from_graph(g)
    assert np.diff(g.row_ptr).max() > 2000
    xs, _ = O.irls(prob, 8)
    with solver(P, g) as s:
        s.set_x(xs[-1])
        side, value, tau = s.cut()
    check_cut(prob, xs[-1], side, value, tau)
    with P.Batch([g, gen.random_graph(40, 0.1, 12), g], pcg_tol=1e-13) as b:
        b.solve(8, O.eps_schedule(8))
        for i in (0, 2):
            side_b, value_b, tau_b = b.cut(i)
            assert abs(value_b - O.sweep_cut(prob, b.get_x(i))["value"]) <= 1e-9 * value_b


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("form", [0, 1])
def test_steps_with_a_hub_row(P, form, precision):
    """Teacher-forced IRLS steps on CSR with a hub row, FP64 and mixed: the
    reweighting, assembly, scaling, residual and SpMV kernels give the hub a
    block of its own.  The mixed solver runs to 1e-11: on the late steps of this
    graph its FP64 residual, recomputed from x, levels off near 2e-13 (the same
    before the hub blocks), while x already agrees with the oracle to 1e-12."""
    g = _hub_graph()
    prob = O.Problem.from_graph(g)
    T = 8
    eps = O.eps_schedule(T)
    xs, _ = O.irls(prob, T, eps, form=form)
    tol = 1e-13 if precision == 0 else 1e-11
    with solver(P, g, format=2, reweight_form=form, precision=precision, pcg_tol=tol) as s:
        for l in range(1, T + 1):
            s.set_x(xs[l - 1])
            info = s.irls_step(eps[l - 1])
            assert info.status == 0
            assert np.max(np.abs(s.get_x() - xs[l])) <= XTOL, l


def test_one_vertex_and_no_source_edges(P):
    """n = 3 (s-v-t) closed form; and b = 0 (no s edges) gives x = 0."""
    rp, col, c = gen.csr_from_edges(3, [0, 1], [1, 2], [3.0, 1.0])
    g = gen.Graph(3, rp, col, c, 0, 2)
    with solver(P, g) as s:
        s.initial()
        assert abs(s.get_x()[1] - 0.75) < 1e-15
        side, value, tau = s.cut()
        assert value == 1.0 and list(side) == [1, 1, 0]
    rp, col, c = gen.csr_from_edges(4, [0, 1, 2], [1, 2, 3], [1.0, 1.0, 1.0])
    with solver(P, gen.Graph(4, rp, col, c, 3, 0)) as s:   # s and t swapped on a path
        s.initial()
        x = s.get_x()
        assert abs(x[2] - 2.0 / 3.0) < 1e-15 and abs(x[1] - 1.0 / 3.0) < 1e-15
    rp, col, c = gen.csr_from_edges(4, [1, 1, 2], [2, 3, 3], [1.0, 1.0, 1.0])
    g = gen.Graph(4, rp, col, c, 0, 3)                 # s = 0 isolated: b = 0
    with solver(P, g) as s:
        info = s.initial()
        x = s.get_x()
        assert np.all(x[[1, 2]] == 0.0) and info.status == 0
        info = s.irls_step(0.1)
        assert np.all(s.get_x()[[1, 2]] == 0.0)


def test_iteration_cap_and_bad_calls(P):
    from paper_1501_03105_gb300 import binding as B
    g = gen.config_graph(1, scale=24)
    with P.Solver(g, pcg_tol=1e-14, pcg_max_iter=2) as s:
        info = s.initial()
        assert info.status == B.ENOCONV and info.pcg_iters == 2
        assert np.all(np.isfinite(s.get_x()))
        with pytest.raises(B.PirmcutError) as e:
            s.irls_step(-1.0)
        assert e.value.status == B.EINVAL
    with P.Solver(g) as s:
        with pytest.raises(B.PirmcutError) as e:
            s.irls_step(0.1)                           # x not set yet
        assert e.value.status == B.EINVAL
        with pytest.raises(B.PirmcutError):
            s.cut()


def test_deterministic(P):
    g = gen.config_graph(1)
    eps = O.eps_schedule(30)
    outs = []
    for _ in range(2):
        with P.Solver(g) as s:
            infos = s.solve(30, eps)
            outs.append((s.get_x(), [i.pcg_iters for i in infos], s.cut()[1]))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1] and outs[0][2] == outs[1][2]


def test_update_weights_matches_fresh_context(P):
    """A sequence of related problems (Section 6): same structure, new c."""
    g = gen.config_graph(5, scale=12)
    g2 = gen.perturb_capacities(g, seed=9, sigma=0.05)
    eps = O.eps_schedule(10)
    with P.Solver(g) as s:
        s.solve(10, eps)
        s.update_weights(g2.c)
        s.solve(10, eps)
        xa = s.get_x()
        ca = s.cut()[1]
    with P.Solver(g2) as s:
        s.solve(10, eps)
        xb = s.get_x()
        cb = s.cut()[1]
    assert np.array_equal(xa, xb) and ca == cb
    prob = O.Problem.from_graph(g2)
    xs, _ = O.irls(prob, 10, eps)
    assert np.max(np.abs(xa - xs[-1])) <= XTOL


def test_device_buffers(P):
    """Inputs and outputs in CUDA memory (torch tensors)."""
    import torch
    g = gen.config_graph(1, scale=20)
    prob = O.Problem.from_graph(g)
    dev = torch.device("cuda")
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    c = torch.from_numpy(g.c).to(dev)
    h = P.pirmcut_create(g.n, rp, col, c, g.s, g.t, P.pirmcut_default_options(pcg_tol=1e-13))
    try:
        P.pirmcut_solve(h, 5, O.eps_schedule(5))
        xd = torch.empty(g.n, dtype=torch.float64, device=dev)
        P.pirmcut_get_x(h, xd)
        sd = torch.empty(g.n, dtype=torch.uint8, device=dev)
        _, value, tau = P.pirmcut_cut(h, sd)
        torch.cuda.synchronize()
        P.pirmcut_set_x(h, xd)
    finally:
        P.pirmcut_destroy(h)
    xs, _ = O.irls(prob, 5)
    assert np.max(np.abs(xd.cpu().numpy() - xs[-1])) <= XTOL
    check_cut(prob, xs[-1], sd.cpu().numpy(), value, tau)


def test_track_cut_records_each_step(P):
    g = gen.config_graph(1, scale=24)
    prob = O.Problem.from_graph(g)
    eps = O.eps_schedule(8)
    xs, _ = O.irls(prob, 8, eps)
    with P.Solver(g, track_cut=1, pcg_tol=1e-13) as s:
        infos = s.solve(8, eps)
    for l, info in enumerate(infos):
        ref = O.sweep_cut(prob, xs[l])
        assert abs(info.cut_value - ref["value"]) <= CUT_RTOL * ref["value"]


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("make", [lambda: gen.config_graph(1), lambda: gen.config_graph(3, scale=9)],
                         ids=["grid64", "vol9"])
def test_fused_reweight_assembly_is_the_same_computation(P, make, form):
    """options.fuse_reweight forms each row's conductances inside the
    assembly pass (Eq. define-reweight-vector, Eq. reweighted-laplacian; the
    lower edges formed again from the same operands): every iterate,
    iteration count, step statistic and the cut equal the separate passes'
    bit for bit, with graph and host launches; and x against the oracle."""
    g = make()
    T = 8
    eps = O.eps_schedule(T)
    runs = []
    for fuse in (0, 1):
        for launch in (1, 0):
            with solver(P, g, format=1, reweight_form=form, step_stats=1, fuse_reweight=fuse,
                        graph_launch=launch) as s:
                assert s.problem_size()[2] == 1
                infos = s.solve(T, eps)
                side, value, tau = s.cut()
                runs.append((s.get_x(), [(i.pcg_iters, i.rel_residual, i.objective, i.flow_value)
                                         for i in infos], value, tau))
    x0, st0, v0, t0 = runs[0]
    for x, st, v, t in runs[1:]:
        assert np.array_equal(x, x0) and st == st0 and v == v0 and t == t0
    prob = O.Problem.from_graph(g)
    xo, _ = O.irls(prob, T, eps, form=form)
    assert np.max(np.abs(x0 - xo[-1])) <= 1e-9


@pytest.mark.parametrize("fmt", [0, 2])
def test_stream_launch_matches_graph_launch(P, fmt):
    """The same kernels launched from the host (graph_launch = 0) give
    bit-identical iterates, iteration counts and cut."""
    g = gen.config_graph(1, scale=40)
    eps = O.eps_schedule(12)
    out = []
    for mode in (1, 0):
        with P.Solver(g, format=fmt, graph_launch=mode) as s:
            infos = s.solve(12, eps)
            out.append((s.get_x(), [i.pcg_iters for i in infos], s.cut()[1]))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]


# ---------------------------------------------------------------------------
# mixed precision: FP32 inner PCG, FP64 refinement to the same FP64 criterion
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("fmt", [0, 2])
def test_mixed_teacher_forced_steps_grid64(P, fmt):
    """Every IRLS step of the 64x64 workload with the mixed-precision solver:
    the FP64 residual test at 1e-13 makes x agree with the exact WLS solution
    to the same 1e-9 bar as the FP64 path."""
    g = gen.config_graph(1)
    prob = O.Problem.from_graph(g)
    T = 50
    eps = O.eps_schedule(T)
    xs, _ = O.irls(prob, T, eps)
    with solver(P, g, format=fmt, precision=1) as s:
        for l in range(1, T + 1):
            s.set_x(xs[l - 1])
            info = s.irls_step(eps[l - 1])
            assert info.status == 0, (l, info.status)
            assert info.rel_residual <= 1e-13
            assert np.max(np.abs(s.get_x() - xs[l])) <= XTOL, l


@pytest.mark.parametrize("name,make", GRAPHS)
def test_mixed_x0_and_steps_small(P, name, make):
    g = make()
    prob = O.Problem.from_graph(g)
    T = 12
    eps = O.eps_schedule(T)
    xs, _ = O.irls(prob, T, eps)
    with solver(P, g, precision=1) as s:
        info = s.initial()
        assert info.status == 0 and info.refinements >= 1
        assert np.max(np.abs(s.get_x() - xs[0])) <= XTOL
        for l in range(1, T + 1):
            s.set_x(xs[l - 1])
            s.irls_step(eps[l - 1])
            assert np.max(np.abs(s.get_x() - xs[l])) <= XTOL, l


def test_mixed_free_running_matches_fp64(P):
    """Algorithm 1 on grid64 at the workload's tolerance (1e-10): the mixed
    solver's cut equals the oracle's and its iterate stays within 1e-6 of the
    FP64 GPU path's."""
    g = gen.config_graph(1)
    prob = O.Problem.from_graph(g)
    T = 50
    eps = O.eps_schedule(T)
    xs, _ = O.irls(prob, T, eps)
    with P.Solver(g, pcg_tol=1e-10) as s:
        s.solve(T, eps)
        x64 = s.get_x()
    with P.Solver(g, pcg_tol=1e-10, precision=1) as s:
        infos = s.solve(T, eps)
        assert all(i.status == 0 and i.rel_residual <= 1e-10 for i in infos)
        xm = s.get_x()
        side, value, tau = s.cut()
    assert np.max(np.abs(xm - x64)) <= 1e-6
    check_cut(prob, xs[-1], side, value, tau)


@pytest.mark.parametrize("fmt", [0, 2])
def test_mixed_stream_matches_graph(P, fmt):
    g = gen.config_graph(1, scale=40)
    eps = O.eps_schedule(12)
    out = []
    for mode in (1, 0):
        with P.Solver(g, format=fmt, graph_launch=mode, precision=1) as s:
            infos = s.solve(12, eps)
            out.append((s.get_x(), [(i.pcg_iters, i.refinements) for i in infos]))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


# ---------------------------------------------------------------------------
# two-level rounding (Section 3.3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("fmt", [0, 2])
@pytest.mark.parametrize("name,make", GRAPHS)
def test_two_level_rounding_matches_oracle(P, name, make, fmt):
    g = make()
    prob = O.Problem.from_graph(g)
    xs, _ = O.irls(prob, 6)
    for l in (0, 3, 6):
        ref = O.two_level_rounding(prob, xs[l])
        with solver(P, g, format=fmt) as s:
            s.set_x(xs[l])
            side, value, gam, nc = s.cut_two_level()
        assert abs(gam[0] - ref["gamma0"]) <= 1e-12 and abs(gam[1] - ref["gamma1"]) <= 1e-12
        assert nc == ref["coarse_vertices"]
        assert abs(value - ref["value"]) <= CUT_RTOL * ref["value"], (name, l)
        assert abs(O.cut_value(prob, side.astype(bool)) - value) <= 1e-12 * value
        assert side[g.s] == 1 and side[g.t] == 0


def test_two_level_on_grid64_after_irls(P):
    """After the full IRLS run the coarse graph is tiny and the two-level cut
    is the exact min cut (the Edmonds-Karp value of the oracle)."""
    g = gen.config_graph(1)
    prob = O.Problem.from_graph(g)
    mu_star, _ = O.max_flow_min_cut(prob)
    with P.Solver(g) as s:
        s.solve(50, O.eps_schedule(50))
        side, value, gam, nc = s.cut_two_level()
        _, sweep_value, _ = s.cut()
    assert nc < 100
    assert abs(value - mu_star) <= 1e-9 * mu_star
    assert value <= sweep_value * (1 + 1e-12)
