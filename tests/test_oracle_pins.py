"""Pins for the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against a closed form, a hand-worked example, an
invariant the paper proves, or an independent exact algorithm, so that a
dropped term, a wrong sign or a wrong index in the oracle fails at least one
of them (``test_oracle_mutations.py`` plants such mistakes to show it).
"""
import json
import os

import numpy as np
import pytest

import gen
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def problem_from_edges(n, s, t, edges):
    u = [e[0] for e in edges]
    v = [e[1] for e in edges]
    c = [e[2] for e in edges]
    rp, col, cc = gen.csr_from_edges(n, u, v, c)
    return O.Problem(n, rp, col, cc, s, t)


def svt(a, b):
    """s - v - t path with capacities a (s-v) and b (v-t); s=0, v=1, t=2."""
    return problem_from_edges(3, 0, 2, [(0, 1, a), (1, 2, b)])


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("a,b", [(3.0, 1.0), (0.25, 2.0), (1.0, 1.0)])
def test_x0_single_vertex_divider(a, b):
    """x^(0) with g = c on s-v-t: (a + b) v = a, so v = a / (a + b)."""
    P = svt(a, b)
    x, _ = O.wls_step(P, O.initial_conductance(P))
    assert x[0] == 1.0 and x[2] == 0.0
    assert abs(x[1] - a / (a + b)) < 1e-15


def test_x0_series_chain_voltage_divider():
    """Chain s - v1 - ... - vk - t: conductances in series.  The voltage at v_i
    is the share of the total resistance sum_j 1/c_j lying between v_i and t."""
    caps = [2.0, 0.5, 3.0, 1.25, 4.0]          # s-v1, v1-v2, v2-v3, v3-v4, v4-t
    k = len(caps) - 1
    s, t = 0, k + 1
    edges = [(i, i + 1, caps[i]) for i in range(k + 1)]
    P = problem_from_edges(k + 2, s, t, edges)
    x, _ = O.wls_step(P, O.initial_conductance(P))
    R = [1.0 / c for c in caps]
    for i in range(1, k + 1):
        expect = sum(R[i:]) / sum(R)
        assert abs(x[i] - expect) < 1e-14


@pytest.mark.parametrize("form", [O.WEIGHTED_L1, O.PAPER])
@pytest.mark.parametrize("a,b,v,eps", [(3.0, 1.0, 0.75, 0.1), (0.5, 2.0, 0.2, 1e-3),
                                       (1.5, 1.4, 0.5, 1e-6)])
def test_one_irls_step_closed_form(form, a, b, v, eps):
    """One reweight + WLS on s-v-t starting from x_v = v (Step 1 and Step 2).

    The s-v edge has |Bx| = 1 - v, the v-t edge |Bx| = v.  The new voltage is
    the divider g_a / (g_a + g_b) of the reweighted conductances:
    weighted-l1 g = c / sqrt(d^2 + eps^2); paper g = c^2 / sqrt(c^2 d^2 + eps^2).
    """
    P = svt(a, b)
    x = np.array([1.0, v, 0.0])
    if form == O.WEIGHTED_L1:
        ga = a / np.sqrt((1 - v) ** 2 + eps ** 2)
        gb = b / np.sqrt(v ** 2 + eps ** 2)
    else:
        ga = a * a / np.sqrt(a * a * (1 - v) ** 2 + eps ** 2)
        gb = b * b / np.sqrt(b * b * v * v + eps ** 2)
    g = O.reweight(P, x, eps, form)
    x1, _ = O.wls_step(P, g)
    assert abs(x1[1] - ga / (ga + gb)) < 1e-14


@pytest.mark.parametrize("a,b", [(3.0, 1.0), (1.0, 3.0), (1.1, 1.0)])
def test_irls_polarises_towards_min_cut(a, b):
    """On s-v-t the min cut removes the smaller edge; IRLS drives x_v to 1
    when a > b (v joins s) and to 0 when a < b, monotonically.  Near the limit
    (distance d to it, eps << d) one step maps d to about d * min(a,b)/max(a,b)
    (g_a ~ a/(1-v), g_b ~ b/v, 1 - v' = g_b/(g_a+g_b)), until d reaches the
    order of eps."""
    P = svt(a, b)
    xs, _ = O.irls(P, 40)
    v = np.array([x[1] for x in xs])
    dist = 1.0 - v if a > b else v
    assert np.all(np.diff(dist) <= 1e-15)
    ratio = min(a, b) / max(a, b)
    assert dist[-1] <= max(ratio ** 30, 1e-5)


@pytest.mark.parametrize("v,eps", [(0.3, 0.1), (0.9, 1e-3), (0.5, 0.0)])
def test_smoothed_objective_closed_form(v, eps):
    """S_eps on s-v-t at x_v = v (Eq. l1-min-smooth-version):
    paper sum_e sqrt((c_e d_e)^2 + eps^2) = sqrt((a(1-v))^2 + eps^2) + sqrt((b v)^2 + eps^2);
    weighted-l1 sum_e c_e sqrt(d_e^2 + eps^2) = a sqrt((1-v)^2 + eps^2) + b sqrt(v^2 + eps^2).
    At eps = 0 both equal the l1 objective ||C B x||_1 (Eq. l1-min)."""
    a, b = 3.0, 0.5
    P = svt(a, b)
    x = np.array([1.0, v, 0.0])
    paper = np.sqrt((a * (1 - v)) ** 2 + eps ** 2) + np.sqrt((b * v) ** 2 + eps ** 2)
    ns = a * np.sqrt((1 - v) ** 2 + eps ** 2) + b * np.sqrt(v ** 2 + eps ** 2)
    assert abs(O.smoothed_objective(P, x, eps, O.PAPER) - paper) < 1e-14
    assert abs(O.smoothed_objective(P, x, eps, O.WEIGHTED_L1) - ns) < 1e-14
    if eps == 0.0:
        assert abs(ns - (a * (1 - v) + b * v)) < 1e-15


def test_reduced_system_hand_example():
    """Two non-terminals u=1, v=2 with s=0, t=3 and g = c:
    s-u 1, u-v 2, v-t 3, s-v 0.5, u-t 0.25, s-t 0.7.
    L~ = [[1 + 2 + 0.25, -2], [-2, 2 + 3 + 0.5]] and b = [1, 0.5]
    (Eq. reduced-laplacian-system; the s-t edge drops out)."""
    P = problem_from_edges(4, 0, 3, [(0, 1, 1.0), (1, 2, 2.0), (2, 3, 3.0), (0, 2, 0.5),
                                     (1, 3, 0.25), (0, 3, 0.7)])
    L = O.laplacian(P, O.initial_conductance(P))
    Lt, b = O.reduced_system(P, L)
    assert np.array_equal(Lt.toarray(), np.array([[3.25, -2.0], [-2.0, 5.5]]))
    assert np.array_equal(b, np.array([1.0, 0.5]))
    # Cramer's rule on the 2x2 system
    det = 3.25 * 5.5 - 4.0
    u = (1.0 * 5.5 + 2.0 * 0.5) / det
    v = (3.25 * 0.5 + 2.0 * 1.0) / det
    x, _ = O.wls_step(P, O.initial_conductance(P))
    assert abs(x[1] - u) < 1e-15 and abs(x[2] - v) < 1e-15


# ---------------------------------------------------------------------------
# invariants the paper proves
# ---------------------------------------------------------------------------

def random_problems():
    out = []
    for seed in range(6):
        g = gen.random_graph(9 + seed, 0.35, seed, zero_frac=0.2, st_edge=(seed % 2 == 0))
        out.append(O.Problem.from_graph(g))
    return out


@pytest.mark.parametrize("form", [O.WEIGHTED_L1, O.PAPER])
def test_laplacian_structure(form):
    """L is symmetric with zero row sums (it is a Laplacian); L~ keeps the
    off-diagonals, its row sums equal the terminal conductances, and b >= 0
    (Section 2.1, proof of Prop. interval-constraint-satisfaction)."""
    for P in random_problems():
        rng = np.random.default_rng(P.n)
        x = rng.random(P.n)
        x[P.s], x[P.t] = 1.0, 0.0
        g = O.reweight(P, x, 1e-2, form)
        L = O.laplacian(P, g).toarray()
        assert np.allclose(L, L.T, rtol=0, atol=1e-14)
        assert np.max(np.abs(L.sum(axis=1))) < 1e-12 * np.max(np.abs(L))
        Lt, b = O.reduced_system(P, O.laplacian(P, g))
        Lt = Lt.toarray()
        nt = P.nonterminals
        assert np.array_equal(Lt, L[np.ix_(nt, nt)])
        gs = np.zeros(P.n)
        gt = np.zeros(P.n)
        for e in range(P.m):
            u, v = P.eu[e], P.ev[e]
            if P.s in (u, v) and P.t not in (u, v):
                gs[v if u == P.s else u] += g[e]
            if P.t in (u, v) and P.s not in (u, v):
                gt[v if u == P.t else u] += g[e]
        assert np.allclose(Lt.sum(axis=1), gs[nt] + gt[nt], rtol=1e-13, atol=1e-13)
        assert np.array_equal(b, gs[nt])
        assert np.all(b >= 0)


def test_maximum_principle_every_step():
    """0 <= x^(l) <= 1 for every IRLS iterate (Prop. interval-constraint-satisfaction)."""
    for P in random_problems():
        for form in (O.WEIGHTED_L1, O.PAPER):
            xs, _ = O.irls(P, 25, form=form)
            for x in xs:
                assert x.min() >= -1e-12 and x.max() <= 1 + 1e-12


def test_electrical_flow_conservation_and_value():
    """The WLS solution is an electrical flow: (L x)_v = 0 at non-terminals and
    the flow value (L x)_s = -(L x)_t = x^T L x (Prop. wls-equal-electrical-flow)."""
    for P in random_problems():
        xs, _ = O.irls(P, 8)
        for l in (0, 3, 8):
            g = O.initial_conductance(P) if l == 0 else O.reweight(P, xs[l - 1], O.eps_schedule(8)[l - 1])
            L = O.laplacian(P, g)
            y = L @ xs[l]
            scale = np.abs(L).max()
            assert np.max(np.abs(y[P.nonterminals])) < 1e-10 * scale
            mu = O.flow_value(P, xs[l], g)
            assert abs(y[P.s] - mu) < 1e-10 * max(1.0, mu)
            assert abs(y[P.t] + mu) < 1e-10 * max(1.0, mu)


@pytest.mark.parametrize("form", [O.WEIGHTED_L1, O.PAPER])
def test_monotone_majorise_minimise(form):
    """Each IRLS step minimises a majoriser of the smoothed objective, so
    S_eps_l(x^(l)) <= S_eps_l(x^(l-1)) (Section 2.2, Eq. l1-min-smooth-version),
    and S is increasing in eps, so with a non-increasing schedule the sequence
    S_eps_l(x^(l)) never increases."""
    for P in random_problems():
        eps = O.eps_schedule(20)
        xs, _ = O.irls(P, 20, eps, form=form)
        prev = None
        for l in range(1, 21):
            a = O.smoothed_objective(P, xs[l], eps[l - 1], form)
            b = O.smoothed_objective(P, xs[l - 1], eps[l - 1], form)
            assert a <= b + 1e-12 * b
            if prev is not None:
                assert a <= prev + 1e-12 * prev
            prev = a


def test_forms_coincide_for_unit_capacities():
    """With c = 1 the weighted-l1 and the paper reweighting are the same map."""
    g = gen.random_graph(12, 0.3, 7)
    g.c[:] = 1.0
    P = O.Problem.from_graph(g)
    xa, _ = O.irls(P, 10, form=O.WEIGHTED_L1)
    xb, _ = O.irls(P, 10, form=O.PAPER)
    for a, b in zip(xa, xb):
        assert np.max(np.abs(a - b)) < 1e-12


# ---------------------------------------------------------------------------
# exact references and cuts
# ---------------------------------------------------------------------------

def load_hand():
    with open(os.path.join(HERE, "golden", "hand_graphs.json")) as f:
        d = json.load(f)
    return {k: v for k, v in d.items() if not k.startswith("_")}


@pytest.mark.parametrize("name", sorted(load_hand()))
def test_exact_references_on_hand_examples(name):
    h = load_hand()[name]
    P = problem_from_edges(h["n"], h["s"], h["t"], h["edges"])
    want_side = np.zeros(h["n"], dtype=bool)
    want_side[h["source_side"]] = True
    assert abs(O.cut_value(P, want_side) - h["min_cut"]) < 1e-14
    val, mins = O.brute_force_min_cut(P)
    assert abs(val - h["min_cut"]) < 1e-14
    assert len(mins) == 1 and np.array_equal(mins[0], want_side)
    flow, side = O.max_flow_min_cut(P)
    assert abs(flow - h["min_cut"]) < 1e-12
    assert np.array_equal(side, want_side)


@pytest.mark.parametrize("seed", range(8))
def test_brute_force_equals_max_flow(seed):
    """Max-flow value == min-cut value (LP duality), two independent routes."""
    g = gen.random_graph(10 + seed % 5, 0.3, 100 + seed, zero_frac=0.15, st_edge=seed % 3 == 0)
    P = O.Problem.from_graph(g)
    val, mins = O.brute_force_min_cut(P)
    flow, side = O.max_flow_min_cut(P)
    assert abs(flow - val) <= 1e-12 * val
    assert abs(O.cut_value(P, side) - val) <= 1e-12 * val
    assert any(np.array_equal(side, m) for m in mins)


def test_sweep_cut_prefix_sums_match_definition():
    """The prefix-sum sweep picks the same prefix and value as evaluating the
    cut definition for every candidate prefix."""
    for seed in range(10):
        g = gen.random_graph(14, 0.3, 200 + seed, st_edge=seed % 2 == 0)
        P = O.Problem.from_graph(g)
        xs, _ = O.irls(P, 5)
        for x in (xs[0], xs[-1]):
            a = O.sweep_cut(P, x)
            b = O.sweep_cut_by_definition(P, x)
            assert a["k"] == b["k"]
            assert abs(a["value"] - b["value"]) <= 1e-13 * b["value"]
            assert abs(a["prefix_value"] - b["value"]) <= 1e-12 * b["value"]
            assert np.array_equal(a["side"], b["side"])


def test_sweep_cut_ties_and_candidates():
    """Tied x values never split: with x = (s=1, 0.5, 0.5, t=0) on a path
    s - a - b - t, the only candidates are {s} and {s, a, b}."""
    P = problem_from_edges(4, 0, 3, [(0, 1, 3.0), (1, 2, 0.1), (2, 3, 2.0)])
    x = np.array([1.0, 0.5, 0.5, 0.0])
    r = O.sweep_cut(P, x)
    assert r["k"] == 2 and r["value"] == 2.0 and abs(r["tau"] - 0.25) < 1e-15
    d = O.sweep_cut_by_definition(P, x)
    assert d["k"] == 2 and d["value"] == 2.0


def test_sweep_cut_order_hand_example():
    """Path s - a - b - t (capacities 5, 1, 5) with x = (1, 0.8, 0.2, 0): the
    sweep visits a before b; prefixes {s}: 5, {s,a}: 1, {s,a,b}: 5, so the
    sweep returns S = {s, a}, value 1, tau = (0.8 + 0.2) / 2."""
    P = problem_from_edges(4, 0, 3, [(0, 1, 5.0), (1, 2, 1.0), (2, 3, 5.0)])
    x = np.array([1.0, 0.8, 0.2, 0.0])
    for r in (O.sweep_cut(P, x), O.sweep_cut_by_definition(P, x)):
        assert r["k"] == 1 and r["value"] == 1.0 and abs(r["tau"] - 0.5) < 1e-15
        assert list(np.nonzero(r["side"])[0]) == [0, 1]


def curated_unique_gap_graphs():
    """Random graphs whose min cut is unique and at least 10% below the runner-up."""
    out = []
    seed = 300
    while len(out) < 6:
        g = gen.random_graph(12, 0.3, seed)
        seed += 1
        P = O.Problem.from_graph(g)
        val, mins = O.brute_force_min_cut(P, rel_tol=0.1)
        if len(mins) == 1:
            out.append((P, val))
    return out


def test_irls_sweep_cut_finds_unique_min_cut():
    """On instances with a unique, well-separated minimum the IRLS + sweep cut
    returns the exact min cut (delta = 0)."""
    for P, val in curated_unique_gap_graphs():
        xs, _ = O.irls(P, 50)
        r = O.sweep_cut(P, xs[-1])
        assert abs(r["value"] - val) <= 1e-12 * val


def test_cheeger_type_bounds():
    """Theorem cheeger-type-inequality with C = 2 sum c, lambda_2 = 2 mu_0 / C
    (mu_0 = x0^T L x0 with g = c) and phi = mu*/C gives mu_0 <= mu* and
    mu*^2 <= 4 C mu_0."""
    for seed in range(8):
        g = gen.random_graph(11, 0.35, 400 + seed, st_edge=seed % 2 == 0)
        P = O.Problem.from_graph(g)
        mu_star, _ = O.brute_force_min_cut(P)
        g0 = O.initial_conductance(P)
        x0, _ = O.wls_step(P, g0)
        mu0 = O.flow_value(P, x0, g0)
        Ctot = 2.0 * P.cap.sum()
        assert mu0 <= mu_star * (1 + 1e-12)
        assert mu_star ** 2 <= 4.0 * Ctot * mu0 * (1 + 1e-12)


def test_pcg_matches_direct_solve():
    """Jacobi-PCG to 1e-13 agrees with the sparse direct solve."""
    g = gen.config_graph(1, scale=24)
    P = O.Problem.from_graph(g)
    xs, _ = O.irls(P, 6)
    for l in range(1, 7):
        gl = O.reweight(P, xs[l - 1], O.eps_schedule(6)[l - 1])
        Lt, b = O.reduced_system(P, O.laplacian(P, gl))
        vd = O.solve_direct(Lt, b)
        vp, it, rel = O.pcg_jacobi(Lt, b, xs[l - 1][P.nonterminals], tol=1e-13, maxit=100000)
        assert rel <= 1e-13
        assert np.max(np.abs(vp - vd)) < 1e-10


# ---------------------------------------------------------------------------
# invariances
# ---------------------------------------------------------------------------

def test_vertex_permutation_invariance():
    g = gen.random_graph(13, 0.3, 501, st_edge=True)
    P = O.Problem.from_graph(g)
    perm = np.random.default_rng(5).permutation(g.n)
    gp = gen.permute_graph(g, perm)
    Pp = O.Problem.from_graph(gp)
    xs, _ = O.irls(P, 15)
    xps, _ = O.irls(Pp, 15)
    for a, b in zip(xs, xps):
        assert np.max(np.abs(a - b[perm])) < 1e-11
    assert abs(O.sweep_cut(P, xs[-1])["value"] - O.sweep_cut(Pp, xps[-1])["value"]) < 1e-12


def test_capacity_scaling_invariance():
    """Weighted-l1 form: c -> alpha c leaves every iterate unchanged.
    Paper form: (c, eps) -> (alpha c, alpha eps) leaves it unchanged."""
    g = gen.random_graph(13, 0.3, 502)
    P = O.Problem.from_graph(g)
    g2 = gen.Graph(g.n, g.row_ptr, g.col, 3.7 * g.c, g.s, g.t)
    P2 = O.Problem.from_graph(g2)
    eps = O.eps_schedule(12)
    xa, _ = O.irls(P, 12, eps)
    xb, _ = O.irls(P2, 12, eps)
    for a, b in zip(xa, xb):
        assert np.max(np.abs(a - b)) < 1e-11
    xa, _ = O.irls(P, 12, eps, form=O.PAPER)
    xb, _ = O.irls(P2, 12, [3.7 * e for e in eps], form=O.PAPER)
    for a, b in zip(xa, xb):
        assert np.max(np.abs(a - b)) < 1e-11


def test_input_validation():
    with pytest.raises(ValueError):
        problem_from_edges(3, 0, 0, [(0, 1, 1.0), (1, 2, 1.0)])          # s == t
    with pytest.raises(ValueError):
        problem_from_edges(3, 0, 2, [(0, 1, -1.0), (1, 2, 1.0)])         # negative capacity
    with pytest.raises(ValueError):
        problem_from_edges(4, 0, 2, [(0, 1, 1.0), (1, 2, 1.0)])          # vertex 3 isolated
    with pytest.raises(ValueError):
        problem_from_edges(3, 0, 2, [(0, 1, float("nan")), (1, 2, 1.0)])  # NaN
    rp, col, c = gen.csr_from_edges(3, [0, 1], [1, 2], [1.0, 2.0])
    c2 = c.copy()
    c2[0] = 5.0                                                          # asymmetric
    with pytest.raises(ValueError):
        O.Problem(3, rp, col, c2, 0, 2)


# ---------------------------------------------------------------------------
# two-level rounding (Section 3.3)
# ---------------------------------------------------------------------------

def test_kmeans_1d_closed_forms():
    """Symmetric clusters around 0.1 and 0.9 stay put; an outlier moves only
    its own centre: [0, 0, 0.3, 1] from (0.1, 0.9) -> c0 = mean(0, 0, 0.3) = 0.1,
    c1 = 1; a tie at the midpoint goes to the lower centre."""
    c0, c1 = O.kmeans_1d(np.array([0.0, 0.1, 0.2, 0.8, 0.9, 1.0]))
    assert abs(c0 - 0.1) < 1e-15 and abs(c1 - 0.9) < 1e-15
    c0, c1 = O.kmeans_1d(np.array([0.0, 0.0, 0.3, 1.0]))
    assert abs(c0 - 0.1) < 1e-15 and c1 == 1.0
    c0, c1 = O.kmeans_1d(np.array([0.0, 0.5, 1.0]))
    assert abs(c0 - 0.25) < 1e-15 and c1 == 1.0


def _constrained_min_cut(P, lab):
    """Brute force over the free vertices (lab == 2) with lab 1 on the source
    side and lab 0 on the sink side."""
    free = np.nonzero(lab == 2)[0]
    best = np.inf
    for code in range(1 << free.shape[0]):
        side = lab == 1
        side[free] = ((code >> np.arange(free.shape[0])) & 1).astype(bool)
        best = min(best, O.cut_value(P, side))
    return best


def test_two_level_equals_constrained_brute_force():
    """The coarse min cut is the least cut of G among the cuts that keep S1 on
    the source side and S0 on the sink side (contraction preserves those cut
    values; the max-flow is exact)."""
    for seed in range(6):
        g = gen.random_graph(12, 0.3, 600 + seed, st_edge=seed % 2 == 0)
        P = O.Problem.from_graph(g)
        xs, _ = O.irls(P, 6)
        x = xs[2]
        r = O.two_level_rounding(P, x)
        lab = np.full(P.n, 2)
        lab[x <= r["gamma0"]] = 0
        lab[x >= r["gamma1"]] = 1
        lab[P.s], lab[P.t] = 1, 0
        assert (lab == 2).sum() <= 14
        assert abs(r["value"] - _constrained_min_cut(P, lab)) <= 1e-12 * r["value"]
        assert r["coarse_vertices"] == (lab == 2).sum() + 2


def test_two_level_proposition_recovers_min_cut():
    """Proposition (Section 3.3): when S1 lies on the source side and S0 on the
    sink side of some min cut, the coarse min cut induces a min cut of G."""
    hits = 0
    for seed in range(12):
        g = gen.random_graph(11, 0.35, 700 + seed)
        P = O.Problem.from_graph(g)
        mu, mins = O.brute_force_min_cut(P)
        xs, _ = O.irls(P, 30)
        r = O.two_level_rounding(P, xs[-1])
        lab0 = xs[-1] <= r["gamma0"]
        lab1 = xs[-1] >= r["gamma1"]
        if any(np.all(m[lab1]) and not np.any(m[lab0]) for m in mins):
            hits += 1
            assert abs(r["value"] - mu) <= 1e-12 * mu
    assert hits >= 6
