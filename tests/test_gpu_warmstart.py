"""GPU parity of the learned warm start against ``oracle/warmstart.py``.

Bars:
* features: f0-f2, f4, f5 within 2e-6 absolute of the oracle's FP64 values
  (CSR: computed in FP64 and rounded once; DIA: computed in FP32 from
  truncated FP64 inputs, differences formed in FP64, the variance in two
  passes -- a few units of 2^-23 on values of size <= 1 and on logarithms
  / 8), f3 from FP32 logarithms (within 1e-5 absolute);
* inference (tensor cores, BF16 operands, FP32 accumulation): within the
  oracle's bound for that data path (split-BF16 features, BF16 hidden layer);
* line search: alpha and the energy change to relative 1e-9 (1e-7 for the
  change, a quotient of FP64 sums) where the direction is exact on both sides
  (a constant), to relative 1e-5 where it comes from the FP32 network;
* the solve after a learned start: the same 1e-9 bar on x as every step;
* training: after one Adam step from zero moments, each parameter whose oracle
  gradient is clearly signed moved by -lr * sign(gradient).
"""
import numpy as np
import pytest

import gen
import oracle as O
import oracle.warmstart as W

pytestmark = pytest.mark.gpu

XTOL = 1e-9


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


def hub_graph(n_nt=1500, seed=17):
    """A sparse random graph plus one hub joined to every other non-terminal:
    a CSR row longer than max(512, 16 x mean), processed by a block of its own."""
    g = gen.random_graph(n_nt, 4.0 / n_nt, seed)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    m = rows < g.col
    u, v, c = rows[m], g.col[m].astype(np.int64), g.c[m]
    others = np.setdiff1d(np.arange(1, n_nt), np.r_[v[u == 0], u[v == 0]])
    u = np.r_[u, np.zeros(others.shape, dtype=np.int64)]
    v = np.r_[v, others]
    c = np.r_[c, np.random.default_rng(seed).uniform(0.01, 0.05, others.shape[0])]
    rp, col, cc = gen.csr_from_edges(g.n, u, v, c)
    return gen.Graph(g.n, rp, col, cc, g.s, g.t)


GRAPHS = [
    ("grid16", lambda: gen.config_graph(1, scale=16)),
    ("vol8", lambda: gen.config_graph(3, scale=8)),
    ("random40", lambda: gen.random_graph(40, 0.1, 12)),
    ("chunglu", lambda: gen.chung_lu_instance(600, 5)),
    ("hub1500", hub_graph),
]


def reduced(prob, x):
    return x[prob.nonterminals]


def line_search_tolerance(prob, g, v0, d, e):
    """First-order bound on how far alpha and the energy change can move when
    every entry of d may be off by at most e (e >= 0, per node)."""
    Lt, b = O.reduced_system(prob, O.laplacian(prob, g))
    r = b - Lt @ v0
    Ad = Lt @ d
    dr, dad = float(d @ r), float(d @ Ad)
    er, ead = float(e @ np.abs(r)), float(e @ np.abs(Ad))
    ta = (er + 2 * abs(dr / dad) * ead) / dad
    tE = 2 * abs(dr) * er / dad + 2 * dr * dr * ead / dad ** 2
    return ta, tE


FEATURE_ATOL = 2e-6


def jacobi_weights(alpha):
    """Weights whose output is alpha * (f1 - f0): one damped Jacobi step,
    since f1 - f0 = (sum_u g x_u) / d_v - x_v = r_v / d_v.  Two hidden units
    carry the positive and the negative part (relu(f1 - f0), relu(f0 - f1)),
    so that the BF16 hidden layer rounds the difference itself, relatively."""
    w = np.zeros(W.NPARAM, dtype=np.float32)
    W1 = w[W.OFF_W1:W.OFF_B1].reshape(64, 6)
    W1[0, 0], W1[0, 1] = -1.0, 1.0
    W1[1, 0], W1[1, 1] = 1.0, -1.0
    W2 = w[W.OFF_W2:W.OFF_B2].reshape(64, 64)
    W2[0, 0], W2[1, 1] = 1.0, 1.0
    w[W.OFF_W3] = alpha
    w[W.OFF_W3 + 1] = -alpha
    return w


@pytest.mark.parametrize("fmt", [0, 2])
@pytest.mark.parametrize("name,make", GRAPHS)
def test_features_match_oracle(P, name, make, fmt):
    g = make()
    prob = O.Problem.from_graph(g)
    T = 3
    eps = O.eps_schedule(T)
    xs, _ = O.irls(prob, T, eps)
    gprev = O.initial_conductance(prob)
    with P.Solver(g, pcg_tol=1e-13, format=fmt) as s:
        s.initial()
        s.mlp_enable(P.binding.MLP_TRAIN, seed=3)
        s.mlp_configure(0, 1e-3)
        for l in range(1, T + 1):
            s.set_x(xs[l - 1])
            s.irls_step(eps[l - 1])
            gl = O.reweight(prob, xs[l - 1], eps[l - 1])
            ref = W.features(prob, xs[l - 1], gl, gprev, eps[l - 1])
            got = s.mlp_features()
            cols = [0, 1, 2, 4, 5]
            np.testing.assert_allclose(got[:, cols], ref[:, cols], rtol=0, atol=FEATURE_ATOL,
                                       err_msg=f"step {l}")
            np.testing.assert_allclose(got[:, 3], ref[:, 3], rtol=0, atol=1e-5, err_msg=f"step {l}")
            assert np.max(np.abs(s.get_x() - xs[l])) <= XTOL
            gprev = gl


@pytest.mark.parametrize("count", [1, 257, 5000])
def test_inference_within_the_bf16_bound(P, count):
    g = gen.config_graph(1, scale=8)
    rng = np.random.default_rng(count)
    w = rng.normal(0, 0.2, W.NPARAM).astype(np.float32)
    F = rng.normal(0, 1, (count, 6)).astype(np.float32)
    with P.Solver(g) as s:
        s.mlp_enable(P.binding.MLP_PREDICT, seed=1)
        s.mlp_weights(w)
        got = s.mlp_predict(F)
        back = s.mlp_weights()
    assert np.array_equal(back, w)
    out, bound = W.mlp_forward_bf16(w, F)
    assert np.all(np.abs(got.astype(np.float64) - out) <= bound)


def test_inference_device_buffers(P):
    import torch
    g = gen.config_graph(1, scale=8)
    rng = np.random.default_rng(9)
    w = rng.normal(0, 0.2, W.NPARAM).astype(np.float32)
    F = rng.normal(0, 1, (300, 6)).astype(np.float32)
    with P.Solver(g) as s:
        s.mlp_enable(P.binding.MLP_PREDICT, seed=1)
        s.mlp_weights(w)
        dF = torch.from_numpy(F).cuda()
        dd = torch.empty(300, dtype=torch.float32, device="cuda")
        s.mlp_predict(dF, dd)
        got = dd.cpu().numpy()
    out, bound = W.mlp_forward_bf16(w, F)
    assert np.all(np.abs(got.astype(np.float64) - out) <= bound)


@pytest.mark.parametrize("fmt", [0, 2])
def test_untrained_model_is_bit_identical_to_the_plain_start(P, fmt):
    """A fresh model has a zero output layer: d = 0, alpha = 0, and every step
    is bit-identical to the plain warm start."""
    g = gen.config_graph(1)
    T = 10
    eps = O.eps_schedule(T)
    with P.Solver(g, format=fmt) as a, P.Solver(g, format=fmt) as b:
        ia = a.solve(T, eps)
        b.mlp_enable(P.binding.MLP_PREDICT, seed=5)
        ib = b.solve(T, eps)
        assert np.array_equal(a.get_x(), b.get_x())
        assert [i.pcg_iters for i in ia] == [i.pcg_iters for i in ib]
        st = b.mlp_stats()
        assert st.steps == T and st.used == 0 and st.alpha == 0.0


@pytest.mark.parametrize("fmt", [0, 2])
@pytest.mark.parametrize("delta", [-1 / 32, 1 / 64])
@pytest.mark.parametrize("name", ["grid24", "hub1500"])
def test_constant_direction_line_search(P, fmt, delta, name):
    """d = const (only b3 set): the line search is exact on both sides; alpha,
    the energy change, the plain residual and the solution follow the oracle."""
    g = gen.config_graph(1, scale=24) if name == "grid24" else hub_graph()
    prob = O.Problem.from_graph(g)
    T = 6
    eps = O.eps_schedule(T)
    xs, _ = O.irls(prob, T, eps)
    w = np.zeros(W.NPARAM, dtype=np.float32)
    w[W.OFF_B3] = delta
    with P.Solver(g, pcg_tol=1e-13, format=fmt) as s:
        s.initial()
        s.mlp_enable(P.binding.MLP_PREDICT, seed=1)
        s.mlp_weights(w)
        for l in range(1, T + 1):
            s.set_x(xs[l - 1])
            s.irls_step(eps[l - 1])
            gl = O.reweight(prob, xs[l - 1], eps[l - 1])
            v0 = reduced(prob, xs[l - 1])
            alpha, dE = W.line_search(prob, gl, v0, np.full(v0.shape, delta))
            st = s.mlp_stats()
            assert st.alpha == pytest.approx(alpha, rel=1e-9)
            assert st.energy_change == pytest.approx(dE, rel=1e-7)
            assert st.energy_change <= 0.0
            assert st.res_plain == pytest.approx(W.residual_norm(prob, gl, v0), rel=1e-9)
            assert st.used == l
            assert np.max(np.abs(s.get_x() - xs[l])) <= XTOL, l


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("fmt", [0, 2])
def test_jacobi_direction_and_the_solve_stays_exact(P, fmt, precision):
    """Weights that output half a Jacobi correction: the GPU's line search
    follows the oracle's on the network's output, the energy decreases, and
    every step still meets the 1e-9 bar on x (FP64 and mixed solvers)."""
    g = gen.config_graph(1, scale=32)
    prob = O.Problem.from_graph(g)
    T = 8
    eps = O.eps_schedule(T)
    xs, _ = O.irls(prob, T, eps)
    gprev = O.initial_conductance(prob)
    w = jacobi_weights(0.5)
    with P.Solver(g, pcg_tol=1e-13, format=fmt, precision=precision) as s:
        s.initial()
        s.mlp_enable(P.binding.MLP_PREDICT, seed=1)
        s.mlp_weights(w)
        for l in range(1, T + 1):
            s.set_x(xs[l - 1])
            info = s.irls_step(eps[l - 1])
            assert info.status == 0
            gl = O.reweight(prob, xs[l - 1], eps[l - 1])
            F = W.features(prob, xs[l - 1], gl, gprev, eps[l - 1])
            out, bound = W.mlp_forward_bf16(w, F)
            v0 = reduced(prob, xs[l - 1])
            alpha, dE = W.line_search(prob, gl, v0, out)
            # d = 0.5 (f1 - f0): the data path's bound plus the feature
            # tolerance of f0 and f1 on the GPU's side
            e = bound + 0.5 * 2 * FEATURE_ATOL
            ta, tE = line_search_tolerance(prob, gl, v0, out, e)
            st = s.mlp_stats()
            assert abs(st.alpha - alpha) <= 2 * ta + 1e-12 * abs(alpha), (st.alpha, alpha, ta)
            assert abs(st.energy_change - dE) <= 2 * tE + 1e-9 * abs(dE), (st.energy_change, dE, tE)
            assert abs(st.alpha - alpha) <= 1e-2 * abs(alpha)
            assert st.energy_change < 0.0
            assert np.max(np.abs(s.get_x() - xs[l])) <= XTOL, l
            gprev = gl


@pytest.mark.parametrize("fmt", [0, 2])
def test_first_adam_step_follows_the_oracle_gradient(P, fmt):
    """One Adam step from zero moments moves each parameter by -lr * sign(g):
    the signs of the GPU's minibatch gradient (hand-written backward pass,
    SplitMix64-drawn nodes) against the oracle's exact gradient."""
    g = gen.config_graph(1, scale=32)
    prob = O.Problem.from_graph(g)
    xs, _ = O.irls(prob, 1, [0.1])
    rng = np.random.default_rng(21)
    w0 = rng.normal(0, 0.2, W.NPARAM).astype(np.float32)
    seed = 77
    lr = 1e-3
    with P.Solver(g, pcg_tol=1e-13, format=fmt) as s:
        s.initial()
        s.mlp_enable(P.binding.MLP_TRAIN, seed=seed)
        s.mlp_configure(1, lr)
        s.mlp_weights(w0)
        s.set_x(xs[0])
        s.irls_step(0.1)
        w1 = s.mlp_weights()
        st = s.mlp_stats()
        assert st.train_steps == 1
    g1 = O.reweight(prob, xs[0], 0.1)
    F = W.features(prob, xs[0], g1, O.initial_conductance(prob), 0.1)
    nodes = W.sample_nodes(seed, 0, prob.nt)
    target = (reduced(prob, xs[1]) - reduced(prob, xs[0]))[nodes].astype(np.float32)
    grad, loss = W.mlp_gradient(w0, F[nodes], target)
    assert st.loss == pytest.approx(loss, rel=1e-3)
    clear = np.abs(grad) > 1e-3 * np.abs(grad).max()
    assert clear.sum() > 0.3 * W.NPARAM
    step = (w1.astype(np.float64) - w0.astype(np.float64))[clear]
    np.testing.assert_allclose(step, -lr * np.sign(grad[clear]), rtol=0, atol=2e-6)
    assert np.all(np.abs(w1 - w0) <= lr * (1 + 1e-5) + 1e-6)


def test_training_is_deterministic_and_graph_equals_stream(P):
    g = gen.config_graph(1)
    T = 12
    eps = O.eps_schedule(T)
    runs = []
    for launch in (1, 1, 0):
        with P.Solver(g, graph_launch=launch) as s:
            s.mlp_enable(P.binding.MLP_PREDICT | P.binding.MLP_TRAIN, seed=11)
            infos = s.solve(T, eps)
            runs.append((s.get_x(), s.mlp_weights(), [i.pcg_iters for i in infos],
                         s.mlp_stats().as_dict()))
    for r in runs[1:]:
        assert np.array_equal(r[0], runs[0][0])
        assert np.array_equal(r[1], runs[0][1])
        assert r[2] == runs[0][2]
        assert r[3] == runs[0][3]
    assert runs[0][3]["train_steps"] == 8 * T


def test_training_lowers_the_loss_on_a_repeated_sequence(P):
    """Fit on the trajectory of one problem, then run it again: the second
    pass's minibatch losses are below the first pass's."""
    g = gen.config_graph(1, scale=48)
    T = 12
    eps = O.eps_schedule(T)
    passes = []
    with P.Solver(g) as s:
        s.mlp_enable(P.binding.MLP_TRAIN, seed=2)
        for _ in range(3):
            s.initial()
            losses = []
            for l in range(T):
                s.irls_step(eps[l])
                losses.append(s.mlp_stats().loss)
            passes.append(np.mean(losses))
    assert passes[2] < passes[0]


def test_mlp_call_errors(P):
    B = P.binding
    g = gen.config_graph(1, scale=8)
    with P.Solver(g) as s:
        for fn in (lambda: s.mlp_weights(), lambda: s.mlp_stats(), lambda: s.mlp_features(),
                   lambda: s.mlp_predict(np.zeros((2, 6), np.float32))):
            with pytest.raises(B.PirmcutError) as ei:
                fn()
            assert ei.value.status == B.EINVAL
        with pytest.raises(B.PirmcutError):
            s.mlp_enable(4)
        with pytest.raises(B.PirmcutError):
            s.mlp_configure(-1, 1e-3)
        with pytest.raises(B.PirmcutError):
            s.mlp_configure(1, 0.0)
        s.mlp_enable(B.MLP_PREDICT)
        assert s.mlp_predict(np.zeros((0, 6), np.float32)).shape == (0,)
        with pytest.raises(ValueError):
            s.mlp_weights(np.zeros(5, np.float32))
        s.mlp_enable(0)
        s.solve(3, O.eps_schedule(3))
        assert s.mlp_stats().steps == 0
