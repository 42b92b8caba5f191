"""Pins of the learned-warm-start oracle (``oracle/warmstart.py``) against
values fixed by hand, by published definitions and by the mathematics, and
mutants (planted on the CPU) that the pins must catch."""
import math

import numpy as np
import pytest

import gen
import oracle as O
import oracle.warmstart as W


# --- SplitMix64: the published output sequence -----------------------------

def test_splitmix64_published_sequence():
    """SplitMix64 seeded with 1234567: the first five outputs as printed in
    the reference implementation accompanying the xoshiro generators."""
    gamma = 0x9E3779B97F4A7C15
    expect = [6457827717110365317, 3203168211198807973, 9817491932198370423,
              4593380528125082431, 16408922859458223821]
    got = [W.splitmix64((1234567 + k * gamma) & W.MASK64) for k in range(5)]
    assert got == expect


def test_sample_nodes_range_spread_and_stream():
    nt = 1000
    a = W.sample_nodes(7, 0, nt)
    b = W.sample_nodes(7, 1, nt)
    assert a.shape == (W.BATCH,) and a.min() >= 0 and a.max() < nt
    assert not np.array_equal(a, b)
    assert np.array_equal(a, W.sample_nodes(7, 0, nt))
    # 2048 draws over 10 bins of 100 nodes: chi-square far below its 1e-6 tail (~45)
    h = np.bincount(a // 100, minlength=10)
    chi2 = float(np.sum((h - W.BATCH / 10) ** 2 / (W.BATCH / 10)))
    assert chi2 < 45.0


# --- BF16 rounding ----------------------------------------------------------

def test_bf16_round_cases():
    f = np.float32
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 3 * 2 ** -9, 1 + 2 ** -8 + 2 ** -20,
                     -2.5, 2 ** -130, 65504.0], dtype=f)
    # exact / tie to even (down) / tie to even (up) / nearest / above the tie /
    # exact negative / subnormal kept / 65504 = 1.999 * 2^15 -> 65536 (nearest)
    expect = np.array([1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, 1 + 2 ** -7, -2.5, 2 ** -130, 65536.0], dtype=f)
    assert np.array_equal(W.bf16_round(vals), expect)
    r = W.bf16_round(np.random.default_rng(1).normal(size=1000).astype(f))
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)


# --- features: a hand-computed example ------------------------------------

def _hand_problem():
    # s=0, a=1, b=2, t=3; edges s-a (1), a-b (2), b-t (1), a-t (3)
    edges = [(0, 1, 1.0), (1, 2, 2.0), (2, 3, 1.0), (1, 3, 3.0)]
    n = 4
    rows = [[] for _ in range(n)]
    for u, v, c in edges:
        rows[u].append((v, c))
        rows[v].append((u, c))
    rp, col, cap = [0], [], []
    for r in rows:
        for v, c in r:
            col.append(v)
            cap.append(c)
        rp.append(len(col))
    return O.Problem(n, rp, col, cap, 0, 3)


def test_features_hand_example():
    prob = _hand_problem()
    # prob.eu/ev list pairs in (u < v) order: (0,1) (1,2) (1,3) (2,3)
    assert list(zip(prob.eu, prob.ev)) == [(0, 1), (1, 2), (1, 3), (2, 3)]
    x = np.array([1.0, 0.6, 0.2, 0.0])
    g = np.array([1.0, 2.0, 4.0, 1.0])
    gp = np.array([1.0, 0.5, 1.0, 1.0])
    eps = 0.01
    f = W.features(prob, x, g, gp, eps)
    # vertex a: neighbours s (g 1, x 1), b (g 2, x 0.2), t (g 4, x 0)
    # mean 1.4/7 = 0.2, E[x^2] = 1.08/7, var = 0.08/0.7 = 4/35
    # vertex b: neighbours a (g 2, x 0.6), t (g 1, x 0): mean 0.4, var 0.24 - 0.16
    expect = np.array([
        [0.6, 0.2, math.sqrt(4 / 35), math.log(4) / 8, math.log(7) / 8, math.log(0.01) / 8],
        [0.2, 0.4, math.sqrt(0.08), math.log(4) / 8, math.log(3) / 8, math.log(0.01) / 8],
    ])
    np.testing.assert_allclose(f, expect, rtol=1e-6, atol=1e-7)


def test_features_constant_field_and_unchanged_conductances():
    """x constant on the non-terminals and g = g_prev: the neighbour mean of a
    vertex with no terminal edge is that constant, its spread 0, f3 = 0."""
    # 8 x 8 grid, s tied to the left column, t to the right column
    k = 8
    u, v, c = [], [], []
    for r in range(k):
        for q in range(k):
            i = r * k + q
            if q + 1 < k:
                u.append(i), v.append(i + 1), c.append(1.0 + 0.1 * r)
            if r + 1 < k:
                u.append(i), v.append(i + k), c.append(2.0 - 0.1 * q)
        u.append(k * k), v.append(r * k), c.append(1.0)
        u.append(k * k + 1), v.append(r * k + k - 1), c.append(1.0)
    rp, col, cap = gen.csr_from_edges(k * k + 2, np.array(u), np.array(v), np.array(c))
    prob = O.Problem(k * k + 2, rp, col, cap, k * k, k * k + 1)
    x = np.full(prob.n, 0.375)
    x[prob.s], x[prob.t] = 1.0, 0.0
    g = O.reweight(prob, x, 0.1)
    f = W.features(prob, x, g, g, 0.1)
    touches = np.zeros(prob.n, dtype=bool)
    for e in range(prob.m):
        if prob.s in (prob.eu[e], prob.ev[e]) or prob.t in (prob.eu[e], prob.ev[e]):
            touches[prob.eu[e]] = touches[prob.ev[e]] = True
    inner = ~touches[prob.nonterminals]
    assert inner.sum() > 10
    np.testing.assert_allclose(f[inner, 1], 0.375, rtol=0, atol=1e-7)
    np.testing.assert_allclose(f[inner, 2], 0.0, atol=1e-4)
    assert np.all(f[:, 3] == 0.0)
    # f4 is log of the diagonal of L~ / 8
    Lt, _ = O.reduced_system(prob, O.laplacian(prob, g))
    np.testing.assert_allclose(f[:, 4], np.log(Lt.diagonal()) / 8, rtol=1e-6)


# --- the network ------------------------------------------------------------

def _rand_params(seed, scale=0.3):
    return np.random.default_rng(seed).normal(0, scale, W.NPARAM).astype(np.float32)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    w = _rand_params(3)
    F = rng.normal(0, 1, (40, 6)).astype(np.float32)
    y = rng.normal(0, 1, 40)
    g, loss = W.mlp_gradient(w, F, y, batch=40)
    p = W.bf16_round(w).astype(np.float64)

    def L(q):
        o, _ = W.forward64(q, F.astype(np.float64))
        return float(np.sum((o - y) ** 2) / 40)

    assert abs(loss - L(p)) <= 1e-12 * max(1.0, L(p))
    idx = np.concatenate([np.arange(W.OFF_W1, W.OFF_W1 + 30), np.arange(W.OFF_B1, W.OFF_B1 + 20),
                          rng.choice(np.arange(W.OFF_W2, W.OFF_B2), 200, replace=False),
                          np.arange(W.OFF_B2, W.NPARAM)])
    h = 1e-6
    for i in idx:
        e = np.zeros(W.NPARAM)
        e[i] = h
        fd = (L(p + e) - L(p - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i
    # the ReLUs matter here: some hidden units are off for some rows
    _, (_, z1, _, z2, _) = W.forward64(p, F.astype(np.float64))
    assert 0 < (z1 > 0).mean() < 1 and 0 < (z2 > 0).mean() < 1


def _fma32(a, b, c):
    # float32 fused multiply-add: the product of a float32 and a BF16 value is
    # exact in float64; one rounding of the sum to float32
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def test_forward_error_bound_covers_float32_fma_evaluation():
    rng = np.random.default_rng(4)
    w = _rand_params(5)
    F = rng.normal(0, 1, (8, 6)).astype(np.float32)
    out, bound = W.mlp_forward(w, F)
    W1, b1, W2, b2, w3, b3 = W.unpack(W.bf16_round(w))
    for r in range(F.shape[0]):
        h1 = np.zeros(64, dtype=np.float32)
        for k in range(64):
            z = b1[k]
            for m in range(6):
                z = _fma32(W1[k, m], F[r, m], z)
            h1[k] = max(z, np.float32(0))
        o = b3
        for j in range(64):
            z = b2[j]
            for k in range(64):
                z = _fma32(W2[j, k], h1[k], z)
            o = _fma32(w3[j], max(z, np.float32(0)), o)
        assert abs(float(o) - out[r]) <= bound[r]
        assert bound[r] < 2e-3 * (1 + abs(out[r]))  # not vacuous


def _bf16(a):
    return W.bf16_round(np.float32(a)).astype(np.float64)


def _trunc32(v):
    """Round toward zero to float32: a worse accumulator than round to nearest."""
    f = np.float32(v)
    if abs(float(f)) > abs(v):
        f = np.nextafter(f, np.float32(0))
    return f


def test_forward_bf16_bound_covers_the_tensor_core_data_path():
    """The tensor-core evaluation emulated step by step: split-BF16 features,
    exact BF16 products, FP32 partial sums (rounded to nearest, or truncated)
    in a shuffled order, ReLU rounded to BF16, an FP32 output layer.  Every
    emulation lies within the bound, which is not vacuous."""
    rng = np.random.default_rng(14)
    w = _rand_params(15)
    F = rng.normal(0, 1, (6, 6)).astype(np.float32)
    F[:, 1] = F[:, 0] + np.float32(1e-3)          # a near-cancelling pair (f1 - f0)
    out, bound = W.mlp_forward_bf16(w, F)
    W1, b1, W2, b2, w3, b3 = (a.astype(np.float64) for a in W.unpack(W.bf16_round(w)))
    for trunc in (False, True):
        acc = _trunc32 if trunc else np.float32
        for r in range(F.shape[0]):
            hi = np.array([_bf16(v) for v in F[r]])
            lo = np.array([_bf16(np.float64(F[r, m]) - hi[m]) for m in range(6)])
            h1 = np.zeros(64)
            for k in range(64):
                terms = [W1[k, m] * hi[m] for m in range(6)] + [W1[k, m] * lo[m] for m in range(6)]
                terms.append(b1[k])
                z = np.float32(0)
                for j in rng.permutation(len(terms)):
                    z = acc(np.float64(z) + terms[j])
                h1[k] = _bf16(max(float(z), 0.0))
            o = np.float32(b3)
            for j in range(64):
                z = np.float32(b2[j])
                for k in rng.permutation(64):
                    z = acc(np.float64(z) + W2[j, k] * h1[k])
                o = _fma32(np.float32(w3[j]), np.float32(max(float(z), 0.0)), o)
            assert abs(float(o) - out[r]) <= bound[r], (trunc, r)
            # not vacuous: the BF16 hidden layer costs about 2^-9 times the
            # absolute path sums (64 x 64 weights of size ~0.2 here)
            assert bound[r] < 0.2 * (1 + abs(out[r]))


def test_forward_zero_output_layer_predicts_zero():
    w = _rand_params(6)
    w[W.OFF_W3:] = 0
    out, bound = W.mlp_forward(w, np.random.default_rng(0).normal(size=(20, 6)).astype(np.float32))
    assert np.all(out == 0) and np.all(bound == 0)


# --- Adam -------------------------------------------------------------------

def test_adam_moves_by_lr_times_sign_for_a_constant_gradient():
    """With m = v = 0 and a constant gradient, the bias-corrected moments are
    g and g^2 at every step, so each step moves by lr * sign(g)."""
    rng = np.random.default_rng(7)
    w0 = rng.normal(size=50).astype(np.float32)
    g = rng.normal(size=50).astype(np.float32)
    g[0] = 0.0
    w, m, v = w0.copy(), np.zeros(50, np.float32), np.zeros(50, np.float32)
    for k in range(1, 4):
        w, m, v = W.adam_step(w, m, v, g, k, lr=1e-3)
        np.testing.assert_allclose(w, w0 - k * 1e-3 * np.sign(g), rtol=0, atol=2e-6)
    assert w[0] == w0[0]


# --- residuals and the candidate ------------------------------------------

def test_residual_norm_at_zero_and_at_the_solution():
    g0 = gen.config_graph(1, scale=10)
    prob = O.Problem.from_graph(g0)
    g = O.initial_conductance(prob)
    Lt, b = O.reduced_system(prob, O.laplacian(prob, g))
    v = O.solve_direct(Lt, b)
    assert W.residual_norm(prob, g, np.zeros(prob.nt)) == pytest.approx(np.linalg.norm(b), rel=1e-14)
    assert W.residual_norm(prob, g, v) <= 1e-12 * np.linalg.norm(b)


def test_energy_identity_and_line_search_optimality():
    """E(v) - E(v*) = ||v - v*||^2_{L~}; the line search's alpha minimises E
    along d and its energy change is E(v0 + alpha d) - E(v0)."""
    g0 = gen.config_graph(1, scale=10)
    prob = O.Problem.from_graph(g0)
    rng = np.random.default_rng(3)
    x = np.clip(O.wls_step(prob, O.initial_conductance(prob))[0] + rng.normal(0, 0.05, prob.n), 0, 1)
    x[prob.s], x[prob.t] = 1.0, 0.0
    g = O.reweight(prob, x, 0.05)
    Lt, b = O.reduced_system(prob, O.laplacian(prob, g))
    vs = O.solve_direct(Lt, b)
    v = x[prob.nonterminals]
    e = v - vs
    assert W.energy(prob, g, v) - W.energy(prob, g, vs) == pytest.approx(e @ (Lt @ e), rel=1e-9)
    d = rng.normal(0, 1, prob.nt)
    alpha, dE = W.line_search(prob, g, v, d)
    E0 = W.energy(prob, g, v)
    assert W.energy(prob, g, v + alpha * d) - E0 == pytest.approx(dE, rel=1e-6)
    assert dE < 0
    for h in (1e-3, -1e-3):
        assert W.energy(prob, g, v + (alpha + h) * d) > E0 + dE
    # the exact error direction: alpha = 1 and the solution is reached
    alpha, dE = W.line_search(prob, g, v, vs - v)
    assert alpha == pytest.approx(1.0, rel=1e-9)
    assert dE == pytest.approx(-(e @ (Lt @ e)), rel=1e-9)
    assert W.line_search(prob, g, v, np.zeros(prob.nt)) == (0.0, 0.0)


# --- mutants ------------------------------------------------------------------

PINS = [test_features_hand_example, test_features_constant_field_and_unchanged_conductances,
        test_gradient_matches_finite_differences, test_forward_error_bound_covers_float32_fma_evaluation,
        test_adam_moves_by_lr_times_sign_for_a_constant_gradient, test_bf16_round_cases,
        test_splitmix64_published_sequence, test_energy_identity_and_line_search_optimality]


def _features_no_terminals(prob, x, g, g_prev, eps):
    x = np.array(x, dtype=np.float64)
    keep = np.ones(prob.m, dtype=bool)
    for e in range(prob.m):
        if prob.s in (prob.eu[e], prob.ev[e]) or prob.t in (prob.eu[e], prob.ev[e]):
            keep[e] = False
    return _ORIG["features"](prob, x, np.where(keep, g, 0.0), np.where(keep, g_prev, 0.0), eps)


def _features_ratio_inverted(prob, x, g, g_prev, eps):
    return _ORIG["features"](prob, x, g_prev, g, eps)


def _gradient_no_relu_mask(w, F, target, batch=W.BATCH):
    p = W.bf16_round(w).astype(np.float64)
    W1, b1, W2, b2, w3, b3 = W.unpack(p)
    out, (F64, z1, h1, z2, h2) = W.forward64(p, np.asarray(F, np.float64))
    dout = 2.0 * (out - target) / batch
    g = np.zeros(W.NPARAM)
    g[W.OFF_W3:W.OFF_B3] = h2.T @ dout
    g[W.OFF_B3] = dout.sum()
    dz2 = np.outer(dout, w3)
    g[W.OFF_W2:W.OFF_B2] = (dz2.T @ h1).ravel()
    g[W.OFF_B2:W.OFF_W3] = dz2.sum(axis=0)
    dz1 = (z1 > 0) * (dz2 @ W2)
    g[W.OFF_W1:W.OFF_B1] = (dz1.T @ F64).ravel()
    g[W.OFF_B1:W.OFF_W2] = dz1.sum(axis=0)
    return g, float(np.sum((out - target) ** 2) / batch)


def _gradient_transposed_w2(w, F, target, batch=W.BATCH):
    g, loss = _ORIG["mlp_gradient"](w, F, target, batch)
    blk = g[W.OFF_W2:W.OFF_B2].reshape(64, 64).T.ravel()
    g = g.copy()
    g[W.OFF_W2:W.OFF_B2] = blk
    return g, loss


def _adam_no_bias_correction(master, m, v, grad, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    return _ORIG["adam_step"](master, m, v, grad, 10 ** 6, lr, b1, b2, eps)


def _bf16_truncate(a):
    u = np.asarray(a, dtype=np.float32).view(np.uint32)
    return (u & 0xFFFF0000).astype(np.uint32).view(np.float32)


def _line_search_sign(prob, g, v0, d):
    alpha, dE = _ORIG["line_search"](prob, g, v0, d)
    return -alpha, dE


def _energy_without_factor_two(prob, g, v):
    Lt, b = O.reduced_system(prob, O.laplacian(prob, g))
    return float(v @ (Lt @ v) - b @ v)


def _splitmix_wrong_shift(z):
    z = (z + 0x9E3779B97F4A7C15) & W.MASK64
    z = ((z ^ (z >> 31)) * 0xBF58476D1CE4E5B9) & W.MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & W.MASK64
    return z ^ (z >> 31)


_ORIG = {k: getattr(W, k) for k in ("features", "mlp_gradient", "adam_step", "bf16_round", "splitmix64",
                                    "line_search", "energy")}

MUTANTS = [
    ("features", _features_no_terminals),
    ("features", _features_ratio_inverted),
    ("mlp_gradient", _gradient_no_relu_mask),
    ("mlp_gradient", _gradient_transposed_w2),
    ("adam_step", _adam_no_bias_correction),
    ("bf16_round", _bf16_truncate),
    ("splitmix64", _splitmix_wrong_shift),
    ("line_search", _line_search_sign),
    ("energy", _energy_without_factor_two),
]


@pytest.mark.parametrize("name,mutant", MUTANTS, ids=[m.__name__ for _, m in MUTANTS])
def test_pins_catch_mutant(monkeypatch, name, mutant):
    monkeypatch.setattr(W, name, mutant)
    caught = False
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            caught = True
            break
    assert caught, f"no pin caught the mutant {mutant.__name__}"
