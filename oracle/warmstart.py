"""CPU oracle of the learned warm start (an extension of Section 3.1).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and never by the product
path.  It shares no code with the CUDA library.

The paper starts the PCG of IRLS step l from the previous iterate v^(l-1)
(Section 3.1) and aims at sequences and batches of related problems
(Section 6).  The library can also move the start along a learned direction: a per-node
MLP predicts x^(l) - x^(l-1) from six features of step l, and an exact line
search on the energy that CG minimises sets the step length, so the start is
never worse than x^(l-1) in that norm.  This module
writes every piece of that out plainly:

* ``features``        the six per-node features, from their definitions;
* ``bf16_round``      IEEE binary32 -> bfloat16, round to nearest even;
* ``mlp_forward``     the network evaluated exactly (FP64) on BF16 weights
                      and FP32 inputs, with a rigorous bound on the error of
                      an FP32 evaluation (fused multiply-add per term);
* ``mlp_forward_bf16`` the same exact value with a bound for the tensor-core
                      data path (BF16 operands, FP32 accumulation);
* ``mlp_gradient``    the exact gradient of the minibatch mean squared error;
* ``splitmix64``      the SplitMix64 generator (Steele, Lea & Flood, 2014),
                      ``sample_nodes`` the minibatch it draws;
* ``adam_step``       one Adam update (Kingma & Ba, 2015) in FP32;
* ``residual_norm``   ||b - L~ v||_2 of a start v, conductances from x^(l-1);
* ``energy``, ``line_search``  the quadratic energy E(v) = v^T L~ v - 2 b^T v
                      and the exact minimiser of E along the learned direction.

Parity status: pinned by hand-computed features on a small graph, by finite
differences of the gradient, by SplitMix64's published output, by BF16
rounding cases, by the Adam first-step identity and by the energy identity
E(v) - E(v*) = ||v - v*||^2 (see
``tests/test_oracle_warmstart.py``).
"""
from __future__ import annotations

import numpy as np

from .pirmcut import Problem, laplacian, reduced_system

H = 64
NF = 6
OFF_W1 = 0
OFF_B1 = OFF_W1 + H * NF
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
NPARAM = OFF_B3 + 1           # 4673
TRAIN_BLOCKS = 32
SAMPLES_PER_BLOCK = 64
BATCH = TRAIN_BLOCKS * SAMPLES_PER_BLOCK
MASK64 = (1 << 64) - 1


def unpack(w):
    """Split a flat parameter vector into (W1, b1, W2, b2, w3, b3)."""
    w = np.asarray(w)
    return (w[OFF_W1:OFF_B1].reshape(H, NF), w[OFF_B1:OFF_W2], w[OFF_W2:OFF_B2].reshape(H, H),
            w[OFF_B2:OFF_W3], w[OFF_W3:OFF_B3], w[OFF_B3])


def features(prob: Problem, x: np.ndarray, g: np.ndarray, g_prev: np.ndarray, eps: float):
    """Per-node features of one IRLS step, float32 [n~, 6] in the order of
    ``prob.nonterminals``.

    x       full voltage vector x^(l-1) (x_s = 1, x_t = 0)
    g       per-edge conductances of step l (``prob.eu``/``prob.ev`` order)
    g_prev  per-edge conductances of step l-1
    eps     eps_l

    For a non-terminal v with incident edges e = (v, u):
      f0 = x_v
      f1 = sum_e g_e x_u / sum_e g_e          (all incident edges, s and t included)
      f2 = sqrt(max(sum_e g_e x_u^2 / sum_e g_e - f1^2, 0))
      f3 = mean of log(g_e / g_prev_e) over edges with u non-terminal and
           both conductances positive (0 if there is none), divided by 8
      f4 = log(sum_e g_e) / 8                 (the diagonal entry of L~)
      f5 = log(eps) / 8
    """
    n = prob.n
    x = np.asarray(x, dtype=np.float64)
    wsum = np.zeros(n)
    wx = np.zeros(n)
    wxx = np.zeros(n)
    lr = np.zeros(n)
    nlr = np.zeros(n)
    terminal = np.zeros(n, dtype=bool)
    terminal[[prob.s, prob.t]] = True
    for e in range(prob.m):
        for a, b in ((prob.eu[e], prob.ev[e]), (prob.ev[e], prob.eu[e])):
            wsum[a] += g[e]
            wx[a] += g[e] * x[b]
            wxx[a] += g[e] * x[b] * x[b]
            if not terminal[b] and g[e] > 0 and g_prev[e] > 0:
                lr[a] += np.log(g[e] / g_prev[e])
                nlr[a] += 1
    v = prob.nonterminals
    mean = wx[v] / wsum[v]
    var = np.maximum(wxx[v] / wsum[v] - mean * mean, 0.0)
    f = np.zeros((v.shape[0], NF))
    f[:, 0] = x[v]
    f[:, 1] = mean
    f[:, 2] = np.sqrt(var)
    f[:, 3] = np.where(nlr[v] > 0, lr[v] / np.maximum(nlr[v], 1), 0.0) / 8.0
    f[:, 4] = np.log(wsum[v]) / 8.0
    f[:, 5] = np.log(eps) / 8.0
    return f.astype(np.float32)


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest, ties to even); returns float32."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)


def forward64(params, F):
    """The network 6 -> 64 -> 64 -> 1 with ReLU on the hidden layers, in FP64,
    on parameters ``params`` as given (no rounding).  Returns (out, cache)."""
    W1, b1, W2, b2, w3, b3 = (np.asarray(p, dtype=np.float64) for p in unpack(params))
    F = np.asarray(F, dtype=np.float64)
    z1 = F @ W1.T + b1
    h1 = np.maximum(z1, 0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0)
    out = h2 @ w3 + b3
    return out, (F, z1, h1, z2, h2)


def mlp_forward(w, F):
    """The network on feature rows F (float32 [N, 6]) with the BF16 rounding of
    the float32 weights w, evaluated exactly in FP64.

    Returns (out, bound): ``out`` the outputs, ``bound`` a rigorous bound on
    |FP32 evaluation - out| when every dot product starts from its bias and
    adds its n terms with one fused multiply-add each: the result is within
    gamma_n = n u / (1 - n u) (u = 2^-24) times the sum of the absolute values
    of bias and terms (Higham, Accuracy and Stability of Numerical Algorithms,
    Section 3.1), ReLU is 1-Lipschitz, and the error of a layer's inputs
    reaches its output through the absolute weights.
    """
    p = bf16_round(w).astype(np.float64)
    F = np.asarray(F, dtype=np.float32).astype(np.float64)
    out, (F, z1, h1, z2, h2) = forward64(p, F)
    W1, b1, W2, b2, w3, b3 = unpack(p)
    u = 2.0 ** -24

    def gamma(k):
        return k * u / (1 - k * u)

    # layer 1 from exact inputs; each later layer adds its own rounding to the
    # propagated error of its (perturbed) inputs
    e1 = gamma(NF) * (np.abs(F) @ np.abs(W1).T + np.abs(b1))
    e2 = gamma(H) * (np.abs(b2) + (np.abs(h1) + e1) @ np.abs(W2).T) + e1 @ np.abs(W2).T
    eo = gamma(H) * (abs(b3) + (np.abs(h2) + e2) @ np.abs(w3)) + e2 @ np.abs(w3)
    return out, eo


def mlp_forward_bf16(w, F, u_acc: float = 2.0 ** -22):
    """The network on feature rows F with the BF16 rounding of the weights w,
    evaluated exactly in FP64, and a bound on |result of the tensor-core data
    path - exact| for the evaluation that:

    * enters each feature as a BF16 head plus a BF16 tail, f ~ hi + lo with
      |f - hi - lo| <= 2^-18 |f| (each rounding to nearest BF16 is within
      2^-9 relative);
    * accumulates layer 1 (six features, the bias as a seventh term) and
      layer 2 (64 terms, starting from b2) in FP32 with any order of
      additions, each within u_acc relative (2^-22: round to nearest would
      give 2^-24; the model also covers truncated partial sums);
    * rounds ReLU(layer 1) to BF16 (2^-9 relative) before layer 2;
    * evaluates layer 3 in FP32 with fused multiply-adds (2^-24).

    The bound follows the forward error analysis of dot products
    (Higham, Accuracy and Stability of Numerical Algorithms, Section 3.1:
    gamma_n = n u / (1 - n u) times the sum of the absolute terms); ReLU is
    1-Lipschitz; an input error reaches the output through |weights|.
    """
    p = bf16_round(w).astype(np.float64)
    F = np.asarray(F, dtype=np.float32).astype(np.float64)
    out, (F, z1, h1, z2, h2) = forward64(p, F)
    W1, b1, W2, b2, w3, b3 = unpack(p)

    def gamma(k, u):
        return k * u / (1 - k * u)

    aW1, aW2, aw3 = np.abs(W1), np.abs(W2), np.abs(w3)
    eF = 2.0 ** -18 * np.abs(F)
    e1 = eF @ aW1.T + gamma(NF + 1, u_acc) * ((np.abs(F) + eF) @ aW1.T + np.abs(b1))
    eh1 = e1 + 2.0 ** -9 * (np.abs(h1) + e1)
    e2 = eh1 @ aW2.T + gamma(H + 1, u_acc) * (np.abs(b2) + (np.abs(h1) + eh1) @ aW2.T)
    eo = e2 @ aw3 + gamma(H + 1, 2.0 ** -24) * (abs(b3) + (np.abs(h2) + e2) @ aw3)
    return out, eo


def mlp_gradient(w, F, target, batch: int = BATCH):
    """Gradient of (1/batch) * sum_i (out_i - target_i)^2 with respect to the
    parameters, at their BF16 rounding; flat float64 [NPARAM], exact FP64
    backward pass (chain rule through the two ReLU layers).  Returns (grad, loss)."""
    p = bf16_round(w).astype(np.float64)
    W1, b1, W2, b2, w3, b3 = unpack(p)
    out, (F64, z1, h1, z2, h2) = forward64(p, np.asarray(F, dtype=np.float32).astype(np.float64))
    err = out - np.asarray(target, dtype=np.float64)
    dout = 2.0 * err / batch
    g = np.zeros(NPARAM)
    g[OFF_W3:OFF_B3] = h2.T @ dout
    g[OFF_B3] = dout.sum()
    dz2 = (z2 > 0) * np.outer(dout, w3)
    g[OFF_W2:OFF_B2] = (dz2.T @ h1).ravel()
    g[OFF_B2:OFF_W3] = dz2.sum(axis=0)
    dz1 = (z1 > 0) * (dz2 @ W2)
    g[OFF_W1:OFF_B1] = (dz1.T @ F64).ravel()
    g[OFF_B1:OFF_W2] = dz1.sum(axis=0)
    return g, float(np.sum(err * err) / batch)


def splitmix64(z: int) -> int:
    """SplitMix64 output for the state z (the state is advanced by the golden
    gamma 0x9e3779b97f4a7c15 before mixing), as published by Steele, Lea and
    Flood (2014) and used to seed the xoshiro generators."""
    z = (z + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def sample_nodes(seed: int, train_step: int, nt: int):
    """The minibatch of Adam step ``train_step`` (0-based count of the steps
    taken before it): node = splitmix64(stream + b * 64 + j) mod n~ for block
    b < 32 and sample j < 64, with stream = splitmix64(seed xor (train_step << 20))."""
    stream = splitmix64((seed ^ (train_step << 20)) & MASK64)
    nodes = []
    for b in range(TRAIN_BLOCKS):
        for j in range(SAMPLES_PER_BLOCK):
            nodes.append(splitmix64((stream + b * SAMPLES_PER_BLOCK + j) & MASK64) % nt)
    return np.array(nodes, dtype=np.int64)


def adam_step(master, m, v, grad, step: int, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update in float32 (step counts from 1).  Returns (master, m, v)."""
    f = np.float32
    master = np.asarray(master, dtype=f)
    grad = np.asarray(grad, dtype=f)
    m = f(b1) * np.asarray(m, dtype=f) + f(1 - f(b1)) * grad
    v = f(b2) * np.asarray(v, dtype=f) + f(1 - f(b2)) * grad * grad
    c1 = f(1) - f(b1) ** f(step)
    c2 = f(1) - f(b2) ** f(step)
    master = master - f(lr) * (m / c1) / (np.sqrt(v / c2) + f(eps))
    return master.astype(f), m.astype(f), v.astype(f)


def residual_norm(prob: Problem, g: np.ndarray, v: np.ndarray) -> float:
    """||b - L~ v||_2 of the reduced system built from conductances g
    (Eq. reduced-laplacian-system); v in reduced numbering."""
    Lt, b = reduced_system(prob, laplacian(prob, g))
    return float(np.linalg.norm(b - Lt @ v))


def energy(prob: Problem, g: np.ndarray, v: np.ndarray) -> float:
    """E(v) = v^T L~ v - 2 b^T v, which equals ||v - v*||^2_{L~} - v*^T b for
    the solution v* of L~ v* = b."""
    Lt, b = reduced_system(prob, laplacian(prob, g))
    return float(v @ (Lt @ v) - 2.0 * (b @ v))


def line_search(prob: Problem, g: np.ndarray, v0: np.ndarray, d: np.ndarray):
    """Exact minimiser of E(v0 + alpha d) over alpha: alpha = d^T r / d^T L~ d
    with r = b - L~ v0 (alpha = 0 when d^T L~ d <= 0).  Returns (alpha, the
    energy change E(v0 + alpha d) - E(v0) = -(d^T r) alpha)."""
    Lt, b = reduced_system(prob, laplacian(prob, g))
    d = np.asarray(d, dtype=np.float64)
    r = b - Lt @ v0
    dad = float(d @ (Lt @ d))
    if not dad > 0.0:
        return 0.0, 0.0
    alpha = float(d @ r) / dad
    return alpha, -float(d @ r) * alpha
