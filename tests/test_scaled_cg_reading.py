"""The FP64 CUDA path runs Jacobi-preconditioned CG (Section 3.1) as plain CG
on the symmetrically scaled system D^-1/2 L~ D^-1/2 x^ = D^-1/2 b started from
x^ = D^1/2 x0, and maps back with x = D^-1/2 x^.  In exact arithmetic the two
recurrences give the same iterates and the same unpreconditioned residuals.
This CPU check pins that reading against the oracle's PCG, iteration by
iteration, on small workloads (no GPU)."""
import numpy as np
import pytest

import gen
import oracle as O


def scaled_cg(A, b, x0, iters):
    """CG on S A S with S = diag(A)^-1/2, as the CUDA path orders it: returns
    the iterates x (mapped back) and ||r|| = ||S^-1 r^|| after each step."""
    A = A.tocsr()
    d = A.diagonal()
    s = 1.0 / np.sqrt(d)
    Ah = (A.multiply(s[:, None]).multiply(s[None, :])).tocsr()
    xh = x0 / s
    rh = s * b - Ah @ xh
    p = rh.copy()
    rz = rh @ rh
    xs, norms = [], []
    for _ in range(iters):
        q = Ah @ p
        alpha = rz / (p @ q)
        xh = xh + alpha * p
        rh = rh - alpha * q
        rz_new = rh @ rh
        p = rh + (rz_new / rz) * p
        rz = rz_new
        xs.append(s * xh)
        norms.append(np.sqrt(np.sum(d * rh * rh)))
    return xs, norms


@pytest.mark.parametrize("name,make,step", [
    ("grid16", lambda: gen.config_graph(1, scale=16), 3),
    ("vol6", lambda: gen.config_graph(3, scale=6), 5),
    ("random60", lambda: gen.random_graph(60, 0.08, 3), 2),
])
def test_scaled_cg_has_the_iterates_of_jacobi_pcg(name, make, step):
    g = make()
    prob = O.Problem.from_graph(g)
    eps = O.eps_schedule(step)
    xs, _ = O.irls(prob, step, eps)
    gl = O.reweight(prob, xs[step - 1], eps[step - 1])
    Lt, b = O.reduced_system(prob, O.laplacian(prob, gl))
    x0 = xs[step - 1][prob.nonterminals]          # the warm start of step l
    k_max = 12
    ys, norms = scaled_cg(Lt, b, x0, k_max)
    bn = np.linalg.norm(b)
    for k in range(1, k_max + 1):
        # the oracle's PCG stopped after exactly k iterations (tol below reach)
        xk, it, rel = O.pcg_jacobi(Lt, b, x0, tol=1e-300, maxit=k)
        assert it == k
        scale = max(1.0, np.max(np.abs(xk)))
        assert np.max(np.abs(ys[k - 1] - xk)) <= 1e-11 * scale, (name, k)
        assert abs(norms[k - 1] / bn - rel) <= 1e-8 * rel + 1e-15, (name, k)


def test_a_plain_cg_on_the_unscaled_system_differs():
    """The check above is not vacuous: CG without the Jacobi scaling (z = r)
    takes other iterates on the same system."""
    g = gen.config_graph(1, scale=16)
    prob = O.Problem.from_graph(g)
    eps = O.eps_schedule(3)
    xs, _ = O.irls(prob, 3, eps)
    gl = O.reweight(prob, xs[2], eps[2])
    Lt, b = O.reduced_system(prob, O.laplacian(prob, gl))
    x0 = xs[2][prob.nonterminals]
    xk, _, _ = O.pcg_jacobi(Lt, b, x0, tol=1e-300, maxit=4)
    # plain CG: the same recurrence with the identity as preconditioner
    x, r = x0.copy(), b - Lt @ x0
    p, rr = r.copy(), r @ r
    for _ in range(4):
        q = Lt @ p
        a = rr / (p @ q)
        x, r = x + a * p, r - a * q
        rr_new = r @ r
        p, rr = r + (rr_new / rr) * p, rr_new
    assert np.max(np.abs(x - xk)) > 1e-6
