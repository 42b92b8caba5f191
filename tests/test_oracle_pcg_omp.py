"""The OpenMP build of the oracle's Jacobi-PCG (oracle/pcg_omp.c), used for
the all-core CPU baseline, pinned like the Python oracle: closed forms of the
reduced system (Section 2.1), the exact solve, and the Python recurrence it
restates (Section 3.1), on one thread and on several."""
import numpy as np
import pytest
import scipy.sparse as sp

import gen
import oracle as O
from oracle import pcg_omp


def test_series_voltage_divider():
    # s - v - t with capacities a, b: the reduced system is (a + b) v = a
    a, b = 3.0, 1.5
    A = sp.csr_matrix(np.array([[a + b]]))
    x, it, rel = pcg_omp.pcg_jacobi(A, np.array([a]), tol=1e-14, threads=1)
    assert x[0] == pytest.approx(a / (a + b), rel=1e-15)
    # a chain s - v1 - v2 - t with unit capacities: voltages 2/3, 1/3
    A = sp.csr_matrix(np.array([[2.0, -1.0], [-1.0, 2.0]]))
    x, it, rel = pcg_omp.pcg_jacobi(A, np.array([1.0, 0.0]), tol=1e-14, threads=2)
    assert np.allclose(x, [2 / 3, 1 / 3], rtol=0, atol=1e-15)
    assert it <= 2                                 # CG is exact in n steps


@pytest.mark.parametrize("threads", [1, 4])
@pytest.mark.parametrize("make", [lambda: gen.config_graph(1, scale=24),
                                  lambda: gen.random_graph(60, 0.08, 3, zero_frac=0.1),
                                  lambda: gen.chung_lu_instance(2000, 7)])
def test_matches_python_recurrence_and_exact_solve(make, threads):
    g = make()
    prob = O.Problem.from_graph(g)
    xs, _ = O.irls(prob, 2, O.eps_schedule(2))
    gl = O.reweight(prob, xs[1], O.eps_schedule(2)[1])
    Lt, b = O.reduced_system(prob, O.laplacian(prob, gl))
    v0 = xs[1][prob.nonterminals]
    x_py, it_py, rel_py = O.pcg_jacobi(Lt, b, v0, tol=1e-12)
    x_c, it_c, rel_c = pcg_omp.pcg_jacobi(Lt, b, v0, tol=1e-12, threads=threads)
    assert abs(it_c - it_py) <= 1
    assert rel_c <= 1e-12
    assert np.max(np.abs(x_c - x_py)) <= 1e-10
    assert np.max(np.abs(x_c - O.solve_direct(Lt, b))) <= 1e-9


def test_zero_rhs_and_converged_start():
    A = sp.csr_matrix(np.array([[2.0, -1.0], [-1.0, 3.0]]))
    x, it, rel = pcg_omp.pcg_jacobi(A, np.zeros(2), x0=np.ones(2))
    assert it == 0 and np.all(x == 0.0)
    xe = np.linalg.solve(A.toarray(), [1.0, 2.0])
    x, it, rel = pcg_omp.pcg_jacobi(A, np.array([1.0, 2.0]), x0=xe, tol=1e-10)
    assert it == 0 and rel <= 1e-10
