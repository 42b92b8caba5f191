"""Plain FP64 CPU oracle for the PIRMCut hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call or execute this package; only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.
It shares no code with the CUDA path.

See :mod:`oracle.pirmcut` for the method (reduced Laplacian, IRLS, PCG,
sweep cut) and :mod:`oracle.exact` for the exact references (brute-force cut
enumeration and an augmenting-path max-flow).
"""
from .pirmcut import (  # noqa: F401
    WEIGHTED_L1,
    PAPER,
    Problem,
    eps_schedule,
    initial_conductance,
    reweight,
    laplacian,
    reduced_system,
    solve_direct,
    pcg_jacobi,
    wls_step,
    irls,
    smoothed_objective,
    flow_value,
    cut_value,
    sweep_cut,
    sweep_cut_by_definition,
    kmeans_1d,
    two_level_rounding,
)
from .exact import brute_force_min_cut, max_flow_min_cut  # noqa: F401
