"""The C ABI library builds for sm_103a, loads, exports every entry point that
include/pirmcut.h declares, and rejects bad input on the host (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pirmcut.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1501_03105_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pirmcut_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("pirmcut_create", "pirmcut_irls_step", "pirmcut_solve", "pirmcut_cut",
                 "pirmcut_get_x", "pirmcut_set_x", "pirmcut_update_weights",
                 "pirmcut_last_error", "pirmcut_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1501_03105_gb300 import binding
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pirmcut_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_default_options(lib):
    from paper_1501_03105_gb300 import binding as B
    o = B.pirmcut_default_options()
    assert o.reweight_form == B.REWEIGHT_WEIGHTED_L1 and o.precision == B.PREC_FP64
    assert o.pcg_tol == 1e-10 and o.pcg_max_iter == 20000 and o.warm_start == 1
    assert o.track_cut == 0 and o.graph_launch == 1 and o.inner_tol == 1e-5
    assert o.time_spmv == 0 and o.reduce_on_host == 0
    assert (o.batch_threads_per_row, o.batch_tile_rows, o.batch_medium_deg) == (0, 0, 0)


def test_batch_options_are_checked_before_any_gpu_work(lib):
    from paper_1501_03105_gb300 import binding as B
    g = gen.random_graph(10, 0.3, 1)
    for kw in (dict(precision=B.PREC_MIXED), dict(batch_threads_per_row=3),
               dict(batch_tile_rows=32), dict(batch_tile_rows=70000), dict(batch_medium_deg=513)):
        _expect(B.EINVAL, B.Batch, [g], **kw)


def _expect(status, fn, *a, **k):
    from paper_1501_03105_gb300 import binding as B
    with pytest.raises(B.PirmcutError) as ei:
        fn(*a, **k)
    assert ei.value.status == status, str(ei.value)
    return ei.value


def test_host_validation_errors(lib):
    """Malformed input is rejected on the host before any GPU work."""
    from paper_1501_03105_gb300 import binding as B
    g = gen.random_graph(10, 0.3, 1)
    _expect(B.EINVAL, B.pirmcut_create, g.n, g.row_ptr, g.col, g.c, g.s, g.s)      # s == t
    _expect(B.EINVAL, B.pirmcut_create, g.n, g.row_ptr, g.col, g.c, g.s, g.n)      # t out of range
    c = g.c.copy()
    c[0] = -1.0
    _expect(B.EINVAL, B.pirmcut_create, g.n, g.row_ptr, g.col, c, g.s, g.t)        # negative
    c[0] = np.nan
    _expect(B.EINVAL, B.pirmcut_create, g.n, g.row_ptr, g.col, c, g.s, g.t)        # NaN
    c = g.c.copy()
    c[0] += 1.0
    _expect(B.EINVAL, B.pirmcut_create, g.n, g.row_ptr, g.col, c, g.s, g.t)        # asymmetric
    col = g.col.copy()
    col[0] = g.n + 3
    _expect(B.EINVAL, B.pirmcut_create, g.n, g.row_ptr, col, g.c, g.s, g.t)        # column range
    rp = g.row_ptr.copy()
    rp[3] = rp[2] - 1
    _expect(B.EINVAL, B.pirmcut_create, g.n, rp, g.col, g.c, g.s, g.t)             # row_ptr order
    rp, cl, cc = gen.csr_from_edges(4, [0, 1, 1], [1, 1, 2], [1.0, 1.0, 1.0])     # self-loop
    _expect(B.EINVAL, B.pirmcut_create, 4, rp, cl, cc, 0, 2)
    _expect(B.EINVAL, B.pirmcut_create, 2, np.array([0, 1, 2]), np.array([1, 0], np.int32),
            np.array([1.0, 1.0]), 0, 1)                                            # n < 3
    opt = B.pirmcut_default_options(pcg_tol=-1.0)
    _expect(B.EINVAL, B.pirmcut_create, g.n, g.row_ptr, g.col, g.c, g.s, g.t, opt)


def test_disconnected_component_is_reported(lib):
    """Prop. nonsingular: a component reaching neither terminal is an error."""
    from paper_1501_03105_gb300 import binding as B
    rp, col, c = gen.csr_from_edges(5, [0, 1, 3], [1, 2, 4], [1.0, 1.0, 1.0])
    e = _expect(B.EDISCONNECTED, B.pirmcut_create, 5, rp, col, c, 0, 2)
    assert "vertex 3" in e.message
    # zero-capacity bridge: structurally connected, electrically not
    rp, col, c = gen.csr_from_edges(4, [0, 1, 1], [1, 2, 3], [1.0, 1.0, 0.0])
    _expect(B.EDISCONNECTED, B.pirmcut_create, 4, rp, col, c, 0, 2)


def test_entry_points_reject_null_context(lib):
    assert lib.pirmcut_initial(None, None) == 1
    assert lib.pirmcut_irls_step(None, ctypes.c_double(0.1), None) == 1
    assert lib.pirmcut_solve(None, 1, None, None) == 1
    assert lib.pirmcut_cut(None, None, None, None, 0) == 1
    assert lib.pirmcut_get_x(None, None, 0) == 1
    assert lib.pirmcut_set_x(None, None, 0) == 1
    assert lib.pirmcut_update_weights(None, None, 0) == 1
    assert lib.pirmcut_kernel_launches(None) == 0
    lib.pirmcut_destroy(None)
