"""The input reduction on the GPU (reduce_on_host = 0) against the host one
(reduce_on_host = 1): the same problem, so bit-identical solves and cuts; the
same error statuses and messages for invalid inputs; capacity updates and the
two-level rounding on a problem built on the device."""
import numpy as np
import pytest

import gen
import oracle as O

pytestmark = pytest.mark.gpu


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


GRAPHS = [
    ("grid64", lambda: gen.config_graph(1)),
    ("grid37x41", lambda: gen.segmentation_grid(
        np.clip(gen.image_disks_2d(37, 41, [(18, 20, 9)]) + np.random.default_rng(7).normal(0, .05, (41, 37)), 0, 1))),
    ("vol12", lambda: gen.config_graph(3, scale=12)),
    ("chunglu", lambda: gen.chung_lu_instance(3000, 5)),
    ("random40", lambda: gen.random_graph(40, 0.1, 12)),   # vertices without terminal edges: host path
]


def run(P, g, host, fmt=0, precision=0, T=6):
    eps = O.eps_schedule(T)
    with P.Solver(g, pcg_tol=1e-12, reduce_on_host=host, format=fmt, precision=precision) as s:
        infos = s.solve(T, eps)
        side, value, tau = s.cut()
        return dict(x=s.get_x(), side=side, value=value, tau=tau, size=s.problem_size(),
                    iters=[i.pcg_iters for i in infos])


@pytest.mark.parametrize("fmt", [0, 2])
@pytest.mark.parametrize("name,make", GRAPHS)
def test_device_reduction_gives_the_host_problem(P, name, make, fmt):
    g = make()
    a, b = run(P, g, 0, fmt), run(P, g, 1, fmt)
    assert a["size"] == b["size"]
    assert np.array_equal(a["x"], b["x"])
    assert a["iters"] == b["iters"]
    assert a["value"] == b["value"] and a["tau"] == b["tau"]
    assert np.array_equal(a["side"], b["side"])


def test_device_reduction_mixed_precision(P):
    g = gen.config_graph(1)
    a, b = run(P, g, 0, precision=1), run(P, g, 1, precision=1)
    assert np.array_equal(a["x"], b["x"]) and a["value"] == b["value"]


def test_device_reduction_from_device_arrays(P):
    import torch
    g = gen.config_graph(1, scale=40)
    ref = run(P, g, 1)
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    c = torch.from_numpy(g.c).cuda()
    h = P.pirmcut_create(g.n, rp, col, c, g.s, g.t, P.pirmcut_default_options(pcg_tol=1e-12))
    try:
        P.pirmcut_solve(h, 6, np.asarray(O.eps_schedule(6)))
        x = np.empty(g.n)
        P.pirmcut_get_x(h, x)
    finally:
        P.pirmcut_destroy(h)
    assert np.array_equal(x, ref["x"])


@pytest.mark.parametrize("fmt", [0, 2])
def test_update_weights_on_a_device_built_problem(P, fmt):
    g = gen.config_graph(1, scale=48)
    cs = list(gen.capacity_sequence(g, 3, seed=9))
    eps = O.eps_schedule(5)
    res = []
    for host in (0, 1):
        with P.Solver(g, pcg_tol=1e-12, reduce_on_host=host, format=fmt) as s:
            out = []
            for cc in cs:
                s.update_weights(cc)
                s.solve(5, eps)
                out.append((s.get_x(), s.cut()[1]))
            res.append(out)
    for (xa, va), (xb, vb) in zip(*res):
        assert np.array_equal(xa, xb) and va == vb
    # a fresh context on the last capacities gives the same
    g3 = gen.Graph(g.n, g.row_ptr, g.col, cs[-1], g.s, g.t)
    fresh = run(P, g3, 0, fmt, T=5)
    assert np.array_equal(fresh["x"], res[0][-1][0])


def test_update_weights_that_drop_a_terminal_edge(P):
    """A capacity update that leaves a vertex without terminal capacity: the
    device reduction hands over to the host (solvability search)."""
    g = gen.config_graph(1, scale=20)
    c2 = g.c.copy()
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    v = 5
    c2[(rows == v) & ((g.col == g.s) | (g.col == g.t))] = 0.0
    c2[(g.col == v) & ((rows == g.s) | (rows == g.t))] = 0.0
    with P.Solver(g, pcg_tol=1e-12) as a, P.Solver(g, pcg_tol=1e-12, reduce_on_host=1) as b:
        for s in (a, b):
            s.update_weights(c2)
            s.solve(4, O.eps_schedule(4))
        assert np.array_equal(a.get_x(), b.get_x())


def test_two_level_on_a_device_built_problem(P):
    g = gen.config_graph(1)
    out = []
    for host in (0, 1):
        with P.Solver(g, pcg_tol=1e-12, reduce_on_host=host) as s:
            s.solve(20, O.eps_schedule(20))
            out.append(s.cut_two_level())
    assert out[0][1] == out[1][1] and np.array_equal(out[0][0], out[1][0])


def _bad_graphs():
    g = gen.config_graph(1, scale=8)
    bad_col = g.col.copy()
    bad_col[3] = g.n + 5
    neg = g.c.copy()
    neg[7] = -1.0
    asym = g.c.copy()
    asym[11] *= 2.0
    return [("column", gen.Graph(g.n, g.row_ptr, bad_col, g.c, g.s, g.t)),
            ("capacity", gen.Graph(g.n, g.row_ptr, g.col, neg, g.s, g.t)),
            ("symmetry", gen.Graph(g.n, g.row_ptr, g.col, asym, g.s, g.t))]


@pytest.mark.parametrize("name,g", _bad_graphs(), ids=lambda v: v if isinstance(v, str) else "")
def test_invalid_inputs_report_the_same_error(P, name, g):
    msgs = []
    for host in (0, 1):
        with pytest.raises(P.PirmcutError) as ei:
            P.Solver(g, reduce_on_host=host)
        msgs.append((ei.value.status, ei.value.message))
    assert msgs[0] == msgs[1]


@pytest.mark.parametrize("host", [0, 1])
@pytest.mark.parametrize("name,make", GRAPHS)
def test_float32_capacities_give_the_same_problem(P, name, make, host):
    """options.capacity_fp32: float capacities (host and device buffers) are
    widened exactly, so the solve equals the one from the doubles of equal
    value bit for bit; update_weights takes floats the same way."""
    import torch
    B = P.binding
    g = make()
    c32 = g.c.astype(np.float32)
    g64 = gen.Graph(g.n, g.row_ptr, g.col, c32.astype(np.float64), g.s, g.t)
    T = 4
    eps = O.eps_schedule(T)
    with P.Solver(g64, pcg_tol=1e-12, reduce_on_host=host) as ref:
        ref.solve(T, eps)
        x_ref = ref.get_x()
        cut_ref = ref.cut()[1]
    opt = B.pirmcut_default_options(pcg_tol=1e-12, reduce_on_host=host, capacity_fp32=1)
    with P.Solver(g, opt) as s:               # host float32 array
        s.solve(T, eps)
        assert np.array_equal(s.get_x(), x_ref)
        assert s.cut()[1] == cut_ref
        # new capacities as floats
        c2 = (g.c * np.exp(np.random.default_rng(3).normal(0, 0.01, g.c.shape[0]))).astype(np.float32)
        rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
        key = np.minimum(rows, g.col) * g.n + np.maximum(rows, g.col)
        _, first = np.unique(key, return_index=True)
        inv = np.unique(key, return_inverse=True)[1]
        c2 = c2[first][inv]                   # symmetric: both directions equal
        s.update_weights(c2)
        s.solve(T, eps)
        x2 = s.get_x()
    g2 = gen.Graph(g.n, g.row_ptr, g.col, c2.astype(np.float64), g.s, g.t)
    with P.Solver(g2, pcg_tol=1e-12, reduce_on_host=host) as ref2:
        ref2.solve(T, eps)
        assert np.array_equal(ref2.get_x(), x2)
    # device buffers
    d = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    h = B.pirmcut_create(g.n, d(g.row_ptr), d(g.col), d(c32), g.s, g.t, opt)
    try:
        B.pirmcut_solve(h, T, np.asarray(eps))
        x = np.empty(g.n)
        B.pirmcut_get_x(h, x)
        assert np.array_equal(x, x_ref)
    finally:
        B.pirmcut_destroy(h)
