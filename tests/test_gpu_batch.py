"""Batched solves (one launch per kernel for all instances) against
single-instance contexts and the FP64 oracle."""
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
    import os
    import paper_1501_03105_gb300 as pkg
    from paper_1501_03105_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return pkg


def star_graph(k, seed):
    """A hub joined to k leaves (hub degree > the heavy-row threshold) plus a
    ring through the leaves; s tied to the hub, t to every leaf."""
    rng = np.random.default_rng(seed)
    hub = 0
    leaves = np.arange(1, k + 1)
    s, t = k + 1, k + 2
    u = list(np.zeros(k, dtype=int)) + list(leaves) + [hub] + list(leaves)
    v = list(leaves) + list(np.roll(leaves, 1)) + [s] + [t] * k
    c = list(rng.uniform(0.5, 1.5, len(u)))
    rp, col, cc = gen.csr_from_edges(k + 3, u, v, c)
    return gen.Graph(k + 3, rp, col, cc, s, t, name=f"star{k}")


def batch_graphs():
    return [gen.chung_lu_instance(3000, 11, float32_caps=True),
            gen.config_graph(1, scale=20),
            gen.random_graph(15, 0.3, 5, st_edge=True),
            star_graph(1500, 3),
            gen.chung_lu_instance(800, 12, float32_caps=True),
            gen.Graph(3, *gen.csr_from_edges(3, [0, 1], [1, 2], [2.0, 1.0]), 0, 2)]


# (threads per short row, rows per range tile, warp-row threshold); None:
# the autotuner's choice.  The star's hub (1500 entries) is a block row in
# every case; thresholds 4 and 16 send many Chung-Lu rows to the warp tier,
# 512 turns it off.
TILINGS = [None, (2, 512, 16), (1, 64, 4), (4, 2048, 512), (32, 512, 32)]


@pytest.mark.parametrize("tiling", TILINGS, ids=lambda t: "auto" if t is None else "g%d-t%d-m%d" % t)
def test_batch_matches_single_contexts_and_oracle(P, tiling):
    graphs = batch_graphs()
    T = 15
    eps = O.eps_schedule(T)
    kw = {} if tiling is None else dict(batch_threads_per_row=tiling[0], batch_tile_rows=tiling[1],
                                        batch_medium_deg=tiling[2])
    with P.Batch(graphs, pcg_tol=1e-13, **kw) as b:
        info = b.info()
        assert info["rows"] == sum(g.n - 2 for g in graphs)
        assert info["threads_per_row"] in (1, 2, 4, 8, 16, 32)
        assert 1 <= info["medium_deg"] <= 512
        if tiling is not None:
            assert (info["threads_per_row"], info["tile_rows"], info["medium_deg"]) == tiling
        infos = b.solve(T, eps)
        xs_b = [b.get_x(i) for i in range(len(graphs))]
        cuts_b = [b.cut(i) for i in range(len(graphs))]
        assert b.kernel_launches() > 0
    iters = [sum(i.pcg_iters for i in inf) for inf in infos]
    assert len(set(iters)) > 1                        # instances converge independently
    for i, g in enumerate(graphs):
        assert all(x.status == 0 for x in infos[i]), g.name
        with P.Solver(g, pcg_tol=1e-13, format=2) as s:
            s.solve(T, eps)
            xs = s.get_x()
            side, value, tau = s.cut()
        assert np.max(np.abs(xs_b[i] - xs)) <= 1e-9, g.name
        sb, vb, tb = cuts_b[i]
        assert abs(vb - value) <= 1e-9 * max(value, 1e-300), g.name
        if abs(tb - tau) < 1e-12:
            assert np.array_equal(sb, side), g.name
        if g.n < 5000:
            prob = O.Problem.from_graph(g)
            xo, _ = O.irls(prob, T, eps)
            assert np.max(np.abs(xs_b[i] - xo[-1])) <= 1e-9, g.name


def test_batch_single_instance_and_repeat(P):
    g = gen.chung_lu_instance(2000, 21, float32_caps=True)
    eps = O.eps_schedule(8)
    with P.Batch([g]) as b:
        a1 = b.solve(8, eps)
        x1 = b.get_x(0)
        a2 = b.solve(8, eps)
        x2 = b.get_x(0)
    assert np.array_equal(x1, x2)                      # deterministic
    assert [i.pcg_iters for i in a1[0]] == [i.pcg_iters for i in a2[0]]


def test_batch_stream_launch_matches_graph_launch(P):
    """graph_launch = 0 runs the same kernels from the host (chunks of 8
    iterations): bit-identical iterates, iteration counts and cuts."""
    graphs = [gen.chung_lu_instance(1500, 31, float32_caps=True), gen.config_graph(1, scale=18),
              gen.random_graph(30, 0.2, 4)]
    T = 6
    eps = O.eps_schedule(T)
    out = []
    for mode in (1, 0):
        with P.Batch(graphs, pcg_tol=1e-12, graph_launch=mode, batch_threads_per_row=2,
                     batch_tile_rows=512, batch_medium_deg=16) as b:
            infos = b.solve(T, eps)
            out.append(([b.get_x(i) for i in range(len(graphs))],
                        [[x.pcg_iters for x in inf] for inf in infos],
                        [b.cut(i)[1] for i in range(len(graphs))]))
    for xa, xb in zip(out[0][0], out[1][0]):
        assert np.array_equal(xa, xb)
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]


def test_batch_rejects_bad_tiling_options(P):
    from paper_1501_03105_gb300 import binding as B
    g = gen.random_graph(10, 0.3, 1)
    for kw in (dict(batch_threads_per_row=3), dict(batch_tile_rows=32), dict(batch_medium_deg=513),
               dict(batch_medium_deg=-1)):
        with pytest.raises(B.PirmcutError) as e:
            P.Batch([g], **kw)
        assert e.value.status == B.EINVAL, kw


def test_batch_reports_bad_instance(P):
    from paper_1501_03105_gb300 import binding as B
    good = gen.random_graph(10, 0.3, 1)
    rp, col, c = gen.csr_from_edges(5, [0, 1, 3], [1, 2, 4], [1.0, 1.0, 1.0])
    bad = gen.Graph(5, rp, col, c, 0, 2)
    with pytest.raises(B.PirmcutError) as e:
        P.Batch([good, bad])
    assert e.value.status == B.EDISCONNECTED and "instance 1" in str(e.value)
