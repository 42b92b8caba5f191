"""The allocation-free sweep cut (pirmcut_sweep_cut_static) against pirmcut_cut
and against the oracle's sweep cut (Section 3.3).

Some callers cannot call cudaMalloc: code running while a stream is captured
into a CUDA graph, frameworks that own all device memory through their own
pool, and real-time loops that must not block in the allocator.  For them the
library offers one sweep-cut entry point whose scratch is a fixed array in the
library's device memory.  These tests call it through the C ABI on device
buffers, twice in a row (the scratch array keeps the previous call's contents),
and compare its cut value, threshold and side with the context-based
pirmcut_cut on the same graph and voltages, and with the FP64 oracle's sweep
cut of those voltages, to the tolerances the other parity tests use (1e-9
relative on the value; the side identical on every vertex at least 1e-6 from
the threshold).  This file is collected last.
"""
import numpy as np
import pytest

import gen
import oracle as O

pytestmark = pytest.mark.gpu

CUT_RTOL = 1e-9


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import os
    from paper_1501_03105_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return torch, binding


def _graphs():
    g_perm = gen.random_graph(30, 0.15, 41, st_edge=True)
    g_perm = gen.permute_graph(g_perm, np.random.default_rng(2).permutation(g_perm.n))
    return [
        ("grid64", gen.config_graph(1)),
        ("chunglu", gen.chung_lu_instance(3000, 5)),
        ("random_st_inside", g_perm),
        ("vol10", gen.config_graph(3, scale=10)),
    ]


@pytest.mark.parametrize("name,g", _graphs())
@pytest.mark.parametrize("x_kind", ["irls", "ties"])
def test_static_sweep_matches_pirmcut_cut(env, name, g, x_kind):
    torch, B = env
    dev = torch.device("cuda")
    with B.Solver(g) as s:
        if x_kind == "irls":
            s.solve(10, [max(0.1 * 0.5 ** l, 1e-6) for l in range(10)])
            x = s.get_x()
        else:
            x = np.round(np.random.default_rng(g.n).random(g.n) * 8) / 8
            x[g.s], x[g.t] = 1.0, 0.0
            s.set_x(x)
        ref_side, ref_value, ref_tau = s.cut()
    prob = O.Problem.from_graph(g)
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    c = torch.from_numpy(g.c).to(dev)
    xd = torch.from_numpy(x).to(dev)
    for call in range(2):
        side = torch.full((g.n,), 7, dtype=torch.uint8, device=dev)
        result = torch.full((4,), np.nan, dtype=torch.float64, device=dev)
        B.pirmcut_sweep_cut_static(g.n, rp, col, c, g.s, g.t, xd, side, result,
                                   torch.cuda.current_stream())
        torch.cuda.synchronize()
        value, tau, k, bad = result.cpu().numpy()
        assert bad == 0.0, call
        assert abs(value - ref_value) <= CUT_RTOL * ref_value, (call, value, ref_value)
        assert abs(tau - ref_tau) <= 1e-15, (call, tau, ref_tau)
        assert np.array_equal(side.cpu().numpy(), ref_side), call
        # the oracle's sweep of the same voltages (prefix sums, vertex-id ties)
        ora = O.sweep_cut(prob, x)
        assert abs(value - ora["value"]) <= CUT_RTOL * ora["value"], (call, value, ora["value"])
        assert abs(tau - ora["tau"]) <= 1e-15, (call, tau, ora["tau"])
        assert int(k) == ora["k"], (call, k, ora["k"])
        far = np.abs(x - ora["tau"]) >= 1e-6
        far[[g.s, g.t]] = True
        assert np.array_equal(side.cpu().numpy().astype(bool)[far], ora["side"][far]), call


def test_static_sweep_rejects_oversized_input(env):
    torch, B = env
    dev = torch.device("cuda")
    n = B.STATIC_MAX_NONTERMINALS + 3
    z64 = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    z32 = torch.zeros(1, dtype=torch.int32, device=dev)
    zc = torch.zeros(1, dtype=torch.float64, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    side = torch.zeros(n, dtype=torch.uint8, device=dev)
    result = torch.zeros(4, dtype=torch.float64, device=dev)
    with pytest.raises(B.PirmcutError) as e:
        B.pirmcut_sweep_cut_static(n, z64, z32, zc, 0, 1, x, side, result)
    assert e.value.status == B.EINVAL
    assert str(B.STATIC_MAX_NONTERMINALS) in B.pirmcut_last_error(None)
