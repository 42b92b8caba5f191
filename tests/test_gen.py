"""The input generators: the direct (sort-free) CSR construction of the
segmentation grids equals the plain edge-list construction entry for entry."""
import numpy as np
import pytest

import gen
from gen.graphs import segmentation_grid, segmentation_grid_from_edges


@pytest.mark.parametrize("shape", [(5, 7), (1, 9), (16, 16), (4, 5, 6), (3, 1, 4), (8, 8, 8)])
def test_direct_segmentation_csr_equals_edge_list_build(shape):
    I = np.clip(np.random.default_rng(len(shape) * 100 + shape[0]).random(shape), 0, 1)
    I.reshape(-1)[::5] = 0.0                      # clipped pixels: zero terminal capacities
    a = segmentation_grid(I, name="x")
    b = segmentation_grid_from_edges(I, name="x")
    assert a.n == b.n and a.s == b.s and a.t == b.t
    assert np.array_equal(a.row_ptr, b.row_ptr)
    assert np.array_equal(a.col, b.col) and a.col.dtype == b.col.dtype
    assert np.array_equal(a.c, b.c)


def test_config_graphs_have_the_stated_sizes():
    g = gen.config_graph(2, scale=64)
    assert g.n == 64 * 64 + 2
    g = gen.config_graph(3, scale=16)
    assert g.n == 16 ** 3 + 2
    assert g.c.dtype == np.float64 and np.all(g.c == g.c.astype(np.float32))
