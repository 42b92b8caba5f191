"""Seeded graph generators (input data only; no IRLS arithmetic here).

Every generator returns a :class:`Graph`: an undirected graph stored as a full
symmetric CSR over all ``n`` vertices, terminals included, with both directions
of every edge present and carrying the same capacity.  Rows are sorted by
column.  Capacities are float64.

Workload recipes (the paper evaluates on N-D segmentation grids and
FlowImprove instances of road networks, Section 5.1 / Table 1; those datasets
are not available, so the synthetic recipes below stand in for them):

* 2-D segmentation grid: a W x H image ``I`` (background 0.3, disks at 0.7,
  Gaussian noise, clipped to [0, 1]); pixel p = x + W*y; 4-neighbour edges with
  c_pq = exp(-(I_p - I_q)^2 / (2 * 0.1^2)); terminal edges c_sp = 2*I_p and
  c_pt = 2*(1 - I_p); s = N, t = N + 1.
* 3-D segmentation volume: the same with an ellipsoid (0.65 inside, 0.35
  outside, noise 0.08) and 6-neighbour edges; p = x + W*y + W*H*z.
* Chung-Lu power-law instance in FlowImprove style (s tied to a BFS-grown
  seed set, t to the rest, weights proportional to weighted degree).
* Small random connected graphs for exhaustive checks.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Graph:
    """Full undirected graph in symmetric CSR form (terminals included)."""

    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray      # int32 [nnz]
    c: np.ndarray        # float64 [nnz]
    s: int
    t: int
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def edges(self):
        """Undirected edge list (u < v) with capacities, in CSR order of u."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))
        m = rows < self.col
        return rows[m], self.col[m].astype(np.int64), self.c[m]


def csr_from_edges(n: int, u, v, c) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Symmetric CSR (rows sorted by column) from an undirected edge list.

    Each undirected edge {u, v} is written in both rows with the same
    capacity. Duplicate pairs are kept as separate entries (callers that
    want them merged must merge first).
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    c = np.asarray(c, dtype=np.float64)
    rows = np.concatenate([u, v])
    cols = np.concatenate([v, u])
    vals = np.concatenate([c, c])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32), vals


# ----------------------------------------------------------------------------
# images
# ----------------------------------------------------------------------------

def image_disks_2d(W: int, H: int, disks, bg: float = 0.3,
                   fg: float = 0.7) -> np.ndarray:
    """Noise-free 2-D test image, shape (H, W).

    ``disks`` is a list of (cx, cy, r): pixel (x, y) is set to ``fg`` when
    (x - cx)^2 + (y - cy)^2 <= r^2 (pixel centres at integer coordinates,
    boundary inclusive); every other pixel is ``bg``.
    """
    I = np.full((H, W), bg, dtype=np.float64)
    yy, xx = np.mgrid[0:H, 0:W]
    for cx, cy, r in disks:
        I[(xx - cx) ** 2 + (yy - cy) ** 2 <= r * r] = fg
    return I


def _noisy(I: np.ndarray, rng: np.random.Generator, sigma: float) -> np.ndarray:
    """Add N(0, sigma) noise drawn in C (row-major) order, clip to [0, 1]."""
    I = I + rng.normal(0.0, sigma, size=I.shape)
    return np.clip(I, 0.0, 1.0)


def image_ellipsoid_3d(W: int, H: int, D: int, semi_axes, seed: int,
                       inside: float = 0.65, outside: float = 0.35,
                       noise: float = 0.08) -> np.ndarray:
    """Seeded 3-D volume, shape (D, H, W): a centred ellipsoid plus noise."""
    rng = np.random.default_rng(seed)
    a, b, cz = semi_axes
    z = (np.arange(D) - (D - 1) / 2.0)[:, None, None]
    y = (np.arange(H) - (H - 1) / 2.0)[None, :, None]
    x = (np.arange(W) - (W - 1) / 2.0)[None, None, :]
    inside_mask = (x / a) ** 2 + (y / b) ** 2 + (z / cz) ** 2 <= 1.0
    I = np.where(inside_mask, inside, outside).astype(np.float64)
    return _noisy(I, rng, noise)


def segmentation_grid(I: np.ndarray, sigma: float = 0.1, tscale: float = 2.0,
                      name: str = "") -> Graph:
    """4-connected (2-D) or 6-connected (3-D) segmentation graph of image I.

    Pixel p = x + W*y (+ W*H*z).  Neighbour capacity
    c_pq = exp(-(I_p - I_q)^2 / (2 sigma^2)); terminal capacities
    c_sp = tscale * I_p and c_pt = tscale * (1 - I_p); s = N, t = N + 1.
    Terminal edges whose capacity is 0 (clipped pixels) are still stored.

    The CSR is written row by row in column order without a sort: a pixel
    row lists its lower neighbours (largest stride first), its upper
    neighbours (smallest stride first), then s and t; rows s and t list every
    pixel.  Equal, entry for entry, to :func:`segmentation_grid_from_edges`.
    """
    shape = I.shape
    flat = I.reshape(-1)
    N = flat.shape[0]
    nd = I.ndim
    strides = [int(np.prod(shape[ax + 1:], dtype=np.int64)) for ax in range(nd)]
    p = np.arange(N, dtype=np.int64)
    coord = [(p // strides[ax]) % shape[ax] for ax in range(nd)]
    slots = []  # (valid, column) in column order
    for ax in range(nd):                      # p - stride, largest stride first
        slots.append((coord[ax] > 0, p - strides[ax]))
    for ax in reversed(range(nd)):            # p + stride, smallest stride first
        slots.append((coord[ax] < shape[ax] - 1, p + strides[ax]))
    k = len(slots) + 2
    valid = np.ones((N, k), dtype=bool)
    cols = np.empty((N, k), dtype=np.int32)
    caps = np.empty((N, k), dtype=np.float64)
    for j, (ok, q) in enumerate(slots):
        qq = np.where(ok, q, p)
        valid[:, j] = ok
        cols[:, j] = qq
        caps[:, j] = np.exp(-((flat - flat[qq]) ** 2) / (2.0 * sigma * sigma))
    cols[:, k - 2] = N
    caps[:, k - 2] = tscale * flat
    cols[:, k - 1] = N + 1
    caps[:, k - 1] = tscale * (1.0 - flat)
    counts = np.concatenate([valid.sum(axis=1), [N, N]]).astype(np.int64)
    row_ptr = np.zeros(N + 3, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    vm = valid.reshape(-1)
    col = np.concatenate([cols.reshape(-1)[vm], np.arange(N, dtype=np.int32),
                          np.arange(N, dtype=np.int32)])
    c = np.concatenate([caps.reshape(-1)[vm], tscale * flat, tscale * (1.0 - flat)])
    return Graph(N + 2, row_ptr, col, c, N, N + 1, name=name)


def segmentation_grid_from_edges(I: np.ndarray, sigma: float = 0.1, tscale: float = 2.0,
                                 name: str = "") -> Graph:
    """The graph of :func:`segmentation_grid` built from an edge list and a
    global sort (the plain construction; kept to check the direct one).

    Pixel p = x + W*y (+ W*H*z).  Neighbour capacity
    c_pq = exp(-(I_p - I_q)^2 / (2 sigma^2)); terminal capacities
    c_sp = tscale * I_p and c_pt = tscale * (1 - I_p); s = N, t = N + 1.
    Terminal edges whose capacity is 0 (clipped pixels) are still stored.
    """
    flat = I.reshape(-1)
    N = flat.shape[0]
    us, vs = [], []
    idx = np.arange(N, dtype=np.int64).reshape(I.shape)
    # neighbour pairs along each axis (last axis = x, stride 1)
    for ax in range(I.ndim):
        sl_a = [slice(None)] * I.ndim
        sl_b = [slice(None)] * I.ndim
        sl_a[ax] = slice(0, -1)
        sl_b[ax] = slice(1, None)
        us.append(idx[tuple(sl_a)].reshape(-1))
        vs.append(idx[tuple(sl_b)].reshape(-1))
    u = np.concatenate(us)
    v = np.concatenate(vs)
    cpq = np.exp(-((flat[u] - flat[v]) ** 2) / (2.0 * sigma * sigma))
    s, t = N, N + 1
    pix = np.arange(N, dtype=np.int64)
    u_all = np.concatenate([u, pix, pix])
    v_all = np.concatenate([v, np.full(N, s, np.int64), np.full(N, t, np.int64)])
    c_all = np.concatenate([cpq, tscale * flat, tscale * (1.0 - flat)])
    row_ptr, col, c = csr_from_edges(N + 2, u_all, v_all, c_all)
    return Graph(N + 2, row_ptr, col, c, s, t, name=name)


# ----------------------------------------------------------------------------
# small random graphs (exhaustive checks) and power-law instances
# ----------------------------------------------------------------------------

def random_graph(n_nt: int, p_edge: float, seed: int, p_term: float = 0.5,
                 cmin: float = 0.5, cmax: float = 1.5, st_edge: bool = False,
                 zero_frac: float = 0.0) -> Graph:
    """Random connected graph with ``n_nt`` non-terminals plus s and t.

    Non-terminals are 0..n_nt-1, s = n_nt, t = n_nt + 1.  A random spanning
    path over the non-terminals keeps the non-terminal graph connected; other
    pairs are edges with probability ``p_edge``.  Each non-terminal is tied to
    s and/or t with probability ``p_term`` each, and vertex 0 is always tied to
    s and vertex n_nt-1 to t so both terminals are reached.  Capacities are
    U[cmin, cmax]; a fraction ``zero_frac`` of terminal capacities is set to 0.
    """
    rng = np.random.default_rng(seed)
    n = n_nt + 2
    s, t = n_nt, n_nt + 1
    perm = rng.permutation(n_nt)
    pairs = set()
    for a, b in zip(perm[:-1], perm[1:]):
        pairs.add((min(a, b), max(a, b)))
    for a in range(n_nt):
        for b in range(a + 1, n_nt):
            if rng.random() < p_edge:
                pairs.add((a, b))
    u = [p[0] for p in sorted(pairs)]
    v = [p[1] for p in sorted(pairs)]
    c = list(rng.uniform(cmin, cmax, len(u)))
    tu, tv, tc = [], [], []
    for a in range(n_nt):
        for term in (s, t):
            forced = (a == 0 and term == s) or (a == n_nt - 1 and term == t)
            if forced or rng.random() < p_term:
                w = rng.uniform(cmin, cmax)
                if not forced and rng.random() < zero_frac:
                    w = 0.0
                tu.append(a)
                tv.append(term)
                tc.append(w)
    if st_edge:
        tu.append(s)
        tv.append(t)
        tc.append(rng.uniform(cmin, cmax))
    row_ptr, col, cc = csr_from_edges(n, u + tu, v + tv, c + tc)
    return Graph(n, row_ptr, col, cc, s, t, name=f"random{n_nt}_{seed}")


def chung_lu_instance(n: int, seed: int, exponent: float = 2.5,
                      avg_degree: float = 10.0, seed_frac: float = 0.05,
                      s_scale: float = 1.0, t_scale: float = 0.05,
                      cmin: float = 0.5, cmax: float = 1.5, float32_caps: bool = False) -> Graph:
    """FlowImprove-style instance on a Chung-Lu power-law graph.

    Expected degrees w_i proportional to (i + 1)^(-1/(exponent-1)), scaled to
    mean ``avg_degree``; edge {i, j} is drawn with probability
    min(1, w_i w_j / sum(w)) via a per-vertex Bernoulli sweep (sampled as a
    Poisson number of endpoint draws, duplicates and self-loops removed).
    The largest connected component is kept and relabelled.  Edge capacities
    are U[cmin, cmax] (rounded to float32 when ``float32_caps``).  A seed set
    is grown by BFS from a random vertex (neighbours in index order, the
    vertex count taken over the kept component) until ceil(seed_frac * n)
    vertices; s ties to
    every seed vertex with capacity s_scale * d_v and t ties to every other
    vertex with capacity t_scale * d_v, d_v being the weighted degree.
    """
    rng = np.random.default_rng(seed)
    w = (np.arange(n) + 1.0) ** (-1.0 / (exponent - 1.0))
    w *= avg_degree / w.mean()
    S = w.sum()
    m_exp = int(round(S / 2))
    prob = w / S
    a = rng.choice(n, size=m_exp, p=prob)
    b = rng.choice(n, size=m_exp, p=prob)
    keep = a != b
    a, b = a[keep], b[keep]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key = np.unique(lo.astype(np.int64) * n + hi)
    u, v = key // n, key % n
    # largest connected component
    import scipy.sparse as sp
    import scipy.sparse.csgraph as csg
    adj = sp.csr_matrix((np.ones(u.shape[0]), (u, v)), shape=(n, n))
    ncomp, lab = csg.connected_components(adj, directed=False)
    big = np.bincount(lab).argmax()
    keepv = np.nonzero(lab == big)[0]
    relabel = -np.ones(n, dtype=np.int64)
    relabel[keepv] = np.arange(keepv.shape[0])
    ke = (relabel[u] >= 0) & (relabel[v] >= 0)
    u, v = relabel[u[ke]], relabel[v[ke]]
    nn = keepv.shape[0]
    cap = rng.uniform(cmin, cmax, u.shape[0])
    if float32_caps:
        cap = cap.astype(np.float32).astype(np.float64)
    deg = np.bincount(u, weights=cap, minlength=nn) + np.bincount(v, weights=cap, minlength=nn)
    rp, cl, _ = csr_from_edges(nn, u, v, cap)
    start = int(rng.integers(nn))
    want = int(np.ceil(seed_frac * nn))
    # BFS order from the start vertex, neighbours in index order
    sym = sp.csr_matrix((np.ones(cl.shape[0]), cl, rp), shape=(nn, nn))
    order = csg.breadth_first_order(sym, start, directed=False, return_predecessors=False)[:want]
    in_seed = np.zeros(nn, dtype=bool)
    in_seed[order] = True
    s, t = nn, nn + 1
    pix = np.arange(nn, dtype=np.int64)
    seedv, rest = pix[in_seed], pix[~in_seed]
    u_all = np.concatenate([u, seedv, rest])
    v_all = np.concatenate([v, np.full(seedv.shape[0], s, np.int64),
                            np.full(rest.shape[0], t, np.int64)])
    c_all = np.concatenate([cap, s_scale * deg[seedv], t_scale * deg[rest]])
    row_ptr, col, c = csr_from_edges(nn + 2, u_all, v_all, c_all)
    return Graph(nn + 2, row_ptr, col, c, s, t, name=f"chunglu{n}_{seed}")


def chung_lu_batch(count: int = 64, seed: int = 4, nmin: float = 1e4, nmax: float = 1e6,
                   **kw) -> list:
    """``count`` Chung-Lu FlowImprove-style instances with sizes n_i drawn
    log-uniformly in [nmin, nmax] (rounded), instance i seeded with seed*1000+i,
    float32 capacities."""
    rng = np.random.default_rng(seed)
    sizes = np.round(10.0 ** rng.uniform(np.log10(nmin), np.log10(nmax), count)).astype(np.int64)
    return [chung_lu_instance(int(sizes[i]), seed * 1000 + i, float32_caps=True, **kw)
            for i in range(count)]


def perturb_capacities(g: Graph, seed: int, sigma: float = 0.01) -> Graph:
    """Multiply every undirected capacity by exp(N(0, sigma)) (same structure).

    Both stored directions of an edge get the same factor.
    """
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    lo = np.minimum(rows, g.col.astype(np.int64))
    hi = np.maximum(rows, g.col.astype(np.int64))
    key = lo * g.n + hi
    uk, inv = np.unique(key, return_inverse=True)
    f = np.exp(rng.normal(0.0, sigma, uk.shape[0]))
    return Graph(g.n, g.row_ptr.copy(), g.col.copy(), g.c * f[inv], g.s, g.t, g.name + "+p")


def capacity_sequence(g: Graph, count: int, seed: int, sigma: float = 0.01):
    """Capacity arrays of a sequence of ``count`` related problems on the
    structure of ``g``: problem 0 has g's capacities and problem k+1
    multiplies every undirected capacity of problem k by exp(N(0, sigma))
    (both stored directions by the same factor).  Yields float64 arrays in
    g's CSR order; the edge pairing is computed once."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    lo = np.minimum(rows, g.col.astype(np.int64))
    hi = np.maximum(rows, g.col.astype(np.int64))
    uk, inv = np.unique(lo * g.n + hi, return_inverse=True)
    rng = np.random.default_rng(seed)
    c = g.c.astype(np.float64).copy()
    for k in range(count):
        if k > 0:
            c = c * np.exp(rng.normal(0.0, sigma, uk.shape[0]))[inv]
        yield c


def permute_graph(g: Graph, perm: np.ndarray) -> Graph:
    """Relabel vertex v as perm[v]; returns a new sorted CSR."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    m = rows < g.col
    u = perm[rows[m]]
    v = perm[g.col[m].astype(np.int64)]
    rp, cl, cc = csr_from_edges(g.n, u, v, g.c[m])
    return Graph(g.n, rp, cl, cc, int(perm[g.s]), int(perm[g.t]), g.name + "+perm")


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

CONFIGS = {
    1: "grid64: 64x64 4-connected segmentation grid, one disk, T=50",
    2: "grid2048: 2048x2048 4-connected segmentation grid, 12 disks, T=50",
    3: "vol256: 256^3 6-connected segmentation volume, ellipsoid, float32 capacities, T=30",
    5: "vol128: 128^3 6-connected segmentation volume (sequence base), float32 capacities, T=30",
}


def config_graph(k: int, scale: int | None = None) -> Graph:
    """Graph of workload ``k`` (seed = k).  ``scale`` shrinks the side length
    (same recipe, smaller image) for tests that need a quick case."""
    if k == 1:
        W = scale or 64
        I = image_disks_2d(W, W, [(W // 2, W // 2, W // 4)])
        I = _noisy(I, np.random.default_rng(1), 0.05)
        return segmentation_grid(I, name=f"grid{W}")
    if k == 2:
        W = scale or 2048
        rng = np.random.default_rng(2)
        cx = rng.uniform(0, W, 12)
        cy = rng.uniform(0, W, 12)
        r = rng.uniform(32, 256, 12) * (W / 2048.0)
        I = image_disks_2d(W, W, list(zip(cx, cy, r)))
        I = _noisy(I, rng, 0.05)
        return segmentation_grid(I, name=f"grid{W}")
    if k in (3, 5):
        # capacities stored as float32 values (widened back to float64)
        W = scale or (256 if k == 3 else 128)
        f = W / 256.0
        I = image_ellipsoid_3d(W, W, W, (96 * f, 80 * f, 64 * f), seed=k)
        g = segmentation_grid(I, name=f"vol{W}")
        g.c = g.c.astype(np.float32).astype(np.float64)
        return g
    raise ValueError(f"unknown workload {k}")
