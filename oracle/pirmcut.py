"""FP64 CPU oracle of the PIRMCut IRLS hot path (Zhu & Gleich, arXiv:1501.03105).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``, never by the product path.  It shares
no code with the CUDA library.

Everything here is written the slow and literal way: the incidence matrix B,
the capacity matrix C and the reweighting matrix W are formed explicitly, the
reweighted Laplacian is the sparse product B^T C W^-1 C B, and the reduced
system is obtained by deleting rows and columns with the null basis Z.  Library
primitives used as single steps: sparse matrix products, a sparse direct solve
(SuperLU), a stable sort and a cumulative sum.

Readings of points the paper leaves open (each one is also listed in the
design notes of the repository):

* reweighting form: the default ``WEIGHTED_L1`` form gives edge e the
  conductance g_e = c_e / sqrt(d_e^2 + eps^2), d = B x.  The ``PAPER`` form is
  the literal Eq. (define-reweight-vector) + Eq. (reweighted-laplacian):
  w_e = sqrt((C B x)_e^2 + eps^2) and g_e = c_e^2 / w_e.
* x^(0) solves the WLS with W^(0) = C (Section 2.1, after Prop. 2), i.e.
  g = c, for both forms; a zero capacity gives a zero conductance.
* eps schedule for a run of T steps: eps_l = max(1e-1 * 2^-(l-1), 1e-6).
* PCG stops when ||b - A x||_2 <= tol * ||b||_2 (unpreconditioned residual,
  relative to b).
* sweep cut: vertices sorted by x descending, vertex index ascending on ties;
  only prefixes that end between two strictly different x values are
  candidates, plus the empty and the full prefix; the smallest cut value wins
  and, among exactly equal values, the shortest prefix.

Parity status: x^(0), one IRLS step, the reduced system, the sweep cut, the cut
value and the exact references are pinned by closed forms, invariants and
brute force (see ``tests/test_oracle_*.py``).  Later-step iterates on the large
synthetic workloads have no independent pin beyond the invariants
(maximum principle, electrical-flow conservation, monotone objective).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph
import scipy.sparse.linalg as spla

WEIGHTED_L1 = 0
PAPER = 1


class Problem:
    """An undirected s-t min-cut instance (Section 2).

    Input: a full symmetric CSR over all n vertices (terminals included), both
    directions of each edge stored with the same capacity, no self-loops,
    capacities finite and >= 0, s != t.  Parallel entries of one pair are
    summed.  Raises ``ValueError`` on invalid input and when some connected
    component of the positive-capacity graph holds non-terminals but neither
    terminal (the reduced Laplacian would be singular, Prop. (nonsingular)).
    """

    def __init__(self, n, row_ptr, col, c, s, t):
        n = int(n)
        row_ptr = np.asarray(row_ptr, dtype=np.int64)
        col = np.asarray(col, dtype=np.int64)
        c = np.asarray(c, dtype=np.float64)
        s, t = int(s), int(t)
        if n < 2 or row_ptr.shape != (n + 1,) or row_ptr[0] != 0:
            raise ValueError("bad row_ptr")
        if np.any(np.diff(row_ptr) < 0) or row_ptr[-1] != col.shape[0]:
            raise ValueError("bad row_ptr")
        if col.shape != c.shape:
            raise ValueError("col/c length mismatch")
        if not (0 <= s < n and 0 <= t < n) or s == t:
            raise ValueError("bad terminals")
        if np.any((col < 0) | (col >= n)):
            raise ValueError("column out of range")
        if not np.all(np.isfinite(c)) or np.any(c < 0):
            raise ValueError("capacities must be finite and >= 0")
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
        if np.any(rows == col):
            raise ValueError("self-loop")
        # group entries by vertex pair, summing parallel entries; keep pairs
        # whose capacity is zero (they are part of the structure)
        up = rows < col
        key_up = rows[up] * n + col[up]
        key_lo = col[~up] * n + rows[~up]
        ku, inv_u = np.unique(key_up, return_inverse=True)
        kl, inv_l = np.unique(key_lo, return_inverse=True)
        cu = np.bincount(inv_u, weights=c[up], minlength=ku.shape[0])
        cl = np.bincount(inv_l, weights=c[~up], minlength=kl.shape[0])
        # symmetric: both directions list the same pairs with the same total capacity
        if ku.shape != kl.shape or np.any(ku != kl) or np.any(cu != cl):
            raise ValueError("CSR is not symmetric")
        self.n = n
        self.s = s
        self.t = t
        self.eu = ku // n
        self.ev = ku % n
        self.cap = cu.astype(np.float64)
        m = self.eu.shape[0]
        self.m = m
        # B: m x n incidence matrix, orientation u -> v (+1 at u, -1 at v)  [Section 2]
        ar = np.arange(m)
        self.B = sp.csr_matrix(
            (np.concatenate([np.ones(m), -np.ones(m)]),
             (np.concatenate([ar, ar]), np.concatenate([self.eu, self.ev]))),
            shape=(m, n))
        # C = diag(c)
        self.C = sp.diags(self.cap)
        # Z: the identity I_n with its s and t columns deleted  [Section 2.1, Prop. 3]
        keep = np.ones(n, dtype=bool)
        keep[[s, t]] = False
        self.nonterminals = np.nonzero(keep)[0].astype(np.int64)
        nn = self.nonterminals.shape[0]
        self.nt = nn
        self.Z = sp.csr_matrix((np.ones(nn), (self.nonterminals, np.arange(nn))), shape=(n, nn))
        self.e_s = np.zeros(n)
        self.e_s[s] = 1.0
        self._check_solvable()

    def _check_solvable(self):
        pos = self.cap > 0
        A = sp.csr_matrix((np.ones(int(pos.sum())), (self.eu[pos], self.ev[pos])),
                          shape=(self.n, self.n))
        ncomp, lab = csgraph.connected_components(A, directed=False)
        ok = np.zeros(ncomp, dtype=bool)
        ok[lab[self.s]] = True
        ok[lab[self.t]] = True
        if not np.all(ok[lab[self.nonterminals]]):
            raise ValueError("disconnected: a non-terminal component reaches neither s nor t")

    @classmethod
    def from_graph(cls, g):
        return cls(g.n, g.row_ptr, g.col, g.c, g.s, g.t)

    def full_x(self, v):
        """x = Z v + e_s: the full voltage vector with x_s = 1, x_t = 0."""
        return self.Z @ v + self.e_s


def eps_schedule(T: int, eps0: float = 1e-1, eps_min: float = 1e-6):
    """eps_l = max(eps0 * 2^-(l-1), eps_min) for l = 1..T (halving schedule)."""
    return [max(eps0 * 0.5 ** (l - 1), eps_min) for l in range(1, T + 1)]


def initial_conductance(prob: Problem) -> np.ndarray:
    """Conductances of the first WLS, W^(0) = C (Section 2.1): C W^-1 C = C."""
    return prob.cap.copy()


def reweight(prob: Problem, x: np.ndarray, eps: float, form: int = WEIGHTED_L1) -> np.ndarray:
    """Per-edge conductance of the next WLS (Step 1, Eq. define-reweight-vector).

    PAPER form: w = sqrt((C B x)^2 + eps^2) and the Laplacian weight is the
    diagonal of C W^-1 C (Eq. reweighted-laplacian), i.e. c^2 / w.
    WEIGHTED_L1 form: c / sqrt((B x)^2 + eps^2).
    """
    d = prob.B @ x
    if form == PAPER:
        w = np.sqrt((prob.cap * d) ** 2 + eps ** 2)
        return prob.cap * prob.cap / w
    if form == WEIGHTED_L1:
        return prob.cap / np.sqrt(d ** 2 + eps ** 2)
    raise ValueError("unknown reweighting form")


def laplacian(prob: Problem, g: np.ndarray) -> sp.csr_matrix:
    """Reweighted Laplacian L = B^T diag(g) B (Eq. reweighted-laplacian)."""
    return (prob.B.T @ sp.diags(g) @ prob.B).tocsr()


def reduced_system(prob: Problem, L: sp.csr_matrix):
    """Reduced Laplacian system (Eq. reduced-laplacian-system).

    Returns (Ltilde, b) with Ltilde = Z^T L Z and b = -Z^T L e_s.
    """
    Lt = (prob.Z.T @ L @ prob.Z).tocsr()
    b = -(prob.Z.T @ (L @ prob.e_s))
    return Lt, b


def solve_direct(Lt: sp.csr_matrix, b: np.ndarray) -> np.ndarray:
    """Exact (to rounding) solution of Ltilde v = b by a sparse LU solve."""
    return spla.spsolve(Lt.tocsc(), b)


def pcg_jacobi(A, b, x0=None, tol=1e-10, maxit=20000):
    """Preconditioned conjugate gradient with M = diag(A) (Section 3.1).

    Follows the textbook PCG recurrence: alpha = (r, z) / (A p, p),
    x += alpha p, r -= alpha A p, z = M^-1 r, beta = (r_new, z_new) / (r, z),
    p = z + beta p.  Stops when ||r||_2 <= tol * ||b||_2 (checked on entry
    too, so a warm start that already satisfies it costs no iteration) or
    after ``maxit`` iterations.  Returns (x, iterations, ||r||/||b||).
    """
    A = A.tocsr()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    dinv = 1.0 / A.diagonal()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    r = b - A @ x
    if np.linalg.norm(r) <= tol * bnorm:
        return x, 0, np.linalg.norm(r) / bnorm
    z = dinv * r
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxit:
        q = A @ p
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rnorm = np.linalg.norm(r)
        if rnorm <= tol * bnorm:
            break
        z = dinv * r
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, it, np.linalg.norm(r) / bnorm


def wls_step(prob: Problem, g: np.ndarray, solver: str = "direct", v0=None,
             tol: float = 1e-12, maxit: int = 1000000):
    """Step 2 (Eq. constrained-wls) with conductances g, via the reduced system.

    Returns (x, info) with x the full voltage vector (x_s = 1, x_t = 0).
    """
    L = laplacian(prob, g)
    Lt, b = reduced_system(prob, L)
    info = {}
    if solver == "direct":
        v = solve_direct(Lt, b)
    elif solver == "pcg":
        v, it, rel = pcg_jacobi(Lt, b, v0, tol, maxit)
        info.update(pcg_iters=it, rel_residual=rel)
    elif solver == "pcg_omp":
        # the same recurrence written out in C, over every host core
        from .pcg_omp import pcg_jacobi as pcg_jacobi_omp
        v, it, rel = pcg_jacobi_omp(Lt, b, v0, tol, maxit)
        info.update(pcg_iters=it, rel_residual=rel)
    else:
        raise ValueError(solver)
    x = prob.full_x(v)
    return x, info


def irls(prob: Problem, T: int, eps=None, form: int = WEIGHTED_L1, solver: str = "direct",
         tol: float = 1e-12, maxit: int = 1000000, warm_start: bool = True):
    """The IRLS loop (Section 2.1 and Algorithm 1, rounding excluded).

    x^(0) solves the WLS with W^(0) = C; then for l = 1..T the conductances
    are reweighted from x^(l-1) with eps_l and the WLS is solved again.
    Returns (xs, infos): xs[l] is x^(l) for l = 0..T.
    """
    if eps is None:
        eps = eps_schedule(T)
    eps = list(eps)
    if len(eps) != T:
        raise ValueError("need one eps per step")
    g = initial_conductance(prob)
    x, info = wls_step(prob, g, solver, None, tol, maxit)
    xs, infos = [x], [info]
    for l in range(1, T + 1):
        g = reweight(prob, xs[-1], eps[l - 1], form)
        v0 = xs[-1][prob.nonterminals] if warm_start else None
        x, info = wls_step(prob, g, solver, v0, tol, maxit)
        info["eps"] = eps[l - 1]
        xs.append(x)
        infos.append(info)
    return xs, infos


def smoothed_objective(prob: Problem, x: np.ndarray, eps: float, form: int = WEIGHTED_L1) -> float:
    """Smoothed l1 objective (Eq. l1-min-smooth-version).

    PAPER: sum_e sqrt((C B x)_e^2 + eps^2).  WEIGHTED_L1: sum_e c_e sqrt((B x)_e^2 + eps^2),
    the function whose majorise-minimise iteration is the WEIGHTED_L1 reweighting.
    """
    d = prob.B @ x
    if form == PAPER:
        return float(np.sum(np.sqrt((prob.cap * d) ** 2 + eps ** 2)))
    return float(np.sum(prob.cap * np.sqrt(d ** 2 + eps ** 2)))


def flow_value(prob: Problem, x: np.ndarray, g: np.ndarray) -> float:
    """Electrical flow value x^T L x of the WLS solution (Prop. wls-equal-electrical-flow)."""
    L = laplacian(prob, g)
    return float(x @ (L @ x))


def cut_value(prob: Problem, side: np.ndarray) -> float:
    """cut(S, S-bar): total capacity of edges with one end in S (Section 2).

    ``side`` is a boolean vector over all n vertices, True on S (s in S, t not).
    """
    side = np.asarray(side, dtype=bool)
    if not side[prob.s] or side[prob.t]:
        raise ValueError("side must hold s and not t")
    crossing = side[prob.eu] != side[prob.ev]
    return float(np.sum(prob.cap[crossing]))


def _sweep_order(prob: Problem, x: np.ndarray) -> np.ndarray:
    """Non-terminals ordered by x descending, vertex index ascending on ties."""
    v = prob.nonterminals
    return v[np.lexsort((v, -x[v]))]


def _candidates(xs_sorted: np.ndarray) -> np.ndarray:
    """Prefix lengths k that end between strictly different x values, plus 0 and n~."""
    nn = xs_sorted.shape[0]
    ks = [0]
    for k in range(1, nn):
        if xs_sorted[k - 1] > xs_sorted[k]:
            ks.append(k)
    if nn > 0:
        ks.append(nn)
    return np.array(ks, dtype=np.int64)


def _threshold(xs_sorted: np.ndarray, k: int) -> float:
    """tau = (x_(k) + x_(k+1)) / 2 with x_(0) = 1 and x_(n~+1) = 0 (1-based ranks)."""
    nn = xs_sorted.shape[0]
    hi = 1.0 if k == 0 else xs_sorted[k - 1]
    lo = 0.0 if k == nn else xs_sorted[k]
    return 0.5 * (hi + lo)


def sweep_cut_by_definition(prob: Problem, x: np.ndarray):
    """Sweep cut (Section 3.3) with every candidate prefix evaluated by the
    cut definition.  O(n~ m): for small graphs and for pinning ``sweep_cut``.

    Returns dict(value, side, k, tau, order).
    """
    order = _sweep_order(prob, x)
    xs_sorted = x[order]
    best = None
    for k in _candidates(xs_sorted):
        side = np.zeros(prob.n, dtype=bool)
        side[prob.s] = True
        side[order[:k]] = True
        val = cut_value(prob, side)
        if best is None or val < best[0]:
            best = (val, int(k), side)
    val, k, side = best
    return dict(value=val, side=side, k=k, tau=_threshold(xs_sorted, k), order=order)


def sweep_cut(prob: Problem, x: np.ndarray):
    """Sweep cut (Section 3.3) by prefix sums.

    Moving vertex v from the sink side to the source side changes the cut by
    delta_v = c(v,t) - c(s,v) + sum_{u after v} c(u,v) - sum_{u before v} c(u,v)
    (u over non-terminal neighbours, "before" = earlier in the sweep order).
    cut(0) = sum_v c(s,v) + c(s,t); cut(k) = cut(0) + sum_{i<k} delta_(i).
    The chosen prefix's value is then recomputed by the cut definition.
    Returns dict(value, prefix_value, side, k, tau, order).
    """
    order = _sweep_order(prob, x)
    nn = order.shape[0]
    rank = np.full(prob.n, -1, dtype=np.int64)
    rank[order] = np.arange(nn)
    s, t = prob.s, prob.t
    eu, ev, cap = prob.eu, prob.ev, prob.cap
    st = ((eu == s) & (ev == t)) | ((eu == t) & (ev == s))
    to_s = ((eu == s) | (ev == s)) & ~st
    to_t = ((eu == t) | (ev == t)) & ~st
    inner = ~(st | to_s | to_t)
    delta = np.zeros(prob.n)
    # terminal edges: s-v stops being cut when v joins, v-t starts being cut
    ws = np.where(eu[to_s] == s, ev[to_s], eu[to_s])
    wt = np.where(eu[to_t] == t, ev[to_t], eu[to_t])
    np.add.at(delta, ws, -cap[to_s])
    np.add.at(delta, wt, cap[to_t])
    cut0 = float(np.sum(cap[to_s]) + np.sum(cap[st]))
    # non-terminal edges: cut while exactly one end has joined
    u, v, c = eu[inner], ev[inner], cap[inner]
    first = np.where(rank[u] < rank[v], u, v)
    second = np.where(rank[u] < rank[v], v, u)
    np.add.at(delta, first, c)
    np.add.at(delta, second, -c)
    prefix = np.concatenate([[cut0], cut0 + np.cumsum(delta[order])])
    xs_sorted = x[order]
    ks = _candidates(xs_sorted)
    vals = prefix[ks]
    j = int(np.argmin(vals))          # first minimum: shortest prefix on exact ties
    k = int(ks[j])
    side = np.zeros(prob.n, dtype=bool)
    side[s] = True
    side[order[:k]] = True
    return dict(value=cut_value(prob, side), prefix_value=float(vals[j]), side=side, k=k,
                tau=_threshold(xs_sorted, k), order=order)


def kmeans_1d(values: np.ndarray, c0: float = 0.1, c1: float = 0.9, max_iter: int = 100):
    """Two-centre K-means (Lloyd) on a 1-D sample, started at c0 and c1 (Section 3.3).

    Each value goes to the nearer centre (the lower one on an exact tie); each
    centre becomes the mean of its values (kept when it has none); stops when
    the assignment no longer changes.  Returns (c0, c1).
    """
    v = np.asarray(values, dtype=np.float64)
    assign = None
    for _ in range(max_iter):
        new = np.abs(v - c1) < np.abs(v - c0)           # True -> upper centre
        if assign is not None and np.array_equal(new, assign):
            break
        assign = new
        if np.any(~assign):
            c0 = float(np.mean(v[~assign]))
        if np.any(assign):
            c1 = float(np.mean(v[assign]))
    return c0, c1


def two_level_rounding(prob: Problem, x: np.ndarray, delta: float = 0.05):
    """Two-level rounding (Section 3.3).

    gamma0 = c0 + delta and gamma1 = c1 - delta from 1-D K-means on x (centres
    started at 0.1 and 0.9); S0 = {x <= gamma0} (holds t), S1 = {x >= gamma1}
    (holds s), Sc = the rest.  The coarse graph G_c has the vertices of Sc
    plus s_c (S1 contracted) and t_c (S0 contracted), with the four kinds of
    edges of the paper: Sc-Sc edges kept, {s_c, u} of weight sum_{v in S1} c(u,v),
    {t_c, u} of weight sum_{v in S0} c(u,v), {s_c, t_c} of weight
    sum_{u in S1, v in S0} c(u,v).  An s_c-t_c min cut of G_c (max-flow) induces
    the cut S1 + (its source side within Sc) of G.
    Returns dict(value, side, gamma0, gamma1, coarse_vertices).
    """
    from .exact import max_flow_min_cut
    c0, c1 = kmeans_1d(x)
    g0, g1 = c0 + delta, c1 - delta
    lab = np.full(prob.n, 2, dtype=np.int64)
    lab[x <= g0] = 0
    lab[x >= g1] = 1
    lab[prob.s] = 1
    lab[prob.t] = 0
    sc = np.nonzero(lab == 2)[0]
    cid = np.full(prob.n, -1, dtype=np.int64)
    cid[sc] = np.arange(sc.shape[0])
    nc = sc.shape[0] + 2
    sC, tC = sc.shape[0], sc.shape[0] + 1
    # map every edge to its coarse endpoints; drop edges inside S0 or S1
    def coarse(vtx):
        return np.where(lab[vtx] == 2, cid[vtx], np.where(lab[vtx] == 1, sC, tC))
    cu, cv = coarse(prob.eu), coarse(prob.ev)
    keep = cu != cv
    u, v, c = cu[keep], cv[keep], prob.cap[keep]
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    key = lo * nc + hi
    uk, inv = np.unique(key, return_inverse=True)
    w = np.bincount(inv, weights=c, minlength=uk.shape[0])
    ru, rv = uk // nc, uk % nc
    rows = np.concatenate([ru, rv])
    cols = np.concatenate([rv, ru])
    vals = np.concatenate([w, w])
    order = np.lexsort((cols, rows))
    rp = np.zeros(nc + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=nc), out=rp[1:])
    coarse_prob = Problem(nc, rp, cols[order], vals[order], sC, tC)
    _, cside = max_flow_min_cut(coarse_prob)
    side = lab == 1
    side[sc] = cside[:sc.shape[0]]
    return dict(value=cut_value(prob, side), side=side, gamma0=g0, gamma1=g1,
                coarse_vertices=nc)
