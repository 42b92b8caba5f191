"""Exact s-t min-cut references for the oracle (test infrastructure only).

Two independent routes to the optimum of the s-t min-cut problem (Section 2),
so that each checks the other (max-flow min-cut duality):

* ``brute_force_min_cut``: evaluates the cut definition on every one of the
  2^n~ vertex sets S that hold s and not t (n~ <= 22).
* ``max_flow_min_cut``: the Edmonds-Karp augmenting-path max-flow (shortest
  augmenting paths found by breadth-first search) in FP64 on the undirected
  graph, each edge being a pair of opposite arcs of capacity c; the source
  side of the min cut is the set reachable from s in the final residual graph.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def brute_force_min_cut(prob, rel_tol: float = 1e-12):
    """Minimum of cut(S, S-bar) over all S with s in S, t not in S.

    Returns (value, minimisers) where minimisers is a list of boolean side
    vectors (over all n vertices) whose value is within ``rel_tol`` of the
    minimum.
    """
    nt = prob.nonterminals
    k = nt.shape[0]
    if k > 22:
        raise ValueError("brute force is limited to 22 non-terminals")
    total = 1 << k
    best = np.inf
    values = np.empty(total)
    chunk = 1 << 16
    for start in range(0, total, chunk):
        codes = np.arange(start, min(total, start + chunk), dtype=np.int64)
        bits = ((codes[:, None] >> np.arange(k)[None, :]) & 1).astype(bool)
        side = np.zeros((codes.shape[0], prob.n), dtype=bool)
        side[:, prob.s] = True
        side[:, nt] = bits
        crossing = side[:, prob.eu] != side[:, prob.ev]
        vals = crossing.astype(np.float64) @ prob.cap
        values[start:start + codes.shape[0]] = vals
        best = min(best, float(vals.min()))
    tol = rel_tol * max(abs(best), 1e-300)
    mins = []
    for code in np.nonzero(values <= best + tol)[0]:
        side = np.zeros(prob.n, dtype=bool)
        side[prob.s] = True
        side[nt] = ((int(code) >> np.arange(k)) & 1).astype(bool)
        mins.append(side)
    return best, mins


def max_flow_min_cut(prob, rel_tol: float = 1e-12):
    """Edmonds-Karp max-flow from s to t; returns (flow_value, source_side).

    Residual capacities below ``rel_tol`` times the largest capacity are
    treated as saturated.
    """
    n = prob.n
    s, t = prob.s, prob.t
    # arc arrays: arc 2e is u->v, arc 2e+1 is v->u, both with capacity c_e
    head = np.empty(2 * prob.m, dtype=np.int64)
    head[0::2] = prob.ev
    head[1::2] = prob.eu
    res = np.repeat(prob.cap, 2).astype(np.float64)
    tail = np.empty(2 * prob.m, dtype=np.int64)
    tail[0::2] = prob.eu
    tail[1::2] = prob.ev
    adj = [[] for _ in range(n)]
    for a in range(2 * prob.m):
        adj[int(tail[a])].append(a)
    head = head.tolist()
    res = res.tolist()
    tiny = rel_tol * (max(prob.cap) if prob.m else 1.0)
    flow = 0.0
    while True:
        pred = [-1] * n
        seen = [False] * n
        seen[s] = True
        dq = deque([s])
        while dq and not seen[t]:
            u = dq.popleft()
            for a in adj[u]:
                v = head[a]
                if not seen[v] and res[a] > tiny:
                    seen[v] = True
                    pred[v] = a
                    dq.append(v)
        if not seen[t]:
            break
        # bottleneck along the path
        bott = np.inf
        v = t
        while v != s:
            a = pred[v]
            bott = min(bott, res[a])
            v = head[a ^ 1]
        v = t
        while v != s:
            a = pred[v]
            res[a] -= bott
            res[a ^ 1] += bott
            v = head[a ^ 1]
        flow += bott
    side = np.array(seen, dtype=bool)
    return flow, side
