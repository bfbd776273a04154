"""Per-edge light-cone evaluation with the full oracle (test infrastructure).

At depth p the expectation <Z_u Z_v> depends only on the qubits within graph
distance p of {u, v}: in the Heisenberg picture each of the p cost layers
widens the support by one neighbourhood, and every gate outside that ball
commutes through and cancels (this is the reverse causal cone of Sec. 5.1,
Eqs. (rcc1)-(rcc4)). Edges between two vertices at distance exactly p also
cancel, so the induced subgraph on the ball gives the same value.

That lets the oracle produce exact FP64 per-edge values, energies and
gradients of graphs far larger than a 2^n statevector on the host allows,
whenever each ball is small (e.g. a 3-regular graph on 30 vertices at p = 2
has balls of at most 14 vertices).
"""
from __future__ import annotations

from collections import deque

import numpy as np

from . import oracle


def ball(n, edges, u, v, p):
    """Vertices within distance p of {u, v}, sorted."""
    adj = [[] for _ in range(n)]
    for a, b in np.asarray(edges).reshape(-1, 2):
        adj[int(a)].append(int(b))
        adj[int(b)].append(int(a))
    dist = {u: 0, v: 0}
    q = deque([u, v])
    while q:
        a = q.popleft()
        if dist[a] == p:
            continue
        for b in adj[a]:
            if b not in dist:
                dist[b] = dist[a] + 1
                q.append(b)
    return sorted(dist)


def edge_subproblem(n, edges, u, v, p):
    """(n_sub, sub_edges, u_sub, v_sub) of the induced subgraph on the ball."""
    verts = ball(n, edges, u, v, p)
    index = {a: i for i, a in enumerate(verts)}
    sub = [(index[int(a)], index[int(b)]) for a, b in np.asarray(edges).reshape(-1, 2)
           if int(a) in index and int(b) in index]
    sub = np.array(sorted((min(a, b), max(a, b)) for a, b in sub), dtype=np.int32).reshape(-1, 2)
    return len(verts), sub, index[u], index[v]


def max_ball(n, edges, p):
    return max(len(ball(n, edges, int(a), int(b), p)) for a, b in np.asarray(edges).reshape(-1, 2))


def edge_energy_grad(n, edges, u, v, gamma, beta):
    """(<1/2(1 - Z_u Z_v)>, d/dgamma, d/dbeta) from the edge's light cone."""
    p = len(np.asarray(gamma).reshape(-1))
    ns, se, us, vs = edge_subproblem(n, edges, u, v, p)
    obs = (np.array([[min(us, vs), max(us, vs)]], dtype=np.int32), np.ones(1))
    return oracle.energy_grad(ns, se, gamma, beta, obs)


def energy_grad(n, edges, gamma, beta, weights=None, edge_subset=None):
    """Sum of weighted per-edge light-cone values: E and its gradient.

    ``edge_subset`` (indices into ``edges``) with ``weights`` evaluates an
    observable such as H_red (representatives weighted by orbit size).
    """
    edges = np.asarray(edges).reshape(-1, 2)
    idx = range(len(edges)) if edge_subset is None else edge_subset
    w = np.ones(len(edges)) if weights is None else None
    p = len(np.asarray(gamma).reshape(-1))
    E, dg, db = 0.0, np.zeros(p), np.zeros(p)
    for k, e in enumerate(idx):
        wk = w[e] if w is not None else float(weights[k])
        a, b = int(edges[e][0]), int(edges[e][1])
        Ee, dge, dbe = edge_energy_grad(n, edges, a, b, gamma, beta)
        E += wk * Ee
        dg += wk * dge
        db += wk * dbe
    return E, dg, db


def ising_energy_grad(n, edges, weights, fields, gamma, beta):
    """E and gradient of an Ising-form objective (real couplings per edge,
    real fields per vertex or None), term by term: each ZZ term sees the
    radius-p ball around its edge, each field term Z_i the radius-p ball
    around i, and the subproblem carries the couplings and fields inside the
    ball (the reverse causal cone of Sec. 5.1 holds for any diagonal cost:
    terms outside the cone commute through and cancel)."""
    edges = np.asarray(edges).reshape(-1, 2)
    w = np.asarray(weights, dtype=np.float64)
    h = np.zeros(n) if fields is None else np.asarray(fields, dtype=np.float64)
    p = len(np.asarray(gamma).reshape(-1))
    E, dg, db = 0.0, np.zeros(p), np.zeros(p)
    terms = [((int(u), int(v)), wk, None) for (u, v), wk in zip(edges, w)]
    if fields is not None:
        terms += [((i, i), None, h[i]) for i in range(n)]
    for (u, v), wk, hk in terms:
        verts = ball(n, edges, u, v, p)
        index = {a: k for k, a in enumerate(verts)}
        inside = [k for k, (a, b) in enumerate(edges) if {int(a), int(b)} <= index.keys()]
        sub = np.array([(index[int(edges[k][0])], index[int(edges[k][1])]) for k in inside],
                       dtype=np.int32).reshape(-1, 2)
        fn = oracle.ising(sub, w[inside], np.array([h[a] for a in verts]))
        if hk is None:
            obs = oracle.ising(np.array([[index[u], index[v]]]), np.array([wk]), np.zeros(len(verts)))
        else:
            oh = np.zeros(len(verts))
            oh[index[u]] = hk
            obs = oracle.ising(np.zeros((0, 2)), np.zeros(0), oh)
        Et, dgt, dbt = oracle.ising_energy_grad(len(verts), fn, gamma, beta, obs)
        E, dg, db = E + Et, dg + dgt, db + dbt
    return E, dg, db
