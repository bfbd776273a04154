"""Brute-force automorphism group and edge orbits (test infrastructure).

For small graphs (n <= 8) every one of the n! vertex permutations is tested
against the definition of an automorphism (Sec. 3, "Graph Automorphisms": (phi(u), phi(v)) is an edge
iff (u, v) is). The edge orbits are then the classes of edges under the whole
group, which pins the generator search plus Algorithm 1 of the package's
orbit finder.
"""
from __future__ import annotations

from itertools import permutations

import numpy as np


def automorphism_group(n, edges, weights=None, fields=None):
    """All vertex permutations mapping edges to edges (of equal weight when
    edge weights are given, integer or real) and, when vertex fields are
    given, every vertex to one of equal field."""
    e = np.asarray(edges).reshape(-1, 2)
    w = [1.0] * len(e) if weights is None else [float(x) for x in np.asarray(weights).reshape(-1)]
    h = None if fields is None else [float(x) for x in np.asarray(fields).reshape(-1)]
    es = {(min(int(u), int(v)), max(int(u), int(v))): wi for (u, v), wi in zip(e, w)}
    group = []
    for perm in permutations(range(n)):
        if h is not None and any(h[perm[i]] != h[i] for i in range(n)):
            continue
        if all(es.get((min(perm[u], perm[v]), max(perm[u], perm[v]))) == wi for (u, v), wi in es.items()):
            group.append(perm)
    return group


def edge_orbit_partition(n, edges, weights=None):
    """The set of edge orbits, each a frozenset of (u, v) tuples."""
    es = sorted({(min(int(u), int(v)), max(int(u), int(v))) for u, v in np.asarray(edges).reshape(-1, 2)})
    group = automorphism_group(n, edges, weights)
    seen, orbits = set(), []
    for e in es:
        if e in seen:
            continue
        orb = frozenset((min(g[e[0]], g[e[1]]), max(g[e[0]], g[e[1]])) for g in group)
        seen |= orb
        orbits.append(orb)
    return set(orbits), group


def ising_orbit_partition(n, edges, weights, fields):
    """Edge orbits and vertex orbits (frozensets) of the automorphisms that
    preserve edge weights and vertex fields."""
    group = automorphism_group(n, edges, weights, fields)
    es = sorted({(min(int(u), int(v)), max(int(u), int(v))) for u, v in np.asarray(edges).reshape(-1, 2)})
    seen, eorb = set(), []
    for e in es:
        if e in seen:
            continue
        orb = frozenset((min(g[e[0]], g[e[1]]), max(g[e[0]], g[e[1]])) for g in group)
        seen |= orb
        eorb.append(orb)
    seenv, vorb = set(), []
    for i in range(n):
        if i in seenv:
            continue
        orb = frozenset(g[i] for g in group)
        seenv |= orb
        vorb.append(orb)
    return eorb, vorb
