"""Host-side edge-orbit computation (the input to the reduced observable H_red).

The paper obtains generators of Aut(G) from nauty's ``sparsenauty`` and then
groups edges into equivalence classes by a breadth-first closure under those
generators (Sec. 4, Algorithm 1). nauty is third-party, so the generators here
come from this module's own individualisation-refinement search:

* colour refinement to the coarsest equitable ordered partition (an
  isomorphism-invariant labelling step);
* a first path of individualisations down to a discrete partition, giving a
  reference leaf;
* for every level of that path, a search of each sibling subtree (pruned by
  the orbits of the generators found so far) for a leaf that differs from the
  reference leaf by an automorphism. The automorphisms found this way form a
  generating set of Aut(G) (one transversal per level of the stabiliser chain).

Every generator is checked to map the edge set onto itself before it is used.
The edge classes are the orbits, on unordered edges, of the group the
generators span (the method of Sec. 4, Algorithm 1), found by a breadth-first
closure: each edge not yet classified seeds a class, and the images of its
members under every generator, normalised to (min, max), join it.

The representative of each class is its seed edge, which is the lowest-indexed
edge of the class (the paper picks a random representative, Sec. 5.4; any
member gives the same expectation because of Eq. (A3)).
"""
from __future__ import annotations

from collections import deque
from dataclasses import dataclass

import numpy as np

__all__ = ["EdgeOrbits", "automorphism_generators", "edge_orbits", "edge_orbits_native", "eta", "eta_mean",
           "is_automorphism"]


def _adjacency(n, edges):
    adj = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(v)
        adj[v].append(u)
    return adj


def _rank(keys):
    order = {k: i for i, k in enumerate(sorted(set(keys)))}
    return [order[k] for k in keys]


def _refine(adj, col, wadj=None):
    """Colour refinement to the coarsest equitable partition refining ``col``
    (with edge weights, a neighbour counts with the weight of its edge)."""
    ncells = len(set(col))
    while True:
        if wadj is None:
            sig = [(col[v], tuple(sorted(col[u] for u in adj[v]))) for v in range(len(col))]
        else:
            sig = [(col[v], tuple(sorted((col[u], w) for u, w in wadj[v]))) for v in range(len(col))]
        new = _rank(sig)
        k = len(set(new))
        if k == ncells:
            return new
        col, ncells = new, k


def _individualise(adj, col, v, wadj=None):
    keys = [(col[u], 0 if u == v else 1) for u in range(len(col))]
    return _refine(adj, _rank(keys), wadj)


def _target_cell(col):
    sizes = {}
    for v, c in enumerate(col):
        sizes.setdefault(c, []).append(v)
    for c in sorted(sizes):
        if len(sizes[c]) > 1:
            return sizes[c]
    return None


def _cell_sizes(col):
    sizes = [0] * len(col)
    for c in col:
        sizes[c] += 1
    return tuple(sizes)


def is_automorphism(perm, edge_set) -> bool:
    """True when the vertex permutation maps the edge set onto itself (and,
    when ``edge_set`` maps edges to weights, every edge to one of equal weight)."""
    weighted = isinstance(edge_set, dict)
    for u, v in edge_set:
        a, b = perm[u], perm[v]
        img = (min(a, b), max(a, b))
        if img not in edge_set:
            return False
        if weighted and edge_set[img] != edge_set[(u, v)]:
            return False
    return True


def _orbit_ids(n, gens):
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for g in gens:
        for a in range(n):
            ra, rb = find(a), find(g[a])
            if ra != rb:
                parent[ra] = rb
    return [find(a) for a in range(n)]


def automorphism_generators(n, edges, weights=None, fields=None):
    """A generating set of Aut(G) as a list of permutations (lists of length n);
    with edge weights (integer or real), of the weight-preserving
    automorphisms; with vertex fields, of those that also map every vertex to
    one of equal field (the fields colour the initial partition)."""
    edges = [tuple(map(int, e)) for e in np.asarray(edges).reshape(-1, 2)]
    if weights is None:
        edge_set = {(min(u, v), max(u, v)) for u, v in edges}
        wadj = None
    else:
        wl = [float(w) for w in np.asarray(weights).reshape(-1)]
        edge_set = {(min(u, v), max(u, v)): w for (u, v), w in zip(edges, wl)}
        wadj = [[] for _ in range(n)]
        for (u, v), w in zip(edges, wl):
            wadj[u].append((v, w))
            wadj[v].append((u, w))
    adj = _adjacency(n, edges)
    if n == 0:
        return []
    hl = None if fields is None else [float(h) for h in np.asarray(fields).reshape(-1)]

    def is_aut(g):
        return is_automorphism(g, edge_set) and (hl is None or all(hl[g[u]] == hl[u] for u in range(n)))

    col = _refine(adj, [0] * n if hl is None else _rank(hl), wadj)
    path = []
    while True:
        cell = _target_cell(col)
        if cell is None:
            break
        path.append((col, cell, cell[0]))
        col = _individualise(adj, col, cell[0], wadj)
    leaf0 = col
    inv0 = [0] * n
    for v, c in enumerate(leaf0):
        inv0[c] = v
    depth_sizes = [_cell_sizes(c) for c, _, _ in path] + [_cell_sizes(leaf0)]

    def leaf_map(leaf):
        # the permutation taking the reference leaf to this leaf: a vertex of
        # colour c in leaf0 goes to the vertex of colour c in ``leaf``
        inv = [0] * n
        for v, c in enumerate(leaf):
            inv[c] = v
        return [inv[leaf0[u]] for u in range(n)]

    def search(col, depth):
        if _cell_sizes(col) != depth_sizes[depth]:
            return None
        cell = _target_cell(col)
        if cell is None:
            g = leaf_map(col)
            return g if is_aut(g) else None
        for x in cell:
            r = search(_individualise(adj, col, x, wadj), depth + 1)
            if r is not None:
                return r
        return None

    gens = []
    for level in range(len(path) - 1, -1, -1):
        col_k, cell, v_k = path[level]
        for w in cell:
            if w == v_k:
                continue
            orb = _orbit_ids(n, gens)
            if orb[w] == orb[v_k]:
                continue
            g = search(_individualise(adj, col_k, w, wadj), level + 1)
            if g is not None:
                assert is_aut(g)
                gens.append(g)
    return gens


@dataclass
class EdgeOrbits:
    """Edge classes of Algorithm 1.

    ``edge_orbit[e]`` is the class of edge e (edges in canonical sorted order),
    ``rep[m]`` the edge index of the representative of class m (its seed) and
    ``weight[m]`` the class size |S~_m|.
    """
    edge_orbit: np.ndarray
    rep: np.ndarray
    weight: np.ndarray
    generators: list

    @property
    def num_orbits(self) -> int:
        return len(self.rep)


def edge_orbits(n, edges, generators=None, weights=None) -> EdgeOrbits:
    """Algorithm 1: breadth-first closure of the edges under the generators
    (of the weight-preserving automorphisms when integer edge weights are given)."""
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    canon = [(int(min(u, v)), int(max(u, v))) for u, v in edges]
    if canon != sorted(canon):
        raise ValueError("edges must be in canonical sorted order (u < v, lexicographic)")
    index = {e: i for i, e in enumerate(canon)}
    if generators is None:
        generators = automorphism_generators(n, edges, weights)
    m = len(canon)
    cls = np.full(m, -1, dtype=np.int64)
    reps, weights = [], []
    for seed in range(m):
        if cls[seed] >= 0:
            continue
        c = len(reps)
        cls[seed] = c
        reps.append(seed)
        size = 1
        queue = deque([canon[seed]])
        while queue:
            a, b = queue.popleft()
            for g in generators:
                ga, gb = g[a], g[b]
                img = (min(ga, gb), max(ga, gb))
                j = index.get(img)
                if j is not None and cls[j] < 0:
                    cls[j] = c
                    size += 1
                    queue.append(img)
        weights.append(size)
    return EdgeOrbits(cls.astype(np.int32), np.asarray(reps, dtype=np.int32),
                      np.asarray(weights, dtype=np.int32), generators)


@dataclass
class IsingOrbits(EdgeOrbits):
    """Edge classes plus vertex classes of the automorphisms that preserve the
    couplings and the fields: ``vertex_orbit[u]`` is the class of vertex u,
    ``vrep[c]`` its smallest vertex, ``vweight[c]`` the class size."""
    vertex_orbit: np.ndarray = None
    vrep: np.ndarray = None
    vweight: np.ndarray = None


def vertex_classes(n, generators):
    """Orbits of the generated group on vertices, numbered by smallest member."""
    root = _orbit_ids(n, generators)
    first = {}
    for u in range(n):
        first.setdefault(root[u], u)
    reps = sorted(first.values())
    index = {root[r]: c for c, r in enumerate(reps)}
    vo = np.array([index[root[u]] for u in range(n)], dtype=np.int32)
    vw = np.bincount(vo, minlength=len(reps)).astype(np.int32)
    return vo, np.asarray(reps, dtype=np.int32), vw


def ising_orbits(n, edges, couplings, fields=None) -> IsingOrbits:
    """Edge and vertex classes for an Ising-form objective (real couplings
    per edge, optional real fields per vertex): the orbits of the group of
    automorphisms that keep both."""
    gens = automorphism_generators(n, edges, couplings, fields)
    eo = edge_orbits(n, edges, generators=gens)
    vo, vr, vw = vertex_classes(n, gens)
    return IsingOrbits(eo.edge_orbit, eo.rep, eo.weight, gens, vo, vr, vw)


def edge_orbits_native(n, edges, weights=None) -> EdgeOrbits:
    """The same classes from the library's C++ implementation
    (``aaqaoa_edge_orbits``: same refinement, search order and closure).
    Generators are not returned (``generators`` is empty)."""
    import ctypes

    from . import _native as N

    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    m = len(e) // 2
    eo = np.zeros(max(m, 1), dtype=np.int32)
    rep = np.zeros(max(m, 1), dtype=np.int32)
    w = np.zeros(max(m, 1), dtype=np.int32)
    k = ctypes.c_int32()
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    wt = None if weights is None else np.ascontiguousarray(np.asarray(weights, dtype=np.int32).reshape(-1))
    N.check(N.aaqaoa_edge_orbits(int(n), m, P(e), P(wt) if wt is not None else None, P(eo), ctypes.byref(k), P(rep),
                                 P(w)), "aaqaoa_edge_orbits")
    return EdgeOrbits(eo[:m].copy(), rep[:k.value].copy(), w[:k.value].copy(), [])


def ising_orbits_native(n, edges, couplings, fields=None) -> IsingOrbits:
    """The classes of ising_orbits from the library's C++ implementation
    (``aaqaoa_ising_orbits``). Generators are not returned."""
    import ctypes

    from . import _native as N

    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    m = len(e) // 2
    cw = np.ascontiguousarray(np.asarray(couplings, dtype=np.float64).reshape(-1))
    fh = None if fields is None else np.ascontiguousarray(np.asarray(fields, dtype=np.float64).reshape(-1))
    eo, rep, w = (np.zeros(max(m, 1), dtype=np.int32) for _ in range(3))
    vo, vr, vw = (np.zeros(n, dtype=np.int32) for _ in range(3))
    k, kv = ctypes.c_int32(), ctypes.c_int32()
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    D = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    N.check(N.aaqaoa_ising_orbits(int(n), m, P(e), D(cw) if m else None, D(fh) if fh is not None else None, P(eo),
                                  ctypes.byref(k), P(rep), P(w), P(vo), ctypes.byref(kv), P(vr), P(vw)),
            "aaqaoa_ising_orbits")
    return IsingOrbits(eo[:m].copy(), rep[:k.value].copy(), w[:k.value].copy(), [], vo.copy(),
                       vr[:kv.value].copy(), vw[:kv.value].copy())


# ------------------------------------------------ structural descriptor eta_p
# Eq. (eta): eta_p = 1 - |union over representatives e of RCC_p(e)| / |E|, the
# fraction of edges outside the combined reverse causal cone of the orbit
# representatives at depth p (Sec. 5.1). Reading of RCC_p(e) as an edge set:
# the ZZ gates that can reach <Z_i Z_j> through p layers, i.e. the edges with
# an endpoint within graph distance p - 1 of {i, j} (on trees the same as the
# edges with both endpoints within distance p). Tables 1-2 print means over a
# random representative per orbit; eta_mean is that expectation, exactly.

def _adj_lists(n, edges):
    adj = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(v)
        adj[v].append(u)
    return adj


def _rcc_edges(adj, edges, i, j, p):
    dist = {i: 0, j: 0}
    frontier = [i, j]
    for d in range(p - 1):
        nxt = []
        for u in frontier:
            for v in adj[u]:
                if v not in dist:
                    dist[v] = d + 1
                    nxt.append(v)
        frontier = nxt
    return {k for k, (u, v) in enumerate(edges) if u in dist or v in dist}


def eta(n, edges, p, reps):
    """eta_p for one choice of representative edges (indices into ``edges``)."""
    e = [tuple(map(int, x)) for x in np.asarray(edges).reshape(-1, 2)]
    if not e:
        return 0.0
    adj = _adj_lists(n, e)
    covered = set()
    for r in reps:
        covered |= _rcc_edges(adj, e, e[int(r)][0], e[int(r)][1], p)
    return 1.0 - len(covered) / len(e)


def eta_mean(n, edges, p, orbits=None):
    """Expected eta_p when each orbit's representative is drawn uniformly and
    independently: 1 - (1/|E|) sum_f P(f covered), P(f covered) =
    1 - prod_m (1 - |{e in S~_m : f in RCC_p(e)}| / |S~_m|)."""
    e = [tuple(map(int, x)) for x in np.asarray(edges).reshape(-1, 2)]
    if not e:
        return 0.0
    if orbits is None:
        orbits = edge_orbits(n, np.asarray(e))
    adj = _adj_lists(n, e)
    rcc = [_rcc_edges(adj, e, u, v, p) for u, v in e]
    miss = np.ones(len(e))
    for c in range(orbits.num_orbits):
        members = [k for k in range(len(e)) if orbits.edge_orbit[k] == c]
        hit = np.zeros(len(e))
        for k in members:
            for f in rcc[k]:
                hit[f] += 1
        miss *= 1.0 - hit / len(members)
    return float(1.0 - np.sum(1.0 - miss) / len(e))
