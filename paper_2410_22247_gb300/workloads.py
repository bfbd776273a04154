"""Seeded synthetic inputs: graph families and QAOA angles.

This module only builds inputs (edge lists, angle vectors, batches). It holds
none of the QAOA arithmetic, so both the CUDA path and the CPU oracle may take
their inputs from it.

Graph families follow the ones the paper benchmarks on (Sec. 6, Tables 1-5 and
the diagnostic-control / non-tree tables of Sec. 6.1): heap-ordered binary
trees, complete r-ary ("balanced") trees, stars, complete graphs K_n, cycles,
the generalized Petersen graph GP(5,2), circulants, random 3-regular graphs and
uniformly random labelled trees (Pruefer sequences). The paper does not publish
its random instances, so the random families here are seeded stand-ins drawn
from the textbook definitions of each family.

Every graph is returned as ``(n, edges)`` with ``edges`` an int32 array of
shape (m, 2), each row (u, v) with u < v, rows sorted lexicographically.
Vertex i is qubit i, i.e. bit i of a basis-state index.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "canonical_edges", "complete_graph", "star_graph", "cycle_graph",
    "heap_binary_tree", "balanced_tree", "prufer_tree", "random_regular",
    "generalized_petersen", "circulant_graph", "random_angles", "angle_grid",
    "mixed_graph_batch", "rng",
]


def rng(seed: int) -> np.random.Generator:
    """The one PRNG used for every seeded input: numpy PCG64."""
    return np.random.Generator(np.random.PCG64(seed))


def canonical_edges(edges) -> np.ndarray:
    """Normalise to rows (min, max), drop nothing, sort lexicographically."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    e = np.sort(e, axis=1)
    if len(e):
        order = np.lexsort((e[:, 1], e[:, 0]))
        e = e[order]
    return e.astype(np.int32)


def complete_graph(n: int):
    """K_n: every pair of the n vertices is an edge."""
    return n, canonical_edges([(i, j) for i in range(n) for j in range(i + 1, n)])


def star_graph(n: int):
    """Star on n vertices: centre 0, leaves 1..n-1 (S_{n-1} has n vertices)."""
    return n, canonical_edges([(0, j) for j in range(1, n)])


def cycle_graph(n: int):
    """Cycle C_n on vertices 0..n-1."""
    return n, canonical_edges([(i, (i + 1) % n) for i in range(n)])


def heap_binary_tree(n: int):
    """Heap-ordered binary tree on n vertices: children of i are 2i+1, 2i+2.

    This is the construction whose edge-orbit counts match Table 1 of the
    paper ("Binary Tree graph instances"): n = 5, 10, 15, 20, 25, 30, 31, 34.
    """
    return n, canonical_edges([(i, c) for i in range(n) for c in (2 * i + 1, 2 * i + 2) if c < n])


def balanced_tree(r: int, h: int):
    """Complete r-ary tree of height h in breadth-first numbering.

    Vertex i has children r*i+1 .. r*i+r. (r, h) = (2,2), (3,2), (2,3), (2,4)
    give the n = 7, 13, 15, 31 instances of Table 2 of the paper.
    """
    n = sum(r ** k for k in range(h + 1))
    return n, canonical_edges([(i, r * i + k) for i in range(n) for k in range(1, r + 1) if r * i + k < n])


def prufer_tree(n: int, seed: int):
    """Uniformly random labelled tree on n >= 2 vertices.

    Draws a Pruefer sequence of n-2 labels uniformly from [0, n) with the
    seeded PCG64 generator and decodes it with the standard smallest-leaf rule.
    """
    if n < 2:
        raise ValueError("a tree needs n >= 2")
    if n == 2:
        return n, canonical_edges([(0, 1)])
    seq = rng(seed).integers(0, n, size=n - 2)
    degree = np.ones(n, dtype=np.int64)
    for a in seq:
        degree[a] += 1
    edges = []
    for a in seq:
        leaf = int(np.flatnonzero(degree == 1)[0])
        edges.append((leaf, int(a)))
        degree[leaf] -= 1
        degree[a] -= 1
    u, v = np.flatnonzero(degree == 1)
    edges.append((int(u), int(v)))
    return n, canonical_edges(edges)


def random_regular(n: int, d: int, seed: int, max_tries: int = 100000):
    """Random d-regular simple graph by the configuration model.

    n*d half-edges ("stubs") are paired by a uniformly random permutation; a
    pairing with a self-loop or a repeated edge is rejected and redrawn.
    """
    if (n * d) % 2:
        raise ValueError("n*d must be even")
    g = rng(seed)
    stubs = np.repeat(np.arange(n), d)
    for _ in range(max_tries):
        perm = g.permutation(stubs)
        pairs = perm.reshape(-1, 2)
        if np.any(pairs[:, 0] == pairs[:, 1]):
            continue
        e = canonical_edges(pairs)
        if len(np.unique(e, axis=0)) != len(e):
            continue
        return n, e
    raise RuntimeError("configuration model did not produce a simple graph")


def generalized_petersen(k: int, s: int):
    """Generalized Petersen graph GP(k, s); GP(5, 2) is the Petersen graph.

    Outer cycle 0..k-1, spokes i -- k+i, inner star polygon k+i -- k+(i+s mod k).
    """
    e = []
    for i in range(k):
        e.append((i, (i + 1) % k))
        e.append((i, k + i))
        e.append((k + i, k + (i + s) % k))
    return 2 * k, canonical_edges(e)


def circulant_graph(n: int, jumps):
    """Circulant C_n(j1, j2, ...): i -- i+j (mod n) for every jump j."""
    e = {tuple(sorted((i, (i + j) % n))) for i in range(n) for j in jumps}
    return n, canonical_edges(sorted(e))


def random_angles(p: int, seed: int):
    """Seeded angles: gamma_l ~ U[0, pi], beta_l ~ U[0, pi/2], l = 1..p."""
    g = rng(seed)
    gamma = g.uniform(0.0, math.pi, size=p)
    beta = g.uniform(0.0, math.pi / 2, size=p)
    return gamma, beta


def angle_grid(k: int):
    """Inclusive k x k grid gamma_i = i*pi/(k-1), beta_j = j*(pi/2)/(k-1).

    Returns arrays of shape (k*k,) ordered gamma-major.
    """
    gs = np.linspace(0.0, math.pi, k)
    bs = np.linspace(0.0, math.pi / 2, k)
    G, B = np.meshgrid(gs, bs, indexing="ij")
    return G.reshape(-1).copy(), B.reshape(-1).copy()


def mixed_graph_batch(count: int, n_lo: int, n_hi: int, seed: int):
    """A seeded batch of graphs of uneven size.

    n ~ U{n_lo..n_hi}; family ~ U{Pruefer tree, cycle, K_n, 3-regular}; K_n is
    only drawn for n <= 16 and 3-regular only for even n, otherwise the family
    is redrawn. Returns a list of (family, n, edges).
    """
    g = rng(seed)
    out = []
    fams = ("prufer", "cycle", "complete", "regular3")
    while len(out) < count:
        n = int(g.integers(n_lo, n_hi + 1))
        fam = fams[int(g.integers(0, len(fams)))]
        sub = int(g.integers(0, 2 ** 31 - 1))
        if fam == "complete" and n > 16:
            continue
        if fam == "regular3" and n % 2:
            continue
        if fam == "prufer":
            _, e = prufer_tree(n, sub)
        elif fam == "cycle":
            _, e = cycle_graph(n)
        elif fam == "complete":
            _, e = complete_graph(n)
        else:
            _, e = random_regular(n, 3, sub)
        out.append((fam, n, e))
    return out


def ising_couplings(n: int, edges, seed: int, symmetric: bool = False, fields: bool = True):
    """Seeded real couplings (one per edge) and fields (one per vertex, or
    None) for an Ising-form objective.

    symmetric=False: couplings ~ U[-1, 2], fields ~ U[-1, 1] (generic, the
    automorphism group is usually trivial). symmetric=True: values drawn per
    class of an automorphism-invariant key (the sorted degree pair of an edge,
    the degree of a vertex), so every automorphism of the graph keeps them and
    H_red stays nontrivial."""
    e = np.asarray(edges).reshape(-1, 2)
    r = rng(seed)
    if not symmetric:
        w = r.uniform(-1.0, 2.0, size=len(e))
        h = r.uniform(-1.0, 1.0, size=n) if fields else None
        return w, h
    deg = np.bincount(e.reshape(-1), minlength=n) if len(e) else np.zeros(n, dtype=np.int64)
    table_w = r.uniform(-1.0, 2.0, size=(n + 1, n + 1))
    table_h = r.uniform(-1.0, 1.0, size=n + 1)
    w = np.array([table_w[min(deg[u], deg[v]), max(deg[u], deg[v])] for u, v in e], dtype=np.float64)
    h = np.array([table_h[deg[i]] for i in range(n)], dtype=np.float64) if fields else None
    return w, h
