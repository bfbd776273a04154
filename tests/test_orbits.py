"""The host orbit finder against the paper's printed orbit counts and brute force."""
import os

import numpy as np
import pytest

from oracle import automorphisms as AUT
from paper_2410_22247_gb300 import orbits as ORB
from paper_2410_22247_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_edge_orbit_counts.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        fam, params, n, m, orbits, *cite = line.split()
        prm = dict(kv.split("=") for kv in params.split(";"))
        rows.append((fam, prm, int(n), int(m), int(orbits), " ".join(cite)))
    return rows


def _graph(fam, prm):
    if fam == "binary":
        return W.heap_binary_tree(int(prm["n"]))
    if fam == "balanced":
        return W.balanced_tree(int(prm["r"]), int(prm["h"]))
    if fam == "complete":
        return W.complete_graph(int(prm["n"]))
    if fam == "star":
        return W.star_graph(int(prm["n"]))
    if fam == "cycle":
        return W.cycle_graph(int(prm["n"]))
    if fam == "petersen":
        return W.generalized_petersen(int(prm["k"]), int(prm["s"]))
    if fam == "circulant":
        return W.circulant_graph(int(prm["n"]), [int(j) for j in prm["j"].split("+")])
    raise KeyError(fam)


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: r[5])
def test_orbit_counts_match_paper(row):
    fam, prm, n, m, orbits, cite = row
    nn, e = _graph(fam, prm)
    assert (nn, len(e)) == (n, m), cite
    res = ORB.edge_orbits(nn, e)
    assert res.num_orbits == orbits, cite
    assert int(res.weight.sum()) == m
    for g in res.generators:
        assert ORB.is_automorphism(g, {tuple(map(int, x)) for x in e})


SMALL = [W.cycle_graph(6), W.star_graph(7), W.complete_graph(5), W.prufer_tree(8, 3), W.random_regular(8, 3, 4),
         W.heap_binary_tree(8), W.balanced_tree(2, 2), W.circulant_graph(8, (1, 3)),
         (6, W.canonical_edges([(0, 1), (1, 2), (2, 0), (3, 4)])), (5, W.canonical_edges([]))]


@pytest.mark.parametrize("k", range(len(SMALL)))
def test_orbits_match_brute_force(k):
    n, e = SMALL[k]
    res = ORB.edge_orbits(n, e)
    canon = [tuple(map(int, x)) for x in e]
    mine = {frozenset(canon[i] for i in range(len(canon)) if res.edge_orbit[i] == c) for c in range(res.num_orbits)}
    ref, group = AUT.edge_orbit_partition(n, e)
    assert mine == ref
    # representative is the seed = lowest edge of its class; weight = class size
    for c in range(res.num_orbits):
        members = [i for i in range(len(canon)) if res.edge_orbit[i] == c]
        assert res.rep[c] == min(members)
        assert res.weight[c] == len(members)


def test_group_order_matches_networkx():
    nx = pytest.importorskip("networkx")
    from networkx.algorithms.isomorphism import GraphMatcher
    for n, e in SMALL[:8]:
        g = nx.Graph()
        g.add_nodes_from(range(n))
        g.add_edges_from(map(tuple, e))
        count = sum(1 for _ in GraphMatcher(g, g).isomorphisms_iter())
        assert count == len(AUT.automorphism_group(n, e))


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: "native-" + r[5])
def test_native_orbit_counts_match_paper(row):
    """The library's C++ finder (aaqaoa_edge_orbits, no GPU) on the printed counts."""
    fam, prm, n, m, orbits, cite = row
    nn, e = _graph(fam, prm)
    res = ORB.edge_orbits_native(nn, e)
    assert res.num_orbits == orbits, cite
    assert int(res.weight.sum()) == m


@pytest.mark.parametrize("k", range(len(SMALL)))
def test_native_orbits_match_brute_force(k):
    n, e = SMALL[k]
    res = ORB.edge_orbits_native(n, e)
    canon = [tuple(map(int, x)) for x in e]
    mine = {frozenset(canon[i] for i in range(len(canon)) if res.edge_orbit[i] == c) for c in range(res.num_orbits)}
    ref, _ = AUT.edge_orbit_partition(n, e)
    assert mine == ref


def test_native_and_python_finders_agree():
    graphs = [W.heap_binary_tree(34), W.complete_graph(16), W.star_graph(30), W.random_regular(30, 3, 0),
              W.generalized_petersen(5, 2), W.prufer_tree(32, 0), W.circulant_graph(12, (1, 3))]
    graphs += [(n, e) for _, n, e in W.mixed_graph_batch(40, 12, 22, 7)]
    for n, e in graphs:
        a, b = ORB.edge_orbits(n, e), ORB.edge_orbits_native(n, e)
        assert np.array_equal(a.edge_orbit, b.edge_orbit) and np.array_equal(a.rep, b.rep)
        assert np.array_equal(a.weight, b.weight)


def test_native_finder_rejects_bad_edges():
    import ctypes
    from paper_2410_22247_gb300 import _native as N
    out = np.zeros(4, dtype=np.int32)
    k = ctypes.c_int32()
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    for bad in ([0, 0, 1, 2], [0, 1, 1, 0], [0, 5, 1, 2]):
        e = np.array(bad, dtype=np.int32)
        assert N.aaqaoa_edge_orbits(4, 2, P(e), None, P(out), ctypes.byref(k), P(out), P(out)) == -1
    e = np.array([0, 1], dtype=np.int32)
    assert N.aaqaoa_edge_orbits(65, 1, P(e), None, P(out), ctypes.byref(k), P(out), P(out)) == -1
    w0 = np.array([0], dtype=np.int32)
    assert N.aaqaoa_edge_orbits(4, 1, P(e), P(w0), P(out), ctypes.byref(k), P(out), P(out)) == -1


@pytest.mark.parametrize("k", range(8))
def test_weighted_orbits_match_brute_force(k):
    """Weight-preserving automorphisms (weighted MaxCut): the finder's classes
    against brute force over all permutations, for seeded integer weights and
    for weights constant on the unweighted orbits (where nothing splits)."""
    n, e = SMALL[k]
    for mode in ("random", "orbit"):
        if mode == "random":
            w = W.rng(40 + k).integers(1, 3, size=len(e))
        else:
            base = ORB.edge_orbits(n, e)
            w = (base.edge_orbit % 3 + 1).astype(np.int64)
        res = ORB.edge_orbits(n, e, weights=w)
        canon = [tuple(map(int, x)) for x in e]
        mine = {frozenset(canon[i] for i in range(len(canon)) if res.edge_orbit[i] == c)
                for c in range(res.num_orbits)}
        ref, _ = AUT.edge_orbit_partition(n, e, w)
        assert mine == ref, mode
        for c in range(res.num_orbits):  # one weight per class
            assert len({int(w[i]) for i in range(len(e)) if res.edge_orbit[i] == c}) == 1
        if mode == "orbit":
            assert res.num_orbits == ORB.edge_orbits(n, e).num_orbits



def test_native_weighted_orbits_match_python_and_brute_force():
    for k_, (n, e) in enumerate(SMALL[:8]):
        w = W.rng(60 + k_).integers(1, 3, size=len(e))
        a, b = ORB.edge_orbits(n, e, weights=w), ORB.edge_orbits_native(n, e, weights=w)
        assert np.array_equal(a.edge_orbit, b.edge_orbit) and np.array_equal(a.weight, b.weight)
    n, e = W.heap_binary_tree(31)
    w = np.array([1 + int(np.floor(np.log2(int(v) + 1))) % 3 for _, v in e])
    a, b = ORB.edge_orbits(n, e, weights=w), ORB.edge_orbits_native(n, e, weights=w)
    assert np.array_equal(a.edge_orbit, b.edge_orbit) and a.num_orbits == ORB.edge_orbits(n, e).num_orbits


ETA_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_eta_values.txt")


def _eta_rows():
    rows = []
    for line in open(ETA_GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        fam, params, n, m, e1, e2, *cite = line.split()
        prm = dict(kv.split("=") for kv in params.split(";"))
        rows.append((fam, prm, int(n), int(m), float(e1), float(e2), " ".join(cite)))
    return rows


@pytest.mark.parametrize("row", _eta_rows(), ids=lambda r: r[6])
def test_eta_matches_paper_tables(row):
    """The exact expectation over random representatives against the printed
    means (two decimals of a sampled mean: within 0.011)."""
    fam, prm, n, m, e1, e2, cite = row
    nn, e = _graph(fam, prm)
    assert (nn, len(e)) == (n, m)
    assert abs(ORB.eta_mean(nn, e, 1) - e1) <= 0.011, cite
    assert abs(ORB.eta_mean(nn, e, 2) - e2) <= 0.011, cite


def test_eta_mean_is_the_enumerated_mean_and_bounds():
    import itertools
    for n, e in (W.balanced_tree(2, 3), W.heap_binary_tree(20), W.cycle_graph(9), W.generalized_petersen(5, 2)):
        orb = ORB.edge_orbits(n, e)
        classes = [[k for k in range(len(e)) if orb.edge_orbit[k] == c] for c in range(orb.num_orbits)]
        for p in (1, 2):
            vals = [ORB.eta(n, e, p, reps) for reps in itertools.product(*classes)]
            assert abs(np.mean(vals) - ORB.eta_mean(n, e, p, orb)) < 1e-12
            assert all(0.0 <= v <= 1.0 for v in vals)
        assert ORB.eta_mean(n, e, 2, orb) <= ORB.eta_mean(n, e, 1, orb) + 1e-12
    # closed forms: K_n, one representative touching 2n-3 edges at p = 1; the
    # star's centre makes every cone span all edges; a cycle's cone has 3 edges
    for n in (5, 8, 12):
        nn, e = W.complete_graph(n)
        assert abs(ORB.eta_mean(nn, e, 1) - (1 - (2 * n - 3) / (n * (n - 1) / 2))) < 1e-12
        assert ORB.eta_mean(*W.star_graph(n), 1) == 0.0
        assert abs(ORB.eta_mean(*W.cycle_graph(n), 1) - (1 - 3 / n)) < 1e-12


def _ising_symmetric_instance(n, e, seed):
    """Couplings and fields that depend on vertex degrees (kept by every
    automorphism) plus a field that singles out vertex 0."""
    deg = np.bincount(np.asarray(e).reshape(-1), minlength=n)
    r = W.rng(seed)
    vals = r.uniform(-2, 2, size=2 * n + 2)
    w = np.array([vals[(deg[u] + deg[v]) % len(vals)] for u, v in e])
    h = np.array([vals[-1] if i == 0 else vals[n + deg[i] % n] for i in range(n)])
    return w, h


@pytest.mark.parametrize("maker", [lambda: W.cycle_graph(6), lambda: W.star_graph(7), lambda: W.complete_graph(5),
                                   lambda: W.heap_binary_tree(7), lambda: W.prufer_tree(8, 2),
                                   lambda: W.random_regular(8, 3, 1)],
                         ids=["c6", "star7", "k5", "bintree7", "prufer8", "reg8"])
def test_ising_orbits_match_brute_force(maker):
    """Edge and vertex classes of the coupling- and field-preserving
    automorphisms equal the brute-force orbits (all permutations), from both
    finders."""
    from oracle import automorphisms as AUT
    n, e = maker()
    for seed in (1, 2):
        w, h = _ising_symmetric_instance(n, e, seed)
        eorb, vorb = AUT.ising_orbit_partition(n, e, w, h)
        io = ORB.ising_orbits(n, e, w, h)
        canon = [tuple(map(int, x)) for x in e]
        got_e = {frozenset(canon[i] for i in range(len(e)) if io.edge_orbit[i] == c) for c in range(io.num_orbits)}
        got_v = {frozenset(u for u in range(n) if io.vertex_orbit[u] == c) for c in range(len(io.vrep))}
        assert got_e == set(eorb) and got_v == set(vorb)
        assert all(io.vertex_orbit[io.vrep[c]] == c and io.vweight[c] == len([u for u in range(n)
                   if io.vertex_orbit[u] == c]) for c in range(len(io.vrep)))
        nat = ORB.ising_orbits_native(n, e, w, h)
        for k in ("edge_orbit", "rep", "weight", "vertex_orbit", "vrep", "vweight"):
            assert np.array_equal(getattr(io, k), getattr(nat, k)), k
