"""Checks that pin the CPU oracle to things other than itself.

Each check returns the largest relative discrepancy it saw, so the same checks
serve the pin tests (discrepancy must be tiny) and the planted-mistake tests
(a mutated oracle must make at least one of them large).

What pins what:
  * dense brute force: scipy.linalg.expm of the 2^n x 2^n matrices of H_C and
    H_M built from Kronecker products of Pauli matrices (Eq. (1), Eq. (A2) for
    the layer order, qubit i = bit i) -- pins the state amplitude by amplitude;
  * the published p = 1 closed form (degrees and triangles) -- pins E and its
    gradient on arbitrary graphs;
  * the Dicke / star symmetric-subspace models -- pin E and gradient at p > 1;
  * central finite differences -- pin the adjoint gradient;
  * invariants that hold for every graph (norm, gamma = 0, beta = 0, periods,
    time reversal, global bit flip, <Z_i> = 0, automorphism invariance of the
    state (Eq. (A2)), equal <ZZ> within an edge orbit (Eq. (A3)),
    <H_red> = <H_C> (Eq. (exact)), term-by-term aggregation (Eq. (agg))
    equal to the diagonal sum, bounds 0 <= E <= C_max).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import expm

from oracle import oracle as O
from oracle import closed_form as CF
from oracle import symmetric as SYM
from oracle import automorphisms as AUT
from oracle import lightcone as LC
from paper_2410_22247_gb300 import workloads as W


def _rel(a, b, scale=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = np.maximum(np.abs(b), 1.0) if scale is None else scale
    return float(np.max(np.abs(a - b) / s)) if a.size else 0.0


def _op_on(n, q, a):
    """Dense operator acting with 2x2 matrix a on qubit q (qubit q = bit q)."""
    m = np.array([[1.0]])
    for k in range(n - 1, -1, -1):
        m = np.kron(m, a if k == q else np.eye(2))
    return m


def dense_state(n, edges, gamma, beta, weights=None, fields=None):
    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    dim = 1 << n
    HC = np.zeros((dim, dim), dtype=np.complex128)
    e = np.asarray(edges).reshape(-1, 2)
    w = np.ones(len(e)) if weights is None else np.asarray(weights, dtype=np.float64)
    for (u, v), we in zip(e, w):
        HC += 0.5 * we * (np.eye(dim) - _op_on(n, int(u), Z) @ _op_on(n, int(v), Z))
    if fields is not None:  # sum_i h_i 1/2 (1 - Z_i)
        for i, hi in enumerate(np.asarray(fields, dtype=np.float64)):
            HC += 0.5 * hi * (np.eye(dim) - _op_on(n, i, Z))
    HM = sum(_op_on(n, q, X) for q in range(n))
    psi = np.ones(dim, dtype=np.complex128) / math.sqrt(dim)
    for g, b in zip(gamma, beta):
        psi = expm(-1j * g * HC) @ psi
        psi = expm(-1j * b * HM) @ psi
    return psi


def small_graphs():
    return [
        W.cycle_graph(5), W.complete_graph(4), W.star_graph(6), W.prufer_tree(7, 3),
        W.random_regular(6, 3, 1), (3, W.canonical_edges([(0, 2)])), W.heap_binary_tree(7),
    ]


def check_bruteforce():
    worst = 0.0
    for k, (n, e) in enumerate(small_graphs()):
        g, b = W.random_angles(2, 100 + k)
        ref = dense_state(n, e, g, b)
        got = O.qaoa_state(n, e, g, b)
        worst = max(worst, float(np.max(np.abs(got - ref))))
    return worst


def closed_form_graphs():
    gs = [W.random_regular(12, 3, 5), W.prufer_tree(11, 2), W.complete_graph(9), W.cycle_graph(10),
          W.generalized_petersen(5, 2), W.circulant_graph(11, (1, 3)), W.star_graph(9)]
    r = W.rng(77)
    # an Erdos-Renyi-style graph with triangles and uneven degrees
    e = [(i, j) for i in range(10) for j in range(i + 1, 10) if r.uniform() < 0.4]
    gs.append((10, W.canonical_edges(e)))
    return gs


def check_closed_form():
    worst = 0.0
    for k, (n, e) in enumerate(closed_form_graphs()):
        g, b = W.random_angles(1, 200 + k)
        E, dg, db = O.energy_grad(n, e, g, b)
        Ec, dgc, dbc = CF.energy_grad_p1(n, e, g, b)
        scale = max(abs(Ec), 1.0)
        worst = max(worst, abs(E - Ec) / scale, _rel(dg, dgc, scale), _rel(db, dbc, scale))
    return worst


def check_symmetric():
    worst = 0.0
    for k, (kind, n) in enumerate((("complete", 7), ("complete", 10), ("star", 8), ("star", 11))):
        p = 1 + k % 3
        g, b = W.random_angles(p, 300 + k)
        if kind == "complete":
            _, e = W.complete_graph(n)
            model = SYM.complete_graph_model(n)
        else:
            _, e = W.star_graph(n)
            model = SYM.star_model(n)
        E, dg, db = O.energy_grad(n, e, g, b)
        Es, dgs, dbs = SYM.energy_grad(model, g, b)
        scale = max(abs(Es), 1.0)
        worst = max(worst, abs(E - Es) / scale, _rel(dg, dgs, scale), _rel(db, dbs, scale))
    return worst


def check_finite_difference():
    worst = 0.0
    for k, (n, e) in enumerate((W.random_regular(10, 3, 8), W.prufer_tree(9, 4))):
        g, b = W.random_angles(3, 400 + k)
        E, dg, db = O.energy_grad(n, e, g, b)
        fg, fb = O.finite_difference_grad(n, e, g, b, h=1e-5)
        scale = max(abs(E), 1.0)
        worst = max(worst, _rel(dg, fg, scale), _rel(db, fb, scale))
    return worst


def check_invariants():
    """Largest violation over a set of exact identities (all should be ~1e-13)."""
    worst = 0.0
    cases = [W.cycle_graph(7), W.prufer_tree(8, 1), W.random_regular(8, 3, 2), W.star_graph(7),
             W.complete_graph(6), W.heap_binary_tree(8)]
    for k, (n, e) in enumerate(cases):
        m = len(e)
        g, b = W.random_angles(2, 500 + k)
        psi = O.qaoa_state(n, e, g, b)
        E = O.energy(n, e, g, b)
        worst = max(worst, abs(np.vdot(psi, psi).real - 1.0))
        worst = max(worst, abs(O.energy(n, e, np.zeros(2), b) - m / 2) / m)
        worst = max(worst, abs(O.energy(n, e, g, np.zeros(2)) - m / 2) / m)
        worst = max(worst, abs(O.energy(n, e, g, b + np.array([math.pi / 2, 0.0])) - E) / m)
        worst = max(worst, abs(O.energy(n, e, g + np.array([0.0, 2 * math.pi]), b) - E) / m)
        worst = max(worst, abs(O.energy(n, e, -g, -b) - E) / m)
        flip = (1 << n) - 1
        worst = max(worst, float(np.max(np.abs(psi - psi[np.arange(1 << n) ^ flip]))))
        for i in range(n):
            zi = np.sum(np.abs(psi) ** 2 * (1 - 2 * ((np.arange(1 << n) >> i) & 1)))
            worst = max(worst, abs(zi))
        # Eq. (A2): psi(pi x) = psi(x) for each automorphism pi
        group = AUT.automorphism_group(n, e)
        xs = np.arange(1 << n)
        for perm in group[: min(len(group), 12)]:
            px = np.zeros_like(xs)
            for i in range(n):
                px |= ((xs >> i) & 1) << perm[i]
            worst = max(worst, float(np.max(np.abs(psi[px] - psi))))
        # Eq. (A3): equal <ZZ> inside an edge orbit; Eq. (exact): <H_red> = <H_C>
        orbits, _ = AUT.edge_orbit_partition(n, e)
        for orb in orbits:
            vals = [O.zz(n, psi, u, v) for u, v in orb]
            worst = max(worst, max(vals) - min(vals))
        idx = {tuple(map(int, x)): i for i, x in enumerate(e)}
        reps = [idx[min(orb)] for orb in orbits]
        wts = [len(orb) for orb in orbits]
        red = O.reduced_observable(e, reps, wts)
        Ered, dgr, dbr = O.energy_grad(n, e, g, b, red)
        Efull, dgf, dbf = O.energy_grad(n, e, g, b)
        worst = max(worst, abs(Ered - Efull) / m, _rel(dgr, dgf, m), _rel(dbr, dbf, m))
        # Eq. (agg): term-by-term aggregation equals the diagonal sum
        worst = max(worst, abs(O.expect_terms(n, psi, O.full_observable(e)) - E) / m)
        worst = max(worst, abs(O.expect_terms(n, psi, red) - E) / m)
        # 0 <= E <= C_max (max cut by brute force)
        cmax = max(O.cut_value(e, x) for x in range(1 << n))
        worst = max(worst, max(0.0, -E), max(0.0, E - cmax))
    return worst


def check_max_cut():
    """C_max by exhaustion against textbook values: a tree (bipartite) cuts
    every edge; K_n cuts floor(n/2) * ceil(n/2); a cycle cuts n edges if n
    is even, n - 1 if odd; K_{a,b} cuts a*b; the Petersen graph's maximum cut
    is 12. The maximiser returned is the smallest: on C_6, x = 0b010101 and
    every smaller x cuts less. Returns the largest violation (in edges)."""
    worst = 0.0
    for n, e in (W.prufer_tree(12, 4), W.heap_binary_tree(15), W.balanced_tree(3, 2), W.star_graph(9)):
        c, x = O.max_cut(n, e)
        worst = max(worst, abs(c - len(e)), abs(O.cut_value(e, x) - c))
    for n in range(2, 10):
        worst = max(worst, abs(O.max_cut(*W.complete_graph(n))[0] - (n // 2) * ((n + 1) // 2)))
    for n in range(3, 12):
        worst = max(worst, abs(O.max_cut(*W.cycle_graph(n))[0] - (n - n % 2)))
    kab = W.canonical_edges([(i, 3 + j) for i in range(3) for j in range(4)])
    worst = max(worst, abs(O.max_cut(7, kab)[0] - 12), abs(O.max_cut(*W.generalized_petersen(5, 2))[0] - 12))
    n, e = W.cycle_graph(6)
    c, x = O.max_cut(n, e)
    worst = max(worst, float(x != 0b010101), float(any(O.cut_value(e, y) >= c for y in range(x))))
    return float(worst)


def check_sampler():
    """Inverse-CDF sampling with given uniforms: a basis state always
    returns itself; |+>^6 returns floor(u 2^6); 100000 stratified uniforms
    reproduce every probability of an unnormalised random state to one
    count. Returns the largest violation (in states or counts)."""
    n = 6
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[37] = 1.0
    worst = float(np.max(np.abs(O.sample(psi, np.linspace(0.0, 0.999, 50)).astype(np.int64) - 37)))
    u = (np.arange(640) + 0.37) / 640
    got = O.sample(O.plus_state(n), u).astype(np.int64)
    worst = max(worst, float(np.max(np.abs(got - np.floor(u * 64).astype(np.int64)))))
    rng = W.rng(3)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    pr = np.abs(psi) ** 2 / np.sum(np.abs(psi) ** 2)
    K = 100000
    counts = np.bincount(O.sample(psi, (np.arange(K) + 0.5) / K).astype(np.int64), minlength=1 << n)
    worst = max(worst, float(np.max(np.abs(counts - K * pr))) - 1.0 - 1e-9)
    return max(worst, 0.0)


ALL_CHECKS = {
    "bruteforce": check_bruteforce,
    "closed_form": check_closed_form,
    "symmetric": check_symmetric,
    "finite_difference": check_finite_difference,
    "invariants": check_invariants,
    "max_cut": check_max_cut,
    "sampler": check_sampler,
}


def check_weighted():
    """Integer edge weights: the oracle's state against dense exponentials of
    the weighted H_C, and the scaling E_{c w}(gamma, beta) = c E_w(c gamma, beta)
    for a uniform factor c (the phase sees c*gamma, the observable c)."""
    worst = 0.0
    for k, (n, e) in enumerate(small_graphs()):
        w = W.rng(200 + k).integers(1, 5, size=len(e))
        g, b = W.random_angles(2, 300 + k)
        ref = dense_state(n, e, g, b, w)
        worst = max(worst, float(np.max(np.abs(O.qaoa_state_w(n, e, w, g, b) - ref))))
        E1 = O.energy_grad_w(n, e, w, g, b)[0]
        E3 = O.energy_grad_w(n, e, 3 * w, np.asarray(g) / 3.0, b)[0]
        worst = max(worst, abs(E3 - 3.0 * E1) / max(abs(E1), 1.0))
    return worst


# ------------------------------------------------------------ light cones
def path_graph(n):
    return n, W.canonical_edges([(i, i + 1) for i in range(n - 1)])


def caterpillar_graph():
    """Spine 0..6 with one leg per spine vertex (7..13): a tree of 14 vertices
    whose vertices have degrees 1..3 and whose balls differ in shape."""
    spine = [(i, i + 1) for i in range(6)]
    legs = [(i, 7 + i) for i in range(7)]
    return 14, W.canonical_edges(spine + legs)


def lightcone_cases():
    """(graph, depths): every radius-p ball is strictly smaller than the graph,
    except for the star, whose ball is the whole graph (a control)."""
    return [
        (W.cycle_graph(14), (1, 2)),
        (W.random_regular(14, 3, 6), (1,)),
        (path_graph(14), (1, 2, 3)),
        (caterpillar_graph(), (1, 2, 3)),
        (W.star_graph(9), (1, 2)),
    ]


def _distances(n, edges, u, v):
    adj = [[] for _ in range(n)]
    for a, b in np.asarray(edges).reshape(-1, 2):
        adj[int(a)].append(int(b))
        adj[int(b)].append(int(a))
    dist = {u: 0, v: 0}
    frontier = [u, v]
    while frontier:
        nxt = []
        for a in frontier:
            for b in adj[a]:
                if b not in dist:
                    dist[b] = dist[a] + 1
                    nxt.append(b)
        frontier = nxt
    return dist


def check_lightcone(lc=None):
    """Per-edge light cones (Sec. 5.1, reverse causal cone) against the full
    statevector: E and every gradient component of H_C, and of a weighted
    subset of edges (the form H_red takes), on graphs whose balls leave
    vertices out. Also the cone's own claim that the edges joining two
    vertices at distance exactly p do not matter: removing them from the
    subproblem leaves every per-edge value unchanged."""
    lc = LC if lc is None else lc
    worst = 0.0
    for k, ((n, e), depths) in enumerate(lightcone_cases()):
        for p in depths:
            g, b = W.random_angles(p, 600 + 10 * k + p)
            E, dg, db = O.energy_grad(n, e, g, b)
            El, dgl, dbl = lc.energy_grad(n, e, g, b)
            scale = max(abs(E), 1.0)
            worst = max(worst, abs(El - E) / scale, _rel(dgl, dg, scale), _rel(dbl, db, scale))
            r = W.rng(700 + 10 * k + p)
            idx = np.sort(r.choice(len(e), size=max(1, len(e) // 3), replace=False))
            wts = r.integers(1, 6, size=len(idx)).astype(np.float64)
            obs = (np.asarray(e)[idx], wts)
            Ew, dgw, dbw = O.energy_grad(n, e, g, b, obs)
            Elw, dglw, dblw = lc.energy_grad(n, e, g, b, weights=wts, edge_subset=idx)
            sw = max(abs(Ew), 1.0)
            worst = max(worst, abs(Elw - Ew) / sw, _rel(dglw, dgw, sw), _rel(dblw, dbw, sw))
            # edges whose two ends are both at distance p cancel
            u, v = (int(x) for x in np.asarray(e)[len(e) // 2])
            dist = _distances(n, e, u, v)
            verts = sorted(a for a in dist if dist[a] <= p)
            index = {a: i for i, a in enumerate(verts)}
            keep = [(index[int(a)], index[int(c)]) for a, c in np.asarray(e)
                    if int(a) in index and int(c) in index and not (dist[int(a)] == p and dist[int(c)] == p)]
            sub = W.canonical_edges(keep)
            one = (W.canonical_edges([(index[u], index[v])]), np.ones(1))
            Eb, dgb, dbb = O.energy_grad(len(verts), sub, g, b, one)
            Ee, dge, dbe = lc.edge_energy_grad(n, e, u, v, g, b)
            worst = max(worst, abs(Eb - Ee), _rel(dgb, dge, 1.0), _rel(dbb, dbe, 1.0))
    return worst


ALL_CHECKS["lightcone"] = check_lightcone


def lightcone_cases_leave_vertices_out():
    """How many (graph, p) light-cone cases have a ball smaller than the graph."""
    return sum(1 for (n, e), depths in lightcone_cases() for p in depths if LC.max_ball(n, e, p) < n)


# ------------------------------------------------ Ising-form objectives
def ising_cases():
    """Small graphs with real edge weights of both signs and real fields."""
    out = []
    for k, (n, e) in enumerate(small_graphs()):
        r = W.rng(900 + k)
        w = r.uniform(-2.0, 3.0, size=len(e))
        h = r.uniform(-1.5, 1.5, size=n)
        out.append((n, e, w, h))
    return out


def check_ising_dense():
    """The Ising oracle's state against dense exponentials of
    H = sum w_e 1/2 (1 - Z_u Z_v) + sum h_i 1/2 (1 - Z_i), amplitude by amplitude."""
    worst = 0.0
    for k, (n, e, w, h) in enumerate(ising_cases()):
        g, b = W.random_angles(2, 950 + k)
        ref = dense_state(n, e, g, b, w, h)
        got = O.ising_state(n, O.ising(e, w, h), g, b)
        worst = max(worst, float(np.max(np.abs(got - ref))))
    return worst


def fields_only_p1(h, gamma, beta):
    """No edges, p = 1: the qubits evolve independently and
    <x_i> = 1/2 (1 + sin(2 beta) sin(gamma h_i)), so
    E = sum_i h_i/2 (1 + sin 2b sin(g h_i)) with its two derivatives."""
    h = np.asarray(h, dtype=np.float64)
    s2, c2 = math.sin(2 * beta), math.cos(2 * beta)
    E = float(np.sum(0.5 * h * (1 + s2 * np.sin(gamma * h))))
    dg = float(np.sum(0.5 * h * s2 * np.cos(gamma * h) * h))
    db = float(np.sum(h * c2 * np.sin(gamma * h)))
    return E, dg, db


def check_ising_fields_closed_form():
    worst = 0.0
    for k in range(4):
        n = 3 + k
        h = W.rng(970 + k).uniform(-2.0, 2.0, size=n)
        g, b = W.random_angles(1, 980 + k)
        E, dg, db = O.ising_energy_grad(n, O.ising(np.zeros((0, 2)), np.zeros(0), h), g, b)
        Ec, dgc, dbc = fields_only_p1(h, g[0], b[0])
        worst = max(worst, abs(E - Ec), abs(dg[0] - dgc), abs(db[0] - dbc))
    return worst


def check_ising_reductions():
    """Without fields and with unit weights the Ising routines give the MaxCut
    oracle's energy and gradient; with integer weights, the weighted-MaxCut
    route (edge e repeated w_e times); scaling every weight and field by c
    is the same as scaling gamma by c and the energy by c."""
    worst = 0.0
    for k, (n, e) in enumerate(small_graphs()):
        g, b = W.random_angles(2, 990 + k)
        E1, dg1, db1 = O.ising_energy_grad(n, O.ising(e, np.ones(len(e)), None), g, b)
        E0, dg0, db0 = O.energy_grad(n, e, g, b)
        s = max(abs(E0), 1.0)
        worst = max(worst, abs(E1 - E0) / s, _rel(dg1, dg0, s), _rel(db1, db0, s))
        wi = W.rng(995 + k).integers(1, 4, size=len(e))
        E2 = O.ising_energy_grad(n, O.ising(e, wi.astype(float), None), g, b)[0]
        E3 = O.energy_grad_w(n, e, wi, g, b)[0]
        worst = max(worst, abs(E2 - E3) / max(abs(E3), 1.0))
    for k, (n, e, w, h) in enumerate(ising_cases()):
        g, b = W.random_angles(2, 1000 + k)
        c = 2.5
        E1 = O.ising_energy_grad(n, O.ising(e, w, h), g, b)[0]
        Ec = O.ising_energy_grad(n, O.ising(e, c * w, c * h), np.asarray(g) / c, b)[0]
        worst = max(worst, abs(Ec - c * E1) / max(abs(E1), 1.0))
    return worst


def check_ising_finite_difference():
    worst = 0.0
    for k, (n, e, w, h) in enumerate(ising_cases()[:4]):
        fn = O.ising(e, w, h)
        # an observable that is not the cost function (other weights, fields)
        r = W.rng(1015 + k)
        obs = O.ising(e, r.uniform(-1, 2, size=len(e)), r.uniform(-1, 1, size=n))
        g, b = (np.array(x) for x in W.random_angles(3, 1010 + k))
        E, dg, db = O.ising_energy_grad(n, fn, g, b, obs)
        hh = 1e-5
        for vec, got in ((g, dg), (b, db)):
            for i in range(len(vec)):
                old = vec[i]
                vec[i] = old + hh
                ep = O.ising_energy(n, fn, g, b, obs)
                vec[i] = old - hh
                em = O.ising_energy(n, fn, g, b, obs)
                vec[i] = old
                worst = max(worst, abs((ep - em) / (2 * hh) - got[i]) / max(abs(E), 1.0))
    return worst


def check_ising_invariants():
    """Automorphisms that preserve weights and fields (brute force) leave the
    state invariant (Eq. A2), give equal <Z_u Z_v> within an edge orbit and
    equal <Z_i> within a vertex orbit (Eq. A3), and H_red built from both
    kinds of orbits has the energy and gradient of H (Eq. exact)."""
    worst = 0.0
    cases = [W.cycle_graph(6), W.star_graph(7), W.complete_graph(5), W.heap_binary_tree(7)]
    for k, (n, e) in enumerate(cases):
        r = W.rng(1020 + k)
        # weights and fields that depend on vertex degrees (kept by every
        # automorphism), plus a field singling out vertex 0, which breaks
        # part of the group
        deg = np.bincount(np.asarray(e).reshape(-1), minlength=n)
        w = np.array([1.5 if (deg[u] + deg[v]) % 2 else -0.75 for u, v in e]) * (1 + 0.1 * r.uniform())
        h = np.array([0.6 if i == 0 else -0.4 * deg[i] / deg.max() for i in range(n)])
        group = AUT.automorphism_group(n, e, w, h)
        assert len(group) > 1
        fn = O.ising(e, w, h)
        g, b = W.random_angles(2, 1030 + k)
        psi = O.ising_state(n, fn, g, b)
        xs = np.arange(1 << n)
        for perm in group[: min(len(group), 12)]:
            px = np.zeros_like(xs)
            for i in range(n):
                px |= ((xs >> i) & 1) << perm[i]
            worst = max(worst, float(np.max(np.abs(psi[px] - psi))))
        eorb, vorb = AUT.ising_orbit_partition(n, e, w, h)
        pr = np.abs(psi) ** 2
        for orb in eorb:
            vals = [O.zz(n, psi, u, v) for u, v in orb]
            worst = max(worst, max(vals) - min(vals))
        for orb in vorb:
            vals = [float(np.sum(pr * (1 - 2 * ((xs >> i) & 1)))) for i in orb]
            worst = max(worst, max(vals) - min(vals))
        idx = {tuple(map(int, x)): i for i, x in enumerate(e)}
        erep = [idx[min(o)] for o in eorb]
        ewt = [len(o) for o in eorb]
        vrep = [min(o) for o in vorb]
        vwt = [len(o) for o in vorb]
        red = O.ising_reduced_observable(fn, erep, ewt, vrep, vwt)
        Er, dgr, dbr = O.ising_energy_grad(n, fn, g, b, red)
        Ef, dgf, dbf = O.ising_energy_grad(n, fn, g, b)
        s = max(abs(Ef), 1.0)
        worst = max(worst, abs(Er - Ef) / s, _rel(dgr, dgf, s), _rel(dbr, dbf, s))
    return worst


ALL_CHECKS["ising_dense"] = check_ising_dense
ALL_CHECKS["ising_fields_closed_form"] = check_ising_fields_closed_form
ALL_CHECKS["ising_reductions"] = check_ising_reductions
ALL_CHECKS["ising_invariants"] = check_ising_invariants
ALL_CHECKS["ising_finite_difference"] = check_ising_finite_difference


def check_ising_lightcone(lc=None):
    """Per-term light cones of Ising objectives against the full Ising
    oracle, on graphs whose radius-p balls leave vertices out."""
    lc = LC if lc is None else lc
    worst = 0.0
    for k, ((n, e), depths) in enumerate(lightcone_cases()[:4]):
        w, h = W.ising_couplings(n, e, 1100 + k)
        for p in depths[:2]:
            g, b = W.random_angles(p, 1110 + 10 * k + p)
            E, dg, db = O.ising_energy_grad(n, O.ising(e, w, h), g, b)
            El, dgl, dbl = lc.ising_energy_grad(n, e, w, h, g, b)
            s = max(abs(E), 1.0)
            worst = max(worst, abs(El - E) / s, _rel(dgl, dg, s), _rel(dbl, db, s))
    return worst
