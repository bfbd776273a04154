"""Closed-form p = 1 MaxCut QAOA energy (test infrastructure).

For one layer, the expectation of a single edge term 1/2 (1 - Z_u Z_v) has a
closed form in the degrees of u and v and the number of triangles through the
edge (Wang, Hadfield, Jiang and Rieffel, Phys. Rev. A 97, 022304 (2018),
Theorem 1). With d = deg(u) - 1, e = deg(v) - 1, f = #common neighbours:

    <C_uv> = 1/2 + 1/4 sin(4b) sin(g) (cos^d g + cos^e g)
                 - 1/4 sin^2(2b) cos^{d+e-2f}(g) (1 - cos^f(2g))

under the ansatz exp(-i b H_M) exp(-i g H_C) |+>^n of Eq. (1). Summing over
all edges gives E_C at any n, which pins the oracle (and, at full size, the
CUDA path) for p = 1. Derivatives come from complex-step differentiation of
the same expression, exact to rounding.
"""
from __future__ import annotations

import numpy as np


def _edge_terms(n, edges):
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    nbr = [set() for _ in range(n)]
    for u, v in edges:
        nbr[u].add(int(v))
        nbr[v].add(int(u))
    out = []
    for u, v in edges:
        d = len(nbr[u]) - 1
        e = len(nbr[v]) - 1
        f = len(nbr[u] & nbr[v])
        out.append((d, e, f))
    return out


def edge_expectation(d, e, f, gamma, beta):
    """<1/2 (1 - Z_u Z_v)> at p = 1 for an edge with the given (d, e, f)."""
    g, b = gamma, beta
    cg = np.cos(g)
    t1 = 0.25 * np.sin(4 * b) * np.sin(g) * (cg ** d + cg ** e)
    t2 = 0.25 * np.sin(2 * b) ** 2 * cg ** (d + e - 2 * f) * (1 - np.cos(2 * g) ** f)
    return 0.5 + t1 - t2


def energy_p1(n, edges, gamma, beta, weights=None):
    """sum over edges (optionally weighted) of the p = 1 edge expectation."""
    terms = _edge_terms(n, edges)
    w = np.ones(len(terms)) if weights is None else np.asarray(weights, dtype=np.float64)
    return sum(wk * edge_expectation(d, e, f, gamma, beta) for wk, (d, e, f) in zip(w, terms))


def energy_grad_p1(n, edges, gamma, beta, h=1e-30):
    """(E, dE/dgamma, dE/dbeta) at p = 1 via complex-step differentiation."""
    g = float(np.asarray(gamma).reshape(-1)[0])
    b = float(np.asarray(beta).reshape(-1)[0])
    E = float(np.real(energy_p1(n, edges, g, b)))
    dg = float(np.imag(energy_p1(n, edges, g + 1j * h, b)) / h)
    db = float(np.imag(energy_p1(n, edges, g, b + 1j * h)) / h)
    return E, np.array([dg]), np.array([db])
