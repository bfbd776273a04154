"""Symmetric-subspace QAOA for K_n and stars (test infrastructure).

On K_n the QAOA state is invariant under every vertex permutation (Eq. (A2)),
so it lives in the (n+1)-dimensional span of the Dicke states |D_k> (uniform
superpositions of the basis states of Hamming weight k). There:
  * |+>^n has components sqrt(binom(n, k)) / 2^{n/2};
  * H_C is diagonal with C = k (n - k);
  * H_M = sum_i X_i is tridiagonal with <D_{k+1}| H_M |D_k> = sqrt((k+1)(n-k)).

For the star (centre 0, L = n-1 leaves) the state is invariant under leaf
permutations, so it lives in span{|x_0> (x) |D_k^{(L)}>}, 2(L+1) dimensions,
with C = k if x_0 = 0 else L - k and H_M = X_0 (x) 1 + 1 (x) H_M^{(L)}.

Energy and gradient are computed with the same adjoint recursion as the full
oracle but on these small dense matrices (matrix exponentials by the
eigendecomposition of the real symmetric H_M), so K_16 and S_29 (n = 30) have
exact FP64 reference values at any p.
"""
from __future__ import annotations

from math import comb

import numpy as np


def _dicke_mixer(L):
    h = np.zeros((L + 1, L + 1))
    for k in range(L):
        h[k + 1, k] = h[k, k + 1] = np.sqrt((k + 1) * (L - k))
    return h


def complete_graph_model(n):
    """(c0, cost diagonal, H_M) of K_n in the Dicke basis."""
    k = np.arange(n + 1)
    c0 = np.sqrt(np.array([comb(n, int(j)) for j in k], dtype=np.float64)) / 2.0 ** (n / 2)
    cost = (k * (n - k)).astype(np.float64)
    return c0.astype(np.complex128), cost, _dicke_mixer(n)


def star_model(n):
    """(c0, cost diagonal, H_M) of the star on n vertices (centre 0)."""
    L = n - 1
    k = np.arange(L + 1)
    leaf0 = np.sqrt(np.array([comb(L, int(j)) for j in k], dtype=np.float64)) / 2.0 ** (n / 2)
    c0 = np.concatenate([leaf0, leaf0]).astype(np.complex128)  # index x0*(L+1) + k
    cost = np.concatenate([k, L - k]).astype(np.float64)
    hl = _dicke_mixer(L)
    x0 = np.array([[0.0, 1.0], [1.0, 0.0]])
    hm = np.kron(x0, np.eye(L + 1)) + np.kron(np.eye(2), hl)
    return c0, cost, hm


class _Expm:
    """exp(-i t H) for a fixed real symmetric H through one eigendecomposition."""

    def __init__(self, h):
        self.w, self.v = np.linalg.eigh(h)

    def __call__(self, t, c):
        return self.v @ (np.exp(-1j * t * self.w) * (self.v.T @ c))


def energy_grad(model, gamma, beta):
    """(E, dE/dgamma, dE/dbeta) of H_C in the symmetric subspace, FP64."""
    c0, cost, hm = model
    ex = _Expm(hm)
    gamma = np.asarray(gamma, dtype=np.float64).reshape(-1)
    beta = np.asarray(beta, dtype=np.float64).reshape(-1)
    p = len(gamma)
    phi = c0.copy()
    for l in range(p):
        phi = np.exp(-1j * gamma[l] * cost) * phi
        phi = ex(beta[l], phi)
    E = float(np.sum(np.abs(phi) ** 2 * cost))
    lam = cost * phi
    dg, db = np.zeros(p), np.zeros(p)
    for l in range(p - 1, -1, -1):
        db[l] = 2.0 * np.imag(np.vdot(lam, hm @ phi))
        phi = ex(-beta[l], phi)
        lam = ex(-beta[l], lam)
        dg[l] = 2.0 * np.imag(np.vdot(lam, cost * phi))
        phi = np.exp(1j * gamma[l] * cost) * phi
        lam = np.exp(1j * gamma[l] * cost) * lam
    return E, dg, db


def energy(model, gamma, beta):
    return energy_grad(model, gamma, beta)[0]


def cut_distribution(model, gamma, beta):
    """{cut value: probability} of the final state, FP64. In the symmetric
    basis each component is one normalised Dicke state (times a centre bit for
    the star) whose basis states all share one cut value, so its probability
    is |component|^2."""
    c0, cost, hm = model
    ex = _Expm(hm)
    phi = c0.copy()
    for l in range(len(np.atleast_1d(gamma))):
        phi = np.exp(-1j * np.atleast_1d(gamma)[l] * cost) * phi
        phi = ex(np.atleast_1d(beta)[l], phi)
    out = {}
    for c, a in zip(cost.astype(int), np.abs(phi) ** 2):
        out[int(c)] = out.get(int(c), 0.0) + float(a)
    return out
