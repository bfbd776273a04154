"""CPU oracle: ctypes front end of ``qaoa_oracle.c`` (test infrastructure).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this module. It never calls into the CUDA library and the CUDA
library never calls into it.

Observables are given as weighted edge lists ``(obs_edges, weights)`` standing
for 1/2 sum_k w_k (1 - Z_{u_k} Z_{v_k}): all edges at weight 1 is H_C, the
orbit representatives at weight |S~_m| is H_red (Sec. 5, "Reducing the Hamiltonian").
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qaoa_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_OMP_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_omp.so")
_lib = None


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain -O2, no fast-math).

    openmp=True builds the same source with -fopenmp into a second library,
    used only to time the oracle on all host cores; the pinned oracle that
    the tests load is always the plain build."""
    path = _OMP_LIB_PATH if openmp else _LIB_PATH
    if not force and os.path.exists(path) and os.path.getmtime(path) >= os.path.getmtime(_SRC):
        return path
    os.makedirs(_OUT_DIR, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared"] + (["-fopenmp"] if openmp else [])
    subprocess.check_call(cmd + ["-o", tmp, _SRC, "-lm"])
    os.replace(tmp, path)
    return path


def load_library(path):
    """Bind the oracle's C entry points from the shared object at ``path``."""
    lib = ctypes.CDLL(path)
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    c128p = np.ctypeslib.ndpointer(np.complex128, flags="C_CONTIGUOUS")
    lib.oracle_cut_value.restype = ctypes.c_int64
    lib.oracle_cut_value.argtypes = [ctypes.c_int, i32p, ctypes.c_uint64]
    lib.oracle_observable_value.restype = ctypes.c_double
    lib.oracle_observable_value.argtypes = [ctypes.c_int, i32p, f64p, ctypes.c_uint64]
    lib.oracle_plus_state.restype = None
    lib.oracle_plus_state.argtypes = [ctypes.c_int, c128p]
    lib.oracle_apply_cost.restype = None
    lib.oracle_apply_cost.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_double, c128p]
    lib.oracle_apply_rx.restype = None
    lib.oracle_apply_rx.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, c128p]
    lib.oracle_apply_mixer.restype = None
    lib.oracle_apply_mixer.argtypes = [ctypes.c_int, ctypes.c_double, c128p]
    lib.oracle_qaoa_state.restype = None
    lib.oracle_qaoa_state.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, f64p, f64p, c128p]
    lib.oracle_expect_diag.restype = ctypes.c_double
    lib.oracle_expect_diag.argtypes = [ctypes.c_int, c128p, ctypes.c_int, i32p, f64p]
    lib.oracle_zz.restype = ctypes.c_double
    lib.oracle_zz.argtypes = [ctypes.c_int, c128p, ctypes.c_int, ctypes.c_int]
    lib.oracle_expect_terms.restype = ctypes.c_double
    lib.oracle_expect_terms.argtypes = [ctypes.c_int, c128p, ctypes.c_int, i32p, f64p]
    lib.oracle_energy_grad.restype = ctypes.c_double
    lib.oracle_energy_grad.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, f64p, f64p,
                                       ctypes.c_int, i32p, f64p, f64p, f64p, c128p, c128p]
    lib.oracle_max_cut.restype = ctypes.c_int64
    lib.oracle_max_cut.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.POINTER(ctypes.c_uint64)]
    lib.oracle_ising_value.restype = ctypes.c_double
    lib.oracle_ising_value.argtypes = [ctypes.c_int, i32p, f64p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64]
    lib.oracle_ising_state.restype = None
    lib.oracle_ising_state.argtypes = [ctypes.c_int, ctypes.c_int, i32p, f64p, ctypes.c_void_p, ctypes.c_int, f64p,
                                       f64p, c128p]
    lib.oracle_ising_energy_grad.restype = ctypes.c_double
    lib.oracle_ising_energy_grad.argtypes = [ctypes.c_int, ctypes.c_int, i32p, f64p, ctypes.c_void_p, ctypes.c_int,
                                             f64p, f64p, ctypes.c_int, i32p, f64p, ctypes.c_void_p, f64p, f64p,
                                             c128p, c128p]
    lib.oracle_threads.restype = ctypes.c_int
    lib.oracle_threads.argtypes = []
    lib.oracle_sample.restype = ctypes.c_int
    lib.oracle_sample.argtypes = [ctypes.c_int, c128p, ctypes.c_int, f64p, ctypes.POINTER(ctypes.c_uint64)]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


class use_library:
    """Context manager: run the oracle functions of this module on another
    build of qaoa_oracle.c (the OpenMP timing build) inside the block."""

    def __init__(self, lib):
        self.lib = lib

    def __enter__(self):
        global _lib
        self.saved = _load()
        _lib = self.lib
        return self.lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def threads() -> int:
    """Threads the currently loaded build runs its loops on."""
    return int(_load().oracle_threads())


def _edges(e):
    return np.ascontiguousarray(np.asarray(e, dtype=np.int32).reshape(-1, 2))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))


def full_observable(edges):
    """H_C as a weighted edge list: every edge at weight 1."""
    e = _edges(edges)
    return e, np.ones(len(e), dtype=np.float64)


def reduced_observable(edges, rep, weight):
    """H_red (Sec. 5, equation for H_red): one representative edge per orbit at weight |S~_m|."""
    e = _edges(edges)
    return _edges(e[np.asarray(rep, dtype=np.int64)]), _f64(weight)


def cut_value(edges, x: int) -> int:
    e = _edges(edges)
    return int(_load().oracle_cut_value(len(e), e, x))


def observable_value(obs, x: int) -> float:
    oe, w = obs
    return float(_load().oracle_observable_value(len(oe), _edges(oe), _f64(w), x))


def plus_state(n):
    psi = np.empty(1 << n, dtype=np.complex128)
    _load().oracle_plus_state(n, psi)
    return psi


def apply_cost(n, edges, gamma, psi):
    e = _edges(edges)
    _load().oracle_apply_cost(n, len(e), e, float(gamma), psi)
    return psi


def apply_rx(n, q, beta, psi):
    _load().oracle_apply_rx(n, q, float(beta), psi)
    return psi


def apply_mixer(n, beta, psi):
    _load().oracle_apply_mixer(n, float(beta), psi)
    return psi


def qaoa_state(n, edges, gamma, beta):
    """The p-layer state of Eq. (1) as a complex128 vector of 2^n amplitudes."""
    e = _edges(edges)
    g, b = _f64(gamma), _f64(beta)
    psi = np.empty(1 << n, dtype=np.complex128)
    _load().oracle_qaoa_state(n, len(e), e, len(g), g, b, psi)
    return psi


def expect_diag(n, psi, obs):
    oe, w = obs
    return float(_load().oracle_expect_diag(n, psi, len(oe), _edges(oe), _f64(w)))


def zz(n, psi, u, v):
    return float(_load().oracle_zz(n, psi, int(u), int(v)))


def expect_terms(n, psi, obs):
    oe, w = obs
    return float(_load().oracle_expect_terms(n, psi, len(oe), _edges(oe), _f64(w)))


def energy(n, edges, gamma, beta, obs=None):
    """E = <psi|O|psi>; O defaults to H_C."""
    if obs is None:
        obs = full_observable(edges)
    return expect_diag(n, qaoa_state(n, edges, gamma, beta), obs)


def energy_grad(n, edges, gamma, beta, obs=None):
    """(E, dE/dgamma, dE/dbeta) by the adjoint recursion, FP64."""
    if obs is None:
        obs = full_observable(edges)
    e = _edges(edges)
    g, b = _f64(gamma), _f64(beta)
    p = len(g)
    oe, w = obs
    dg = np.zeros(p)
    db = np.zeros(p)
    phi = np.empty(1 << n, dtype=np.complex128)
    lam = np.empty(1 << n, dtype=np.complex128)
    E = _load().oracle_energy_grad(n, len(e), e, p, g, b, len(oe), _edges(oe), _f64(w), dg, db, phi, lam)
    return float(E), dg, db


def finite_difference_grad(n, edges, gamma, beta, obs=None, h=1e-6):
    """Central finite differences of the oracle energy (FP64)."""
    g, b = _f64(gamma).copy(), _f64(beta).copy()
    dg, db = np.zeros_like(g), np.zeros_like(b)
    for vec, out in ((g, dg), (b, db)):
        for i in range(len(vec)):
            old = vec[i]
            vec[i] = old + h
            ep = energy(n, edges, g, b, obs)
            vec[i] = old - h
            em = energy(n, edges, g, b, obs)
            vec[i] = old
            out[i] = (ep - em) / (2 * h)
    return dg, db


def max_cut(n, edges):
    """(C_max, smallest maximising x) by exhaustion over 2^n states."""
    e = _edges(edges)
    arg = ctypes.c_uint64()
    c = _load().oracle_max_cut(n, len(e), e, ctypes.byref(arg))
    return int(c), int(arg.value)


def sample(psi, u):
    """Inverse-CDF samples of basis states from |psi|^2 for uniforms u in [0, 1)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    n = int(round(np.log2(len(psi))))
    u = _f64(u)
    out = np.zeros(len(u), dtype=np.uint64)
    r = _load().oracle_sample(n, psi, len(u), u, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    if r != 0:
        raise MemoryError("oracle_sample: no memory for the cumulative sums")
    return out


# ------------------------------------------------ integer edge weights
# Weighted MaxCut, H_C = 1/2 sum_e w_e (1 - Z_u Z_v) with integer w_e >= 1: the
# weighted cut sum_e w_e [x_u != x_v] is the plain cut of the edge list in
# which edge e appears w_e times, so the C routines above serve unchanged with
# that list as the cost and (edges, w) as the observable.

def weighted_cost_edges(edges, weights):
    e = _edges(edges)
    w = np.asarray(weights, dtype=np.int64).reshape(-1)
    return _edges(np.repeat(e, w, axis=0))


def full_observable_w(edges, weights):
    return _edges(edges), _f64(weights)


def qaoa_state_w(n, edges, weights, gamma, beta):
    return qaoa_state(n, weighted_cost_edges(edges, weights), gamma, beta)


def energy_grad_w(n, edges, weights, gamma, beta, obs=None):
    """(E, dE/dgamma, dE/dbeta) of weighted MaxCut; obs defaults to the weighted H_C."""
    if obs is None:
        obs = full_observable_w(edges, weights)
    return energy_grad(n, weighted_cost_edges(edges, weights), gamma, beta, obs)


def max_cut_w(n, edges, weights):
    return max_cut(n, weighted_cost_edges(edges, weights))


# ------------------------------------------------ Ising-form objectives
# H = sum_e w_e 1/2 (1 - Z_u Z_v) + sum_i h_i 1/2 (1 - Z_i) with real w_e, h_i;
# diagonal C(x) = sum_e w_e [x_u != x_v] + sum_i h_i x_i. An Ising function is
# (edges, w, h), h None for no fields; it serves as cost and as observable.

def ising(edges, w, h=None):
    """Normalise an Ising function: int32 edges, float64 weights and fields (or None)."""
    e = _edges(edges)
    wv = _f64(w) if w is not None else np.ones(len(e))
    hv = None if h is None else _f64(h)
    if len(wv) != len(e):
        raise ValueError("one weight per edge")
    return e, wv, hv


def _hptr(h):
    return None if h is None else h.ctypes.data_as(ctypes.c_void_p)


def ising_value(fn, n, x: int) -> float:
    e, w, h = fn
    return float(_load().oracle_ising_value(len(e), e, w, n, _hptr(h), x))


def ising_state(n, fn, gamma, beta):
    """The p-layer state of Eq. (1) with cost layers exp(-i gamma_l H)."""
    e, w, h = fn
    g, b = _f64(gamma), _f64(beta)
    psi = np.empty(1 << n, dtype=np.complex128)
    _load().oracle_ising_state(n, len(e), e, w, _hptr(h), len(g), g, b, psi)
    return psi


def ising_energy_grad(n, fn, gamma, beta, obs=None):
    """(E, dE/dgamma, dE/dbeta) of the Ising observable obs (default: the cost
    function itself) by the adjoint recursion, FP64."""
    e, w, h = fn
    oe, ow, oh = fn if obs is None else obs
    g, b = _f64(gamma), _f64(beta)
    p = len(g)
    dg, db = np.zeros(p), np.zeros(p)
    phi = np.empty(1 << n, dtype=np.complex128)
    lam = np.empty(1 << n, dtype=np.complex128)
    E = _load().oracle_ising_energy_grad(n, len(e), e, w, _hptr(h), p, g, b, len(oe), oe, ow, _hptr(oh), dg, db,
                                         phi, lam)
    return float(E), dg, db


def ising_energy(n, fn, gamma, beta, obs=None):
    """E = <psi|O|psi>, O the Ising observable obs (default: the cost function)."""
    return ising_energy_grad(n, fn, gamma, beta, obs)[0]


def ising_reduced_observable(fn, edge_rep, edge_weight, vertex_rep=None, vertex_weight=None, n=None):
    """H_red of an Ising function: one representative edge per edge orbit at
    weight |orbit| w_rep, one representative vertex per vertex orbit at weight
    |orbit| h_rep (no fields when the function has none)."""
    e, w, h = fn
    rep = np.asarray(edge_rep, dtype=np.int64)
    oe = _edges(e[rep]) if len(rep) else np.zeros((0, 2), dtype=np.int32)
    ow = _f64(np.asarray(edge_weight, dtype=np.float64) * w[rep]) if len(rep) else np.zeros(0)
    oh = None
    if h is not None:
        oh = np.zeros(len(h))
        for v, k in zip(np.asarray(vertex_rep, dtype=np.int64), np.asarray(vertex_weight, dtype=np.float64)):
            oh[v] = k * h[v]
    return oe, ow, oh
