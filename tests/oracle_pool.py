"""Oracle evaluations spread over the host cores (test infrastructure).

The workers are started with the "spawn" method, never by fork: a process
forked after the parent has touched the CUDA driver can hang. Each worker
imports the oracle afresh and evaluates one job at a time.
"""
from __future__ import annotations

import multiprocessing as mp
import os


def _energy_job(args):
    from oracle import oracle as O
    n, edges, gamma, beta, obs = args
    return O.energy(n, edges, gamma, beta, obs)


def _energy_grad_job(args):
    from oracle import oracle as O
    n, edges, gamma, beta, obs = args
    E, dg, db = O.energy_grad(n, edges, gamma, beta, obs)
    return E, dg, db


def workers() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def _map(fn, jobs):
    jobs = list(jobs)
    if len(jobs) <= 1:
        return [fn(j) for j in jobs]
    order = sorted(range(len(jobs)), key=lambda i: -int(jobs[i][0]))  # largest n first
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(workers(), len(jobs))) as pool:
        res = pool.map(fn, [jobs[i] for i in order], chunksize=1)
    out = [None] * len(jobs)
    for i, r in zip(order, res):
        out[i] = r
    return out


def energies(jobs):
    """[(n, edges, gamma, beta, obs or None)] -> oracle energies, in order."""
    return _map(_energy_job, jobs)


def energy_grads(jobs):
    """[(n, edges, gamma, beta, obs or None)] -> (E, dE/dgamma, dE/dbeta), in order."""
    return _map(_energy_grad_job, jobs)
