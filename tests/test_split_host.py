"""A single statevector split across ranks by its top k qubits, on the host:
2 and 4 gloo ranks on the CPU, each holding a slab of 2^(n-k) amplitudes,
exchanging through all-to-all as paper_2410_22247_gb300.split lays out, and
all-reducing the partial sums once. Energy and adjoint gradient must equal
the full FP64 oracle's to 1e-12; each slab's cost as an Ising-form function
of its local bits (the form a device kernel applies) must reproduce C(x).

The per-slab arithmetic here is plain FP64 numpy (test infrastructure): the
phase exp(-i gamma C(x)) with C at the logical index, RX(2 beta) on a local
physical bit, and the inner products of the adjoint recursion.
"""
import os
import socket

import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_22247_gb300 import split as SP
from paper_2410_22247_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rx_bit(slab, b, beta):
    """RX(2 beta) = [[c, -i s], [-i s, c]] on physical bit b of the slab."""
    v = slab.reshape(-1, 2, 1 << b)
    a, d = v[:, 0, :].copy(), v[:, 1, :].copy()
    c, s = np.cos(beta), np.sin(beta)
    v[:, 0, :] = c * a - 1j * s * d
    v[:, 1, :] = -1j * s * a + c * d


def _x_inner(lam, phi, b):
    """<lambda| X_b |phi> over the slab (pairs differing in local bit b)."""
    ph = phi.reshape(-1, 2, 1 << b)
    fl = np.stack([ph[:, 1, :], ph[:, 0, :]], axis=1).reshape(-1)
    return np.vdot(lam, fl)


def _worker(rank, world, port, n, edges, gamma, beta, obs_edges, obs_w, ret):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    k = int(np.log2(world))
    L = SP.SplitLayout(n, k)
    C = np.array([O.cut_value(edges, x) for x in range(1 << n)], dtype=np.float64)
    Ob = np.array([O.observable_value((obs_edges, obs_w), x) for x in range(1 << n)], dtype=np.float64)
    p = len(gamma)

    def exchange(slab):
        send = torch.from_numpy(np.ascontiguousarray(slab))
        recv = torch.empty_like(send)
        dist.all_to_all_single(torch.view_as_real(recv), torch.view_as_real(send))
        return recv.numpy().copy()

    # forward
    phi = np.full(1 << L.local_bits, 2.0 ** (-n / 2), dtype=np.complex128)
    layout = 0
    for st in SP.layer_schedule(p):
        if st[0] == "phase":
            _, l, layout = st
            phi *= np.exp(-1j * gamma[l] * C[L.logical_index(rank, layout)])
        elif st[0] == "mix":
            _, l, which, layout = st
            qs = L.local_qubits(layout) if which == "local" else L.swapped_in(layout)
            pos = L.pos(layout)
            for q in qs:
                _rx_bit(phi, int(pos[q]), beta[l])
        else:
            phi = exchange(phi)
            layout = st[1]
    xs = L.logical_index(rank, layout)
    part = np.zeros(1 + 2 * p)
    part[0] = float(np.sum(np.abs(phi) ** 2 * Ob[xs]))
    lam = Ob[xs] * phi
    # adjoint: the same steps in reverse on (phi, lambda)
    for st in SP.layer_schedule(p, adjoint=True):
        if st[0] == "mix":
            _, l, which, lay = st
            qs = L.local_qubits(lay) if which == "local" else L.swapped_in(lay)
            pos = L.pos(lay)
            for q in qs:
                part[1 + p + l] += 2.0 * _x_inner(lam, phi, int(pos[q])).imag
                _rx_bit(phi, int(pos[q]), -beta[l])
                _rx_bit(lam, int(pos[q]), -beta[l])
        elif st[0] == "exchange":
            phi, lam = exchange(phi), exchange(lam)
        else:
            _, l, lay = st
            cx = C[L.logical_index(rank, lay)]
            part[1 + l] += 2.0 * np.vdot(lam, cx * phi).imag
            ph = np.exp(1j * gamma[l] * cx)
            phi, lam = phi * ph, lam * ph
    t = torch.from_numpy(part)
    dist.all_reduce(t)  # the one collective of the reduction
    if rank == 0:
        ret.put(t.numpy().tolist())
    dist.barrier()
    dist.destroy_process_group()


def _run_split(world, n, edges, gamma, beta, obs):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, n, edges, np.asarray(gamma), np.asarray(beta), obs[0], obs[1], q),
                       nprocs=world, start_method="spawn")
    return np.array(q.get(timeout=60))


@pytest.mark.parametrize("world,case", [(2, "reg10"), (4, "prufer9"), (2, "star8"), (4, "cycle8")])
def test_split_state_energy_and_gradient_match_oracle(world, case, oracle_lib):
    n, e = {"reg10": lambda: W.random_regular(10, 3, 2), "prufer9": lambda: W.prufer_tree(9, 3),
            "star8": lambda: W.star_graph(8), "cycle8": lambda: W.cycle_graph(8)}[case]()
    p = 2
    g, b = W.random_angles(p, 60 + n)
    obs = O.full_observable(e)
    got = _run_split(world, n, e, g, b, obs)
    E, dg, db = O.energy_grad(n, e, g, b, obs)
    ref = np.concatenate([[E], dg, db])
    assert np.max(np.abs(got - ref)) < 1e-12 * max(abs(E), 1.0), (got, ref)


def test_split_layouts_cover_every_qubit_once_per_layer():
    for n, k in ((8, 1), (8, 2), (9, 3), (34, 3)):
        L = SP.SplitLayout(n, k)
        for lay in (0, 1):
            mixed = list(L.local_qubits(lay)) + list(L.swapped_in(1 - lay))
            assert sorted(mixed) == list(range(n))
            assert sorted(L.pos(lay)) == list(range(n))
        sched = SP.layer_schedule(3)
        assert [s[0] for s in sched].count("exchange") == 3
        rev = SP.layer_schedule(3, adjoint=True)
        assert len(rev) == len(sched)


@pytest.mark.parametrize("n,k", [(8, 1), (9, 2), (10, 2)])
def test_slab_cost_reproduces_the_cut_at_every_index(n, k, oracle_lib):
    """Each slab's cost, as an Ising-form function of its local bits
    (couplings, fields from edges to rank bits, a constant), equals C(x) at
    the logical index of every amplitude, in both layouts; with fields too."""
    _, e = W.random_regular(n, 3, n) if n % 2 == 0 else W.prufer_tree(n, 1)
    r = W.rng(n + k)
    w = r.uniform(-1, 2, size=len(e))
    h = r.uniform(-1, 1, size=n)
    fn = O.ising(e, w, h)
    L = SP.SplitLayout(n, k)
    for rank in range(L.ranks):
        for lay in (0, 1):
            le, lw, lh, c0 = L.slab_cost(e, w, h, rank, lay)
            sub = O.ising(le, lw, lh)
            xs = L.logical_index(rank, lay)
            for i in range(0, 1 << L.local_bits, 3):
                assert abs(O.ising_value(sub, L.local_bits, i) + c0 - O.ising_value(fn, n, int(xs[i]))) < 1e-12
