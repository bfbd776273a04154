"""One statevector split across 2^k devices by its top k qubits (host logic).

When 2^n amplitudes outgrow one device (Sec. 5.3: the state size is the
wall), rank r of W = 2^k ranks holds the slab of 2^(n-k) amplitudes whose top
k physical index bits equal r. Logical qubit q sits at physical bit pos[q];
two layouts alternate:

  layout 0: pos[q] = q, so logical qubits n-k..n-1 are the rank bits;
  layout 1: logical qubits n-k..n-1 sit at physical bits n-2k..n-k-1 and
            logical qubits n-2k..n-k-1 are the rank bits.

One QAOA layer (Eq. 1) on the split state:
  1. the cost phase exp(-i gamma C(x)): diagonal, so it is applied in any
     layout, with C evaluated at the logical index (for a device kernel: the
     slab's cost as an Ising-form function of its local bits, slab_cost);
  2. RX(2 beta) on every logical qubit at a local bit (local butterflies);
  3. one exchange: an all-to-all in which rank r sends its chunk c (top local
     bits = c) to rank c and receives rank s's chunk into block s, which
     swaps the rank bits with the top k local bits (the layout toggles);
  4. RX(2 beta) on the k logical qubits that just became local.
The energy is a sum over amplitudes: per-rank partial sums and one
all-reduce. The adjoint gradient runs the same steps in reverse on phi and
lambda (the inverse exchange is the same all-to-all) and all-reduces the
2p partial inner products once at the end.

Nothing here touches amplitudes: the module gives layouts, index maps, the
exchange's chunking, each slab's cost function and the step schedule; the
compute per slab is a device kernel's (or, in tests, the oracle's).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class SplitLayout:
    n: int  # logical qubits
    k: int  # rank bits: 2^k ranks

    def __post_init__(self):
        if self.k < 1 or 2 * self.k > self.n:
            raise ValueError(f"need 1 <= k and 2k <= n (n={self.n}, k={self.k})")

    @property
    def ranks(self) -> int:
        return 1 << self.k

    @property
    def local_bits(self) -> int:
        return self.n - self.k

    def pos(self, layout: int) -> np.ndarray:
        """Physical bit of every logical qubit in the given layout (0 or 1)."""
        p = np.arange(self.n)
        if layout == 1:
            n, k = self.n, self.k
            p[n - k:] = np.arange(n - 2 * k, n - k)
            p[n - 2 * k:n - k] = np.arange(n - k, n)
        return p

    def local_qubits(self, layout: int) -> np.ndarray:
        """Logical qubits at local physical bits, in increasing physical bit."""
        p = self.pos(layout)
        q = np.argsort(p)
        return q[: self.local_bits]

    def swapped_in(self, layout_after: int) -> np.ndarray:
        """The k logical qubits the exchange into layout_after made local."""
        n, k = self.n, self.k
        return np.arange(n - k, n) if layout_after == 1 else np.arange(n - 2 * k, n - k)

    def logical_index(self, rank: int, layout: int) -> np.ndarray:
        """Logical basis index of each of rank's 2^(n-k) amplitudes (small n)."""
        phys = (np.uint64(rank) << np.uint64(self.local_bits)) + np.arange(1 << self.local_bits, dtype=np.uint64)
        p = self.pos(layout)
        x = np.zeros_like(phys)
        for q in range(self.n):
            x |= ((phys >> np.uint64(p[q])) & np.uint64(1)) << np.uint64(q)
        return x

    def exchange_splits(self):
        """all-to-all chunking of a slab: 2^k equal contiguous chunks (the top
        k local bits), chunk c to rank c, rank s's chunk into block s."""
        size = 1 << (self.n - 2 * self.k)
        return [size] * self.ranks, [size] * self.ranks

    def relabel(self, edges, layout: int) -> np.ndarray:
        """Edges in physical-bit labels (vertex q -> pos[q])."""
        p = self.pos(layout)
        e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
        return np.stack([p[e[:, 0]], p[e[:, 1]]], axis=1) if len(e) else e

    def slab_cost(self, edges, weights, fields, rank: int, layout: int):
        """The cost C(x) restricted to rank's slab as an Ising-form function of
        its n-k local bits: couplings between two local bits, fields on local
        bits (an edge to a rank bit b adds +w when b = 0 and -w with a
        constant +w when b = 1), and a constant (edges between two rank bits,
        fields of rank bits). Returns (local_edges, couplings, fields, const)."""
        nl = self.local_bits
        e = self.relabel(edges, layout)
        w = np.ones(len(e)) if weights is None else np.asarray(weights, dtype=np.float64)
        hfield = np.zeros(self.n) if fields is None else np.asarray(fields, dtype=np.float64)
        p = self.pos(layout)
        bit = lambda b: (rank >> (b - nl)) & 1  # value of physical rank bit b
        le, lw = [], []
        h = np.zeros(nl)
        const = 0.0
        for (a, b), we in zip(e, w):
            a, b = int(a), int(b)
            if a < nl and b < nl:
                le.append((min(a, b), max(a, b)))
                lw.append(we)
            elif a < nl or b < nl:
                u, g = (a, b) if a < nl else (b, a)
                if bit(g):
                    h[u] -= we
                    const += we
                else:
                    h[u] += we
            else:
                const += we * (bit(a) != bit(b))
        for q in range(self.n):
            b = int(p[q])
            if b < nl:
                h[b] += hfield[q]
            elif bit(b):
                const += hfield[q]
        order = np.argsort([a * 64 + b for a, b in le], kind="stable")
        le = np.asarray([le[i] for i in order], dtype=np.int32).reshape(-1, 2)
        lw = np.asarray([lw[i] for i in order], dtype=np.float64)
        return le, lw, h, const


def layer_schedule(p: int, adjoint: bool = False):
    """Steps of the split circuit: ("phase", l, layout), ("mix", l, qubits),
    ("exchange", layout_after). The forward sweep starts in layout 0; every
    layer ends one exchange later, so layer l runs in layout l % 2. The
    adjoint sweep is the exact reverse (an inverse exchange is the same
    all-to-all), its mixer steps carrying the layer's dE/dbeta."""
    steps = []
    for l in range(p):
        lay = l % 2
        steps.append(("phase", l, lay))
        steps.append(("mix", l, "local", lay))
        steps.append(("exchange", 1 - lay))
        steps.append(("mix", l, "swapped_in", 1 - lay))
    if adjoint:
        rev = []
        for st in reversed(steps):
            if st[0] == "exchange":
                rev.append(("exchange", 1 - st[1]))  # back to the layout before it
            else:
                rev.append(st)
        return rev
    return steps
