"""A seeded randomized sweep through the CUDA path against the FP64 oracle:
graph family, size (several tiles, one to three high passes), layer count,
pass plan (any the autotuner may pick), layer-boundary fusion on or off,
precision and observable are drawn per case. Tolerances as in
test_gpu_parity (complex128 1e-10, complex64 1e-5, gradients relative to
max(|g|, 1e-3 |E|) resp. max(|g|, |E|)).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_22247_gb300 import workloads as W
from paper_2410_22247_gb300 import orbits as ORB

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "c128": 1e-10}
# (L, K) candidates per pass kind: tile bits and two-stage low-pass bits
LOW = {("c64", 1): (13, 9), ("c64", 2): (12, 8), ("c128", 1): (12, 8), ("c128", 2): (11, 7)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _graph(rng, n):
    fam = rng.integers(0, 4)
    if fam == 0:
        return W.prufer_tree(n, int(rng.integers(1 << 30)))
    if fam == 1 and n % 2 == 0:
        return W.random_regular(n, 3, int(rng.integers(1 << 30)))
    if fam == 2:
        return W.circulant_graph(n, (1, int(rng.integers(2, n // 2))))
    return W.cycle_graph(n)


def _plan_choice(rng, pl, prec):
    """Draw a valid (L, K) for the forward and the adjoint passes."""
    from paper_2410_22247_gb300._native import AAQAOAError
    for _ in range(50):
        f = LOW[(prec, 1)][rng.integers(0, 2)], int(rng.integers(1, 4))
        b = LOW[(prec, 2)][rng.integers(0, 2)], int(rng.integers(1, 5))
        try:
            pl.set_pass_plan(f[0], f[1], b[0], b[1])
            return pl.pass_plan()
        except AAQAOAError:
            continue
    pl.set_pass_plan(0, 0, 0, 0)
    return pl.pass_plan()


@pytest.mark.parametrize("seed", range(48))
def test_random_case_matches_oracle(seed):
    from paper_2410_22247_gb300.api import Plan
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(14, 21))
    n, e = _graph(rng, n)
    p = int(rng.integers(1, 5))
    prec = ("c64", "c128")[seed % 2]
    obs = ("red", "full")[(seed // 2) % 2]
    g = rng.uniform(-np.pi, np.pi, size=p)
    b = rng.uniform(-np.pi, np.pi, size=p)
    pl = Plan(n, e, p, orbits=ORB.edge_orbits(n, e), precision=prec, with_grad=True)
    plan4 = _plan_choice(rng, pl, prec)
    pl.set_layer_fusion(bool(rng.integers(0, 2)))
    Er, dgr, dbr = O.energy_grad(n, e, g, b)
    E, dg, db = pl.grad(g, b, obs)
    tol = TOL[prec]
    where = (seed, n, len(e), p, prec, obs, plan4, pl.layer_fusion())
    assert abs(E - Er) <= tol * max(abs(Er), 1.0), where
    floor = (1.0 if prec == "c64" else 1e-3) * max(abs(Er), 1.0)
    gerr = np.abs(np.concatenate([dg, db]) - np.concatenate([dgr, dbr]))
    assert np.all(gerr <= tol * np.maximum(np.abs(np.concatenate([dgr, dbr])), floor)), where
    assert abs(pl.expect(g, b, obs) - Er) <= tol * max(abs(Er), 1.0), where
    pl.close()


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_maximum_layer_count_through_fused_boundaries(precision):
    """p = 64, the largest layer count the library takes: 63 fused
    boundaries in each sweep (plan with two high passes per layer)."""
    from paper_2410_22247_gb300.api import Plan
    n, e = W.prufer_tree(16, 3)
    p = 64
    rng = np.random.default_rng(64)
    g = rng.uniform(-0.4, 0.4, size=p)
    b = rng.uniform(-0.4, 0.4, size=p)
    pl = Plan(n, e, p, orbits=ORB.edge_orbits(n, e), precision=precision, with_grad=True)
    pl.set_pass_plan(9, 2, 8, 2) if precision == "c64" else pl.set_pass_plan(8, 2, 7, 2)
    assert sum(1 for st in pl.schedule(False) if st[3] >= 0) == p - 1
    Er, dgr, dbr = O.energy_grad(n, e, g, b)
    E, dg, db = pl.grad(g, b, "red")
    tol = TOL[precision]
    floor = (1.0 if precision == "c64" else 1e-3) * max(abs(Er), 1.0)
    assert abs(E - Er) <= tol * max(abs(Er), 1.0)
    gerr = np.abs(np.concatenate([dg, db]) - np.concatenate([dgr, dbr]))
    assert np.all(gerr <= tol * np.maximum(np.abs(np.concatenate([dgr, dbr])), floor))


def test_isolated_qubits():
    """Vertices without edges (a 12-vertex tree inside n = 18): their qubits
    still go through the mixer, and the oracle sees the same register."""
    from paper_2410_22247_gb300.api import Plan
    _, e = W.prufer_tree(12, 8)
    n = 18
    g, b = W.random_angles(3, 12)
    Er, dgr, dbr = O.energy_grad(n, e, g, b)
    for precision in ("c64", "c128"):
        pl = Plan(n, e, 3, orbits=ORB.edge_orbits(n, e), precision=precision, with_grad=True)
        E, dg, db = pl.grad(g, b, "full")
        tol = TOL[precision]
        assert abs(E - Er) <= tol * max(abs(Er), 1.0)
        floor = (1.0 if precision == "c64" else 1e-3) * max(abs(Er), 1.0)
        gerr = np.abs(np.concatenate([dg, db]) - np.concatenate([dgr, dbr]))
        assert np.all(gerr <= tol * np.maximum(np.abs(np.concatenate([dgr, dbr])), floor))
