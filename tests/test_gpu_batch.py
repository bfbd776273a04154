"""Batched evaluation (parameter landscapes, uneven graph batches) and the
failure path of the tiled passes, on the GPU through the C ABI.

Tolerances as in test_gpu_parity: complex128 1e-10, complex64 1e-5 relative
to max(|E|, 1).
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import symmetric as SYM
from paper_2410_22247_gb300 import workloads as W
from paper_2410_22247_gb300 import orbits as ORB

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "c128": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _uneven_graphs(seed, count, n_lo, n_hi):
    out = []
    for fam, n, e in W.mixed_graph_batch(count, n_lo, n_hi, seed):
        out.append((n, e, ORB.edge_orbits(n, e)))
    return out


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_uneven_batch_matches_oracle(precision):
    from paper_2410_22247_gb300.api import MultiPlan
    graphs = _uneven_graphs(5, 18, 4, 15) + _uneven_graphs(6, 4, 16, 17)
    p = 2
    mp = MultiPlan(graphs, p, precision=precision)
    info = mp.info()
    assert 0 < info["small_graphs"] < len(graphs)
    for call in range(2):  # the second call replays the captured CUDA graph
        rng = W.rng(100 + call)
        gs = rng.uniform(0, np.pi, size=(len(graphs), p))
        bs = rng.uniform(0, np.pi / 2, size=(len(graphs), p))
        for obs in ("red", "full"):
            E = mp.expect(gs, bs, obs)
            for k, (n, e, orb) in enumerate(graphs):
                ref = O.energy(n, e, gs[k], bs[k])
                assert abs(E[k] - ref) <= TOL[precision] * max(abs(ref), 1.0), (k, n, obs, E[k], ref)
    assert mp.info()["launches_per_call"] >= 1


def test_uneven_batch_of_256_graphs_matches_single_plans():
    # the batch shape of 256 graphs with n in 12..22 (three families plus K_n),
    # compared with one plan per graph on the same device
    from paper_2410_22247_gb300.api import MultiPlan, Plan
    graphs = _uneven_graphs(7, 256, 12, 22)
    p = 2
    mp = MultiPlan(graphs, p, precision="c64")
    rng = W.rng(3)
    gs = rng.uniform(0, np.pi, size=(len(graphs), p))
    bs = rng.uniform(0, np.pi / 2, size=(len(graphs), p))
    E = mp.expect(gs, bs, "red")
    for k in list(range(0, 256, 17)) + [255]:
        n, e, orb = graphs[k]
        single = Plan(n, e, p, orbits=orb, precision="c64", with_grad=False).expect(gs[k], bs[k], "red")
        assert abs(E[k] - single) <= 1e-5 * max(abs(single), 1.0)
        if n <= 14:
            ref = O.energy(n, e, gs[k], bs[k])
            assert abs(E[k] - ref) <= 1e-5 * max(abs(ref), 1.0)


def test_landscape_of_4096_points_on_star_s19():
    # star S_19 (n = 20), p = 1, the inclusive 64 x 64 grid over [0, pi] x [0, pi/2]
    import torch
    from paper_2410_22247_gb300.api import Plan
    n, e = W.star_graph(20)
    gs, bs = W.angle_grid(64)
    pl = Plan(n, e, 1, orbits=ORB.edge_orbits(n, e), precision="c64", batch=4096, with_grad=False)
    dg = torch.tensor(gs, device="cuda")
    db = torch.tensor(bs, device="cuda")
    out = torch.zeros(4096, dtype=torch.float64, device="cuda")
    pl.expect_device(dg, db, out, "red")
    pl.sync()
    E = out.cpu().numpy()
    model = SYM.star_model(20)
    idx = np.arange(0, 4096, 7)
    ref = np.array([SYM.energy(model, [gs[i]], [bs[i]]) for i in idx])
    assert np.max(np.abs(E[idx] - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-5


def test_expired_wait_is_reported_and_the_plan_recovers():
    from paper_2410_22247_gb300 import _native as N
    from paper_2410_22247_gb300._native import AAQAOAError
    from paper_2410_22247_gb300.api import Plan
    n, e = W.random_regular(18, 3, 2)
    g, b = W.random_angles(2, 4)
    pl = Plan(n, e, 2, orbits=None, precision="c64", with_grad=False)
    ref = O.energy(n, e, g, b)
    assert abs(pl.expect(g, b) - ref) < 1e-5 * ref
    N.check(N.aaqaoa_inject_fault(pl.handle, N.AAQAOA_FAULT_DROP_TILE), "inject")
    with pytest.raises(AAQAOAError, match="TIMEOUT"):
        pl.expect(g, b)
    # the context and the plan still work
    assert abs(pl.expect(g, b) - ref) < 1e-5 * ref
    small = Plan(*W.cycle_graph(6), 1, with_grad=False)
    assert N.aaqaoa_inject_fault(small.handle, N.AAQAOA_FAULT_DROP_TILE) == -6


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_uneven_batch_with_graphs_beyond_one_high_pass(precision):
    """Graphs large enough for two high passes per layer (n = 23, 24) in an
    uneven batch: each group of equal n runs the per-point-graph passes
    (a graph per point) with the multi-pass plan, against the exact
    symmetric-subspace energy of stars."""
    from paper_2410_22247_gb300.api import MultiPlan
    sizes = [23, 24, 23, 24, 14]
    graphs = []
    for n in sizes:
        nn, e = W.star_graph(n)
        graphs.append((nn, e, ORB.edge_orbits(nn, e)))
    p = 2
    mp = MultiPlan(graphs, p, precision=precision)
    rng = W.rng(31)
    gs = rng.uniform(0, np.pi, size=(len(graphs), p))
    bs = rng.uniform(0, np.pi / 2, size=(len(graphs), p))
    for obs in ("red", "full"):
        E = mp.expect(gs, bs, obs)
        for k, n in enumerate(sizes):
            ref = SYM.energy(SYM.star_model(n), gs[k], bs[k])
            assert abs(E[k] - ref) <= TOL[precision] * max(abs(ref), 1.0), (k, n, obs, E[k], ref)
    mp.close()


@pytest.mark.parametrize("precision", ["c64", "c128"])
@pytest.mark.parametrize("n_case", ["small12", "tiled18", "fused22"])
def test_gradient_batch_matches_oracle_and_single_calls(n_case, precision):
    """aaqaoa_grad_batch: B points through the whole-circuit kernel (n = 12),
    the tiled passes (n = 18) and fused layer boundaries (n = 22), in two
    waves of the workspace's batch size, against the oracle and against
    one-point calls."""
    from paper_2410_22247_gb300.api import Plan
    n = {"small12": 12, "tiled18": 18, "fused22": 22}[n_case]
    nn, e = W.prufer_tree(n, 6)
    p, B = 3, 5
    rng = W.rng(40 + n)
    gs = rng.uniform(0, np.pi, size=(B, p))
    bs = rng.uniform(-np.pi / 2, np.pi / 2, size=(B, p))
    pl = Plan(nn, e, p, orbits=ORB.edge_orbits(nn, e), precision=precision, batch=3, with_grad=True)
    if n_case == "fused22":
        pl.set_pass_plan(*((13, 2, 12, 2) if precision == "c64" else (12, 2, 11, 2)))
    E, dg, db = pl.grad_batch(gs, bs, "red")
    tol = TOL[precision]
    floor = (1.0 if precision == "c64" else 1e-3)
    for k in range(B):
        Er, dgr, dbr = O.energy_grad(nn, e, gs[k], bs[k])
        s = max(abs(Er), 1.0)
        assert abs(E[k] - Er) <= tol * s, (k, E[k], Er)
        ref = np.concatenate([dgr, dbr])
        got = np.concatenate([dg[k], db[k]])
        assert np.all(np.abs(got - ref) <= tol * np.maximum(np.abs(ref), floor * s)), k
        E1, dg1, db1 = pl.grad(gs[k], bs[k], "red")
        assert abs(E1 - E[k]) <= tol * s
        assert np.max(np.abs(np.concatenate([dg1, db1]) - got)) <= tol * s
