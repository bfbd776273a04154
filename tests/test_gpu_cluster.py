"""The complex64 adjoint's 14-qubit low pass by a cluster of 4 CTAs
(distributed shared memory exchange), through the C ABI, against the FP64
oracle and against the plain pass plan.

Tolerances as in test_gpu_parity: energies 1e-5 relative to max(|E|, 1),
gradient components 1e-5 relative to max(|g_ref|, |E|).
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import symmetric as SYM
from paper_2410_22247_gb300 import workloads as W
from paper_2410_22247_gb300 import orbits as ORB

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22247_gb300 import _native
    _native.load()


def g_err(g, gref, E):
    return float(np.max(np.abs(np.asarray(g) - gref) / np.maximum(np.abs(gref), max(abs(E), 1.0))))


def cluster_plan(n, e, p, batch=1, orbits=True):
    from paper_2410_22247_gb300.api import Plan
    orb = ORB.edge_orbits(n, e) if orbits else None
    pl = Plan(n, e, p, orbits=orb, precision="c64", batch=batch, with_grad=True)
    K = -(-(n - 14) // 8)
    pl.set_pass_plan(0, 0, 14, K)
    assert pl.pass_plan()[2] == 14
    return pl, orb


@pytest.mark.parametrize("n,p,fuse", [(15, 1, 1), (16, 2, 1), (19, 3, 1), (22, 2, 0), (23, 2, 1), (24, 3, 1)])
def test_cluster_low_pass_gradient_matches_oracle(n, p, fuse):
    _, e = W.prufer_tree(n, 40 + n)
    g, b = W.random_angles(p, 70 + n)
    pl, orb = cluster_plan(n, e, p)
    pl.set_layer_fusion(fuse)
    launches = pl.schedule(True)
    turn = launches[0][2] == launches[0][3]  # a turnaround pass may open the sweep
    assert launches[1 if turn else 0][1] == 14
    for obs in ("red", "full"):
        oobs = O.full_observable(e) if obs == "full" else O.reduced_observable(e, orb.rep, orb.weight)
        Er, dgr, dbr = O.energy_grad(n, e, g, b, oobs)
        E, dg, db = pl.grad(g, b, obs)
        assert abs(E - Er) <= 1e-5 * max(abs(Er), 1.0)
        assert g_err(dg, dgr, Er) < 1e-5, (dg, dgr)
        assert g_err(db, dbr, Er) < 1e-5, (db, dbr)
    pl.close()


def test_cluster_low_pass_launches_are_recorded():
    from paper_2410_22247_gb300 import _native as N
    n, e = W.random_regular(20, 3, 5)
    pl, _ = cluster_plan(n, e, 2)
    N.check(N.aaqaoa_profile_enable(pl.handle, 1), "profile")
    pl.grad(*W.random_angles(2, 1), "red")
    recs = pl.profile_launches()
    N.check(N.aaqaoa_profile_enable(pl.handle, 0), "profile")
    cl = [r for r in recs if r["cluster"]]
    assert len(cl) == 2 and all(r["kind"] == 1 for r in cl)
    pl.close()


def test_cluster_low_pass_boundary_angles():
    """Shifted layers (|sin| > |cos|), beta = pi/2, zero layers through the
    cluster pass."""
    n, e = W.random_regular(18, 3, 7)
    pl, _ = cluster_plan(n, e, 2)
    for g, b in (([0.0, 0.7], [0.3, 0.0]), ([0.9, 1.3], [np.pi / 4, -np.pi / 4]), ([2 * np.pi, -0.4], [np.pi / 2, 1e-9]),
                 ([40.0, -17.3], [2.3, -1.9])):
        Er, dgr, dbr = O.energy_grad(n, e, g, b)
        E, dg, db = pl.grad(g, b, "red")
        assert abs(E - Er) <= 1e-5 * max(abs(Er), 1.0)
        assert g_err(dg, dgr, Er) < 1e-5 and g_err(db, dbr, Er) < 1e-5, (g, b)
    pl.close()


def test_cluster_low_pass_batch_matches_single_points():
    """grad_batch runs the cluster pass once per point of the batch."""
    n, e = W.prufer_tree(20, 3)
    p, B = 2, 5
    rng = W.rng(12)
    gs = rng.uniform(0, np.pi, size=(B, p))
    bs = rng.uniform(-np.pi / 2, np.pi / 2, size=(B, p))
    pl, _ = cluster_plan(n, e, p, batch=3)
    E, dg, db = pl.grad_batch(gs, bs, "red")
    for k in range(B):
        Er, dgr, dbr = O.energy_grad(n, e, gs[k], bs[k])
        assert abs(E[k] - Er) <= 1e-5 * max(abs(Er), 1.0)
        assert g_err(dg[k], dgr, Er) < 1e-5 and g_err(db[k], dbr, Er) < 1e-5, k
    pl.close()


@pytest.mark.parametrize("p", [2, 4])
def test_cluster_low_pass_full_size_star_n30(p):
    """The headline workload shape: the star S_29 at n = 30 through the
    cluster pass plan, against the exact symmetric-subspace oracle."""
    n, e = W.star_graph(30)
    g, b = W.random_angles(p, 29)
    Er, dgr, dbr = SYM.energy_grad(SYM.star_model(30), g, b)
    pl, orb = cluster_plan(n, e, p)
    E, dg, db = pl.grad(g, b, "red")
    assert abs(E - Er) <= 1e-5 * Er
    assert g_err(dg, dgr, Er) < 1e-5 and g_err(db, dbr, Er) < 1e-5
    pl.close()


def test_cluster_and_plain_plans_agree_bitwise_on_the_forward():
    """The forward passes are shared; energies from both adjoint plans are the
    same number, and gradients agree to rounding."""
    n, e = W.random_regular(22, 3, 2)
    g, b = W.random_angles(2, 9)
    pl, _ = cluster_plan(n, e, 2)
    E1, dg1, db1 = pl.grad(g, b, "red")
    pl.set_pass_plan(0, 0, 8, 0)
    E2, dg2, db2 = pl.grad(g, b, "red")
    assert E1 == E2
    assert np.max(np.abs(np.concatenate([dg1 - dg2, db1 - db2]))) < 1e-5 * max(abs(E1), 1.0)
    pl.close()
