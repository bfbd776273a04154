"""Layer-boundary fusion (Eq. (1): the mixer of layer l and the cost layer
of l+1 meet at a diagonal step, so one pass can end layer l and start the
next on the same qubits), through the C ABI.

Fused and unfused schedules compute the same quantities in a different
rounding order: both are compared with the FP64 oracle at the parity
tolerances (complex128 1e-10, complex64 1e-5 relative) and with each other.
The plans below force at least two high passes per layer (the condition for
fusion) at n = 22, and p = 2..5 so that the fused group alternates between
the last two high groups and the adjoint's fused passes carry dE/dbeta of
two layers.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from oracle import symmetric as SYM
from paper_2410_22247_gb300 import workloads as W
from paper_2410_22247_gb300 import orbits as ORB

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "c128": 1e-10}
# forward (L, K) and adjoint (L, K) with K >= 2 at n = 22
PLANS = {"c64": [(13, 2, 12, 2), (9, 2, 8, 2), (9, 3, 8, 3)],
         "c128": [(12, 2, 11, 2), (8, 2, 7, 3)]}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _plan(n, e, p, precision, batch=1, grad=True):
    from paper_2410_22247_gb300.api import Plan
    return Plan(n, e, p, orbits=ORB.edge_orbits(n, e), precision=precision, batch=batch, with_grad=grad)


def _rel(x, ref, scale):
    return float(np.max(np.abs(np.asarray(x) - np.asarray(ref)) / np.maximum(np.abs(np.asarray(ref)), scale)))


def test_fusion_is_on_by_default_and_switchable():
    n, e = W.prufer_tree(22, 9)
    pl = _plan(n, e, 2, "c64")
    assert pl.layer_fusion()
    pl.set_layer_fusion(False)
    assert not pl.layer_fusion()
    pl.set_layer_fusion(True)
    assert pl.layer_fusion()


@pytest.mark.parametrize("precision", ["c64", "c128"])
@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_fused_energy_and_gradient_match_oracle_and_unfused(p, precision):
    n, e = W.prufer_tree(22, 9)
    g, b = W.random_angles(p, 50 + p)
    Er, dgr, dbr = O.energy_grad(n, e, g, b)
    tol = TOL[precision]
    gscale = max(abs(Er), 1.0) if precision == "c64" else 1e-3 * max(abs(Er), 1.0)
    pl = _plan(n, e, p, precision)
    for plan4 in PLANS[precision]:
        pl.set_pass_plan(*plan4)
        res = {}
        for fused in (True, False):
            pl.set_layer_fusion(fused)
            for obs in ("red", "full"):
                E, dg, db = pl.grad(g, b, obs)
                assert abs(E - Er) <= tol * max(abs(Er), 1.0), (plan4, fused, obs, E, Er)
                assert _rel(dg, dgr, gscale) < tol, (plan4, fused, obs)
                assert _rel(db, dbr, gscale) < tol, (plan4, fused, obs)
                Ee = pl.expect(g, b, obs)
                assert abs(Ee - Er) <= tol * max(abs(Er), 1.0), (plan4, fused, obs, Ee, Er)
            res[fused] = np.concatenate([[E], dg, db])
        # the two schedules differ only in rounding order
        assert np.max(np.abs(res[True] - res[False])) <= tol * max(abs(Er), 1.0), plan4


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_fused_statevector_matches_oracle(precision):
    n, e = W.prufer_tree(22, 9)
    p = 3
    g, b = W.random_angles(p, 61)
    ref = O.qaoa_state(n, e, g, b)
    pl = _plan(n, e, p, precision, grad=False)
    pl.set_pass_plan(*PLANS[precision][0][:2], 0, 0)
    assert pl.layer_fusion()
    psi = pl.statevector(g, b).astype(np.complex128)
    err = np.max(np.abs(psi - ref)) / np.max(np.abs(ref))
    assert err < TOL[precision], err


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_fused_batch_matches_single_calls(precision):
    """Batched points with fused passes: a CTA's chunk of tiles crosses
    point boundaries, where both layers' angles and the next phase table
    change together."""
    n, e = W.prufer_tree(22, 9)
    B, p = 5, 3
    rng = W.rng(12)
    gs = rng.uniform(0, np.pi, size=(B, p))
    bs = rng.uniform(-np.pi / 2, np.pi / 2, size=(B, p))
    pl = _plan(n, e, p, precision, batch=B, grad=False)
    pl.set_pass_plan(*PLANS[precision][0][:2], 0, 0)
    E = pl.expect_batch(gs, bs, "red")
    for k in range(B):
        Er = O.energy(n, e, gs[k], bs[k])
        assert abs(E[k] - Er) <= TOL[precision] * max(abs(Er), 1.0), (k, E[k], Er)


def test_fused_full_size_star_n30_p4_c64():
    """The n = 30 star at p = 4 (three fused boundaries each way, default
    plan) against the exact symmetric-subspace oracle."""
    n, e = W.star_graph(30)
    p = 4
    g, b = W.random_angles(p, 77)
    Er, dgr, dbr = SYM.energy_grad(SYM.star_model(30), g, b)
    pl = _plan(n, e, p, "c64")
    assert pl.layer_fusion()
    E, dg, db = pl.grad(g, b, "red")
    s = max(abs(Er), 1.0)
    assert abs(E - Er) <= 1e-5 * s
    assert _rel(dg, dgr, s) < 1e-5 and _rel(db, dbr, s) < 1e-5
    pl.close()


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_fused_static_scratch_energy(precision):
    """aaqaoa_expect_static (no workspace) runs the same fused schedule."""
    from paper_2410_22247_gb300 import _native as N
    n, e = W.prufer_tree(22 if precision == "c64" else 21, 9)  # the static scratch's largest state
    p = 3
    orb = ORB.edge_orbits(n, e)
    ee = np.ascontiguousarray(np.asarray(e, dtype=np.int32).reshape(-1))
    rep = np.ascontiguousarray(orb.rep, dtype=np.int32)
    wt = np.ascontiguousarray(orb.weight, dtype=np.int32)
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    F = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    N.check(N.aaqaoa_prepare(n, len(e), P(ee), len(rep), P(rep), P(wt), None, p, 1 if precision == "c128" else 0,
                             None, ctypes.byref(h)), "aaqaoa_prepare")
    try:
        f, k = PLANS[precision][0][:2]
        N.check(N.aaqaoa_set_pass_plan(h, f, k, 0, 0), "aaqaoa_set_pass_plan")
        g, b = W.random_angles(p, 90)
        Er = O.energy(n, e, g, b)
        for fused in (1, 0):
            N.check(N.aaqaoa_set_layer_fusion(h, fused), "aaqaoa_set_layer_fusion")
            E = ctypes.c_double()
            N.check(N.aaqaoa_expect_static(h, F(np.asarray(g, dtype=np.float64)), F(np.asarray(b, dtype=np.float64)),
                                           N.AAQAOA_OBS_RED, ctypes.byref(E)), "aaqaoa_expect_static")
            assert abs(E.value - Er) <= TOL[precision] * max(abs(Er), 1.0), (fused, E.value, Er)
    finally:
        N.aaqaoa_destroy(h)


def test_aggregate_only_refuses_a_state_overwritten_by_a_fused_energy():
    """A fused energy call streams the state through the passes without
    storing the final state, so the stored state is gone afterwards."""
    from paper_2410_22247_gb300._native import AAQAOAError
    n, e = W.prufer_tree(22, 9)
    p = 2
    g, b = W.random_angles(p, 91)
    pl = _plan(n, e, p, "c64", grad=False)
    E1 = pl.expect(g, b, "red", "singlepass")  # stores the final state
    assert abs(pl.aggregate_only("red") - E1) <= 1e-5 * max(abs(E1), 1.0)
    pl.expect(*W.random_angles(p, 92), "red")  # fused: the passes overwrite it
    with pytest.raises(AAQAOAError, match="INVALID_ARG"):
        pl.aggregate_only("red")
    pl.statevector(g, b)  # stored again
    assert abs(pl.aggregate_only("red") - E1) <= 1e-5 * max(abs(E1), 1.0)


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_fused_weighted_maxcut_matches_oracle(precision):
    """Weighted MaxCut (integer weights 1..3) through fused boundaries: the
    next layer's phase table is indexed by the weighted cut value."""
    from paper_2410_22247_gb300.api import Plan
    n, e = W.prufer_tree(22, 9)
    w = [1 + (k % 3) for k in range(len(e))]
    p = 3
    g, b = W.random_angles(p, 95)
    Er, dgr, dbr = O.energy_grad_w(n, e, w, g, b)
    pl = Plan(n, e, p, orbits=ORB.edge_orbits(n, e, weights=w), precision=precision, with_grad=True, weights=w)
    pl.set_pass_plan(*PLANS[precision][0])
    assert pl.layer_fusion()
    tol = TOL[precision]
    gscale = max(abs(Er), 1.0) if precision == "c64" else 1e-3 * max(abs(Er), 1.0)
    for obs in ("red", "full"):
        E, dg, db = pl.grad(g, b, obs)
        assert abs(E - Er) <= tol * max(abs(Er), 1.0), (obs, E, Er)
        assert _rel(dg, dgr, gscale) < tol and _rel(db, dbr, gscale) < tol, obs


def test_profile_records_each_launch_of_the_schedule():
    """aaqaoa_profile_launches lists the launches of a gradient call in
    order: the parameter tables, the forward sweep, the adjoint sweep, with
    the fused boundaries flagged where the schedule has them."""
    from paper_2410_22247_gb300 import _native as N
    n, e = W.prufer_tree(22, 9)
    p = 3
    g, b = W.random_angles(p, 97)
    pl = _plan(n, e, p, "c64")
    pl.set_pass_plan(*PLANS["c64"][0])
    fwd, adj = pl.schedule(False, gradient=True), pl.schedule(True)
    turn = adj[0][2] == adj[0][3]  # the turnaround pass opens the adjoint sweep
    N.check(N.aaqaoa_profile_enable(pl.handle, 1), "profile")
    pl.grad(g, b, "red")
    recs = pl.profile_launches()
    N.check(N.aaqaoa_profile_enable(pl.handle, 0), "profile")
    kinds = [r["kind"] for r in recs]
    assert kinds == [4] + [0] * len(fwd) + [1] * len(adj)
    fused = [r["fused"] for r in recs[1:]]
    assert fused == [st[3] >= 0 for st in fwd] + [st[3] >= 0 for st in adj]
    assert sum(fused) == 2 * (p - 1) + (1 if turn else 0)
    # phase first; the energy in the forward's last pass or in the turnaround
    assert recs[1]["cut_work"] and recs[len(fwd) + (1 if turn else 0)]["cut_work"]
    assert all(r["ms"] > 0 for r in recs[1:])
    S = (1 << n) * 8
    # |+> store; the adjoint's first launch: phi in, phi and lambda out, or
    # the complex64 turnaround: phi in, lambda out (phi stays as loaded)
    assert recs[1]["bytes"] == S and recs[len(fwd) + 1]["bytes"] == (2 if turn else 3) * S


# pass plans at n = 18..24 whose gradient schedule opens the adjoint with a
# turnaround pass (the forward's last group is one of the adjoint's groups),
# read off the host schedule
TURN_PLANS = [("c64", 18, (8, 2, 8, 2)), ("c64", 20, (7, 2, 8, 2)), ("c64", 22, (7, 2, 8, 2)),
              ("c64", 24, (7, 3, 9, 3)), ("c128", 18, (7, 2, 8, 2)), ("c128", 20, (5, 2, 6, 2)),
              ("c128", 22, (5, 2, 6, 2))]


@pytest.mark.parametrize("precision,n,plan4", TURN_PLANS)
def test_turnaround_gradient_matches_oracle_and_the_unfused_sweeps(n, plan4, precision):
    """The turnaround pass (the forward's last group mixed forward on phi,
    the energy and lambda = O phi, then both vectors mixed back) gives the
    oracle's energy and gradient, for H_red and H_C, p = 1..3, and the same
    as the sweeps without fusion (no turnaround)."""
    _, e = W.prufer_tree(n, 5)
    for p in (1, 2, 3):
        g, b = W.random_angles(p, 40 + n + p)
        pl = _plan(n, e, p, precision)
        pl.set_pass_plan(*plan4)
        adj = pl.schedule(True)
        assert adj[0][2] == adj[0][3], (n, plan4, adj[0])
        orb = ORB.edge_orbits(n, e)
        for obs in ("red", "full"):
            oobs = O.full_observable(e) if obs == "full" else O.reduced_observable(e, orb.rep, orb.weight)
            Er, dgr, dbr = O.energy_grad(n, e, g, b, oobs)
            E, dg, db = pl.grad(g, b, obs)
            gs = max(abs(Er), 1.0) * (1.0 if precision == "c64" else 1e-3)
            assert abs(E - Er) <= TOL[precision] * max(abs(Er), 1.0), (obs, E, Er)
            assert _rel(dg, dgr, gs) < TOL[precision] and _rel(db, dbr, gs) < TOL[precision], obs
        E1, dg1, db1 = pl.grad(g, b, "red")
        pl.set_layer_fusion(False)
        assert not pl.schedule(True)[0][2] == pl.schedule(True)[0][3]
        E0, dg0, db0 = pl.grad(g, b, "red")
        sc = max(abs(E0), 1.0)
        assert abs(E1 - E0) <= TOL[precision] * sc
        assert np.max(np.abs(np.concatenate([dg1 - dg0, db1 - db0]))) <= TOL[precision] * sc
        pl.close()


@pytest.mark.parametrize("n", [20, 21])
def test_turnaround_batch_and_boundary_angles_c64(n):
    """Batched gradients through the turnaround (each point its own
    parameters) and angles with |sin beta| > |cos beta| (the shifted
    rotation in both halves of the turnaround), against the oracle. The
    complex64 turnaround stores lambda times f^(n - 2q) and leaves phi as
    loaded (f the factor one butterfly drops, q the pass's qubits): at
    n = 21 the exponent is odd, and the last layer's f is negative in both
    rotation forms (beta = -pi/4 - 0.2 shifted, beta = 2.8 not)."""
    e = W.prufer_tree(n, 3)[1]
    p, B = 2, 5
    rng = W.rng(21)
    gs = rng.uniform(-np.pi, np.pi, size=(B, p))
    bs = rng.uniform(-np.pi / 2, np.pi / 2, size=(B, p))
    gs[0], bs[0] = [0.9, 1.3], [np.pi / 2 - 0.1, -np.pi / 4 - 0.2]
    bs[1, 1] = 2.8
    pl = _plan(n, e, p, "c64", batch=3)
    pl.set_pass_plan(7, 2, 8, 2)
    turn = pl.schedule(True)[0]
    assert turn[2] == turn[3]  # a turnaround over q = 6 (n = 20) or 7 (n = 21) qubits
    E, dg, db = pl.grad_batch(gs, bs, "red")
    for k in range(B):
        Er, dgr, dbr = O.energy_grad(n, e, gs[k], bs[k])
        sc = max(abs(Er), 1.0)
        assert abs(E[k] - Er) <= 1e-5 * sc
        assert _rel(dg[k], dgr, sc) < 1e-5 and _rel(db[k], dbr, sc) < 1e-5, k
    pl.close()
