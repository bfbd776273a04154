"""Workload configurations checked against the FP64 oracle, through the C ABI.

* The random labelled tree on 24 vertices (seeded uniform Pruefer sequence)
  at p = 3, complex64 and complex128, energy and adjoint gradient of H_C and
  H_red against the full C statevector oracle; complex128 also against
  central finite differences of its own energies (h = 1e-6).
* The batch of 256 graphs of uneven size (n = 12..22, Pruefer trees, cycles,
  K_n up to n = 16, 3-regular), every graph against the oracle's energy.
* The Pruefer tree on 32 vertices at p = 4, complex64, energy and gradient
  against the per-edge light cones (Sec. 5.1): every radius-4 ball of this
  seeded tree has at most 22 vertices, so the oracle is exact there.

Tolerances as in test_gpu_parity: complex128 1e-10, complex64 1e-5, energies
relative to max(|E|, 1); gradient components relative to
max(|g_ref|, floor), floor = 1e-3 |E| for complex128 and |E| for complex64.
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import lightcone as LC
from paper_2410_22247_gb300 import workloads as W
from paper_2410_22247_gb300 import orbits as ORB
from tests import oracle_pool as POOL

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "c128": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22247_gb300 import _native
    _native.load()


def e_rel(a, b):
    return abs(a - b) / max(abs(b), 1.0)


def g_err(g, gref, E, precision):
    floor = (1.0 if precision == "c64" else 1e-3) * max(abs(E), 1.0)
    g, gref = np.asarray(g), np.asarray(gref)
    return float(np.max(np.abs(g - gref) / np.maximum(np.abs(gref), floor)))


# ------------------------------------------------ Pruefer tree n = 24, p = 3
TREE24 = W.prufer_tree(24, 0)
P24 = 3
ANGLES24 = W.random_angles(P24, 24)


@pytest.fixture(scope="module")
def tree24_reference():
    """Oracle energy and gradient of H_C and of H_red (both FP64, adjoint)."""
    n, e = TREE24
    orb = ORB.edge_orbits(n, e)
    g, b = ANGLES24
    red = O.reduced_observable(e, orb.rep, orb.weight)
    full_ref, red_ref = POOL.energy_grads([(n, e, g, b, None), (n, e, g, b, red)])
    return orb, {"full": full_ref, "red": red_ref}


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_prufer_tree_n24_p3_energy_and_gradient_match_oracle(precision, tree24_reference):
    from paper_2410_22247_gb300.api import Plan
    n, e = TREE24
    orb, ref = tree24_reference
    assert orb.num_orbits < len(e)
    g, b = ANGLES24
    pl = Plan(n, e, P24, orbits=orb, precision=precision, with_grad=True)
    tol = TOL[precision]
    for obs in ("full", "red"):
        Er, dgr, dbr = ref[obs]
        E, dg, db = pl.grad(g, b, obs)
        assert e_rel(E, Er) < tol, (obs, E, Er)
        assert g_err(dg, dgr, Er, precision) < tol, (obs, dg, dgr)
        assert g_err(db, dbr, Er, precision) < tol, (obs, db, dbr)
        assert e_rel(pl.expect(g, b, obs), Er) < tol
    # Eq. (exact): <H_red> = <H_C> for the oracle itself
    assert abs(ref["red"][0] - ref["full"][0]) < 1e-10 * ref["full"][0]
    pl.close()


def test_prufer_tree_n24_p3_c128_gradient_matches_finite_differences():
    """Central differences (h = 1e-6) of the library's own complex128 energies:
    round-off ~ eps |E| / h ~ 1e-9 |E| and truncation O(h^2), so 1e-6 |E|."""
    from paper_2410_22247_gb300.api import Plan
    n, e = TREE24
    g, b = (np.array(x, dtype=np.float64) for x in ANGLES24)
    pl = Plan(n, e, P24, orbits=ORB.edge_orbits(n, e), precision="c128", with_grad=True)
    E, dg, db = pl.grad(g, b, "red")
    h = 1e-6
    for vec, got in ((g, dg), (b, db)):
        for i in range(len(vec)):
            old = vec[i]
            vec[i] = old + h
            ep = pl.expect(g, b, "red")
            vec[i] = old - h
            em = pl.expect(g, b, "red")
            vec[i] = old
            assert abs((ep - em) / (2 * h) - got[i]) < 1e-6 * max(abs(E), 1.0), (i, got[i])
    pl.close()


# ------------------------------------------------ 256 graphs of uneven size
def test_uneven_batch_of_256_graphs_matches_oracle_for_every_graph():
    from paper_2410_22247_gb300.api import MultiPlan
    graphs = [(n, e, ORB.edge_orbits(n, e)) for _, n, e in W.mixed_graph_batch(256, 12, 22, 7)]
    p = 2
    rng = W.rng(3)
    gs = rng.uniform(0, np.pi, size=(len(graphs), p))
    bs = rng.uniform(0, np.pi / 2, size=(len(graphs), p))
    ref = np.array(POOL.energies([(n, e, gs[k], bs[k], None) for k, (n, e, _) in enumerate(graphs)]))
    mp = MultiPlan(graphs, p, precision="c64")
    for call in range(2):  # the second call replays the captured CUDA graph
        for obs in ("red", "full"):
            E = mp.expect(gs, bs, obs)
            err = np.abs(E - ref) / np.maximum(np.abs(ref), 1.0)
            assert np.max(err) < 1e-5, (call, obs, int(np.argmax(err)), float(np.max(err)))
    mp.close()


# ------------------------------------------------ Pruefer tree n = 32, p = 4
def test_prufer_tree_n32_p4_gradient_matches_light_cones():
    torch = pytest.importorskip("torch")
    import gc
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < 80e9:
        pytest.skip("needs ~70 GB of free device memory")
    from paper_2410_22247_gb300.api import Plan
    n, e = W.prufer_tree(32, 0)
    p = 4
    assert LC.max_ball(n, e, p) <= 22
    g, b = W.random_angles(p, 32)
    orb = ORB.edge_orbits(n, e)
    Er, dgr, dbr = LC.energy_grad(n, e, g, b, weights=orb.weight, edge_subset=orb.rep)
    pl = Plan(n, e, p, orbits=orb, precision="c64", with_grad=True)
    for obs in ("red", "full"):
        E, dg, db = pl.grad(g, b, obs)
        assert e_rel(E, Er) < 1e-5, (obs, E, Er)
        assert g_err(dg, dgr, Er, "c64") < 1e-5, (obs, dg, dgr)
        assert g_err(db, dbr, Er, "c64") < 1e-5, (obs, db, dbr)
    pl.close()
    torch.cuda.empty_cache()
