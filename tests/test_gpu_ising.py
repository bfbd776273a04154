"""Ising-form objectives (real couplings of either sign and real fields) on the
GPU through the C ABI, against the FP64 oracle's Ising routines.

With mixed signs the energy can cancel to near zero, so errors are measured
on the scale of the operator norm bound S = sum_e |w_e| + sum_i |h_i| of H_C
(the largest |C(x)|): |E - E_ref| <= tol * S, and each gradient component
|g - g_ref| <= tol * max(|g_ref|, floor) with floor = S for complex64 and
1e-3 S for complex128 (tol: 1e-5 complex64, 1e-10 complex128).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_22247_gb300 import workloads as W
from paper_2410_22247_gb300 import orbits as ORB

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "c128": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22247_gb300 import _native
    _native.load()


def plan_for(n, e, w, h, p, precision, orbits=None, batch=1, grad=True):
    from paper_2410_22247_gb300.api import Plan
    return Plan(n, e, p, orbits=orbits, precision=precision, batch=batch, with_grad=grad, couplings=w, fields=h)


def scale(w, h):
    return float(np.sum(np.abs(w)) + (0.0 if h is None else np.sum(np.abs(h))))


def check(got, ref, S, precision):
    E, dg, db = got
    Er, dgr, dbr = ref
    tol = TOL[precision]
    floor = (1.0 if precision == "c64" else 1e-3) * S
    assert abs(E - Er) <= tol * S, (E, Er)
    g, gr = np.concatenate([dg, db]), np.concatenate([dgr, dbr])
    assert np.all(np.abs(g - gr) <= tol * np.maximum(np.abs(gr), floor)), (g, gr)


# whole circuit in one CTA (n <= 12/13), tiled passes with one and two high
# passes per layer (the latter through fused layer boundaries)
CASES = {
    "cycle7": lambda: W.cycle_graph(7),
    "k10": lambda: W.complete_graph(10),
    "reg14": lambda: W.random_regular(14, 3, 3),
    "bintree17": lambda: W.heap_binary_tree(17),
    "prufer20": lambda: W.prufer_tree(20, 4),
}

# angles with |sin beta| > |cos beta| (cot form of the rotation), negative
# angles, and generic ones
ANGLES = [
    ([0.37, -0.81], [0.21, 1.13]),
    ([1.9, 0.44], [-1.2, 0.95]),
]


@pytest.mark.parametrize("precision", ["c64", "c128"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_ising_energy_and_gradient_match_oracle(case, precision):
    n, e = CASES[case]()
    w, h = W.ising_couplings(n, e, 10 + n, symmetric=False)
    fn = O.ising(e, w, h)
    S = scale(w, h)
    pl = plan_for(n, e, w, h, 2, precision)
    jobs = [(g, b) for g, b in ANGLES]
    refs = [O.ising_energy_grad(n, fn, g, b) for g, b in jobs]
    for (g, b), ref in zip(jobs, refs):
        check(pl.grad(g, b, "full"), ref, S, precision)
        assert abs(pl.expect(g, b, "full") - ref[0]) <= TOL[precision] * S
    pl.close()


@pytest.mark.parametrize("precision", ["c64", "c128"])
@pytest.mark.parametrize("case", ["cycle7", "bintree17", "prufer20"])
def test_ising_reduced_observable_matches_full(case, precision):
    """Couplings and fields kept by every automorphism: H_red (edge and vertex
    orbit representatives, Eq. A3) gives the energy and gradient of H_C."""
    n, e = CASES[case]()
    w, h = W.ising_couplings(n, e, 30 + n, symmetric=True)
    orb = ORB.ising_orbits(n, e, w, h)
    assert orb.num_orbits < len(e) and len(orb.vrep) < n
    fn = O.ising(e, w, h)
    S = scale(w, h)
    g, b = ANGLES[1]
    ref = O.ising_energy_grad(n, fn, g, b)
    red = O.ising_reduced_observable(fn, orb.rep, orb.weight, orb.vrep, orb.vweight)
    ref_red = O.ising_energy_grad(n, fn, g, b, red)
    assert abs(ref_red[0] - ref[0]) <= 1e-10 * S
    pl = plan_for(n, e, w, h, 2, precision, orbits=orb)
    check(pl.grad(g, b, "red"), ref, S, precision)
    check(pl.grad(g, b, "full"), ref, S, precision)
    pl.close()


@pytest.mark.parametrize("precision", ["c64", "c128"])
@pytest.mark.parametrize("case", ["cycle7", "reg14", "prufer20"])
def test_ising_statevector_matches_oracle(case, precision):
    n, e = CASES[case]()
    w, h = W.ising_couplings(n, e, 50 + n)
    for g, b in ANGLES:
        pl = plan_for(n, e, w, h, 2, precision, grad=False)
        psi = pl.statevector(g, b)
        ref = O.ising_state(n, O.ising(e, w, h), g, b)
        err = np.max(np.abs(psi.astype(np.complex128) - ref)) / np.max(np.abs(ref))
        assert err < TOL[precision], err
        pl.close()


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_ising_fused_boundaries_and_plans(precision):
    """n = 22 at p = 3 with two high passes per layer, layer boundaries fused
    into one pass and not fused, both against the oracle."""
    n, e = W.prufer_tree(22, 7)
    w, h = W.ising_couplings(n, e, 77)
    g, b = [0.4, -1.1, 2.2], [1.0, 0.3, -0.9]
    ref = O.ising_energy_grad(n, O.ising(e, w, h), g, b)
    S = scale(w, h)
    pl = plan_for(n, e, w, h, 3, precision)
    pl.set_pass_plan(*((13, 2, 12, 2) if precision == "c64" else (12, 2, 11, 2)))
    for fuse in (1, 0):
        pl.set_layer_fusion(fuse)
        fused = any(st[3] >= 0 for st in pl.schedule(False)) and any(st[3] >= 0 for st in pl.schedule(True))
        assert fused == bool(fuse)
        check(pl.grad(g, b, "full"), ref, S, precision)
        psi = pl.statevector(g, b)
        ref_psi = O.ising_state(n, O.ising(e, w, h), g, b)
        assert np.max(np.abs(psi.astype(np.complex128) - ref_psi)) / np.max(np.abs(ref_psi)) < TOL[precision]
    pl.close()


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_ising_batches_match_oracle(precision):
    n, e = W.random_regular(16, 3, 9)
    w, h = W.ising_couplings(n, e, 91)
    fn = O.ising(e, w, h)
    S = scale(w, h)
    B, p = 5, 2
    r = W.rng(92)
    gs = r.uniform(-np.pi, np.pi, size=(B, p))
    bs = r.uniform(-np.pi / 2, np.pi / 2, size=(B, p))
    pl = plan_for(n, e, w, h, p, precision, batch=3)
    E, dg, db = pl.grad_batch(gs, bs, "full")
    Eb = pl.expect_batch(gs, bs, "full")
    for k in range(B):
        ref = O.ising_energy_grad(n, fn, gs[k], bs[k])
        check((E[k], dg[k], db[k]), ref, S, precision)
        assert abs(Eb[k] - ref[0]) <= TOL[precision] * S
    pl.close()


def test_ising_without_fields_and_unit_couplings_is_maxcut():
    from paper_2410_22247_gb300.api import Plan
    n, e = W.random_regular(18, 3, 4)
    g, b = [0.7, 0.2], [0.4, 1.0]
    ising = plan_for(n, e, np.ones(len(e)), None, 2, "c128")
    maxcut = Plan(n, e, 2, precision="c128")
    Ei, dgi, dbi = ising.grad(g, b)
    Em, dgm, dbm = maxcut.grad(g, b)
    assert abs(Ei - Em) < 1e-10 * len(e)
    assert np.max(np.abs(np.concatenate([dgi - dgm, dbi - dbm]))) < 1e-9 * len(e)


def test_ising_unsupported_calls_are_reported():
    from paper_2410_22247_gb300._native import AAQAOAError
    n, e = W.cycle_graph(14)
    w, h = W.ising_couplings(n, e, 5)
    pl = plan_for(n, e, w, h, 1, "c64", grad=False)
    with pytest.raises(AAQAOAError, match="UNSUPPORTED"):
        pl.expect([0.1], [0.2], "full", "perterm")
    with pytest.raises(AAQAOAError, match="UNSUPPORTED"):
        pl.max_cut()
    with pytest.raises(AAQAOAError, match="UNSUPPORTED"):
        pl.sample([0.1], [0.2], [0.5])
    assert np.isfinite(pl.expect([0.1], [0.2]))


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_ising_full_size_regular3_n30_matches_light_cones(precision):
    """The bench's Ising workload: random 3-regular n = 30 with seeded real
    couplings and fields, p = 2, against per-term light cones (Sec. 5.1; a
    ZZ term's ball has at most 14 vertices, a field term's at most 10)."""
    from oracle import lightcone as LC
    n, e = W.random_regular(30, 3, 0)
    w, h = W.ising_couplings(n, e, 30)
    g, b = W.random_angles(2, 5)
    ref = LC.ising_energy_grad(n, e, w, h, g, b)
    pl = plan_for(n, e, w, h, 2, precision)
    check(pl.grad(g, b, "full"), ref, scale(w, h), precision)
    assert abs(pl.expect(g, b, "full") - ref[0]) <= TOL[precision] * scale(w, h)
    pl.close()
