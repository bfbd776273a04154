"""Beyond the evaluation itself, through the C ABI against the oracle:
maximum cut and approximation ratio, sampling of the final state, and a
gradient-driven optimisation loop."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import symmetric as SYM
from oracle import closed_form as CF
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


def plan(n, e, p, precision="c64", grad=False):
    from paper_2410_22247_gb300.api import Plan
    return Plan(n, e, p, orbits=ORB.edge_orbits(n, e), precision=precision, with_grad=grad)


@pytest.mark.parametrize("graph", ["K12", "prufer16", "reg3_18", "petersen", "cycle15", "star20", "reg3_24",
                                   "path5", "k4"])
def test_max_cut_matches_exhaustion(graph):
    g = {"K12": W.complete_graph(12), "prufer16": W.prufer_tree(16, 2), "reg3_18": W.random_regular(18, 3, 1),
         "petersen": W.generalized_petersen(5, 2), "cycle15": W.cycle_graph(15), "star20": W.star_graph(20),
         "reg3_24": W.random_regular(24, 3, 4), "path5": (5, W.canonical_edges([(i, i + 1) for i in range(4)])),
         "k4": W.complete_graph(4)}[graph]
    n, e = g
    for prec in ("c64", "c128"):
        c, x = plan(n, e, 1, prec).max_cut()
        assert (c, x) == O.max_cut(n, e)


def test_max_cut_full_size_closed_forms():
    # bipartite graphs cut every edge; the smallest maximiser is the colour
    # class that avoids the top vertex
    n, e = W.star_graph(30)
    assert plan(n, e, 1).max_cut() == (29, 1)
    n, e = W.heap_binary_tree(34)
    depth = [int(np.floor(np.log2(v + 1))) for v in range(n)]
    even = sum(1 << v for v in range(n) if depth[v] % 2 == 0)
    odd = sum(1 << v for v in range(n) if depth[v] % 2 == 1)
    assert plan(n, e, 1).max_cut() == (33, min(even, odd))
    n, e = W.complete_graph(16)
    c, x = plan(n, e, 1).max_cut()
    assert c == 64 and x == 0xFF and O.cut_value(e, x) == 64


def test_approximation_ratio_reduced_equals_full():
    n, e = W.heap_binary_tree(20)
    pl = plan(n, e, 2, "c128")
    g, b = W.random_angles(2, 6)
    r_full = pl.approximation_ratio(g, b, "full")
    r_red = pl.approximation_ratio(g, b, "red")
    assert abs(r_full - r_red) < 1e-12 and abs(r_full - O.energy(n, e, g, b) / len(e)) < 1e-10


def _away_from_boundaries(cdf, u, margin):
    d = np.min(np.abs(cdf[None, :] - u[:, None]), axis=1)
    return u[d > margin]


@pytest.mark.parametrize("n,family", [(10, "prufer"), (13, "reg3"), (16, "star"), (19, "prufer")])
def test_samples_match_oracle_inverse_cdf(n, family):
    """complex128: the same x as the oracle's inverse CDF for every uniform
    farther than 1e-11 from a CDF step. complex64: every sample lies in its
    uniform's CDF bracket up to 2e-6 (the FP32 state's probability error)."""
    if family == "prufer":
        n, e = W.prufer_tree(n, 7)
    elif family == "reg3":
        n, e = W.random_regular(n + (n % 2), 3, 2)
    else:
        n, e = W.star_graph(n)
    g, b = W.random_angles(2, 11)
    psi = O.qaoa_state(n, e, g, b)
    cdf = np.cumsum(np.abs(psi) ** 2)
    cdf = cdf / cdf[-1]
    u_all = W.rng(5).uniform(0, 1, 2000)
    u = _away_from_boundaries(cdf, u_all, 1e-11)
    x, cut = plan(n, e, 2, "c128").sample(g, b, u)
    assert len(u) > 1900 and np.array_equal(x, O.sample(psi, u))
    assert all(cut[i] == O.cut_value(e, int(x[i])) for i in range(0, len(u), 97))
    x, cut = plan(n, e, 2, "c64").sample(g, b, u_all)
    xi = x.astype(np.int64)
    lo = np.where(xi > 0, cdf[np.maximum(xi - 1, 0)], 0.0)
    assert np.all(lo - 2e-6 <= u_all) and np.all(u_all < cdf[xi] + 2e-6)


def test_samples_full_size_star_follow_cut_distribution():
    # S_29 (n = 30): the cut value of each sample follows the exact FP64
    # distribution of the symmetric-subspace model (seeded uniforms, 5 sigma)
    n, e = W.star_graph(30)
    g, b = W.random_angles(2, 12)
    K = 65536
    u = W.rng(13).uniform(0, 1, K)
    x, cut = plan(n, e, 2).sample(g, b, u)
    dist = SYM.cut_distribution(SYM.star_model(n), g, b)
    counts = np.bincount(cut, minlength=30)
    for c, pr in dist.items():
        assert abs(counts[c] - K * pr) <= 5 * np.sqrt(K * pr * (1 - pr)) + 1
    assert all(O.cut_value(e, int(x[i])) == cut[i] for i in range(0, K, 1031))
    assert abs(cut.mean() - SYM.energy(SYM.star_model(n), g, b)) < 5 * cut.std() / np.sqrt(K)


def test_sampling_rejects_bad_uniforms():
    from paper_2410_22247_gb300._native import AAQAOAError
    n, e = W.cycle_graph(12)
    pl = plan(n, e, 1)
    with pytest.raises(AAQAOAError, match="INVALID_ARG"):
        pl.sample([0.1], [0.2], [0.5, 1.0])
    with pytest.raises(AAQAOAError, match="INVALID_ARG"):
        pl.sample([0.1], [0.2], [-0.1])


def test_adam_reaches_ring_p1_optimum():
    # p = 1 on a triangle-free 2-regular graph: F_1/|E| = 1/2 + sin(4 beta) sin(2 gamma) / 4,
    # maximum 3/4 (closed form)
    from paper_2410_22247_gb300.api import maximize
    n, e = W.cycle_graph(16)
    pl = plan(n, e, 1, "c128", grad=True)
    gam, bet, hist = maximize(pl, [0.3], [0.2], steps=300, lr=0.03)
    assert len(hist) == 301 and abs(hist[-1] - pl.expect(gam, bet, "red")) < 1e-12
    assert abs(hist[-1] / len(e) - 0.75) < 1e-4
    assert abs(CF.energy_p1(n, e, gam[0], bet[0]) / len(e) - 0.75) < 1e-4
    assert hist[10] > hist[0]


def test_multistart_adam_matches_single_runs_and_finds_ring_optimum():
    """maximize_multistart steps 4 starting points together through the
    batched gradient; each trajectory equals the one-point run from the same
    start, and the best reaches the closed-form ring optimum F_1/|E| = 3/4."""
    from paper_2410_22247_gb300.api import Plan, maximize, maximize_multistart
    n, e = W.cycle_graph(16)
    pl = Plan(n, e, 1, orbits=ORB.edge_orbits(n, e), precision="c128", batch=4, with_grad=True)
    g0 = np.array([[0.3], [1.2], [2.0], [-0.4]])
    b0 = np.array([[0.2], [0.5], [-0.3], [0.9]])
    gam, bet, hist, best = maximize_multistart(pl, g0, b0, steps=200, lr=0.03)
    assert hist.shape == (201, 4)
    # the last history row is F_p at the returned points
    assert np.max(np.abs(hist[-1] - pl.expect_batch(gam, bet, "red"))) < 1e-12
    for k in range(4):
        g1, b1, h1 = maximize(pl, g0[k], b0[k], steps=200, lr=0.03)
        assert np.max(np.abs(h1 - hist[:, k])) < 1e-9
        assert abs(g1[0] - gam[k, 0]) < 1e-9 and abs(b1[0] - bet[k, 0]) < 1e-9
    assert abs(hist[-1, best] / len(e) - 0.75) < 1e-3


def wplan(n, e, w, p, precision, orbits=True, grad=True):
    from paper_2410_22247_gb300.api import Plan
    orb = ORB.edge_orbits(n, e, weights=w) if orbits else None
    return Plan(n, e, p, orbits=orb, precision=precision, with_grad=grad, weights=w)


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("case", ["prufer14_rand", "reg3_20_rand", "star22_orbit", "tree24_depth", "k8_rand"])
def test_weighted_maxcut_energy_and_gradient(prec, case):
    """Weighted MaxCut (integer weights): energy and adjoint gradient against the
    weighted oracle, with H_C and with H_red from weight-preserving orbits."""
    if case == "prufer14_rand":
        n, e = W.prufer_tree(14, 5)
        w = W.rng(1).integers(1, 5, size=len(e))
    elif case == "reg3_20_rand":
        n, e = W.random_regular(20, 3, 6)
        w = W.rng(2).integers(1, 4, size=len(e))
    elif case == "star22_orbit":
        n, e = W.star_graph(22)
        w = np.full(len(e), 3)
    elif case == "tree24_depth":
        n, e = W.heap_binary_tree(24)
        w = np.array([1 + int(np.floor(np.log2(int(v) + 1))) % 3 for _, v in e])
    else:
        n, e = W.complete_graph(8)
        w = W.rng(3).integers(1, 6, size=len(e))
    g, b = W.random_angles(2, 17)
    pl = wplan(n, e, w, 2, prec)
    if case == "star22_orbit":
        # uniform weight 3: E_w(gamma, beta) = 3 E(3 gamma, beta) (pinned on the
        # CPU), with E from the exact symmetric-subspace model. The plain C
        # oracle's sequential sums over 2^22 terms carry ~2^n eps relative error
        # on this case's large gradient components, more than 1e-10.
        E1, dg1, db1 = SYM.energy_grad(SYM.star_model(n), 3 * np.asarray(g), b)
        Er, dgr, dbr = 3 * E1, 9 * dg1, 3 * db1
    else:
        Er, dgr, dbr = O.energy_grad_w(n, e, w, g, b)
    tol = {"c64": 1e-5, "c128": 1e-10}[prec]
    scale = max(abs(Er), 1.0) if prec == "c64" else 1e-3 * abs(Er)
    for obs in ("full", "red"):
        E, dg, db = pl.grad(g, b, obs)
        assert abs(E - Er) <= tol * max(abs(Er), 1.0), obs
        for x, r in zip(np.concatenate([dg, db]), np.concatenate([dgr, dbr])):
            assert abs(x - r) <= tol * max(abs(r), scale), obs
        assert abs(pl.expect(g, b, obs) - Er) <= tol * max(abs(Er), 1.0)
    for mode in ("singlepass", "perterm"):
        pl.expect(g, b, "full", "singlepass")
        assert abs(pl.aggregate_only("red", mode) - Er) <= tol * max(abs(Er), 1.0)


def test_weighted_max_cut_and_samples():
    n, e = W.random_regular(18, 3, 7)
    w = W.rng(4).integers(1, 5, size=len(e))
    pl = wplan(n, e, w, 1, "c128", grad=False)
    assert pl.max_cut() == O.max_cut_w(n, e, w)
    g, b = [0.4], [0.3]
    x, cut = pl.sample(g, b, W.rng(6).uniform(0, 1, 500))
    we = O.weighted_cost_edges(e, w)
    assert all(cut[i] == O.cut_value(we, int(x[i])) for i in range(500))


def test_weighted_prepare_errors():
    from paper_2410_22247_gb300._native import AAQAOAError
    from paper_2410_22247_gb300.api import Plan
    n, e = W.cycle_graph(6)
    with pytest.raises(AAQAOAError, match="INVALID_ARG"):
        Plan(n, e, 1, weights=[1, 1, 0, 1, 1, 1], with_grad=False)
    with pytest.raises(AAQAOAError, match="UNSUPPORTED"):
        Plan(n, e, 1, weights=[100] * 6, with_grad=False)
    orb = ORB.edge_orbits(n, e)  # one orbit of the unweighted cycle
    with pytest.raises(AAQAOAError, match="BAD_ORBITS"):
        Plan(n, e, 1, orbits=orb, weights=[1, 2, 1, 2, 1, 2], with_grad=False)
