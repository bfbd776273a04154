"""The energy entry point that allocates no device memory.

Some callers cannot allocate device memory where they evaluate an energy (a
host application owns every allocation, or the device-memory budget is used
up), so they cannot hand the library a workspace. aaqaoa_expect_static keeps
all of its scratch in a static device array inside the library. This test
calls it through the C ABI with a plan that has no workspace, twice in a row
(the second call must not see the first call's leftovers), and checks it
against aaqaoa_expect of a plan with a workspace and against the FP64 oracle
(the symmetric-subspace model for K_12 and the star, the C statevector oracle
for the 3-regular graph), to the same tolerance as the other parity tests
(complex128 1e-10, complex64 1e-5 relative).
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


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _bare_plan(n, e, p, precision, orb):
    """A plan made by aaqaoa_prepare only: no workspace is ever set."""
    from paper_2410_22247_gb300 import _native as N
    ee = np.ascontiguousarray(np.asarray(e, dtype=np.int32).reshape(-1))
    rep = np.ascontiguousarray(orb.rep, dtype=np.int32)
    wt = np.ascontiguousarray(orb.weight, dtype=np.int32)
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    h = ctypes.c_void_p()
    flags = 1 if precision == "c128" else 0
    N.check(N.aaqaoa_prepare(n, len(e), P(ee), len(rep), P(rep), P(wt), None, p, flags, None, ctypes.byref(h)),
            "aaqaoa_prepare")
    return h


def _expect_static(h, g, b, obs):
    from paper_2410_22247_gb300 import _native as N
    g = np.ascontiguousarray(g, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    E = ctypes.c_double()
    F = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    N.check(N.aaqaoa_expect_static(h, F(g), F(b), obs, ctypes.byref(E)), "aaqaoa_expect_static")
    return E.value


GRAPHS = {
    "k12": (lambda: W.complete_graph(12), lambda g, b: SYM.energy(SYM.complete_graph_model(12), g, b)),
    "reg18": (lambda: W.random_regular(18, 3, 4), None),
    "star21": (lambda: W.star_graph(21), lambda g, b: SYM.energy(SYM.star_model(21), g, b)),
}


@pytest.mark.parametrize("precision", ["c64", "c128"])
@pytest.mark.parametrize("case", sorted(GRAPHS))
def test_static_scratch_energy_matches_workspace_energy(case, precision):
    from paper_2410_22247_gb300 import _native as N
    from paper_2410_22247_gb300.api import Plan
    maker, model = GRAPHS[case]
    n, e = maker()
    orb = ORB.edge_orbits(n, e)
    p = 2
    ref_plan = Plan(n, e, p, orbits=orb, precision=precision, with_grad=False)
    h = _bare_plan(n, e, p, precision, orb)
    try:
        for call, seed in enumerate((3, 4)):  # two calls in a row, different angles
            g, b = W.random_angles(p, seed)
            for obs, name in ((N.AAQAOA_OBS_RED, "red"), (N.AAQAOA_OBS_FULL, "full")):
                got = _expect_static(h, g, b, obs)
                want = ref_plan.expect(g, b, name)
                assert abs(got - want) <= TOL[precision] * max(abs(want), 1.0), (call, name, got, want)
                exact = model(g, b) if model is not None else O.energy(n, e, g, b)
                assert abs(got - exact) <= TOL[precision] * max(abs(exact), 1.0), (call, name, got, exact)
    finally:
        N.aaqaoa_destroy(h)


def test_static_scratch_rejects_states_beyond_its_size():
    from paper_2410_22247_gb300 import _native as N
    n, e = W.star_graph(23)
    h = _bare_plan(n, e, 1, "c64", ORB.edge_orbits(n, e))
    try:
        E = ctypes.c_double()
        g = np.array([0.1])
        F = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        rc = N.aaqaoa_expect_static(h, F(g), F(g), N.AAQAOA_OBS_RED, ctypes.byref(E))
        assert rc == -6
        assert b"n <= 22" in N.aaqaoa_last_error_detail()
    finally:
        N.aaqaoa_destroy(h)
