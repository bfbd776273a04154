"""The C-ABI library without a GPU: it loads, exports every declared symbol,
and its host-side validation (no device calls) rejects malformed inputs."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2410_22247_gb300 import _native as N
from paper_2410_22247_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "aaqaoa.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(aaqaoa_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = N.load()
    decl = declared_symbols()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(N.EXPORTED) == decl


def _prepare(n, edges, p=1, orbits=None, flags=0):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    h = ctypes.c_void_p()
    rep = weight = eo = None
    k = 0
    if orbits is not None:
        rep = np.ascontiguousarray(orbits[0], dtype=np.int32)
        weight = np.ascontiguousarray(orbits[1], dtype=np.int32)
        eo = None if len(orbits) < 3 or orbits[2] is None else np.ascontiguousarray(orbits[2], dtype=np.int32)
        k = len(rep)
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if a is not None and a.size else None
    rc = N.aaqaoa_prepare(n, len(e) // 2, P(e), k, P(rep), P(weight), P(eo), p, flags, None, ctypes.byref(h))
    if rc == 0:
        N.aaqaoa_destroy(h)
    return rc


def test_prepare_accepts_valid_graphs():
    n, e = W.star_graph(6)
    assert _prepare(n, e, orbits=([0], [5], [0] * 5)) == 0
    assert _prepare(n, e, orbits=([0], [5])) == 0
    assert _prepare(1, np.zeros((0, 2))) == 0
    assert _prepare(34, W.heap_binary_tree(34)[1], p=4, flags=1) == 0


@pytest.mark.parametrize("case,code", [
    ("n0", -1), ("n35", -1), ("p0", -1), ("selfloop", -1), ("dup", -1), ("dup_rev", -1), ("range", -1),
    ("flags", -1), ("wsum", -2), ("rep_range", -2), ("rep_dup", -2), ("w0", -2), ("eo_rep", -2),
    ("eo_count", -2),
])
def test_prepare_rejects(case, code):
    path = [(0, 1), (1, 2), (2, 3)]
    args = dict(n=4, edges=path)
    if case == "n0":
        args = dict(n=0, edges=np.zeros((0, 2)))
    elif case == "n35":
        args = dict(n=35, edges=[(0, 1)])
    elif case == "p0":
        args["p"] = 0
    elif case == "selfloop":
        args["edges"] = [(0, 1), (2, 2)]
    elif case == "dup":
        args["edges"] = [(0, 1), (0, 1)]
    elif case == "dup_rev":
        args["edges"] = [(0, 1), (1, 0)]
    elif case == "range":
        args["edges"] = [(0, 4)]
    elif case == "flags":
        args["flags"] = 7
    elif case == "wsum":
        args["orbits"] = ([0, 1], [1, 1])
    elif case == "rep_range":
        args["orbits"] = ([0, 5], [2, 1])
    elif case == "rep_dup":
        args["orbits"] = ([0, 0], [2, 1])
    elif case == "w0":
        args["orbits"] = ([0, 1], [3, 0])
    elif case == "eo_rep":
        args["orbits"] = ([0, 1], [2, 1], [1, 1, 0])
    elif case == "eo_count":
        args["orbits"] = ([0, 1], [2, 1], [0, 1, 1])
    assert _prepare(**args) == code
    assert N.aaqaoa_last_error_detail()  # a message was recorded


def test_workspace_size_grows_with_batch_and_gradient():
    n, e = W.random_regular(20, 3, 1)
    ee = np.ascontiguousarray(e.reshape(-1), dtype=np.int32)
    h = ctypes.c_void_p()
    assert N.aaqaoa_prepare(n, len(e), ee.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 0, None, None, None,
                            2, 0, None, ctypes.byref(h)) == 0
    sizes = {}
    for batch in (1, 4):
        for grad in (0, 1):
            s = ctypes.c_size_t()
            assert N.aaqaoa_workspace_bytes(h, batch, grad, ctypes.byref(s)) == 0
            sizes[batch, grad] = s.value
    N.aaqaoa_destroy(h)
    state = (1 << 20) * 8
    assert sizes[1, 0] > state and sizes[1, 1] > 2 * state
    assert sizes[4, 0] > 4 * state


def test_strerror_covers_codes():
    for c in [0, -1, -2, -3, -4, -5, -6]:
        assert N.aaqaoa_strerror(c)


def test_prepare_multi_names_the_bad_graph():
    good = np.ascontiguousarray(np.array([[0, 1], [1, 2]], dtype=np.int32).reshape(-1))
    bad = np.ascontiguousarray(np.array([[0, 0]], dtype=np.int32).reshape(-1))
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    descs = (N.GraphDesc * 3)()
    for i, (n, e) in enumerate([(3, good), (3, good), (2, bad)]):
        descs[i].n = n
        descs[i].num_edges = len(e) // 2
        descs[i].edges = P(e)
        descs[i].num_orbits = 0
    h = ctypes.c_void_p()
    assert N.aaqaoa_prepare_multi(3, descs, 1, 0, None, ctypes.byref(h)) == -1
    assert b"graph 2" in N.aaqaoa_last_error_detail()
    # the optional class of every edge is checked like aaqaoa_prepare's
    rep, wt = (np.ascontiguousarray(np.array(v, dtype=np.int32)) for v in ([0], [2]))
    # (on a host without a GPU a valid batch stops later, at stream creation: ERR_CUDA)
    for eo_vals, codes in (([0, 0], (0, -4)), ([0, 1], (-2,))):
        eo = np.ascontiguousarray(np.array(eo_vals, dtype=np.int32))
        descs = (N.GraphDesc * 1)()
        descs[0].n, descs[0].num_edges, descs[0].edges = 3, 2, P(good)
        descs[0].num_orbits, descs[0].orbit_rep, descs[0].orbit_weight, descs[0].edge_orbit = 1, P(rep), P(wt), P(eo)
        h = ctypes.c_void_p()
        rc = N.aaqaoa_prepare_multi(1, descs, 1, 0, None, ctypes.byref(h))
        assert rc in codes, N.aaqaoa_last_error_detail()
        if rc == 0:
            N.aaqaoa_destroy_multi(h)


def _handle(n, edges, p, flags=0):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    h = ctypes.c_void_p()
    assert N.aaqaoa_prepare(n, len(e) // 2, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 0, None, None, None,
                            p, flags, None, ctypes.byref(h)) == 0
    return h


def test_pass_plans_default_and_validation():
    """Default qubits per pass and the rejection of plans that do not tile n
    (host-side only: no workspace, so no tensor maps are built)."""
    h = _handle(*W.star_graph(30), p=2)
    try:
        out = np.zeros(4, dtype=np.int32)
        assert N.aaqaoa_get_pass_plan(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))) == 0
        assert out.tolist() == [13, 2, 8, 3]   # forward 13 + 9 + 8, adjoint 8 + 8 + 7 + 7
        assert N.aaqaoa_set_pass_plan(h, 9, 3, 12, 3) == 0
        assert N.aaqaoa_get_pass_plan(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))) == 0
        assert out.tolist() == [9, 3, 12, 3]
        assert N.aaqaoa_set_pass_plan(h, 13, 1, 0, 0) == -1   # 17 qubits in one high pass
        assert N.aaqaoa_set_pass_plan(h, 3, 2, 0, 0) == -1    # low pass below one row
        assert N.aaqaoa_set_pass_plan(h, 0, 0, 0, 0) == 0
        assert N.aaqaoa_get_pass_plan(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))) == 0
        assert out.tolist() == [13, 2, 8, 3]
    finally:
        N.aaqaoa_destroy(h)
    h = _handle(*W.cycle_graph(10), p=1)
    try:
        out = np.ones(4, dtype=np.int32)
        assert N.aaqaoa_get_pass_plan(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))) == 0
        assert out.tolist() == [0, 0, 0, 0]
    finally:
        N.aaqaoa_destroy(h)


def _schedule(h, adjoint):
    cnt = ctypes.c_int()
    assert N.aaqaoa_get_schedule(h, adjoint, None, 0, ctypes.byref(cnt)) == 0
    out = np.zeros((max(cnt.value, 1), 5), dtype=np.int32)
    assert N.aaqaoa_get_schedule(h, adjoint, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), cnt.value,
                                 ctypes.byref(cnt)) == 0
    return [tuple(int(v) for v in r) for r in out[:cnt.value]]


def _check_schedule(steps, n, p, adjoint, fused, c128=False, turn_group=None):
    """The launches realise Eq. (1) layer by layer: flattened into (layer,
    qubit group) mixer steps (a fused launch is two steps with the next
    layer's diagonal step between them) the layers come in order, each layer
    mixes every qubit exactly once, j0 counts the layer's qubits mixed
    before, and the sweep's last launch is a high pass (it carries the
    last-stage work: energy, or dE/dgamma of layer 0). adjoint: 0 the
    forward sweep of an energy evaluation, 1 the adjoint sweep, 2 the forward
    sweep of a gradient evaluation. A turnaround pass (a row whose second
    layer is its own layer) opens the adjoint sweep: it mixes the last
    layer's group forward and back, and the gradient's forward sweep leaves
    that group of the last layer to it (turn_group receives (s, q))."""
    order = list(range(p - 1, -1, -1)) if adjoint == 1 else list(range(p))
    turn = adjoint == 1 and len(steps) > 0 and steps[0][2] == steps[0][3]
    flat = []
    for i, (s, q, l, l2, j0) in enumerate(steps):
        done = sum(qq for (ll, ss, qq) in flat if ll == l)
        assert j0 == done
        flat.append((l, s, q))
        if turn and i == 0:
            assert s > 0 and l == p - 1, "the turnaround is a high pass of the last layer"
            continue
        if l2 >= 0:
            assert s > 0, "fused launches are high passes"
            assert order.index(l2) == order.index(l) + 1
            assert all(ll != l2 for (ll, _, _) in flat), "the fused half starts its layer"
            flat.append((l2, s, q))
    pos = [order.index(l) for (l, _, _) in flat]
    assert pos == sorted(pos)
    for l in range(p):
        covered = sorted(b for (ll, s, q) in flat if ll == l for b in range(s, s + q))
        if adjoint == 2 and turn_group is not None and l == p - 1:
            covered = sorted(covered + list(range(turn_group[0], turn_group[0] + turn_group[1])))
        assert covered == list(range(n)), l
    if not (adjoint == 2 and turn_group is not None):  # else the turnaround ends the sweep
        assert steps[-1][0] > 0 and steps[-1][3] == -1
    # a layer's qubit groups (at p = 1 the gradient's forward sweep holds
    # all but the one the turnaround takes)
    groups = {(s, q) for s, q, *_ in steps}
    if adjoint == 2 and turn_group is not None:
        groups.add(tuple(turn_group))
    if adjoint != 1 and not c128 and len(groups) >= 3:
        # the generating pass takes a high group, then the low pass
        assert steps[0][0] > 0 and steps[1][0] == 0 and steps[0][2] == steps[1][2] == 0
    elif turn:
        assert steps[1][0] == 0, "the turnaround, then the low pass"
    else:
        assert steps[0][0] == 0, "the sweep starts with the low pass"
    nf = sum(1 for i, st in enumerate(steps) if st[3] >= 0 and not (turn and i == 0))
    assert nf == (p - 1 if fused else 0)
    return turn


@pytest.mark.parametrize("n,p,plan4", [(30, 2, (0, 0, 0, 0)), (30, 4, (0, 0, 0, 0)), (30, 5, (9, 3, 12, 3)),
                                       (22, 3, (13, 2, 8, 3)), (26, 6, (9, 2, 8, 3)), (32, 3, (0, 0, 0, 0))])
def test_fused_schedule_realises_the_layers_in_order(n, p, plan4):
    h = _handle(*W.star_graph(n), p=p)
    try:
        assert N.aaqaoa_set_pass_plan(h, *plan4) == 0
        plan = np.zeros(4, dtype=np.int32)
        assert N.aaqaoa_get_pass_plan(h, plan.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))) == 0
        en = ctypes.c_int()
        assert N.aaqaoa_get_layer_fusion(h, ctypes.byref(en)) == 0 and en.value == 1
        Kf, Kb = int(plan[1]), int(plan[3])
        steps = _schedule(h, 0)
        _check_schedule(steps, n, p, 0, fused=Kf >= 2)
        assert len(steps) == p * (Kf + 1) - (p - 1 if Kf >= 2 else 0)
        adj = _schedule(h, 1)
        turn = _check_schedule(adj, n, p, 1, fused=Kb >= 2)
        assert len(adj) == p * (Kb + 1) - (p - 1 if Kb >= 2 else 0)  # the turnaround takes the place of a pass
        gf = _schedule(h, 2)
        _check_schedule(gf, n, p, 2, fused=Kf >= 2, turn_group=adj[0][:2] if turn else None)
        assert len(gf) == len(steps) - (1 if turn else 0)
        assert N.aaqaoa_set_layer_fusion(h, 0) == 0
        for mode in (0, 1, 2):
            K = Kb if mode == 1 else Kf
            steps = _schedule(h, mode)
            assert not (mode == 1 and steps[0][2] == steps[0][3]), "no turnaround without fusion"
            _check_schedule(steps, n, p, mode, fused=False)
            assert len(steps) == p * (K + 1)
    finally:
        N.aaqaoa_destroy(h)


def test_random_pass_plans_schedule_every_layer_once():
    """400 seeded pass plans (n = 14..34, p = 1..4, both precisions, layer
    fusion on and off): every sweep the host schedules -- energy, adjoint,
    the gradient's forward sweep -- realises Eq. (1) layer by layer, with
    the launch counts the plan implies; no device needed."""
    rng = np.random.default_rng(7)
    tried = 0
    while tried < 400:
        n, p = int(rng.integers(14, 35)), int(rng.integers(1, 5))
        plan4 = (int(rng.integers(5, 14)), int(rng.integers(1, 4)), int(rng.integers(5, 13)), int(rng.integers(1, 4)))
        for flags in (0, 1):
            h = _handle(*W.star_graph(n), p=p, flags=flags)
            try:
                if N.aaqaoa_set_pass_plan(h, *plan4) != 0:
                    continue
                tried += 1
                Kf, Kb = plan4[1], plan4[3]
                for fuse in (1, 0):
                    assert N.aaqaoa_set_layer_fusion(h, fuse) == 0
                    ff, fb = bool(fuse) and Kf >= 2, bool(fuse) and Kb >= 2
                    fwd = _schedule(h, 0)
                    _check_schedule(fwd, n, p, 0, fused=ff, c128=bool(flags))
                    assert len(fwd) == p * (Kf + 1) - (p - 1 if ff else 0)
                    adj = _schedule(h, 1)
                    turn = _check_schedule(adj, n, p, 1, fused=fb, c128=bool(flags))
                    assert len(adj) == p * (Kb + 1) - (p - 1 if fb else 0)
                    assert not turn or fuse, (n, p, plan4)
                    gf = _schedule(h, 2)
                    _check_schedule(gf, n, p, 2, fused=ff, c128=bool(flags), turn_group=adj[0][:2] if turn else None)
                    assert len(gf) == len(fwd) - (1 if turn else 0)
            finally:
                N.aaqaoa_destroy(h)


def test_turnaround_takes_the_forward_last_group_at_n30():
    """The n = 30 gradient evaluation: the forward's 8-qubit group 22-29 is
    also the adjoint's last group, so one turnaround pass ends the forward
    sweep and opens the adjoint one (p = 2, 3)."""
    for p in (2, 3):
        h = _handle(*W.star_graph(30), p=p)
        try:
            adj, gf, fe = _schedule(h, 1), _schedule(h, 2), _schedule(h, 0)
            assert adj[0][:4] == (22, 8, p - 1, p - 1) and adj[0][4] == 0
            assert gf[-1][:2] != (22, 8) and len(gf) == len(fe) - 1
            assert _check_schedule(adj, 30, p, 1, fused=True)
            _check_schedule(gf, 30, p, 2, fused=True, turn_group=(22, 8))
        finally:
            N.aaqaoa_destroy(h)


def test_complex128_forward_starts_with_the_low_pass():
    """complex128 sweeps keep the low pass first (their kernels generate the
    state in stage 0); complex64 forward sweeps start on the first high group."""
    for flags, first_low in ((N.AAQAOA_C128, True), (0, False)):
        h = _handle(*W.star_graph(30), p=3, flags=flags)
        try:
            steps = _schedule(h, 0)
            _check_schedule(steps, 30, 3, 0, fused=True, c128=bool(flags))
            assert (steps[0][0] == 0) == first_low
            adj = _schedule(h, 1)
            turn = adj[0][2] == adj[0][3]  # a turnaround first, then the low pass
            assert adj[1 if turn else 0][0] == 0
        finally:
            N.aaqaoa_destroy(h)


def test_schedule_without_fusion_cases():
    # one high pass per layer, or one layer: nothing to fuse
    for n, p, plan4 in ((20, 3, (13, 1, 12, 1)), (30, 1, (0, 0, 0, 0))):
        h = _handle(*W.star_graph(n), p=p)
        try:
            assert N.aaqaoa_set_pass_plan(h, *plan4) == 0
            for adjoint in (0, 1):
                steps = _schedule(h, adjoint)
                turn = _check_schedule(steps, n, p, adjoint, fused=False)
                assert all(st[3] == -1 for st in steps[(1 if turn else 0):])  # a turnaround may open the adjoint
        finally:
            N.aaqaoa_destroy(h)
    h = _handle(*W.cycle_graph(10), p=3)  # whole-circuit kernel: no tiled passes
    try:
        assert _schedule(h, 0) == [] and _schedule(h, 1) == []
        assert N.aaqaoa_set_layer_fusion(h, 2) == -1
        assert N.aaqaoa_get_schedule(h, 0, None, -1, ctypes.byref(ctypes.c_int())) == -1
    finally:
        N.aaqaoa_destroy(h)


def test_batch_argument_checks():
    """gamma/beta arrays of a batch call must hold B*p values each, B >= 1,
    and a device output must hold B rows: checked before the C call (no GPU)."""
    import types
    from paper_2410_22247_gb300.api import Plan
    fake = types.SimpleNamespace(p=2)
    assert Plan._batch_points(fake, np.zeros(6), np.zeros(6)) == 3
    for g, b in ((np.zeros(6), np.zeros(4)), (np.zeros(5), np.zeros(5)), (np.zeros(0), np.zeros(0))):
        with pytest.raises(ValueError):
            Plan._batch_points(fake, g, b)
    torch = pytest.importorskip("torch")
    d = torch.zeros(6, dtype=torch.float64)
    assert Plan._device_points(fake, d, d, torch.zeros(15, dtype=torch.float64), 5) == 3
    with pytest.raises(ValueError):
        Plan._device_points(fake, d, d, torch.zeros(14, dtype=torch.float64), 5)
    with pytest.raises(ValueError):
        Plan._device_points(fake, d, torch.zeros(4, dtype=torch.float64), d, 1)


def _prepare_ising(n, edges, w, h=None, eorb=None, vorb=None, p=1):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    m = len(e) // 2
    wv = np.ascontiguousarray(w, dtype=np.float64)
    hv = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if a is not None and a.size else None
    D = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None and a.size else None
    arr = lambda x: None if x is None else np.ascontiguousarray(x, dtype=np.int32)
    er, ew, eo = (arr(x) for x in (eorb or (None, None, None)))
    vr, vw, vo = (arr(x) for x in (vorb or (None, None, None)))
    hdl = ctypes.c_void_p()
    rc = N.aaqaoa_prepare_ising(n, m, P(e), D(wv), D(hv), 0 if er is None else len(er), P(er), P(ew), P(eo),
                                0 if vr is None else len(vr), P(vr), P(vw), P(vo), p, 0, None, ctypes.byref(hdl))
    if rc == 0:
        N.aaqaoa_destroy(hdl)
    return rc


def test_prepare_ising_validation():
    """Ising plans: real couplings and fields, vertex orbits for H_red; the
    host rejects non-finite values, classes that mix couplings or fields,
    vertex classes that do not partition the vertices, and fields with edge
    orbits but no vertex orbits."""
    path = [(0, 1), (1, 2), (2, 3)]
    w = [0.5, -1.25, 0.5]
    h = [0.3, -0.2, -0.2, 0.3]
    eorb = ([0, 1], [2, 1], [0, 1, 0])
    vorb = ([0, 1], [2, 2], [0, 1, 1, 0])
    assert _prepare_ising(4, path, w, h, eorb, vorb) == 0
    assert _prepare_ising(4, path, w, None, eorb) == 0
    assert _prepare_ising(4, path, w, h) == 0                                   # no H_red
    assert _prepare_ising(4, path, [0.5, np.nan, 0.5], h) == -1                # weight not finite
    assert _prepare_ising(4, path, w, [0.3, np.inf, -0.2, 0.3]) == -1          # field not finite
    assert _prepare_ising(4, path, [0.5, -1.25, 0.7], h, eorb, vorb) == -2     # class mixes couplings
    assert _prepare_ising(4, path, w, [0.3, -0.2, -0.2, 0.4], eorb, vorb) == -2  # class mixes fields
    assert _prepare_ising(4, path, w, h, eorb) == -2                           # fields, no vertex orbits
    assert _prepare_ising(4, path, w, h, eorb, ([0, 1], [2, 1], [0, 1, 1, 0])) == -2  # sizes do not sum to n
    assert _prepare_ising(4, path, w, h, eorb, ([0, 1], [2, 2], [0, 1, 0, 1])) == -2  # class {0, 2} mixes fields
    assert _prepare_ising(4, [(0, 0)], [1.0]) == -1                            # edges checked as for MaxCut
    assert N.aaqaoa_last_error_detail()


def test_cluster_low_pass_plan_and_schedule():
    """The complex64 adjoint may take a 14-qubit low pass (cluster of 4 CTAs):
    n = 30 then needs 14 + 8 + 8 qubits per layer; every layer of the
    schedule still mixes every qubit once. complex128 rejects it."""
    n, e = W.star_graph(30)
    ee = np.ascontiguousarray(e.reshape(-1), dtype=np.int32)
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    for flags, ok in ((0, True), (1, False)):
        h = ctypes.c_void_p()
        assert N.aaqaoa_prepare(n, len(e), P(ee), 0, None, None, None, 2, flags, None, ctypes.byref(h)) == 0
        rc = N.aaqaoa_set_pass_plan(h, 0, 0, 14, 2)
        assert (rc == 0) == ok
        if ok:
            plan4 = (ctypes.c_int * 4)()
            assert N.aaqaoa_get_pass_plan(h, plan4) == 0 and list(plan4)[2:] == [14, 2]
            steps = (ctypes.c_int32 * (5 * 16))()
            cnt = ctypes.c_int()
            assert N.aaqaoa_get_schedule(h, 1, steps, 16, ctypes.byref(cnt)) == 0
            rows = [list(steps[5 * i:5 * i + 5]) for i in range(cnt.value)]
            assert cnt.value == 5  # 3 passes per layer, one boundary fused
            turn = rows[0][2] == rows[0][3]  # a turnaround (group 22-29) may open the sweep
            assert rows[1 if turn else 0][:2] == [0, 14]
            for layer in (0, 1):
                mixed = set()
                for s0, q, l, l2, j0 in rows:
                    if l == layer:
                        mixed |= set(range(s0, s0 + q))
                    if l2 == layer:
                        mixed |= set(range(s0, s0 + q))
                assert mixed == set(range(n))
        N.aaqaoa_destroy(h)


def test_stats_summarises_an_unprofiled_plan_as_zero():
    """aaqaoa_stats (host-side only here: a plan without a workspace and
    without recorded launches) fills every kind with zeros; NULL is rejected."""
    h = _handle(*W.cycle_graph(16), p=1)
    try:
        st = N.Stats()
        rc = N.aaqaoa_stats(h, ctypes.byref(st))
        assert rc in (0, -4)  # -4 (CUDA error): no device to synchronise with on this host
        if rc == 0:
            assert list(st.launches) == [0] * 5 and list(st.ms) == [0.0] * 5
        assert N.aaqaoa_stats(h, None) == -1
    finally:
        N.aaqaoa_destroy(h)
