"""Python front end of the C ABI: a plan object and a torch.autograd.Function.

PyTorch supplies device memory (the plan's workspace is a uint8 CUDA tensor)
and the CUDA stream; every computation runs in ``libaaqaoa.so``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as N

OBSERVABLES = {"full": N.AAQAOA_OBS_FULL, "red": N.AAQAOA_OBS_RED,
               N.AAQAOA_OBS_FULL: N.AAQAOA_OBS_FULL, N.AAQAOA_OBS_RED: N.AAQAOA_OBS_RED}
AGG_MODES = {"fused": N.AAQAOA_AGG_FUSED, "perterm": N.AAQAOA_AGG_PERTERM, "singlepass": N.AAQAOA_AGG_SINGLEPASS,
             "perorbit": N.AAQAOA_AGG_PERORBIT}


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t)) if a is not None and a.size else None


class Plan:
    """A prepared graph (and its edge orbits) with a device workspace.

    ``orbits`` is an object with ``rep``, ``weight`` and ``edge_orbit``
    attributes (e.g. :class:`paper_2410_22247_gb300.orbits.EdgeOrbits`), a
    ``(rep, weight[, edge_orbit])`` tuple, or None for no reduced observable.

    ``weights`` (integer, >= 1) makes a weighted-MaxCut plan with exact
    integer cut values. ``couplings`` (real, one per edge) and ``fields``
    (real, one per vertex, or None) make an Ising plan (aaqaoa_prepare_ising);
    its H_red also needs vertex orbits: ``orbits`` with ``vrep``, ``vweight``
    and ``vertex_orbit`` attributes (:class:`paper_2410_22247_gb300.orbits.IsingOrbits`).
    """

    def __init__(self, n, edges, p, orbits=None, precision="c64", batch=1, with_grad=True,
                 stream=None, device=None, weights=None, couplings=None, fields=None):
        import torch

        self._lib = N.load()
        self.n, self.p = int(n), int(p)
        self.precision = precision
        self.edges = _i32(edges).reshape(-1, 2)
        flags = N.AAQAOA_C128 if precision == "c128" else N.AAQAOA_C64
        rep = weight = eo = None
        if orbits is not None:
            if hasattr(orbits, "rep"):
                rep, weight, eo = orbits.rep, orbits.weight, getattr(orbits, "edge_orbit", None)
            else:
                rep, weight = orbits[0], orbits[1]
                eo = orbits[2] if len(orbits) > 2 else None
            rep, weight = _i32(rep), _i32(weight)
            eo = None if eo is None else _i32(eo)
        self.num_orbits = 0 if rep is None else len(rep)
        e = _i32(self.edges)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        handle = ctypes.c_void_p()
        self.weights = None if weights is None else _i32(weights)
        self.ising = couplings is not None
        if self.ising:
            if weights is not None:
                raise ValueError("give integer weights or real couplings, not both")
            cw = _f64(couplings)
            fh = None if fields is None else _f64(fields)
            if len(cw) != len(self.edges) or (fh is not None and len(fh) != self.n):
                raise ValueError("couplings need one value per edge and fields one per vertex")
            vr = vw = vo = None
            if orbits is not None and getattr(orbits, "vrep", None) is not None:
                vr, vw = _i32(orbits.vrep), _i32(orbits.vweight)
                vo = None if getattr(orbits, "vertex_orbit", None) is None else _i32(orbits.vertex_orbit)
            self.couplings, self.fields = cw, fh
            N.check(N.aaqaoa_prepare_ising(self.n, len(self.edges), _ptr(e, ctypes.c_int32),
                                           _ptr(cw, ctypes.c_double), _ptr(fh, ctypes.c_double), self.num_orbits,
                                           _ptr(rep, ctypes.c_int32), _ptr(weight, ctypes.c_int32),
                                           _ptr(eo, ctypes.c_int32), 0 if vr is None else len(vr),
                                           _ptr(vr, ctypes.c_int32), _ptr(vw, ctypes.c_int32),
                                           _ptr(vo, ctypes.c_int32), self.p, flags,
                                           ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(handle)),
                    "aaqaoa_prepare_ising")
        else:
            N.check(N.aaqaoa_prepare_weighted(self.n, len(self.edges), _ptr(e, ctypes.c_int32),
                                              _ptr(self.weights, ctypes.c_int32), self.num_orbits,
                                              _ptr(rep, ctypes.c_int32), _ptr(weight, ctypes.c_int32),
                                              _ptr(eo, ctypes.c_int32), self.p, flags,
                                              ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(handle)),
                    "aaqaoa_prepare_weighted")
        self.handle = handle
        self.batch = int(batch)
        self.with_grad = bool(with_grad)
        size = ctypes.c_size_t()
        N.check(N.aaqaoa_workspace_bytes(self.handle, self.batch, int(self.with_grad), ctypes.byref(size)),
                "aaqaoa_workspace_bytes")
        self.workspace = torch.empty(int(size.value), dtype=torch.uint8, device=self.device)
        N.check(N.aaqaoa_set_workspace(self.handle, ctypes.c_void_p(self.workspace.data_ptr()), size.value,
                                       self.batch, int(self.with_grad)), "aaqaoa_set_workspace")

    # -- host-pointer calls (synchronising) --------------------------------
    def expect(self, gamma, beta, observable="full", agg="fused") -> float:
        g, b = _f64(gamma), _f64(beta)
        out = ctypes.c_double()
        N.check(N.aaqaoa_expect(self.handle, _ptr(g, ctypes.c_double), _ptr(b, ctypes.c_double),
                                OBSERVABLES[observable], AGG_MODES[agg], ctypes.byref(out)), "aaqaoa_expect")
        return out.value

    def grad(self, gamma, beta, observable="full"):
        g, b = _f64(gamma), _f64(beta)
        E = ctypes.c_double()
        dg = np.zeros(self.p)
        db = np.zeros(self.p)
        N.check(N.aaqaoa_grad(self.handle, _ptr(g, ctypes.c_double), _ptr(b, ctypes.c_double),
                              OBSERVABLES[observable], ctypes.byref(E), _ptr(dg, ctypes.c_double),
                              _ptr(db, ctypes.c_double)), "aaqaoa_grad")
        return E.value, dg, db

    def _batch_points(self, g, b):
        """Number of points B of flat (gamma, beta) arrays of B*p values each."""
        if len(g) != len(b) or len(g) == 0 or len(g) % self.p:
            raise ValueError(f"gammas and betas need B*p values each (p = {self.p}); got {len(g)} and {len(b)}")
        return len(g) // self.p

    def expect_batch(self, gammas, betas, observable="full"):
        g = _f64(gammas)
        b = _f64(betas)
        B = self._batch_points(g, b)
        out = np.zeros(B)
        N.check(N.aaqaoa_expect_batch(self.handle, B, _ptr(g, ctypes.c_double), _ptr(b, ctypes.c_double),
                                      OBSERVABLES[observable], _ptr(out, ctypes.c_double)), "aaqaoa_expect_batch")
        return out

    def grad_batch(self, gammas, betas, observable="full"):
        """(E[B], dE/dgamma[B, p], dE/dbeta[B, p]) of B points (rows of
        gammas, betas), in waves of the workspace's batch size."""
        g = _f64(gammas)
        b = _f64(betas)
        B = self._batch_points(g, b)
        E = np.zeros(B)
        dg = np.zeros(B * self.p)
        db = np.zeros(B * self.p)
        N.check(N.aaqaoa_grad_batch(self.handle, B, _ptr(g, ctypes.c_double), _ptr(b, ctypes.c_double),
                                    OBSERVABLES[observable], _ptr(E, ctypes.c_double), _ptr(dg, ctypes.c_double),
                                    _ptr(db, ctypes.c_double)), "aaqaoa_grad_batch")
        return E, dg.reshape(B, self.p), db.reshape(B, self.p)

    def edge_zz(self, gamma, beta):
        g, b = _f64(gamma), _f64(beta)
        out = np.zeros(len(self.edges))
        N.check(N.aaqaoa_edge_zz(self.handle, _ptr(g, ctypes.c_double), _ptr(b, ctypes.c_double),
                                 _ptr(out, ctypes.c_double) if len(out) else ctypes.cast(ctypes.pointer(ctypes.c_double()), ctypes.POINTER(ctypes.c_double))),
                "aaqaoa_edge_zz")
        return out

    def verify_orbits(self, gamma, beta, tol):
        """Check that every edge has its class representative's <ZZ> at
        (gamma, beta) (Eq. A3); returns -1, or raises AAQAOAError with code
        AAQAOA_ERR_BAD_ORBITS naming the first failing class."""
        g, b = _f64(gamma), _f64(beta)
        bad = ctypes.c_int(-1)
        N.check(N.aaqaoa_verify_orbits(self.handle, _ptr(g, ctypes.c_double), _ptr(b, ctypes.c_double),
                                       float(tol), ctypes.byref(bad)), "aaqaoa_verify_orbits")
        return bad.value

    def pass_plan(self):
        """[L, K] of the forward and [L, K] of the adjoint passes per layer."""
        out = np.zeros(4, dtype=np.int32)
        N.check(N.aaqaoa_get_pass_plan(self.handle, _ptr(out, ctypes.c_int32)), "aaqaoa_get_pass_plan")
        return out.tolist()

    def set_pass_plan(self, fwd_low=0, fwd_high=0, bwd_low=0, bwd_high=0):
        N.check(N.aaqaoa_set_pass_plan(self.handle, int(fwd_low), int(fwd_high), int(bwd_low), int(bwd_high)),
                "aaqaoa_set_pass_plan")

    def layer_fusion(self):
        """True when layer boundaries are fused into one pass (the default)."""
        v = ctypes.c_int()
        N.check(N.aaqaoa_get_layer_fusion(self.handle, ctypes.byref(v)), "aaqaoa_get_layer_fusion")
        return bool(v.value)

    def set_layer_fusion(self, enable):
        N.check(N.aaqaoa_set_layer_fusion(self.handle, 1 if enable else 0), "aaqaoa_set_layer_fusion")

    def schedule(self, adjoint=False, gradient=False):
        """The tiled passes of one sweep, in launch order: a list of (first
        qubit, qubits, layer, fused second layer or -1, qubits of the layer
        mixed before this pass). adjoint: the adjoint sweep of a gradient
        evaluation (a first row whose second layer equals its layer is the
        turnaround pass); gradient: the forward sweep of a gradient
        evaluation (it ends before the turnaround's group); neither: the
        forward sweep of an energy evaluation."""
        mode = 1 if adjoint else (2 if gradient else 0)
        cnt = ctypes.c_int()
        N.check(N.aaqaoa_get_schedule(self.handle, mode, None, 0, ctypes.byref(cnt)), "aaqaoa_get_schedule")
        out = np.zeros((max(cnt.value, 1), 5), dtype=np.int32)
        N.check(N.aaqaoa_get_schedule(self.handle, mode, _ptr(out, ctypes.c_int32), cnt.value, ctypes.byref(cnt)),
                "aaqaoa_get_schedule")
        return [tuple(int(v) for v in r) for r in out[:cnt.value]]

    def profile_launches(self):
        """The launches recorded since profiling was enabled
        (aaqaoa_profile_enable), in order: dicts of kind (0 forward pass,
        1 adjoint pass, 2 whole circuit, 3 aggregation, 4 parameter tables),
        cut_work, fused, cluster, turnaround, ms and bytes."""
        cnt = ctypes.c_int()
        N.check(N.aaqaoa_profile_launches(self.handle, 0, ctypes.byref(cnt), None, None, None, None),
                "aaqaoa_profile_launches")
        n = cnt.value
        kind = np.zeros(max(n, 1), dtype=np.int32)
        flags = np.zeros(max(n, 1), dtype=np.int32)
        ms = np.zeros(max(n, 1))
        by = np.zeros(max(n, 1))
        N.check(N.aaqaoa_profile_launches(self.handle, n, ctypes.byref(cnt), _ptr(kind, ctypes.c_int32),
                                          _ptr(flags, ctypes.c_int32), _ptr(ms, ctypes.c_double),
                                          _ptr(by, ctypes.c_double)), "aaqaoa_profile_launches")
        return [{"kind": int(kind[i]), "cut_work": bool(flags[i] & 1), "fused": bool(flags[i] & 2),
                 "cluster": bool(flags[i] & 4), "turnaround": bool(flags[i] & 8),
                 "ms": float(ms[i]), "bytes": float(by[i])} for i in range(n)]

    def autotune(self):
        """Time the candidate pass plans and keep the fastest; returns pass_plan()."""
        out = np.zeros(4, dtype=np.int32)
        N.check(N.aaqaoa_autotune(self.handle, _ptr(out, ctypes.c_int32)), "aaqaoa_autotune")
        return out.tolist()

    def max_cut(self):
        """(C_max, smallest maximising bitstring) by device exhaustion."""
        c = np.zeros(1, dtype=np.int32)
        x = ctypes.c_uint64()
        N.check(N.aaqaoa_max_cut(self.handle, _ptr(c, ctypes.c_int32), ctypes.byref(x)), "aaqaoa_max_cut")
        return int(c[0]), int(x.value)

    def approximation_ratio(self, gamma, beta, observable="red"):
        """F_p / C_max (Sec. 2) with F_p from the given observable."""
        cmax, _ = self.max_cut()
        return self.expect(gamma, beta, observable) / cmax

    def sample(self, gamma, beta, u):
        """Bitstrings drawn from |psi_p|^2 for the caller's uniforms u in [0, 1),
        with their cut values: (x uint64 array, C(x) int32 array)."""
        g, b = _f64(gamma), _f64(beta)
        u = _f64(u)
        x = np.zeros(len(u), dtype=np.uint64)
        cut = np.zeros(len(u), dtype=np.int32)
        N.check(N.aaqaoa_sample(self.handle, _ptr(g, ctypes.c_double), _ptr(b, ctypes.c_double), len(u),
                                _ptr(u, ctypes.c_double), x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                _ptr(cut, ctypes.c_int32)), "aaqaoa_sample")
        return x, cut

    def statevector(self, gamma, beta):
        g, b = _f64(gamma), _f64(beta)
        dt = np.complex128 if self.precision == "c128" else np.complex64
        out = np.zeros(1 << self.n, dtype=dt)
        N.check(N.aaqaoa_statevector(self.handle, _ptr(g, ctypes.c_double), _ptr(b, ctypes.c_double),
                                     ctypes.c_void_p(out.ctypes.data)), "aaqaoa_statevector")
        return out

    def aggregate_only(self, observable="full", agg="singlepass") -> float:
        out = ctypes.c_double()
        N.check(N.aaqaoa_aggregate_only(self.handle, OBSERVABLES[observable], AGG_MODES[agg], ctypes.byref(out)),
                "aaqaoa_aggregate_only")
        return out.value

    # -- device-pointer calls (asynchronous on the plan's stream) ----------
    def _device_points(self, d_gamma, d_beta, d_out, row):
        """B of device (gamma, beta) tensors of B*p doubles; d_out must hold B rows of `row` doubles."""
        ng, nb = d_gamma.numel(), d_beta.numel()
        if ng != nb or ng == 0 or ng % self.p:
            raise ValueError(f"d_gamma and d_beta need B*p values each (p = {self.p}); got {ng} and {nb}")
        B = ng // self.p
        if d_out.numel() < B * row:
            raise ValueError(f"output tensor holds {d_out.numel()} values; {B} points need {B * row}")
        return B

    def expect_device(self, d_gamma, d_beta, d_energy, observable="full"):
        B = self._device_points(d_gamma, d_beta, d_energy, 1)
        N.check(N.aaqaoa_expect_device(self.handle, B, ctypes.c_void_p(d_gamma.data_ptr()),
                                       ctypes.c_void_p(d_beta.data_ptr()), OBSERVABLES[observable],
                                       ctypes.c_void_p(d_energy.data_ptr())), "aaqaoa_expect_device")

    def grad_device(self, d_gamma, d_beta, d_out, observable="full"):
        if self._device_points(d_gamma, d_beta, d_out, 1 + 2 * self.p) != 1:
            raise ValueError("grad_device takes one point; use grad_batch_device for several")
        N.check(N.aaqaoa_grad_device(self.handle, ctypes.c_void_p(d_gamma.data_ptr()),
                                     ctypes.c_void_p(d_beta.data_ptr()), OBSERVABLES[observable],
                                     ctypes.c_void_p(d_out.data_ptr())), "aaqaoa_grad_device")

    def grad_batch_device(self, d_gamma, d_beta, d_out, observable="full"):
        """d_gamma, d_beta: B*p doubles on the device; d_out: B rows of 1 + 2p."""
        B = self._device_points(d_gamma, d_beta, d_out, 1 + 2 * self.p)
        N.check(N.aaqaoa_grad_batch_device(self.handle, B, ctypes.c_void_p(d_gamma.data_ptr()),
                                           ctypes.c_void_p(d_beta.data_ptr()), OBSERVABLES[observable],
                                           ctypes.c_void_p(d_out.data_ptr())), "aaqaoa_grad_batch_device")

    def sync(self):
        N.check(N.aaqaoa_sync(self.handle), "aaqaoa_sync")

    def launch_count(self) -> int:
        c = ctypes.c_int()
        N.check(N.aaqaoa_launch_count(self.handle, ctypes.byref(c)), "aaqaoa_launch_count")
        return c.value

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            N.aaqaoa_destroy(self.handle)
            self.handle = ctypes.c_void_p()
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MultiPlan:
    """An uneven batch of graphs evaluated in one call (``aaqaoa_*_multi``).

    ``graphs`` is a list of ``(n, edges, orbits)`` with ``orbits`` as for
    :class:`Plan` (or None). Energies of all graphs come back from one
    replay of a CUDA graph captured on the first call.
    """

    def __init__(self, graphs, p, precision="c64", stream=None, device=None):
        import torch

        self._lib = N.load()
        self.p = int(p)
        self.G = len(graphs)
        self.precision = precision
        self._keep = []
        descs = (N.GraphDesc * self.G)()
        for i, (n, edges, orbits) in enumerate(graphs):
            e = _i32(edges)
            rep = weight = eo = None
            if orbits is not None:
                rep = _i32(orbits.rep if hasattr(orbits, "rep") else orbits[0])
                weight = _i32(orbits.weight if hasattr(orbits, "weight") else orbits[1])
                eo_src = getattr(orbits, "edge_orbit", None) if hasattr(orbits, "rep") else \
                    (orbits[2] if len(orbits) > 2 else None)
                eo = None if eo_src is None else _i32(eo_src)
            self._keep += [e, rep, weight, eo]
            descs[i].n = int(n)
            descs[i].num_edges = len(e) // 2
            descs[i].edges = _ptr(e, ctypes.c_int32)
            descs[i].num_orbits = 0 if rep is None else len(rep)
            descs[i].orbit_rep = _ptr(rep, ctypes.c_int32)
            descs[i].orbit_weight = _ptr(weight, ctypes.c_int32)
            descs[i].edge_orbit = _ptr(eo, ctypes.c_int32)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        flags = N.AAQAOA_C128 if precision == "c128" else N.AAQAOA_C64
        h = ctypes.c_void_p()
        N.check(N.aaqaoa_prepare_multi(self.G, descs, self.p, flags, ctypes.c_void_p(self.stream.cuda_stream),
                                       ctypes.byref(h)), "aaqaoa_prepare_multi")
        self.handle = h
        size = ctypes.c_size_t()
        N.check(N.aaqaoa_multi_workspace_bytes(self.handle, ctypes.byref(size)), "aaqaoa_multi_workspace_bytes")
        self.workspace = torch.empty(int(size.value), dtype=torch.uint8, device=self.device)
        N.check(N.aaqaoa_multi_set_workspace(self.handle, ctypes.c_void_p(self.workspace.data_ptr()), size.value),
                "aaqaoa_multi_set_workspace")

    def expect(self, gammas, betas, observable="full"):
        g, b = _f64(gammas), _f64(betas)
        out = np.zeros(self.G)
        N.check(N.aaqaoa_expect_multi(self.handle, _ptr(g, ctypes.c_double), _ptr(b, ctypes.c_double),
                                      OBSERVABLES[observable], _ptr(out, ctypes.c_double)), "aaqaoa_expect_multi")
        return out

    def info(self):
        v = [ctypes.c_int() for _ in range(4)]
        N.check(N.aaqaoa_multi_info(self.handle, *[ctypes.byref(x) for x in v]), "aaqaoa_multi_info")
        return dict(zip(("graphs", "small_graphs", "branches", "launches_per_call"), (x.value for x in v)))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            N.aaqaoa_destroy_multi(self.handle)
            self.handle = ctypes.c_void_p()
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class AAQAOAFunction(torch.autograd.Function):
        """E(gamma, beta) with the adjoint gradient of ``aaqaoa_grad_device``.

        ``gamma`` and ``beta`` are float64 CUDA tensors of length p. The
        forward pass computes the energy and both gradients in one call; the
        backward pass only scales them by the incoming gradient.
        """

        @staticmethod
        def forward(ctx, gamma, beta, plan, observable="full"):
            g = gamma.detach().to(dtype=torch.float64).contiguous()
            b = beta.detach().to(dtype=torch.float64).contiguous()
            out = torch.empty(1 + 2 * plan.p, dtype=torch.float64, device=g.device)
            plan.grad_device(g, b, out, observable)
            ctx.save_for_backward(out[1:1 + plan.p].clone(), out[1 + plan.p:].clone())
            return out[0].clone()

        @staticmethod
        def backward(ctx, grad_out):
            dg, db = ctx.saved_tensors
            return grad_out * dg, grad_out * db, None, None

    return AAQAOAFunction


_FN = None


def energy(gamma, beta, plan, observable="full"):
    """Differentiable energy: ``AAQAOAFunction.apply(gamma, beta, plan, observable)``."""
    global _FN
    if _FN is None:
        _FN = _autograd_function()
    return _FN.apply(gamma, beta, plan, observable)


def maximize(plan, gamma0, beta0, steps=200, lr=0.05, observable="red", betas=(0.9, 0.999), eps=1e-8):
    """Adam ascent of F_p(gamma, beta) driven by the adjoint gradient
    (aaqaoa_grad). Returns (gamma, beta, history of F_p). The paper optimises
    with gradient-free COBYLA (Sec. 6); this is the gradient-based form of the
    same outer loop. The last history entry is F_p at the returned point."""
    g = np.array(gamma0, dtype=np.float64)
    b = np.array(beta0, dtype=np.float64)
    x = np.concatenate([g, b])
    m = np.zeros_like(x)
    v = np.zeros_like(x)
    hist = []
    for t in range(1, steps + 1):
        E, dg, db = plan.grad(x[:plan.p], x[plan.p:], observable)
        hist.append(E)
        d = np.concatenate([dg, db])
        m = betas[0] * m + (1 - betas[0]) * d
        v = betas[1] * v + (1 - betas[1]) * d * d
        mh = m / (1 - betas[0] ** t)
        vh = v / (1 - betas[1] ** t)
        x = x + lr * mh / (np.sqrt(vh) + eps)
    hist.append(plan.expect(x[:plan.p], x[plan.p:], observable))
    return x[:plan.p], x[plan.p:], np.array(hist)


def maximize_multistart(plan, gammas0, betas0, steps=200, lr=0.05, observable="red", betas=(0.9, 0.999),
                        eps=1e-8):
    """Adam ascent from B starting points at once, each step one batched
    energy + gradient call (aaqaoa_grad_batch) for all of them. gammas0,
    betas0: arrays of shape (B, p). Returns (gamma, beta) of shape (B, p), the
    history of F_p of shape (steps + 1, B), whose last row is F_p at the
    returned points, and the index of the best returned point."""
    g = np.array(gammas0, dtype=np.float64).reshape(-1, plan.p)
    b = np.array(betas0, dtype=np.float64).reshape(-1, plan.p)
    x = np.concatenate([g, b], axis=1)
    m = np.zeros_like(x)
    v = np.zeros_like(x)
    hist = []
    for t in range(1, steps + 1):
        E, dg, db = plan.grad_batch(x[:, :plan.p], x[:, plan.p:], observable)
        hist.append(E)
        d = np.concatenate([dg, db], axis=1)
        m = betas[0] * m + (1 - betas[0]) * d
        v = betas[1] * v + (1 - betas[1]) * d * d
        mh = m / (1 - betas[0] ** t)
        vh = v / (1 - betas[1] ** t)
        x = x + lr * mh / (np.sqrt(vh) + eps)
    hist.append(plan.expect_batch(x[:, :plan.p], x[:, plan.p:], observable))
    hist = np.array(hist)
    return x[:, :plan.p], x[:, plan.p:], hist, int(np.argmax(hist[-1]))
