"""ctypes binding of the C-ABI FE-LBM library (``include/felbm.h``).

Argument marshalling only: every step of the update runs in the library's
CUDA kernels.  The names mirror the C entry points without the ``felbm_``
prefix.  Device memory (the workspace) and the stream come from PyTorch.
If the library is not built or cannot be loaded, every call raises -- there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MAX_WALL_IDS = 256
LAP_CONSISTENT, LAP_PAPER = 0, 1
FP64, FP32_DEV = 0, 1
DIAG_SLOTS = 16          # FELBM_DIAG_SLOTS: raw sums behind one diagnostics record
SOLVER_MIXED, SOLVER_FP64 = 0, 1
LAPMU_FACE, LAPMU_NODAL = 0, 1

_ERRORS = {
    -1: "invalid argument", -2: "bad mesh", -3: "CUDA error", -4: "workspace",
    -5: "non-finite state", -6: "unsupported", -7: "solve not converged",
}


class FelbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"felbm error {code} ({_ERRORS.get(code, '?')}): {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("tau_l", ctypes.c_double), ("tau_v", ctypes.c_double),
                ("rho_l", ctypes.c_double), ("rho_v", ctypes.c_double),
                ("kappa", ctypes.c_double), ("beta", ctypes.c_double),
                ("mobility", ctypes.c_double), ("phi_c", ctypes.c_double * MAX_WALL_IDS),
                ("n_wall_ids", ctypes.c_int32), ("lap_mode", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("solver_mode", ctypes.c_int32),
                ("solver_iters", ctypes.c_int32), ("solver_rounds", ctypes.c_int32),
                ("lapmu_mode", ctypes.c_int32)]


class MeshInfo(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_tri", ctypes.c_int32),
                ("n_wall_edges", ctypes.c_int32), ("n_groups", ctypes.c_int32), ("nnz", ctypes.c_int32),
                ("max_degree", ctypes.c_int32), ("bandwidth", ctypes.c_int32),
                ("min_area", ctypes.c_double), ("total_area", ctypes.c_double),
                ("n_tiles", ctypes.c_int32), ("max_tile_halo", ctypes.c_int32)]


class MeshDesc(ctypes.Structure):
    _fields_ = [("xy", ctypes.c_void_p), ("n_nodes", ctypes.c_int32), ("tri", ctypes.c_void_p),
                ("n_tri", ctypes.c_int32), ("wall_edges", ctypes.c_void_p), ("wall_id", ctypes.c_void_p),
                ("n_wall_edges", ctypes.c_int32), ("period_x", ctypes.c_double), ("period_y", ctypes.c_double)]


class DiagRequest(ctypes.Structure):
    _fields_ = [("centre", ctypes.c_double * 2), ("radius", ctypes.c_double),
                ("band", ctypes.c_double), ("substrate_wall_id", ctypes.c_int32)]


class Diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("mass", ctypes.c_double), ("mass0", ctypes.c_double),
                ("mass_drift_rel", ctypes.c_double), ("kinetic_energy", ctypes.c_double),
                ("max_u", ctypes.c_double), ("interface_rho_uu", ctypes.c_double),
                ("p_in", ctypes.c_double), ("p_out", ctypes.c_double), ("delta_p", ctypes.c_double),
                ("wetted_length", ctypes.c_double), ("height", ctypes.c_double),
                ("theta_deg", ctypes.c_double), ("status", ctypes.c_int32),
                ("solver_sweeps", ctypes.c_int32), ("solver_residual", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class StepTiming(ctypes.Structure):
    _fields_ = [("collide_ms", ctypes.c_float), ("mu_ms", ctypes.c_float),
                ("gradmu_ms", ctypes.c_float), ("element_ms", ctypes.c_float),
                ("rhs_ms", ctypes.c_float), ("solve_ms", ctypes.c_float),
                ("total_ms", ctypes.c_float), ("solve_launches", ctypes.c_int32),
                ("launches", ctypes.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class TuneResult(ctypes.Structure):
    _fields_ = [("sweep_parts", ctypes.c_int32), ("parts_ms", ctypes.c_float * 4),
                ("sweep_tiled", ctypes.c_int32), ("tiled_ms", ctypes.c_float * 4),
                ("cta_max_nodes", ctypes.c_int32), ("n_candidates", ctypes.c_int32),
                ("candidates", ctypes.c_int32 * 16), ("step_ms", ctypes.c_float * 16)]

    def as_dict(self):
        n = self.n_candidates
        return {"sweep_parts": self.sweep_parts, "sweep_tiled": self.sweep_tiled,
                "parts_ms": dict(zip((1, 2, 3, 6), [round(x, 5) for x in self.parts_ms])),
                "tiled_ms": dict(zip((1, 2, 3, 6), [round(x, 5) for x in self.tiled_ms])),
                "cta_max_nodes": self.cta_max_nodes,
                "candidates": list(self.candidates[:n]), "step_ms": list(self.step_ms[:n])}


_LIB = None
_P = ctypes.c_void_p
_I32 = ctypes.c_int32


def _declare(lib):
    sig = {
        "felbm_last_error": (ctypes.c_char_p, []),
        "felbm_params_derive": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, _P, _I32,
                                               ctypes.POINTER(Params)]),
        "felbm_mesh_create": (ctypes.c_int, [_P, _I32, _P, _I32, _P, _P, _I32, ctypes.c_double,
                                             ctypes.c_double, ctypes.POINTER(_P)]),
        "felbm_mesh_info_get": (ctypes.c_int, [_P, ctypes.POINTER(MeshInfo)]),
        "felbm_mesh_destroy": (None, [_P]),
        "felbm_mesh_groups": (ctypes.c_int, [_P, _P, _P]),
        "felbm_mesh_create_batch": (ctypes.c_int, [_I32, ctypes.POINTER(MeshDesc), ctypes.POINTER(_P)]),
        "felbm_diagnostics_groups": (ctypes.c_int, [_P, _P, _I32, _P]),
        "felbm_workspace_bytes": (ctypes.c_int, [_P, ctypes.POINTER(Params),
                                                 ctypes.POINTER(ctypes.c_size_t)]),
        "felbm_init": (ctypes.c_int, [_P, ctypes.POINTER(Params), _P, _P, _P, _P, ctypes.c_size_t, _P,
                                      ctypes.POINTER(_P)]),
        "felbm_step": (ctypes.c_int, [_P, _I32]),
        "felbm_diagnostics": (ctypes.c_int, [_P, ctypes.POINTER(DiagRequest), ctypes.POINTER(Diag)]),
        "felbm_get_state": (ctypes.c_int, [_P, _P, _P]),
        "felbm_set_state": (ctypes.c_int, [_P, _P, _P]),
        "felbm_get_fields": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
        "felbm_mass_solve": (ctypes.c_int, [_P, _P, _P, _I32]),
        "felbm_mass_solve_static": (ctypes.c_int, [_P, _P, _P, _I32]),
        "felbm_adjoint_seed": (ctypes.c_int, [_P, _P, _P]),
        "felbm_adjoint_step": (ctypes.c_int, [_P]),
        "felbm_adjoint_get": (ctypes.c_int, [_P, _P, _P, _P]),
        "felbm_set_wetting": (ctypes.c_int, [_P, _P, _I32]),
        "felbm_checkpoint_bytes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
        "felbm_checkpoint_save": (ctypes.c_int, [_P, _P]),
        "felbm_checkpoint_load": (ctypes.c_int, [_P, _P]),
        "felbm_batch_schedule": (ctypes.c_int, [_P, _I32]),
        "felbm_sweep_parts": (ctypes.c_int, [_P, _I32]),
        "felbm_sweep_tiled": (ctypes.c_int, [_P, _I32]),
        "felbm_solver_check": (ctypes.c_int, [_P, _I32, ctypes.c_double]),
        "felbm_diagnostics_enqueue": (ctypes.c_int, [_P, ctypes.POINTER(DiagRequest), _P]),
        "felbm_diag_finish": (ctypes.c_int, [_P, ctypes.POINTER(DiagRequest), _P, ctypes.POINTER(Diag)]),
        "felbm_autotune": (ctypes.c_int, [_P, _I32, ctypes.POINTER(TuneResult)]),
        "felbm_timing_enable": (ctypes.c_int, [_P, _I32]),
        "felbm_timing_get": (ctypes.c_int, [_P, ctypes.POINTER(StepTiming)]),
        "felbm_fp64_fma_rate": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
        "felbm_state_destroy": (None, [_P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args


def lib():
    """Load ``libfelbm.so`` (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = _build.lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -m paper_1708_04678_gb300.build`")
        _LIB = ctypes.CDLL(path)
        _declare(_LIB)
    return _LIB


def _check(code):
    if code != 0:
        raise FelbmError(code, lib().felbm_last_error().decode())


def check_slots(slots):
    """A diagnostics slot buffer: contiguous host float64, at least DIAG_SLOTS values."""
    if isinstance(slots, np.ndarray):
        ok = slots.dtype == np.float64 and slots.flags["C_CONTIGUOUS"] and slots.size >= DIAG_SLOTS
    else:
        ok = (not slots.is_cuda and str(slots.dtype) == "torch.float64" and slots.is_contiguous()
              and slots.numel() >= DIAG_SLOTS)
    if not ok:
        raise ValueError("slots: contiguous host float64 buffer of at least DIAG_SLOTS values")


def _ptr(a):
    """Host or device address of a numpy array or torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    return a.data_ptr()


def fp64_fma_rate(stream=None):
    """felbm_fp64_fma_rate: the device's FP64 FMA rate in TFLOP/s (instrument)."""
    v = ctypes.c_double()
    _check(lib().felbm_fp64_fma_rate(ctypes.c_void_p(stream.cuda_stream) if stream is not None else None,
                                     ctypes.byref(v)))
    return v.value


def params_derive(phys, lap_mode=LAP_CONSISTENT, solver_iters=0, precision=FP64,
                  solver_mode=SOLVER_MIXED, solver_rounds=0, lapmu_mode=LAPMU_FACE):
    """felbm_params from a physical description (sigma, xi, contact angles in
    degrees, dt, tau_l, tau_v, rho_l, rho_v, mobility)."""
    p = Params()
    p.dt = phys["dt"]
    p.tau_l, p.tau_v = phys["tau_l"], phys["tau_v"]
    p.rho_l, p.rho_v = phys["rho_l"], phys["rho_v"]
    p.mobility = phys["mobility"]
    th = np.ascontiguousarray(phys.get("theta_deg", ()), dtype=np.float64)
    _check(lib().felbm_params_derive(phys["sigma"], phys["xi"], _ptr(th) if th.size else None,
                                     int(th.size), ctypes.byref(p)))
    p.lap_mode = lap_mode
    p.precision = precision
    p.solver_mode = solver_mode
    p.solver_iters = solver_iters
    p.solver_rounds = solver_rounds
    p.lapmu_mode = lapmu_mode
    return p


class Mesh:
    """felbm_mesh: validated, reordered mesh tables on the host."""

    def __init__(self, xy, tri, wall_edges=None, wall_id=None, period=(0.0, 0.0)):
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        we = np.ascontiguousarray(np.zeros((0, 2)) if wall_edges is None else wall_edges, dtype=np.int32)
        wid = np.ascontiguousarray(np.zeros(0) if wall_id is None else wall_id, dtype=np.int32)
        h = _P()
        _check(lib().felbm_mesh_create(_ptr(xy), len(xy), _ptr(tri), len(tri),
                                       _ptr(we) if len(we) else None, _ptr(wid) if len(wid) else None,
                                       len(we), float(period[0]), float(period[1]), ctypes.byref(h)))
        self.handle = h
        self.n_nodes = len(xy)

    @classmethod
    def from_dict(cls, m):
        return cls(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"])

    @classmethod
    def batch(cls, meshes):
        """felbm_mesh_create_batch over mesh dicts (xy, tri, wall_edges,
        wall_id, period); each member keeps its periodic lengths."""
        keep = []
        descs = (MeshDesc * len(meshes))()
        n_total = 0
        for k, m in enumerate(meshes):
            xy = np.ascontiguousarray(m["xy"], dtype=np.float64)
            tri = np.ascontiguousarray(m["tri"], dtype=np.int32)
            we = np.ascontiguousarray(m["wall_edges"], dtype=np.int32).reshape(-1, 2)
            wid = np.ascontiguousarray(m["wall_id"], dtype=np.int32).reshape(-1)
            keep += [xy, tri, we, wid]
            d = descs[k]
            d.xy, d.n_nodes, d.tri, d.n_tri = xy.ctypes.data, len(xy), tri.ctypes.data, len(tri)
            d.wall_edges = we.ctypes.data if len(we) else None
            d.wall_id = wid.ctypes.data if len(wid) else None
            d.n_wall_edges = len(we)
            d.period_x, d.period_y = float(m["period"][0]), float(m["period"][1])
            n_total += len(xy)
        self = cls.__new__(cls)
        h = _P()
        _check(lib().felbm_mesh_create_batch(len(meshes), descs, ctypes.byref(h)))
        self.handle = h
        self.n_nodes = n_total
        return self

    def info(self):
        i = MeshInfo()
        _check(lib().felbm_mesh_info_get(self.handle, ctypes.byref(i)))
        return {name: getattr(i, name) for name, _ in i._fields_}

    def groups(self):
        """(first caller node id, node count) of each connected component."""
        n = self.info()["n_groups"]
        first = np.empty(n, dtype=np.int32)
        size = np.empty(n, dtype=np.int32)
        _check(lib().felbm_mesh_groups(self.handle, _ptr(first), _ptr(size)))
        return first, size

    def workspace_bytes(self, params):
        n = ctypes.c_size_t()
        _check(lib().felbm_workspace_bytes(self.handle, ctypes.byref(params), ctypes.byref(n)))
        return n.value

    def close(self):
        if self.handle:
            lib().felbm_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


mesh_create = Mesh


class State:
    """felbm_state: the distributions and tables of one mesh on one GPU.

    The workspace is a torch uint8 tensor on ``device``; ``stream`` is a
    ``torch.cuda.Stream`` (default: the current stream).  The state starts at
    the equilibria of C0, p0 (default 0) and u0 ((2, N) or (N, 2); default 0)."""

    def __init__(self, mesh: Mesh, params: Params, C0, device="cuda", stream=None, workspace=None, p0=None,
                 u0=None):
        import torch
        self.torch = torch
        self.params = params
        self.N = mesh.n_nodes
        nbytes = mesh.workspace_bytes(params)
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        elif workspace.numel() * workspace.element_size() < nbytes:
            raise ValueError("workspace too small")
        self.workspace = workspace
        self.stream = stream if stream is not None else torch.cuda.current_stream(workspace.device)
        C0 = np.ascontiguousarray(C0, dtype=np.float64)
        if C0.shape != (self.N,):
            raise ValueError("C0 must have one value per node")
        if p0 is not None:
            p0 = np.ascontiguousarray(p0, dtype=np.float64)
            if p0.shape != (self.N,):
                raise ValueError("p0 must have one value per node")
        if u0 is not None:
            u0 = np.asarray(u0, dtype=np.float64)
            if u0.shape == (self.N, 2):
                u0 = u0.T
            u0 = np.ascontiguousarray(u0)
            if u0.shape != (2, self.N):
                raise ValueError("u0 must have shape (2, N) or (N, 2)")
        h = _P()
        _check(lib().felbm_init(mesh.handle, ctypes.byref(params), _ptr(C0), _ptr(p0), _ptr(u0),
                                workspace.data_ptr(), nbytes, ctypes.c_void_p(self.stream.cuda_stream),
                                ctypes.byref(h)))
        self.handle = h
        self.n_groups = mesh.info()["n_groups"]

    def step(self, n=1):
        _check(lib().felbm_step(self.handle, int(n)))

    def diagnostics(self, centre=None, radius=0.0, band=0.0, substrate=0):
        req = DiagRequest()
        if centre is not None:
            req.centre[0], req.centre[1] = float(centre[0]), float(centre[1])
        req.radius, req.band, req.substrate_wall_id = float(radius), float(band), int(substrate)
        d = Diag()
        code = lib().felbm_diagnostics(self.handle, ctypes.byref(req), ctypes.byref(d))
        if code not in (0, -5, -7):
            _check(code)
        return d.as_dict()

    @staticmethod
    def _request(centre, radius, band, substrate):
        req = DiagRequest()
        if centre is not None:
            req.centre[0], req.centre[1] = float(centre[0]), float(centre[1])
        req.radius, req.band, req.substrate_wall_id = float(radius), float(band), int(substrate)
        return req

    def diagnostics_enqueue(self, slots, centre=None, radius=0.0, band=0.0, substrate=0):
        """Queue the diagnostics and an asynchronous copy of their raw sums
        into `slots` (host float64 array or pinned tensor, DIAG_SLOTS values);
        does not synchronise.  Finish with diag_finish after the stream."""
        check_slots(slots)
        req = self._request(centre, radius, band, substrate)
        _check(lib().felbm_diagnostics_enqueue(self.handle, ctypes.byref(req), _ptr(slots)))

    def diag_finish(self, slots, centre=None, radius=0.0, band=0.0, substrate=0):
        req = self._request(centre, radius, band, substrate)
        d = Diag()
        code = lib().felbm_diag_finish(self.handle, ctypes.byref(req), _ptr(slots), ctypes.byref(d))
        if code not in (0, -5, -7):
            _check(code)
        return d.as_dict()

    def diagnostics_groups(self, requests=None, n_groups=None):
        """Per-group diagnostics; requests: list of dicts with centre, radius,
        band, substrate (or None)."""
        if n_groups is None:
            n_groups = len(requests) if requests is not None else self.n_groups
        reqs = None
        if requests is not None:
            reqs = (DiagRequest * n_groups)()
            for g, r in enumerate(requests):
                c = r.get("centre", (0.0, 0.0))
                reqs[g].centre[0], reqs[g].centre[1] = float(c[0]), float(c[1])
                reqs[g].radius = float(r.get("radius", 0.0))
                reqs[g].band = float(r.get("band", 0.0))
                reqs[g].substrate_wall_id = int(r.get("substrate", 0))
        out = (Diag * n_groups)()
        code = lib().felbm_diagnostics_groups(self.handle, reqs, n_groups, out)
        if code not in (0, -5, -7):
            _check(code)
        return [o.as_dict() for o in out]

    def get_state(self, g=None, h=None):
        if g is None:
            g = np.empty((9, self.N))
        if h is None:
            h = np.empty((9, self.N))
        _check(lib().felbm_get_state(self.handle, _ptr(g), _ptr(h)))
        return g, h

    def set_state(self, g, h):
        if isinstance(g, np.ndarray):
            g = np.ascontiguousarray(g, dtype=np.float64)
            h = np.ascontiguousarray(h, dtype=np.float64)
        _check(lib().felbm_set_state(self.handle, _ptr(g), _ptr(h)))

    def get_fields(self):
        out = {k: np.empty(self.N) for k in ("C", "p", "ux", "uy", "mu")}
        _check(lib().felbm_get_fields(self.handle, *(_ptr(out[k]) for k in ("C", "p", "ux", "uy", "mu"))))
        return out

    def mass_solve(self, B):
        B = np.ascontiguousarray(B, dtype=np.float64)
        k = B.shape[0]
        X = np.empty_like(B)
        _check(lib().felbm_mass_solve(self.handle, _ptr(B), _ptr(X), k))
        return X

    def check_static_solve_args(self, d_B, d_X):
        """Reject, before anything is launched, tensors that the C ABI would
        read or write out of bounds: B and X must be contiguous float64
        tensors of shape (k, n_nodes), 1 <= k <= 18, on the state's device,
        and must not overlap.  Returns k."""
        torch = self.torch
        for name, t in (("B", d_B), ("X", d_X)):
            if not isinstance(t, torch.Tensor):
                raise ValueError(f"{name}: a torch tensor on the state's device is required")
            if t.dtype != torch.float64:
                raise ValueError(f"{name}: dtype must be float64, got {t.dtype}")
            if not t.is_contiguous():
                raise ValueError(f"{name}: must be contiguous")
            if t.device != self.workspace.device:
                raise ValueError(f"{name}: on {t.device}, the state lives on {self.workspace.device}")
            if t.dim() != 2 or t.shape[1] != self.N or not 1 <= t.shape[0] <= 18:
                raise ValueError(f"{name}: shape must be (k, {self.N}) with 1 <= k <= 18, got {tuple(t.shape)}")
        if d_X.shape != d_B.shape:
            raise ValueError(f"X has shape {tuple(d_X.shape)}, B has {tuple(d_B.shape)}")
        nbytes = d_B.numel() * 8
        if d_B.data_ptr() < d_X.data_ptr() + nbytes and d_X.data_ptr() < d_B.data_ptr() + nbytes:
            raise ValueError("X overlaps B")
        return int(d_B.shape[0])

    def mass_solve_static(self, d_B, d_X):
        """felbm_mass_solve_static: device tensors B, X of shape (k, n_nodes),
        float64, caller order; enqueued on the state's stream."""
        k = self.check_static_solve_args(d_B, d_X)
        _check(lib().felbm_mass_solve_static(self.handle, d_B.data_ptr(), d_X.data_ptr(), k))

    # -- adjoint and checkpoints ------------------------------------------
    def set_wetting(self, phi_c):
        phi = np.ascontiguousarray(phi_c, dtype=np.float64)
        _check(lib().felbm_set_wetting(self.handle, _ptr(phi), int(phi.size)))

    def checkpoint_bytes(self):
        n = ctypes.c_size_t()
        _check(lib().felbm_checkpoint_bytes(self.handle, ctypes.byref(n)))
        return n.value

    def checkpoint_save(self, d_buf):
        _check(lib().felbm_checkpoint_save(self.handle, d_buf.data_ptr()))

    def checkpoint_load(self, d_buf):
        _check(lib().felbm_checkpoint_load(self.handle, d_buf.data_ptr()))

    def adjoint_seed(self, dL_dg, dL_dh):
        dg = np.ascontiguousarray(dL_dg, dtype=np.float64)
        dh = np.ascontiguousarray(dL_dh, dtype=np.float64)
        _check(lib().felbm_adjoint_seed(self.handle, _ptr(dg), _ptr(dh)))

    def adjoint_step(self):
        _check(lib().felbm_adjoint_step(self.handle))

    def adjoint_get(self, n_wall_ids=None):
        n_ids = self.params.n_wall_ids if n_wall_ids is None else n_wall_ids
        dg = np.empty((9, self.N))
        dh = np.empty((9, self.N))
        dphi = np.zeros(max(n_ids, 1))
        _check(lib().felbm_adjoint_get(self.handle, _ptr(dg), _ptr(dh), _ptr(dphi)))
        return dg, dh, dphi[:n_ids]

    def batch_schedule(self, cta_max_nodes):
        _check(lib().felbm_batch_schedule(self.handle, int(cta_max_nodes)))

    def sweep_parts(self, parts):
        _check(lib().felbm_sweep_parts(self.handle, int(parts)))

    def sweep_tiled(self, on=True):
        _check(lib().felbm_sweep_tiled(self.handle, 1 if on else 0))

    def solver_check(self, enable=True, tol=1e-6):
        _check(lib().felbm_solver_check(self.handle, 1 if enable else 0, float(tol)))

    def autotune(self, trials=5):
        r = TuneResult()
        _check(lib().felbm_autotune(self.handle, int(trials), ctypes.byref(r)))
        return r.as_dict()

    def timing_enable(self, on=True):
        _check(lib().felbm_timing_enable(self.handle, 1 if on else 0))

    def timing_get(self):
        t = StepTiming()
        _check(lib().felbm_timing_get(self.handle, ctypes.byref(t)))
        return t.as_dict()

    def close(self):
        if getattr(self, "handle", None):
            lib().felbm_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


init = State
