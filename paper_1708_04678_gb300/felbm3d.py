"""ctypes binding of the 3D entry points (``include/felbm3d.h``).

Argument marshalling only: every step runs in the library's CUDA kernels
(D3Q19 on linear tetrahedra).  Names mirror the C entry points without the
``felbm3d_`` prefix; parameters are the shared ``felbm.Params``.  There is
no CPU fallback: a missing library raises.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import felbm as F
from .felbm import FP32_DEV, FP64, LAP_CONSISTENT, LAP_PAPER, SOLVER_FP64, SOLVER_MIXED  # noqa: F401

_P = ctypes.c_void_p
_I32 = ctypes.c_int32


class MeshInfo3D(ctypes.Structure):
    _fields_ = [("n_nodes", _I32), ("n_tet", _I32), ("n_wall_faces", _I32), ("nnz", _I32),
                ("max_degree", _I32), ("bandwidth", _I32), ("max_incidence", _I32),
                ("min_volume", ctypes.c_double), ("total_volume", ctypes.c_double)]


class DiagRequest3D(ctypes.Structure):
    _fields_ = [("centre", ctypes.c_double * 3), ("radius", ctypes.c_double),
                ("band", ctypes.c_double), ("substrate_wall_id", _I32)]


class Diag3D(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("mass", ctypes.c_double), ("mass0", ctypes.c_double),
                ("mass_drift_rel", ctypes.c_double), ("kinetic_energy", ctypes.c_double),
                ("max_u", ctypes.c_double), ("interface_rho_uu", ctypes.c_double),
                ("p_in", ctypes.c_double), ("p_out", ctypes.c_double), ("delta_p", ctypes.c_double),
                ("wetted_area", ctypes.c_double), ("height", ctypes.c_double),
                ("base_diameter", ctypes.c_double), ("theta_deg", ctypes.c_double), ("status", _I32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_DECLARED = False


def lib():
    """The shared library with the 3D signatures declared."""
    global _DECLARED
    L = F.lib()
    if not _DECLARED:
        sig = {
            "felbm3d_mesh_create": (ctypes.c_int, [_P, _I32, _P, _I32, _P, _P, _I32, _P, ctypes.POINTER(_P)]),
            "felbm3d_mesh_info_get": (ctypes.c_int, [_P, ctypes.POINTER(MeshInfo3D)]),
            "felbm3d_mesh_destroy": (None, [_P]),
            "felbm3d_workspace_bytes": (ctypes.c_int, [_P, ctypes.POINTER(F.Params), ctypes.POINTER(ctypes.c_size_t)]),
            "felbm3d_init": (ctypes.c_int, [_P, ctypes.POINTER(F.Params), _P, _P, ctypes.c_size_t, _P,
                                            ctypes.POINTER(_P)]),
            "felbm3d_step": (ctypes.c_int, [_P, _I32]),
            "felbm3d_diagnostics": (ctypes.c_int, [_P, ctypes.POINTER(DiagRequest3D), ctypes.POINTER(Diag3D)]),
            "felbm3d_diagnostics_enqueue": (ctypes.c_int, [_P, ctypes.POINTER(DiagRequest3D), _P]),
            "felbm3d_diag_finish": (ctypes.c_int, [_P, ctypes.POINTER(DiagRequest3D), _P,
                                                   ctypes.POINTER(Diag3D)]),
            "felbm3d_get_state": (ctypes.c_int, [_P, _P, _P]),
            "felbm3d_set_state": (ctypes.c_int, [_P, _P, _P]),
            "felbm3d_get_fields": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
            "felbm3d_timing_enable": (ctypes.c_int, [_P, _I32]),
            "felbm3d_timing_get": (ctypes.c_int, [_P, _P]),
            "felbm3d_step_launches": (ctypes.c_int, [_P, ctypes.POINTER(_I32)]),
            "felbm3d_state_destroy": (None, [_P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _DECLARED = True
    return L


_check = F._check
_ptr = F._ptr


class Mesh3D:
    """felbm3d_mesh: validated, reordered tetrahedral mesh tables on the host."""

    def __init__(self, xyz, tet, wall_faces=None, wall_id=None, period=(0.0, 0.0, 0.0)):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        tet = np.ascontiguousarray(tet, dtype=np.int32)
        wf = np.ascontiguousarray(np.zeros((0, 3)) if wall_faces is None else wall_faces, dtype=np.int32)
        wid = np.ascontiguousarray(np.zeros(0) if wall_id is None else wall_id, dtype=np.int32)
        per = np.ascontiguousarray(period, dtype=np.float64)
        if xyz.ndim != 2 or xyz.shape[1] != 3 or tet.ndim != 2 or tet.shape[1] != 4 or per.shape != (3,):
            raise ValueError("xyz must be (N, 3), tet (T, 4), period (3,)")
        self._keep = (xyz, tet, wf, wid, per)
        h = _P()
        _check(lib().felbm3d_mesh_create(_ptr(xyz), len(xyz), _ptr(tet), len(tet),
                                         _ptr(wf) if len(wf) else None, _ptr(wid) if len(wid) else None,
                                         len(wf), _ptr(per), ctypes.byref(h)))
        self.handle = h
        self.n_nodes = len(xyz)

    @classmethod
    def from_dict(cls, m):
        return cls(m["xyz"], m["tet"], m["wall_faces"], m["wall_id"], m["period"])

    def info(self):
        i = MeshInfo3D()
        _check(lib().felbm3d_mesh_info_get(self.handle, ctypes.byref(i)))
        return {name: getattr(i, name) for name, _ in i._fields_}

    def workspace_bytes(self, params):
        n = ctypes.c_size_t()
        _check(lib().felbm3d_workspace_bytes(self.handle, ctypes.byref(params), ctypes.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "handle", None):
            lib().felbm3d_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State3D:
    """felbm3d_state: distributions and tables of one tetrahedral mesh on one
    GPU; workspace is a torch uint8 tensor, stream a torch.cuda.Stream."""

    def __init__(self, mesh: Mesh3D, params, C0, device="cuda", stream=None, workspace=None):
        import torch
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
        h = _P()
        _check(lib().felbm3d_init(mesh.handle, ctypes.byref(params), _ptr(C0), workspace.data_ptr(), nbytes,
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.handle = h

    def step(self, n=1):
        _check(lib().felbm3d_step(self.handle, int(n)))

    @staticmethod
    def _request(centre, radius, band, substrate):
        req = DiagRequest3D()
        if centre is not None:
            for k in range(3):
                req.centre[k] = float(centre[k])
        req.radius, req.band, req.substrate_wall_id = float(radius), float(band), int(substrate)
        return req

    def diagnostics(self, centre=None, radius=0.0, band=0.0, substrate=0):
        req = self._request(centre, radius, band, substrate)
        d = Diag3D()
        code = lib().felbm3d_diagnostics(self.handle, ctypes.byref(req), ctypes.byref(d))
        if code != 0:
            _check(code)
        return d.as_dict()

    def diagnostics_enqueue(self, slots, centre=None, radius=0.0, band=0.0, substrate=0):
        """Queue the diagnostics and an asynchronous copy of their raw sums into
        `slots` (host float64, F.DIAG_SLOTS values); finish with diag_finish."""
        F.check_slots(slots)
        req = self._request(centre, radius, band, substrate)
        _check(lib().felbm3d_diagnostics_enqueue(self.handle, ctypes.byref(req), _ptr(slots)))

    def diag_finish(self, slots, centre=None, radius=0.0, band=0.0, substrate=0):
        req = self._request(centre, radius, band, substrate)
        d = Diag3D()
        _check(lib().felbm3d_diag_finish(self.handle, ctypes.byref(req), _ptr(slots), ctypes.byref(d)))
        return d.as_dict()

    def get_state(self, g=None, h=None):
        g = np.empty((19, self.N)) if g is None else g
        h = np.empty((19, self.N)) if h is None else h
        _check(lib().felbm3d_get_state(self.handle, _ptr(g), _ptr(h)))
        return g, h

    def set_state(self, g, h):
        if isinstance(g, np.ndarray):
            g = np.ascontiguousarray(g, dtype=np.float64)
            h = np.ascontiguousarray(h, dtype=np.float64)
        _check(lib().felbm3d_set_state(self.handle, _ptr(g), _ptr(h)))

    def get_fields(self):
        keys = ("C", "p", "ux", "uy", "uz", "mu")
        out = {k: np.empty(self.N) for k in keys}
        _check(lib().felbm3d_get_fields(self.handle, *(_ptr(out[k]) for k in keys)))
        return out

    def launches(self):
        n = _I32()
        _check(lib().felbm3d_step_launches(self.handle, ctypes.byref(n)))
        return n.value

    def timing_enable(self, on=True):
        _check(lib().felbm3d_timing_enable(self.handle, 1 if on else 0))

    def timing_get(self):
        ms = np.zeros(6)
        _check(lib().felbm3d_timing_get(self.handle, _ptr(ms)))
        return dict(zip(("collide_mu_ms", "gradmu_ms", "element_ms", "rhs_ms", "solve_ms", "total_ms"), ms))

    def close(self):
        if getattr(self, "handle", None):
            lib().felbm3d_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


mesh_create = Mesh3D
init = State3D
