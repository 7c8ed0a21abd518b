"""Helpers shared by the GPU parity tests: run the same seeded workload
through the CPU oracle and through the CUDA library, compare element by
element.  The relative error of a field is max|gpu - oracle| / max|oracle|
(normwise: g holds values near zero where an elementwise ratio means
nothing)."""
import numpy as np

from oracle import OracleMesh, OracleSim, params_from_physical
from paper_1708_04678_gb300 import felbm as F

LAP = {"consistent": F.LAP_CONSISTENT, "paper": F.LAP_PAPER}


def rel_err(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def oracle_sim(w, lap="consistent"):
    m = w["mesh"]
    om = OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"])
    return OracleSim(om, params_from_physical(w["phys"], lap), w["C0"])


def gpu_state(w, lap="consistent", solver_iters=0, stream=None, solver_mode=F.SOLVER_MIXED,
              precision=F.FP64):
    mesh = F.Mesh.from_dict(w["mesh"])
    prm = F.params_derive(w["phys"], LAP[lap], solver_iters=solver_iters, solver_mode=solver_mode,
                          precision=precision)
    return F.State(mesh, prm, w["C0"], stream=stream)


def compare_states(osim, gst):
    g, h = gst.get_state()
    return {"g": rel_err(g, osim.g), "h": rel_err(h, osim.h),
            "C": rel_err(h.sum(0), osim.h.sum(0))}


def elementwise_c_err(osim, gst, floor=0.05):
    """Largest elementwise relative error of C = sum h over the nodes where
    the oracle's C is at least `floor` (where a ratio means something)."""
    h = gst.get_state()[1]
    C, Co = h.sum(0), osim.h.sum(0)
    sel = np.abs(Co) >= floor
    return float((np.abs(C[sel] - Co[sel]) / np.abs(Co[sel])).max())

