#!/usr/bin/env python
"""Throughput of the FE-LBM contact-line step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl felbm|reference]

A step is one full time step (collision, chemical potential with the wetting
boundary, element Laplacian of mu, P0 forces, streaming right-hand side and
the consistent-mass solve) of the rough-wall droplet: a 2048 x 1024 box whose
bottom wall is y = 8 + 4 sin(2 pi x / 64), meshed body-fitted with 1017 rows
(2,082,816 nodes, 4,161,536 triangles, jitter 0.2h), droplet R 300, contact
angle 60 degrees, density ratio 100.  Its state and solve working set are far
above the 129 MB L2, and L2 is flushed before every timed step (a 256 MiB
write).  The metric is node-updates per second: one node, one step, both D2Q9
sets; each step is timed with CUDA events on the library's stream.  The
headline is the FP32-deviation form; the plain FP64 step of the same workload
is timed beside it, and the 256 x 256 free droplet, the 64-droplet batch, the
adjoint and the 3D step as further sections.

The path has no exchange step across meshes, so N > 1 runs N independent
replicas (one per GPU, weak scaling); value is the sum over ranks, the time
the maximum over ranks.

``--impl reference`` times the FP64 CPU oracle (numpy/scipy) on all host
cores, one single-threaded process per core, each stepping its own copy of
a 128-column periodic strip of the same workload (130,176 nodes, the same
rows, wall, jitter and physics), capped to about two minutes: one
step of the full mesh takes the oracle over a minute and several GB, and
runs slower per node-update than the strip does (more cache misses), so the
strip's rate is an upper bound on the oracle's full-mesh rate.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 256 << 20
METRIC = "node-updates/s (2xD2Q9)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="felbm", choices=["felbm", "reference"])
    ap.add_argument("--cpu-baseline-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--only-3d", action="store_true",
                    help="time only the 3D (D3Q19, tetrahedra) section and print it as one JSON line")
    ap.add_argument("--ncu-case", choices=["fp32", "fp32-tiled", "fp64"],
                    help="run two steps of the 1024-column rough-wall droplet (1,041,408 nodes, above L2, about "
                         "2 GB on the device) and exit: the small case for ncu captures of the step kernels")
    ap.add_argument("--sweep-parts", type=int, default=2, help="threads per node of the solve steps (--ncu-case)")
    return ap.parse_args()


def workload():
    from paper_1708_04678_gb300 import inputs as I
    return I.rough_wall_droplet()


def oracle_sample():
    """The bounded sample of the workload the CPU oracle is timed on."""
    from paper_1708_04678_gb300 import inputs as I
    return I.rough_wall_strip()


def workload_config(w, world=1):
    """The `config` object of both arms: what the workload is."""
    return {"workload": "rough-wall droplet 2048x1024: wall y = 8 + 4 sin(2 pi x/64), 1017 body-fitted rows "
                        "(2,082,816 nodes, 4,161,536 triangles), jitter 0.2h, R 300, 60 deg, density ratio 100, "
                        "dt 0.1",
            "nodes": len(w["mesh"]["xy"]), "triangles": len(w["mesh"]["tri"]), "dt": w["phys"]["dt"],
            "l2": "inputs larger than L2 (about 0.6 GB touched per solve step) and L2 flushed before every "
                  "timed step (256 MiB write)",
            "parallelism": f"replicas x{world}"}


# ------------------------------------------------------------- CPU oracle --
def run_oracle(budget_s, max_steps, warmup):
    """Time the FP64 oracle on steps of the bounded sample of the workload;
    returns (node-updates/s, steps timed, seconds)."""
    from oracle import OracleMesh, OracleSim, params_from_physical
    w = oracle_sample()
    m = w["mesh"]
    sim = OracleSim(OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"]),
                    params_from_physical(w["phys"]), w["C0"])
    for _ in range(warmup):
        sim.step(1)
    t0 = time.perf_counter()
    n = 0
    while n < max_steps:
        sim.step(1)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return len(m["xy"]) * n / dt, n, dt


def _oracle_worker(conn):
    """One host core of the all-cores oracle timing: builds its own copy of
    the strip sample, then runs the number of steps it is sent and answers
    with the wall time they took (None ends it)."""
    from oracle import OracleMesh, OracleSim, params_from_physical
    w = oracle_sample()
    m = w["mesh"]
    sim = OracleSim(OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"]),
                    params_from_physical(w["phys"]), w["C0"])
    conn.send(len(m["xy"]))
    while True:
        k = conn.recv()
        if k is None:
            break
        t0 = time.perf_counter()
        sim.step(k)
        conn.send(time.perf_counter() - t0)
    conn.close()


def host_procs():
    """Processes for the all-cores oracle timing: one per usable host core,
    capped so that their copies of the strip (about 0.75 GB each) fit in
    half of the free host memory."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    try:
        free = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        cores = min(cores, max(1, int(free * 0.5 // (0.75 * 2 ** 30))))
    except (ValueError, OSError):
        pass
    return max(1, min(cores, 64))


def run_oracle_all_cores(budget_s, max_steps, warmup, procs):
    """Time the FP64 oracle on all host cores at once: `procs` processes, one
    per core and single-threaded, each stepping its own copy of the strip
    sample (independent units, as the GPU replicas are).  The processes
    advance in lock step, so each step costs the slowest one's time; returns
    (node-updates/s over all processes, steps timed, seconds)."""
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"                      # inherited by the spawned processes
    ctx = mp.get_context("spawn")
    pipes, workers = [], []
    try:
        for _ in range(procs):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b,), daemon=True)
            p.start()
            b.close()
            pipes.append(a)
            workers.append(p)
        nodes = sum(c.recv() for c in pipes)

        def lockstep():
            for c in pipes:
                c.send(1)
            for c in pipes:
                c.recv()

        for _ in range(warmup):
            lockstep()
        t0 = time.perf_counter()
        n = 0
        while n < max_steps:
            lockstep()
            n += 1
            if time.perf_counter() - t0 > budget_s:
                break
        dt = time.perf_counter() - t0
    finally:
        for c in pipes:
            try:
                c.send(None)
            except (BrokenPipeError, OSError):
                pass
        for p in workers:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    return nodes * n / dt, n, dt


def cpu_baseline_subprocess(seconds):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-only",
                        "--cpu-seconds", str(seconds)], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1:] or ["failed"]}
    return json.loads(r.stdout.strip().splitlines()[-1])


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 9
                          for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


SOURCES_2D = ("felbm.cu", "felbm_dev32.cuh", "felbm_adjoint.cuh", "felbm_internal.h", "mesh.cpp", "felbm.h")
SOURCES_3D = ("felbm3d.cu", "felbm3d_dev32.cuh", "felbm3d_internal.h", "mesh3d.cpp", "felbm_internal.h",
              "felbm3d.h", "felbm.h")


def source_hash(files=SOURCES_2D):
    """sha256 prefix of the CUDA library sources a kernel is built from (to
    tell whether a recorded ncu figure still describes the kernel that runs)."""
    import hashlib
    h = hashlib.sha256()
    for name in files:
        for d in (os.path.join(ROOT, "paper_1708_04678_gb300", "csrc"), os.path.join(ROOT, "include")):
            path = os.path.join(d, name)
            if os.path.exists(path):
                with open(path, "rb") as f:
                    h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, files=SOURCES_2D):
    """DRAM bytes per launch of `kernel` from profiles/roofline_traffic.txt
    (lines: kernel, source hash, bytes), if recorded for these sources."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
    if not os.path.exists(path):
        return None
    h = source_hash(files)
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel and parts[1] == h:
                return float(parts[2])
    return None


def recorded_fp64_flops(files=SOURCES_2D):
    """FP64 flops per unit (triangle or node) of the FP64 step's kernels from
    profiles/fp64_flops.txt (lines: kernel, source hash, flops, unit), for
    these sources: 2 x DFMA + DADD + DMUL thread instructions of one ncu
    capture divided by the units of the launch."""
    path = os.path.join(ROOT, "profiles", "fp64_flops.txt")
    out = {}
    if not os.path.exists(path):
        return out
    h = source_hash(files)
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 4 and not line.startswith("#") and parts[1] == h:
                out[parts[0]] = (float(parts[2]), parts[3])
    return out


def fp64_roofline(r64, n_nodes, n_tri, rate, fp64_peak, flops):
    """FP64-pipe roofline of the FP64 step: the element kernel alone (the
    largest FP64 kernel) and the whole step's FP64 flops per node-update."""
    if not flops or "k_element" not in flops:
        return {"bound": "fp64", "unavailable": "no FP64 flop counts recorded for these sources"}
    per = {"tri": n_tri, "node": n_nodes}
    ph = r64["phase_ms"]
    el = flops["k_element"][0] * per[flops["k_element"][1]]
    ach = el / (ph["element_ms"] * 1e-3) / 1e12
    step = sum(f * per[u] * (2 if k == "k_refine" else 1) for k, (f, u) in flops.items()) / n_nodes
    return {"bound": "fp64", "kernel": "k_element (P0 forces and element residual, FP64)",
            "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
            "flops_per_launch": el, "launch_ms": ph["element_ms"],
            "step_fp64_flops_per_node_update": step,
            "step_achieved": step * rate / 1e12, "step_frac": step * rate / 1e12 / fp64_peak,
            "peak_source": "felbm_fp64_fma_rate (independent FP64 FMA chains on every SM, measured in this run)",
            "source_hash": source_hash()}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                d = json.load(f)
            hbm = d.get("hbm_gbs") or d.get("hbm_GBps")
            if hbm:
                return float(hbm), "measured"
        except (OSError, ValueError):
            pass
    return 6800.0, "fallback"


# ------------------------------------------------------ rank aggregation --
def max_over_ranks(x, torch, dist, world, device):
    """The largest of the ranks' values (the job's time is its slowest rank)."""
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank_step, steps, world, max_ms):
    """Whole-job throughput of N independent replicas: all ranks' units over
    the slowest rank's time."""
    return units_per_rank_step * steps * world / (max_ms * 1e-3)


# --------------------------------------------------------------- GPU arm --
def phase_pass(st, torch, stream, flush, n):
    """Phase split of n steps with the library's phase events switched on
    (kept out of the timed steps: the events sit between the kernels of the
    step graph and break its programmatic-launch chain)."""
    st.timing_enable(True)
    phases = []
    for k in range(n):
        with torch.cuda.stream(stream):
            flush.fill_(k & 255)
        st.step(1)
        phases.append(st.timing_get())
    st.timing_enable(False)
    return phases


def time_precision(F, torch, w, dev, precision, K, W, flush, barrier, world, dist, e2e=True):
    """Build a state of the workload in one precision, run W warm-up steps and
    K timed steps (L2 flushed before each), then K end-to-end steps through
    host buffers, in two forms.  Returns the measurements of this rank."""
    mesh = F.Mesh.from_dict(w["mesh"])
    prm = F.params_derive(w["phys"], precision=precision)
    stream = torch.cuda.Stream(dev)
    st = F.State(mesh, prm, w["C0"], device=dev, stream=stream)
    tune = st.autotune(trials=3)
    for k in range(W):
        with torch.cuda.stream(stream):
            flush.fill_(k & 255)
        st.step(1)
    stream.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    torch.cuda.synchronize()
    barrier()
    # the timed steps run without phase events (they would sit between the
    # kernels of the step graph and break its programmatic-launch chain)
    for k in range(K):
        with torch.cuda.stream(stream):
            flush.fill_(k & 255)
        ev0[k].record(stream)
        st.step(1)
        ev1[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    total_ms = max_over_ranks(sum(ev0[k].elapsed_time(ev1[k]) for k in range(K)), torch, dist, world, dev)
    # phase split (and the solve sweep's launch time) from a separate pass with phase events
    phases = phase_pass(st, torch, stream, flush, min(K, 10))
    diag = st.diagnostics(w["centre"], w["R"], w["phys"]["xi"])
    out = {"total_ms": total_ms, "tune": tune, "diag": diag,
           "phase_ms": {k: statistics.mean(p[k] for p in phases) for k in phases[0] if k.endswith("_ms")},
           "launches": phases[0]["launches"], "solve_launches": phases[0]["solve_launches"]}
    if e2e:
        # end to end through the public API with host buffers, every step: the
        # pinned g, h copied in (set_state copies on its own stream, so the
        # copy overlaps the previous step), one step, and the step's
        # diagnostics read back asynchronously into pinned slots; all K
        # results are read and finished on the host inside the timed region
        g0, h0 = st.get_state()
        gp = torch.from_numpy(g0).pin_memory()
        hp = torch.from_numpy(h0).pin_memory()
        slots = torch.zeros((K, F.DIAG_SLOTS), dtype=torch.float64).pin_memory()
        for k in range(2):
            st.set_state(gp, hp)
            st.step(1)
            st.diagnostics_enqueue(slots[k])
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for k in range(K):
            st.set_state(gp, hp)
            st.step(1)
            st.diagnostics_enqueue(slots[k])
        stream.synchronize()
        e2e_diag = [st.diag_finish(slots[k]) for k in range(K)]
        out["e2e_s"] = max_over_ranks(time.perf_counter() - t0, torch, dist, world, dev)
        if any(d["status"] != 0 for d in e2e_diag):
            raise RuntimeError("end-to-end steps produced a non-finite state")
        # the same with the whole state read back every step (felbm_get_state
        # into pinned host arrays, which synchronises) instead of the metrics
        go = torch.empty_like(gp).pin_memory()
        ho = torch.empty_like(hp).pin_memory()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for k in range(K):
            st.set_state(gp, hp)
            st.step(1)
            st.get_state(go.numpy(), ho.numpy())
        out["e2e_state_s"] = max_over_ranks(time.perf_counter() - t0, torch, dist, world, dev)
        if not (np.isfinite(go.numpy()).all() and np.isfinite(ho.numpy()).all()):
            raise RuntimeError("end-to-end steps produced a non-finite state")
        out["state_bytes"] = int(gp.numel() * 8 + hp.numel() * 8)
    out["info"] = mesh.info()
    st.close()
    return out


def time_batch(F, torch, dev, K, flush, barrier, world, dist):
    """The 64-droplet contact-angle sweep (widths 64..512, 3.46M nodes) as one
    FP32-deviation batch: autotuned schedule, then K timed steps."""
    from paper_1708_04678_gb300 import inputs as I
    b = I.batch(I.droplet_sweep())
    mesh = F.Mesh.batch(b["meshes"])
    prm = F.params_derive(b["phys"], precision=F.FP32_DEV)
    stream = torch.cuda.Stream(dev)
    st = F.State(mesh, prm, b["C0"], device=dev, stream=stream)
    tune = st.autotune(trials=3)
    for k in range(3):
        with torch.cuda.stream(stream):
            flush.fill_(k & 255)
        st.step(1)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    torch.cuda.synchronize()
    barrier()
    for k in range(K):
        with torch.cuda.stream(stream):
            flush.fill_(k & 255)
        ev0[k].record(stream)
        st.step(1)
        ev1[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    total_ms = max_over_ranks(sum(ev0[k].elapsed_time(ev1[k]) for k in range(K)), torch, dist, world, dev)
    reqs = [{"centre": m["centre"], "radius": m["R"], "band": 4.0, "substrate": m["substrate"]}
            for m in b["members"]]
    dg = st.diagnostics_groups(reqs)
    n = mesh.info()["n_nodes"]
    st.timing_enable(True)
    st.step(1)
    sweeps = st.timing_get()["solve_launches"] + 1
    st.timing_enable(False)
    st.close()
    value = job_rate(n, K, world, total_ms)
    # the whole step against the minimum bytes per node-update of the FP32
    # form, as for the rough wall (distributions and right-hand side written
    # and read, three 18-float streams per solve step, ~200 B of fields)
    step_bytes = 2 * 18 * 4 + 2 * 18 * 4 + sweeps * 3 * 18 * 4 + 200
    hbm_peak, peak_src = peaks()
    return {"workload": "64-droplet contact-angle sweep, widths 64..512, FP32 deviation storage",
            "nodes": n, "members": len(b["members"]), "steps": K,
            "value": value, "unit": "node-updates/s",
            "ms_per_step": total_ms / K, "schedule": tune,
            "finite": all(d["status"] == 0 for d in dg),
            "max_abs_mass_drift_rel": max(abs(d["mass_drift_rel"]) for d in dg),
            "step_roofline": {"alg_bytes_per_node_update": step_bytes, "sweeps": sweeps,
                              "achieved": value / world * step_bytes / 1e9, "peak": hbm_peak, "unit": "GB/s",
                              "frac": value / world * step_bytes / 1e9 / hbm_peak, "peak_source": peak_src}}


def time_adjoint(F, torch, dev, K):
    """The FP64 forward step and its adjoint on the 128x64 sessile droplet
    (8,320 nodes): device time per step of each."""
    from paper_1708_04678_gb300 import inputs as I
    w = I.sessile_droplet_128x64()
    mesh = F.Mesh.from_dict(w["mesh"])
    stream = torch.cuda.Stream(dev)
    st = F.State(mesh, F.params_derive(w["phys"]), w["C0"], device=dev, stream=stream)
    st.step(5)
    g, h = st.get_state()
    st.adjoint_seed(np.zeros_like(g), np.ones_like(h))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    st.step(K)
    e1.record(stream)
    e1.synchronize()
    fwd_ms = e0.elapsed_time(e1) / K
    e0.record(stream)
    for _ in range(K):
        st.adjoint_step()
    e1.record(stream)
    e1.synchronize()
    adj_ms = e0.elapsed_time(e1) / K
    n = len(w["mesh"]["xy"])
    st.close()
    return {"workload": "sessile droplet 128x64 (8,320 nodes), FP64", "steps": K,
            "forward_ms_per_step": fwd_ms, "adjoint_ms_per_step": adj_ms,
            "adjoint_node_updates_per_s": n / (adj_ms * 1e-3), "adjoint_over_forward": adj_ms / fwd_ms}


def time_free_droplet(F, torch, dev, K, flush, barrier, world, dist, fp64_peak):
    """The 256 x 256 free droplet (131,072 nodes, 4 triangles per cell, jitter
    0.25h, density ratio 100, dt 0.05): FP32-deviation and FP64 steps.  Its
    solve working set fits in L2 inside a step."""
    from paper_1708_04678_gb300 import inputs as I
    w = I.free_droplet_256()
    n = len(w["mesh"]["xy"])
    out = {"workload": "free droplet 256x256 (131,072 nodes, 262,144 triangles), R 48, density ratio 100, dt 0.05"}
    for name, prec in (("fp32_dev", F.FP32_DEV), ("fp64", F.FP64)):
        r = time_precision(F, torch, w, dev, prec, K, 3, flush, barrier, world, dist, e2e=False)
        out[name] = {"value": job_rate(n, K, world, r["total_ms"]), "unit": "node-updates/s",
                     "ms_per_step": r["total_ms"] / K, "steps": K,
                     "phase_ms": {k: round(v, 5) for k, v in r["phase_ms"].items()},
                     "sweep_ms": r["phase_ms"]["solve_ms"] / r["solve_launches"], "autotune": r["tune"],
                     "finite": r["diag"]["status"] == 0}
        if prec == F.FP64:
            out[name]["fp64_roofline"] = fp64_roofline(r, n, len(w["mesh"]["tri"]), out[name]["value"] / world,
                                                       fp64_peak, recorded_fp64_flops())
    return out


def time_3d(torch, dev, K, flush):
    """The paper's own setting: D3Q19 on linear tetrahedra, the 64^3 static
    droplet (262,144 nodes, 1,572,864 tetrahedra; state and solve working
    set above L2).  FP32 deviation storage and FP64 (mixed solve): time per
    step, phases, and the roofline of the FP32 solve sweep."""
    from paper_1708_04678_gb300 import felbm as F
    from paper_1708_04678_gb300 import felbm3d as F3
    from paper_1708_04678_gb300 import inputs3d as I3
    w = I3.static_droplet_64()
    mesh = F3.Mesh3D.from_dict(w["mesh"])
    info = mesh.info()
    n = info["n_nodes"]
    out = {"workload": "static droplet 64^3 (262,144 nodes, 1,572,864 tetrahedra), D3Q19, R=16, xi=4, "
                       "density ratio 2", "nodes": n}
    for name, prec in (("fp32_dev", F.FP32_DEV), ("fp64", F.FP64)):
        stream = torch.cuda.Stream(dev)
        st = F3.State3D(mesh, F.params_derive(w["phys"], precision=prec), w["C0"], device=dev, stream=stream)
        for k in range(3):
            st.step(1)
        tot = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for k in range(K):
            with torch.cuda.stream(stream):
                flush.fill_(k & 255)
            e0.record(stream)
            st.step(1)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        phases = phase_pass(st, torch, stream, flush, min(K, 5))
        d = st.diagnostics(w["centre"], w["R"], w["phys"]["xi"], substrate=-1)
        ph = {k: statistics.mean(p[k] for p in phases) for k in phases[0]}
        r = {"ms_per_step": tot / K, "value": n * K / (tot * 1e-3), "unit": "node-updates/s",
             "phase_ms": {k: round(v, 5) for k, v in ph.items()}, "launches_per_step": st.launches(),
             "after_timed_steps": {k: d[k] for k in ("max_u", "delta_p", "mass_drift_rel", "interface_rho_uu",
                                                     "status")}}
        # end to end through host buffers, as for the 2D headline: every step
        # a pinned FP64 state in (overlapping the previous step), one step,
        # its diagnostics read back asynchronously; all finished in the region
        g0, h0 = st.get_state()
        gp = torch.from_numpy(g0).pin_memory()
        hp = torch.from_numpy(h0).pin_memory()
        slots = torch.zeros((K, F.DIAG_SLOTS), dtype=torch.float64).pin_memory()
        st.set_state(gp, hp)
        st.step(1)
        st.diagnostics_enqueue(slots[0])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(K):
            st.set_state(gp, hp)
            st.step(1)
            st.diagnostics_enqueue(slots[k])
        stream.synchronize()
        e2e = [st.diag_finish(slots[k]) for k in range(K)]
        e2e_s = time.perf_counter() - t0
        if any(x["status"] != 0 for x in e2e):
            raise RuntimeError("3D end-to-end steps produced a non-finite state")
        r["e2e"] = {"value": n * K / e2e_s, "unit": "node-updates/s", "h2d_bytes_per_step": 2 * 19 * n * 8,
                    "d2h_bytes_per_step": 8 * F.DIAG_SLOTS}
        if prec == F.FP32_DEV:
            sweeps = st.launches() - 4                       # mu, grad mu, element, rhs + the solve
            sweep_ms = ph["solve_ms"] / sweeps
            # one solve step: gathered x_k, rhs, new x (3 x 38 floats per node),
            # the mass row (column + FP32 value per entry), 1/m_i per node
            alg = n * (3 * 38 * 4 + 4) + info["nnz"] * (4 + 4)
            hbm_peak, src = peaks()
            ach = alg / (sweep_ms * 1e-3) / 1e9
            r["roofline"] = {"bound": "hbm", "kernel": "k3_sweep_rows32 (one step of the FP32 solve, 38 right-hand "
                                                       "sides, ten lanes per node)",
                             "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                             "traffic": recorded_traffic("k3_sweep_rows32", SOURCES_3D),
                             "source_hash": source_hash(SOURCES_3D), "alg_bytes_per_launch": alg,
                             "launch_ms": sweep_ms, "peak_source": src}
        out[name] = r
        st.close()
    return out


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1708_04678_gb300 import build as B
    from paper_1708_04678_gb300 import felbm as F

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    B.build()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_subprocess(args.cpu_seconds)

    def barrier():
        if world > 1:
            dist.barrier()

    w = workload()
    N = len(w["mesh"]["xy"])
    K, W = args.steps, max(args.warmup, 3)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    fp64_peak = F.fp64_fma_rate()
    with ClockSampler(local) as clk:
        r32 = time_precision(F, torch, w, dev, F.FP32_DEV, K, W, flush, barrier, world, dist)
        r64 = time_precision(F, torch, w, dev, F.FP64, K, W, flush, barrier, world, dist)
        extra = not args.no_batch
        rfd = time_free_droplet(F, torch, dev, K, flush, barrier, world, dist, fp64_peak) if extra else None
        rb = time_batch(F, torch, dev, max(10, K // 2), flush, barrier, world, dist) if extra else None
        radj = time_adjoint(F, torch, dev, max(5, K // 2)) if extra else None
        r3 = time_3d(torch, dev, max(5, K // 5), flush) if extra else None

    for name, r in (("FP32", r32), ("FP64", r64)):
        if r["diag"]["status"] != 0:
            raise SystemExit(f"bench: the {name} state is not finite after the timed steps")
    if rank == 0:
        nnz = r32["info"]["nnz"]
        # dominant kernel of the FP32-deviation step: one step of the FP32
        # solve of the 18 right-hand sides (the last one also updates the
        # fields), timed as the solve phase over its launches
        sweep_ms = r32["phase_ms"]["solve_ms"] / r32["solve_launches"]
        # algorithmic bytes of one solve step x_{k+1} = x_k + tau m^-1 (b - M x_k):
        # gathered x_k, b and the new x (3 x 18 floats per node), the mass
        # row (column index + FP32 value per entry), the inverse lumped mass
        alg_bytes = N * (3 * 18 * 4 + 4) + nnz * (4 + 4)
        hbm_peak, peak_src = peaks()
        achieved = alg_bytes / (sweep_ms * 1e-3) / 1e9
        # whole step, with the minimum bytes per node-update of the FP32 form:
        # distributions read and written (2 x 18 x 4), right-hand side written
        # and read (2 x 18 x 4), per solve step a gathered iterate, the
        # right-hand side and the new iterate (3 x 18 x 4), about 200 B of
        # nodal and element fields
        k_sweeps = r32["solve_launches"] + 1
        step_bytes = 2 * 18 * 4 + 2 * 18 * 4 + k_sweeps * 3 * 18 * 4 + 200

        def summary(r, dtype):
            return {"value": job_rate(N, K, world, r["total_ms"]), "ms_per_step": r["total_ms"] / K,
                    "dtype": dtype, "phase_ms": {k: round(v, 5) for k, v in r["phase_ms"].items()},
                    "launches_per_step": r["launches"], "autotune": r["tune"],
                    "e2e_value": job_rate(N, K, world, r["e2e_s"] * 1e3),
                    "e2e_state_out_value": job_rate(N, K, world, r["e2e_state_s"] * 1e3),
                    "after_timed_steps": {k: r["diag"][k] for k in ("max_u", "delta_p", "mass_drift_rel",
                                                                    "wetted_length", "theta_deg", "status")}}

        s32, s64 = summary(r32, "f32 (FP64 C, mu, reductions)"), summary(r64, "f64")
        s64["fp64_roofline"] = fp64_roofline(r64, N, len(w["mesh"]["tri"]), s64["value"] / world, fp64_peak,
                                             recorded_fp64_flops())
        s64["e2e"] = {"value": s64["e2e_value"], "unit": "node-updates/s", "h2d_bytes_per_step": r64["state_bytes"],
                      "d2h_bytes_per_step": 8 * F.DIAG_SLOTS}
        nominal = 8000.0
        out = {
            "metric": METRIC,
            "value": s32["value"],
            "unit": "node-updates/s",
            "n_gpus": world,
            "steps": K,
            "warmup": W,
            "ms_per_step": s32["ms_per_step"],
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": dict(workload_config(w, world), precision="FP32 deviation storage (fp32_dev); "
                           "plain FP64 in fp64", solver=f"FP32 Richardson steps at the Chebyshev roots, "
                                                         f"{r32['solve_launches'] + 1} per step"),
            "fp32_dev": s32,
            "fp64": s64,
            "free_droplet_256": rfd,
            "batched": rb,
            "adjoint": radj,
            "tetrahedra_3d": r3,
            "step_roofline": {"alg_bytes_per_node_update": step_bytes, "sweeps": k_sweeps,
                              "achieved": s32["value"] * step_bytes / 1e9, "peak": hbm_peak, "unit": "GB/s",
                              "frac": s32["value"] * step_bytes / 1e9 / hbm_peak,
                              "frac_of_nominal_8TBps": s32["value"] * step_bytes / 1e9 / nominal},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": recorded_traffic("k_sweep32"),
                         "kernel": "k_sweep32 (one step of the FP32 solve of the 18 right-hand sides)",
                         "source_hash": source_hash(),
                         "alg_bytes_per_launch": alg_bytes, "launch_ms": sweep_ms,
                         "peak_source": peak_src, "frac_of_nominal_8TBps": achieved / nominal},
            "e2e": {"value": s32["e2e_value"], "unit": "node-updates/s",
                    "h2d_bytes_per_step": r32["state_bytes"], "d2h_bytes_per_step": 8 * F.DIAG_SLOTS},
            "e2e_state_out": {"value": s32["e2e_state_out_value"], "unit": "node-updates/s",
                              "h2d_bytes_per_step": r32["state_bytes"], "d2h_bytes_per_step": r32["state_bytes"]},
            "gpu_launches": r32["launches"] * K,
            "clocks": clk.summary(),
        }
        if cpu is not None:
            out["cpu_baseline"] = cpu
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    budget = 120.0
    warm = min(args.warmup, 1)
    procs = host_procs()
    v, n, secs = run_oracle_all_cores(budget, args.steps, warm, procs)
    why = "the requested steps" if n >= args.steps else f"the first step past {budget:.0f} s"
    sample = (f"{n} steps (after {warm} warm-up) of {procs} copies of the 128-column strip of the rough-wall "
              f"droplet (130,176 nodes each, the same rows, wall, jitter and physics), one single-threaded "
              f"process per host core in lock step, in {secs:.1f} s (stopped after {why}); FP64 numpy/scipy "
              f"oracle")
    out = {"metric": METRIC, "value": v, "unit": "node-updates/s", "n_gpus": world, "steps": n,
           "warmup": warm, "ms_per_step": secs * 1e3 / n, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(workload(), world),
           "impl": "reference",
           "cpu_baseline": {"value": v, "unit": "node-updates/s", "cores": procs, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": "node-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def ncu_case(args):
    """Two steps of the 1024-column rough-wall droplet in one precision, with
    a fixed solve split (no autotuning, so the launches are the step's)."""
    import torch
    from paper_1708_04678_gb300 import build as B
    B.build()
    from paper_1708_04678_gb300 import felbm as F
    from paper_1708_04678_gb300 import inputs as I
    w = I.rough_wall_droplet(width=1024, R=150.0)
    prec = F.FP64 if args.ncu_case == "fp64" else F.FP32_DEV
    st = F.State(F.Mesh.from_dict(w["mesh"]), F.params_derive(w["phys"], precision=prec), w["C0"], device="cuda:0")
    st.sweep_parts(args.sweep_parts)
    if args.ncu_case == "fp32-tiled":
        st.sweep_tiled(True)
    st.step(2)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": args.ncu_case, "nodes": len(w["mesh"]["xy"]), "status": st.diagnostics()["status"]}))


def main():
    args = parse()
    if args.ncu_case:
        ncu_case(args)
        return
    if args.cpu_baseline_only:
        v1, n1, s1 = run_oracle(args.cpu_seconds * 0.5, 10 ** 6, 1)
        procs = host_procs()
        v, n, secs = run_oracle_all_cores(args.cpu_seconds, 10 ** 6, 1, procs)
        print(json.dumps({"value": v, "unit": "node-updates/s", "cores": procs, "kind": "oracle",
                          "sample": f"{procs} single-threaded processes, one per host core, each stepping its "
                                    f"own copy of the 128-column strip of the rough-wall droplet (130,176 nodes, "
                                    f"the same rows, wall, jitter and physics) in lock step: {n} steps after 1 "
                                    f"warm-up, {secs:.1f} s; FP64 numpy/scipy oracle",
                          "single_core": {"value": v1, "steps": n1, "seconds": round(s1, 2)}}))
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.only_3d:
        import torch
        from paper_1708_04678_gb300 import build as B
        B.build()
        dev = torch.device("cuda", 0)
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        with ClockSampler(0) as clk:
            r3 = time_3d(torch, dev, args.steps, flush)
        print(json.dumps({"tetrahedra_3d": r3, "clocks": clk.summary()}), flush=True)
        return
    run_gpu(args)


if __name__ == "__main__":
    main()
