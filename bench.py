"""Benchmark of the particle hot path: RK4 particle-steps/s for
advect + locate + rebin on a 3D Q2 mesh, with its HBM roofline fraction.

Workload (default, c3): 3D unit cube, 128^3 hexes with interior vertices
jittered by up to 0.1 h, Q2 velocity = curl of 8 random-phase sinusoidal
vector potentials (zero wall-normal flow), 20 particles per cell
(41,943,040), three FP64 properties, RK4 at CFL 0.5.  One benchmark step =
one time step of every particle (advect with located stages, final locate,
rebin into the (cell, id)-sorted store).  The particle state (~3.5 GB) is
far larger than L2, so no L2 flush is needed between steps.  `value` is the
FP64 form (double-float arithmetic, FP64 storage); the same line carries the
FP32-basis form's rate on the same workload and its position and cell-average
error against the FP64 form over the configuration's 20 steps, measured on
every particle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config c3|c2|c1|c4|c5|c2p|next]

c2 is the 64^3 FP64 workload; c4 times the adjoint (recorded forward +
reverse sweep) at 32^3 x 32 per cell over 20 steps; c5 times the 64-problem
ensemble (10 steps per persistent graph launch); c2p times c2 with the damage
and deformation-gradient ODEs; next times the rows after the hot path (time
interpolation, property ODEs, transfers, generation) on the c2 workload.

Under torchrun (N > 1) the c2 and c3 mesh is split over the ranks in slabs
of cell layers: each rank advances the particles of its layers and hands
those that leave to its neighbours (NCCL point-to-point; strong scaling);
--partition replicas runs N independent copies instead (weak scaling).  The
64 members of c5 are dealt out to the ranks by particle count (strong
scaling).  The time is the maximum over ranks.  --impl reference times the CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1612_03369_gb300 import workloads as W  # noqa: E402
from paper_1612_03369_gb300 import shard  # noqa: E402

# Algorithmic bytes per particle-step (the method's data movement): each
# particle's state (x, x-hat, u64 id, P properties) read once and written
# once, the new-cell key written and read, and the cell data (8 unique Q2
# nodes x 3 components + one vertex, and a u32 offset) amortised over the
# particles per cell.  The FP32-basis form counts x-hat and the DOFs as FP32.
def step_bytes(dim: int, n_props: int, ppc: float, xhat_bytes: int = 8, dof_bytes: int = 8) -> float:
    state = dim * 8 + dim * xhat_bytes + 8 + n_props * 8
    cell_data = ((2 ** dim) * dim * dof_bytes + dim * 8 + 4) / ppc
    return 2 * state + 8 + cell_data


# The advect kernel's share: it reads x, x-hat, cell, id and the properties and
# writes them in the new order with the new cell; cell data amortised.
def advect_bytes(dim: int, ppc: float, n_props: int, xhat_bytes: int = 8, dof_bytes: int = 8) -> float:
    return 2 * (dim * 8 + dim * xhat_bytes + 4 + 8 + n_props * 8) + ((2 ** dim) * dim * dof_bytes + dim * 8) / ppc


# DRAM bytes (read + write) per particle of one launch of the advect kernel,
# from an ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the
# current kernel on the 64^3 x 20 workload, RK4, in the middle of a
# multi-step call; traffic grows with the particle count, so a launch at
# another size is scaled by its particles.  Keyed by precision (0 FP64
# form, 1 FP32-basis form).
ADVECT_DRAM_BYTES_PER_PARTICLE = {0: 1342.109e6 / 5242880, 1: 1017.072e6 / 5242880}
# Warp instructions per 32 particle-steps and pipe utilisation of the same
# captures: the advect kernel is bound by instruction issue (double-float
# arithmetic on the FP32 pipe) in the FP64 form, and by issue and load
# latency in the FP32-basis form, not by HBM.
ADVECT_ISSUE = {
    0: {"warp_instructions_per_32_particle_steps": 10758, "issue_active_pct": 76.3, "fma_pipe_active_pct": 61.2,
        "top_stall": "not_selected 3.12 per issue (issue-bound)"},
    1: {"warp_instructions_per_32_particle_steps": 4343, "issue_active_pct": 64.5, "fma_pipe_active_pct": 41.1,
        "top_stall": "long_scoreboard 3.83 per issue"},
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def workload(name: str, n: int | None = None):
    """The named workload; n overrides the cells per axis (for profiling a
    kernel at a size ncu can capture), and the result is then no bench line
    of the named configuration."""
    if name == "c1":
        return W.c1() if n is None else W.c1(n=n)
    if name == "c3":
        wl = W.c3() if n is None else W.c3(n=n)
        wl.name = "c3_3d_curl_%d^3" % wl.n[0]
        return wl
    return W.c2() if n is None else W.c2(n=n)


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,clocks.mem,clocks.max.mem")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        """Start sampling every 50 ms and return once the first sample is in
        (nvidia-smi takes a moment to start), so that the samples cover the
        timed region that follows."""
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 10.0 and self.proc.poll() is None:
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.02)
            self.skip = sum(1 for _ in open(self.path))  # samples from before the timed region
        except Exception:
            self.proc = None

    def stop(self):
        """Samples from the last one before the timed region to the first
        one after it (a region shorter than the sampling period still gets
        the two that bracket it)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        t0 = time.time()
        while time.time() - t0 < 1.0 and self.proc.poll() is None:
            if sum(1 for _ in open(self.path)) > getattr(self, "skip", 0):
                break
            time.sleep(0.01)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, mem, mmax, reasons = [], [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in list(open(self.path))[max(getattr(self, "skip", 0) - 1, 0):]:
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            try:
                mem.append(float(f[9]))
                mmax.append(float(f[10]))
            except (ValueError, IndexError):
                pass
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "mem_mhz": statistics.median(mem) if mem else None, "mem_max_mhz": max(mmax) if mmax else None}


def _seed(P, mesh, wl):
    parts = P.Particles(mesh, uniform_count=wl.ppc, seed=wl.pseed, n_props=wl.n_props)
    st = parts.export()
    for q in range(min(wl.n_props, wl.dim)):
        parts.set_property(q, st["x"][q].contiguous())  # property q = initial coordinate q
    del st
    return parts


def _timed_advect(P, parts, wl, precision, steps, warmup, stream, barrier, clocks=None):
    """warmup untimed steps, then `steps` steps between CUDA events on the
    stream, with the library's per-step advect / rebin events on.  Returns
    (ms, advect ms per step, rebin ms per step, particle-steps, counter
    deltas, clock record or None)."""
    import torch

    parts.advect(wl.dt, wl.integrator, warmup, precision)
    torch.cuda.synchronize()
    c0 = parts.stats()
    P.pic_timing_enable(parts.h, True)
    if clocks is not None:
        clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    parts.advect(wl.dt, wl.integrator, steps, precision)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if clocks is not None else None
    P.pic_timing_enable(parts.h, False)
    adv, reb, nsteps = P.pic_timing_read(parts.h)
    c1 = parts.stats()
    d = {k: c1[k] - c0[k] for k in c1}
    return e0.elapsed_time(e1), adv / max(nsteps, 1), reb / max(nsteps, 1), d["particle_steps"], d, clk


def _accuracy_fp32_basis(P, mesh, wl, form=None):
    """Both forms from the same seeded store over the configuration's steps;
    every particle compared by id, and the per-cell averages of property 0.
    The FP64 form is the reference here: it matches the CPU oracle to 1e-12
    in positions and cell averages (the parity tests), far below the FP32
    basis's error.  form: PIC_FP32_BASIS (default) or
    PIC_FP32_BASIS_STAGE_DF."""
    import torch

    out = {}
    runs = []
    for prec in (P.PIC_FP64, P.PIC_FP32_BASIS if form is None else form):
        parts = _seed(P, mesh, wl)
        parts.advect(wl.dt, wl.integrator, wl.n_steps, prec)
        e = parts.export()
        avg, cnt = parts.average(0)
        runs.append((e["x"], e["id"], avg, cnt))
        del e
        parts.close()
    (x64, id64, a64, c64), (x32, id32, a32, c32) = runs
    N0 = wl.n_particles
    pos = torch.full((N0,), -1, dtype=torch.int64, device=x64.device)
    pos[id32 - wl.first_id] = torch.arange(id32.numel(), device=x64.device)
    p32 = pos[id64 - wl.first_id]
    both = p32 >= 0
    dx = (x64[:, both] - x32[:, p32[both]]).abs().amax(dim=0)
    diff_cells = (a64 != a32) | (c64 != c32)
    out.update({
        "reference": "the FP64 form on the GPU (itself within 1e-12 of the CPU oracle in the parity tests)",
        "steps": wl.n_steps, "particles_compared": int(both.sum()),
        "lost_fp64_form": int(N0 - id64.numel()), "lost_fp32_basis_form": int(N0 - id32.numel()),
        "max_position_error": float(dx.max()), "rms_position_error": float(dx.pow(2).mean().sqrt()),
        "cells_with_different_average": int(diff_cells.sum()),
        "max_cell_average_error": float((a64 - a32).abs().max()),
        "cells_with_different_count": int((c64 != c32).sum()),
    })
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1612_03369_gb300 import pic as P

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    wl = workload(args.config, args.mesh)
    precision = P.PIC_FP64
    mesh = P.Mesh(wl.n, wl.X, wl.U)
    parts = _seed(P, mesh, wl)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    launches0 = P.pic_kernel_launches()
    ms, adv_avg_ms, reb_avg_ms, psteps, cdelta, clk = _timed_advect(
        P, parts, wl, precision, args.steps, args.warmup, stream, barrier, ClockSampler(local_rank))
    launches = P.pic_kernel_launches() - launches0
    n1, nlost, status = parts.state()

    # ---- the other particle -> field transfers (Sec. 2.7), timed on their
    # own after the step loop: the cell averages (ii), shape-function-weighted
    # vertex averages (iv) and the per-cell linear least squares (v) of
    # property 0
    xfer = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, fn in (("cell_average_ms", lambda: parts.average(0)),
                     ("vertex_average_ms", lambda: parts.vertex_average(0)),
                     ("project_linear_ms", lambda: parts.project_linear(0))):
        for _ in range(3):
            fn()
        e0.record(stream)
        for _ in range(10):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        xfer[name] = e0.elapsed_time(e1) / 10

    # ---- end to end through the C ABI with host buffers: every step copies
    # the step's velocity DOFs host->device (a flow solver hands over a new
    # field each step), advances one step, averages the properties per cell
    # and reads the averages back to the host.
    Uh = torch.from_numpy(np.ascontiguousarray(wl.U)).pin_memory()
    avg_d = torch.empty((max(wl.n_props, 1), wl.ncells), dtype=torch.float64, device=dev)
    cnt_d = torch.empty(wl.ncells, dtype=torch.int32, device=dev)
    avg_h = torch.empty((max(wl.n_props, 1), wl.ncells), dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 20))

    def step_tail():
        P.pic_advect(parts.h, mesh.h, wl.dt, wl.integrator, precision, 1)
        for q in range(wl.n_props):
            P.pic_interpolate_to_cells(parts.h, mesh.h, q, avg_d[q], cnt_d if q == 0 else None)
        avg_h.copy_(avg_d, non_blocking=True)

    # serial: each step uploads its field, then advances (the copy waits for
    # the previous step)
    stats_e0 = parts.stats()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        P.pic_set_velocity_dofs(mesh.h, Uh)  # host pointer: H2D copy inside the library call
        step_tail()
        stream.synchronize()
    barrier()
    e2e_serial_s = time.perf_counter() - t0
    e2e_serial_psteps = parts.stats()["particle_steps"] - stats_e0["particle_steps"]
    # pipelined: the next step's field is staged on a copy stream while the
    # current step runs, then committed (one upload per step either way); the
    # averages go to one of two device buffers and are read back on a second
    # copy stream while the next step runs, into one of two pinned host
    # buffers, which the host reads one step later
    copy_stream, d2h_stream = torch.cuda.Stream(), torch.cuda.Stream()
    avg_db = [avg_d, torch.empty_like(avg_d)]
    avg_hb = [avg_h, torch.empty_like(avg_h).pin_memory()]
    ready = [torch.cuda.Event(), torch.cuda.Event()]  # averages of step n computed (compute stream)
    done = [torch.cuda.Event(), torch.cuda.Event()]  # averages of step n on the host (copy stream)
    checks = []
    stats_e0 = parts.stats()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    P.pic_stage_velocity_dofs(mesh.h, Uh, copy_stream)
    P.pic_commit_velocity_dofs(mesh.h, stream)
    for n in range(e2e_steps):
        b = n % 2
        P.pic_advect(parts.h, mesh.h, wl.dt, wl.integrator, precision, 1)
        if n >= 2:
            stream.wait_event(done[b])  # step n - 2's read-back of this buffer has finished
        for q in range(wl.n_props):
            P.pic_interpolate_to_cells(parts.h, mesh.h, q, avg_db[b][q], cnt_d if q == 0 else None)
        ready[b].record(stream)
        d2h_stream.wait_event(ready[b])
        with torch.cuda.stream(d2h_stream):
            avg_hb[b].copy_(avg_db[b], non_blocking=True)
        done[b].record(d2h_stream)
        if n + 1 < e2e_steps:
            P.pic_stage_velocity_dofs(mesh.h, Uh, copy_stream)
            P.pic_commit_velocity_dofs(mesh.h, stream)
        if n >= 1:
            done[1 - b].synchronize()  # step n - 1's averages are on the host
            checks.append(float(avg_hb[1 - b][0, 0]))
    done[(e2e_steps - 1) % 2].synchronize()
    checks.append(float(avg_hb[(e2e_steps - 1) % 2][0, 0]))
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_psteps = parts.stats()["particle_steps"] - stats_e0["particle_steps"]
    torch.cuda.synchronize()
    assert len(checks) == e2e_steps

    # ---- the FP32-basis form (precision form) on the same workload, its own
    # store; and its error against the FP64 form over the configuration's steps
    # (after the end-to-end steps: from its first use on, every field update
    # also builds the FP32 coefficient table)
    fp32 = None
    if args.config == "c3":
        p32 = _seed(P, mesh, wl)
        ms32, adv32, reb32, ps32, cd32, _ = _timed_advect(P, p32, wl, P.PIC_FP32_BASIS, args.steps, args.warmup,
                                                         stream, barrier)
        p32.close()
        fp32 = {"value": ps32 / (ms32 / 1e3), "unit": "particle-steps/s", "ms_per_step": ms32 / args.steps,
                "advect_ms_per_step": adv32, "rebin_ms_per_step": reb32,
                "algorithmic_bytes_per_particle_step": step_bytes(wl.dim, wl.n_props, wl.ppc, 4, 4),
                "newton_iterations_per_particle_step": cd32["newton_iterations"] / max(ps32, 1),
                "full_path_particle_steps": cd32["deferred"]}
        hbm, _ = load_peaks()
        fp32["step_fraction_of_hbm_roofline"] = (fp32["value"] * fp32["algorithmic_bytes_per_particle_step"] / 1e9
                                                 / hbm)
        ab32 = advect_bytes(wl.dim, wl.ppc, wl.n_props, 4, 4)
        fp32["roofline"] = roofline_object(1, adv32, ps32 / args.steps, ab32, hbm)
        if not args.no_accuracy:
            fp32["accuracy"] = _accuracy_fp32_basis(P, mesh, wl)
        # the strict reading: the double-float Newton residual step at the
        # stage points too (PIC_FP32_BASIS_STAGE_DF)
        p32 = _seed(P, mesh, wl)
        msd, advd, rebd, psd, cdd, _ = _timed_advect(P, p32, wl, P.PIC_FP32_BASIS_STAGE_DF, args.steps,
                                                      args.warmup, stream, barrier)
        p32.close()
        roof_d = roofline_object(1, advd, psd / args.steps, ab32, hbm)
        roof_d.update({"kernel": "advect_kernel<3,RK4> (FP32-basis form, double-float stage residuals)",
                       "traffic": None, "traffic_source": "not captured for this variant"})
        roof_d.pop("issue_view", None)
        fp32["stage_residuals_double_float"] = {
            "value": psd / (msd / 1e3), "unit": "particle-steps/s", "ms_per_step": msd / args.steps,
            "advect_ms_per_step": advd, "roofline": roof_d,
            "newton_iterations_per_particle_step": cdd["newton_iterations"] / max(psd, 1),
            "what": "the FP32-basis form with the double-float Newton residual and convergence test at every "
                    "stage point, not only at the new position"}
        if not args.no_accuracy:
            fp32["stage_residuals_double_float"]["accuracy"] = _accuracy_fp32_basis(
                P, mesh, wl, P.PIC_FP32_BASIS_STAGE_DF)

    (tmax, e2e_s, e2e_serial_s), (psteps_all, e2e_all, e2e_serial_all) = shard.reduce_timing(
        [ms, e2e_s, e2e_serial_s], [psteps, e2e_psteps, e2e_serial_psteps], device=dev if world > 1 else None)

    hbm, peak_kind = load_peaks()
    value = psteps_all / (tmax / 1e3)
    sbytes = step_bytes(wl.dim, wl.n_props, wl.ppc)
    ab = advect_bytes(wl.dim, wl.ppc, wl.n_props)
    res = {
        "metric": "RK4 particle-steps/s (advect+locate+rebin), 3D Q2 mesh; % of HBM roofline",
        "value": value,
        "unit": "particle-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tmax / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64 storage / df64 arithmetic (double-float on the FP32 pipe, ~2^-48)",
        "data": "synthetic (seeded jittered mesh, curl-of-potential Q2 field, local-coordinate seeding)",
        "config": {"workload": wl.name, "mesh": "x".join(str(v) for v in wl.n), "particles": wl.n_particles,
                   "particles_per_cell": wl.ppc, "n_props": wl.n_props, "integrator": "RK4" if wl.integrator == 4 else
                   ("RK2" if wl.integrator == 2 else "Euler"), "dt": wl.dt, "cfl": 0.5, "form": "FP64",
                   "l2": "state ~%.0f MB > 129 MB L2, no flush" % (wl.n_particles * sbytes / 2 / 1e6),
                   "parallelism": "replicas x%d" % world if world > 1 else "single GPU"},
        "step_fraction_of_hbm_roofline": (value * sbytes / 1e9) / hbm,
        "step_algorithmic_bytes_per_particle_step": sbytes,
        "roofline": roofline_object(0, adv_avg_ms, psteps / args.steps, ab, hbm, peak_kind, reb_avg_ms),
        "fp32_basis_form": fp32,
        "transfers_one_property": xfer,
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": {"value": e2e_all / e2e_s, "unit": "particle-steps/s",
                "h2d_bytes_per_step": int(wl.U.nbytes),
                "d2h_bytes_per_step": int(wl.n_props * wl.ncells * 8), "steps": e2e_steps,
                "what": "per step: velocity DOFs H2D from pinned host memory (staged on a copy stream during the "
                        "previous step, then committed) + pic_advect 1 step + per-cell averages of all properties "
                        "+ D2H of the averages on a second copy stream into one of two pinned buffers; the host "
                        "reads step n's averages while step n+1 runs, and the last step's before the clock stops",
                "serial_value": e2e_serial_all / e2e_serial_s,
                "serial_what": "the same with the upload issued on the compute stream before each step"},
        "state": {"alive": n1, "lost_total": nlost, "status_word": status,
                  "walks": cdelta["walks"], "global_searches": cdelta["global_searches"],
                  "fp64_fallback_particle_steps": cdelta["fallback64"],
                  "fp64_walk_particle_steps": cdelta["walk64"],
                  "full_path_particle_steps": cdelta["deferred"],
                  "newton_iterations_per_particle_step": cdelta["newton_iterations"] / max(psteps, 1)},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(wl, seconds=args.cpu_seconds)
        res["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(wl, seconds=min(args.cpu_seconds, 10.0))
    parts.close()
    mesh.close()
    return res


def run_slab(args, rank, world, local_rank):
    """One mesh split over the ranks in slabs of cell layers (parallel
    transport, Sec. 2.4): every rank seeds and advances the particles of its
    own layers on a sub-mesh with two halo layers, then hands the particles
    that left its layers to its neighbours (NCCL point-to-point, counts then
    payload) and merges what it receives.  The total work is fixed: strong
    scaling.  A rank's particles are seeded with its own generator stream
    (first id = the rank's global offset), the same distribution as the
    single store's."""
    import torch
    import torch.distributed as dist
    from paper_1612_03369_gb300 import pic as P
    from paper_1612_03369_gb300 import slab

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    wl = workload(args.config, args.mesh)
    s = slab.make_slab(wl.n, rank, world, halo=2)
    mesh = P.Mesh(s.local_n, slab.slice_vertices(wl.X, s), slab.slice_nodes(wl.U, s))
    own = wl.ppc * s.owned_cells
    parts = P.Particles(mesh, per_cell=slab.owned_per_cell(s, wl.ppc), seed=wl.pseed + rank,
                        first_id=slab.first_id(s, wl.ppc), n_props=wl.n_props, capacity=int(own * 1.25) + 4096)
    st = parts.export()
    for q in range(min(wl.n_props, wl.dim)):
        parts.set_property(q, st["x"][q].contiguous())
    del st
    stream = torch.cuda.current_stream()
    moved = [0, 0]

    def step():
        parts.advect(wl.dt, wl.integrator, 1)
        d, u = slab.exchange_step(parts, s, dev)
        moved[0] += d
        moved[1] += u

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    c0 = parts.stats()
    def barrier():
        if world > 1:
            dist.barrier()

    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    moved[:] = [0, 0]
    launches0 = P.pic_kernel_launches()
    P.pic_timing_enable(parts.h, True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    P.pic_timing_enable(parts.h, False)
    adv, reb, nst = P.pic_timing_read(parts.h)
    ms = e0.elapsed_time(e1)
    launches = P.pic_kernel_launches() - launches0
    psteps = parts.stats()["particle_steps"] - c0["particle_steps"]

    # end to end: every step uploads the rank's slice of the field from
    # pinned host memory, steps, exchanges, and reads the averages of its own
    # cells back
    Uh = torch.from_numpy(slab.slice_nodes(wl.U, s)).pin_memory()
    avg_h = torch.empty(s.owned_cells, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 10))
    ce = parts.stats()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        P.pic_set_velocity_dofs(mesh.h, Uh)
        step()
        a, _ = parts.average(0)
        avg_h.copy_(a[s.own_lo: s.own_hi])
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_psteps = parts.stats()["particle_steps"] - ce["particle_steps"]
    (tmax, e2e_s), (psteps_all, e2e_all, mv_d, mv_u) = shard.reduce_timing(
        [ms, e2e_s], [psteps, e2e_psteps, moved[0], moved[1]], device=dev if world > 1 else None)
    hbm, peak_kind = load_peaks()
    value = psteps_all / (tmax / 1e3)
    sbytes = step_bytes(wl.dim, wl.n_props, wl.ppc)
    res = {
        "metric": "RK4 particle-steps/s (advect+locate+rebin), 3D Q2 mesh; % of HBM roofline",
        "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f64 storage / df64 arithmetic (double-float on the FP32 pipe, ~2^-48)",
        "data": "synthetic (seeded jittered mesh, curl-of-potential Q2 field, local-coordinate seeding per rank)",
        "config": {"workload": wl.name, "mesh": "x".join(str(v) for v in wl.n), "particles": wl.n_particles,
                   "particles_per_cell": wl.ppc, "n_props": wl.n_props, "integrator": "RK4", "dt": wl.dt, "cfl": 0.5,
                   "form": "FP64", "parallelism": "slab x%d (cell layers along z, 2 halo layers, NCCL exchange of "
                                                   "the particles that leave a slab, with their cells)" % world,
                   "l2": "state > 129 MB L2 per rank, no flush"},
        "step_fraction_of_hbm_roofline": (value / world * sbytes / 1e9) / hbm,
        "exchanged_particles_per_step": (mv_d + mv_u) / args.steps,
        "roofline": roofline_object(0, adv / max(nst, 1), psteps / args.steps, advect_bytes(wl.dim, wl.ppc, wl.n_props),
                                    hbm, peak_kind, reb / max(nst, 1)),
        "roofline_scope": "rank 0's advect kernel on its slab (each rank runs the same kernel on its own slab)",
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": {"value": e2e_all / e2e_s, "unit": "particle-steps/s",
                "h2d_bytes_per_step": int(Uh.numel() * 8) * world, "d2h_bytes_per_step": int(wl.ncells * 8),
                "steps": e2e_steps,
                "what": "per step and rank: the rank's field slice H2D from pinned memory, one step with the "
                        "exchange, the averages of its own cells D2H"},
    }
    parts.close()
    mesh.close()
    return res


# FP32 peak derived from unit counts and the maximum SM clock: 152 SMs x 128
# FP32 lanes x 2 flops (FMA) x 2.07 GHz (the ALU bound of the double-float
# kernels below).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12

# FP32 flops (FADD + FMUL + 2 FFMA) per reverse step of the 32^3 x 32 adjoint
# (1,048,576 particles, RK4), counted by an ncu capture of these kernels:
# reverse_lambda_kernel (G and lambda at 4.19M stage points, double-float)
# and cell_partial_kernel (the per-cell sums, double-float).
ADJOINT_C4_FP32_FLOPS_PER_REVERSE_STEP = 1.572e10 + 6.538e9
# DRAM bytes (read + write) of the same two kernels per reverse step, same capture.
ADJOINT_C4_DRAM_BYTES_PER_REVERSE_STEP = (204.5e6 + 148.8e6) + (220.1e6 + 15.9e6)


def run_adjoint(args):
    """c4: the adjoint (pic_advect_record + pic_tape_adjoint) against the
    plain FP64-form forward of the same run, on one GPU."""
    import torch
    from paper_1612_03369_gb300 import pic as P

    wl = W.c4()
    steps = wl.n_steps
    mesh = P.Mesh(wl.n, wl.X, wl.U)
    N = wl.n_particles

    def fresh():
        return P.Particles(mesh, uniform_count=wl.ppc, seed=wl.pseed)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def gradient(kind):
        # recorded forward, then the reverse sweep: (record ms, reverse ms)
        p = fresh()
        torch.cuda.synchronize()
        e0.record()
        tape = P.pic_advect_record_tape(p.h, mesh.h, wl.dt, 4, steps, kind)
        e1.record()
        torch.cuda.synchronize()
        r = e0.elapsed_time(e1)
        st = p.export()
        lam = 2.0 * (st["x"] - 0.5).contiguous()
        dU = torch.empty((3, wl.U.shape[1]), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        e0.record()
        P.pic_tape_adjoint(tape, lam, dU)
        e1.record()
        torch.cuda.synchronize()
        a = e0.elapsed_time(e1)
        P.pic_destroy_tape(tape)
        p.close()
        return r, a

    fwd_ms, adj_ms, rec_ms = [], [], []
    for rep in range(args.warmup + args.steps):
        p = fresh()
        torch.cuda.synchronize()
        e0.record()
        p.advect(wl.dt, 4, steps)
        e1.record()
        torch.cuda.synchronize()
        f = e0.elapsed_time(e1)
        p.close()
        r, a = gradient(P.PIC_TAPE_STAGES)
        if rep >= args.warmup:
            fwd_ms.append(f)
            rec_ms.append(r)
            adj_ms.append(a)
    f, r, a = statistics.median(fwd_ms), statistics.median(rec_ms), statistics.median(adj_ms)
    rev_tf = ADJOINT_C4_FP32_FLOPS_PER_REVERSE_STEP * steps / (a / 1e3) / 1e12
    # the same gradient through a checkpoint tape (about half the memory)
    ck = [gradient(P.PIC_TAPE_CHECKPOINTS) for _ in range(1 + max(1, args.steps))][1:]
    ck_r, ck_a = statistics.median(c[0] for c in ck), statistics.median(c[1] for c in ck)
    psteps = N * steps
    return {
        "metric": "adjoint particle-steps/s (recorded forward + reverse sweep), 3D Q2 mesh",
        "value": psteps / ((r + a) / 1e3), "unit": "particle-steps/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": (r + a), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "particles": N, "time_steps": steps, "integrator": "RK4",
                   "one_benchmark_step": "one full gradient: %d recorded steps + reverse sweep" % steps},
        "forward_plain_ms": f, "record_ms": r, "reverse_ms": a,
        "roofline": {"kernel": "reverse sweep: reverse_lambda_kernel<3,4> + cell_partial_kernel<3> (with the record "
                               "sort and node sums in the time)", "bound": "alu", "achieved": rev_tf,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": rev_tf / FP32_PEAK_TFLOPS,
                     "fp32_flops_per_reverse_step": ADJOINT_C4_FP32_FLOPS_PER_REVERSE_STEP,
                     "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz",
                     "traffic": ADJOINT_C4_DRAM_BYTES_PER_REVERSE_STEP, "traffic_per": "reverse step, both kernels"},
        "forward_plain_particle_steps_per_s": psteps / (f / 1e3),
        "tape": "stage records (116 B per particle-step)",
        "checkpoint_tape": {"record_ms": ck_r, "reverse_ms": ck_a, "gradient_ms": ck_r + ck_a,
                            "particle_steps_per_s": psteps / ((ck_r + ck_a) / 1e3),
                            "bytes_per_particle_step": 56},
        "accuracy": "dL/dU within 1e-12 of max|dL/dU| of the oracle's reverse mode (tests/test_gpu_adjoint.py)",
    }


def run_ensemble(args, rank=0, world=1, local_rank=0):
    """c5: 64 problems advanced 10 steps per launch of the persistent kernel
    (replayed graph), against the per-step graph and against the problems
    advanced one after another with pic_advect.  Under torchrun the members
    are dealt out to the ranks by particle count (no collective on the data
    path; the total work is fixed, so the scaling is strong)."""
    import torch
    from paper_1612_03369_gb300 import pic as P

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    wls_all = W.c5()
    mine = shard.partition_by_weight([w.n_particles for w in wls_all], world)[rank]
    wls = [wls_all[i] for i in mine]
    steps = wls_all[0].n_steps
    if not wls:  # more ranks than members: this rank idles through the protocol
        shard.reduce_timing([0.0, 0.0, 0.0], [0.0], device=dev if world > 1 else None)
        return None
    meshes = [P.Mesh(w.n, w.X, w.U) for w in wls]
    ens = P.Ensemble(meshes, per_cell=[w.per_cell for w in wls], seeds=[w.pseed for w in wls])
    ens.set_dt([w.dt for w in wls])
    tuned = ens.tune(4)
    N = sum(w.n_particles for w in wls)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(mode):
        for _ in range(args.warmup):
            ens.run(4, steps, mode=mode, use_graph=True)
        torch.cuda.synchronize()
        n0 = ens.state()[0]
        e0.record()
        for _ in range(args.steps):
            ens.run(4, steps, mode=mode, use_graph=True)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps, n0

    persist_ms, n_alive = timed(1)
    multi_ms, _ = timed(0)
    # plain: the problems one after another
    solos = [P.Particles(m, per_cell=w.per_cell, seed=w.pseed) for m, w in zip(meshes, wls)]
    for _ in range(args.warmup):
        for p, w in zip(solos, wls):
            p.advect(w.dt, 4, steps)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        for p, w in zip(solos, wls):
            p.advect(w.dt, 4, steps)
    e1.record()
    torch.cuda.synchronize()
    solo_ms = e0.elapsed_time(e1) / args.steps
    (persist_ms, multi_ms, solo_ms), (n_alive,) = shard.reduce_timing([persist_ms, multi_ms, solo_ms], [n_alive],
                                                                      device=dev if world > 1 else None)
    return {
        "metric": "ensemble RK4 particle-steps/s (advect+locate+rebin), 64 2D Q2 problems, one persistent launch",
        "value": n_alive * steps / (persist_ms / 1e3), "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": persist_ms, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "c5_ensemble_64", "problems": len(wls_all),
                   "particles": sum(w.n_particles for w in wls_all),
                   "sides": [w.n[0] for w in wls_all], "time_steps_per_launch": steps,
                   "one_benchmark_step": "%d time steps of every problem" % steps,
                   "parallelism": ("members dealt to %d ranks by particle count" % world) if world > 1
                   else "single GPU"},
        "autotuned_rank0": {"blocks_per_sm": tuned[0], "tile": tuned[1], "one_step_ms": tuned[2]},
        "per_step_graph_particle_steps_per_s": n_alive * steps / (multi_ms / 1e3),
        "sequential_solo_particle_steps_per_s": n_alive * steps / (solo_ms / 1e3),
    }


def run_props(args):
    """c2 with the Sec. 2.6 property ODEs: every step also integrates the
    damage variable and the 3x3 deformation gradient (double-float velocity
    gradient at every stage) on top of advect+locate+rebin."""
    import torch
    from paper_1612_03369_gb300 import pic as P

    wl = W.c2()
    mesh = P.Mesh(wl.n, wl.X, wl.U)
    n_props = 3 + 1 + 9
    parts = P.Particles(mesh, uniform_count=wl.ppc, seed=wl.pseed, n_props=n_props)
    N = parts.state()[0]
    st = parts.export()
    for q in range(3):
        parts.set_property(q, st["x"][q].contiguous())
    del st
    eye = np.eye(3).reshape(-1)
    for q in range(9):
        parts.set_property(4 + q, torch.full((N,), float(eye[q]), dtype=torch.float64, device="cuda"))
    odes = dict(damage=3, alpha=1.0, beta=0.5, deformation=4)
    parts.advect_properties(wl.dt, wl.integrator, args.warmup, **odes)
    torch.cuda.synchronize()
    s0 = parts.stats()["particle_steps"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    parts.advect_properties(wl.dt, wl.integrator, args.steps, **odes)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ps = parts.stats()["particle_steps"] - s0
    return {
        "metric": "RK4 particle-steps/s with damage + deformation-gradient ODEs (advect+ODEs+locate+rebin), 3D Q2",
        "value": ps / (ms / 1e3), "unit": "particle-steps/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "c2_props_64^3", "particles": N, "n_props": n_props,
                   "odes": "damage (slot 3), F row-major (slots 4-12)"},
    }


# FP32 flops (FADD + FMUL + 2 FFMA) per particle-step of the property-ODE
# work beyond the plain step: the stage-gradient kernel (13,768) and the ODE
# kernel (4,480), both in double-float, counted by ncu on the 64^3 x 20
# workload (an ncu capture of these kernels).
PROPS_ODE_FP32_FLOPS_PER_PARTICLE_STEP = 18248.0

# FP64 operations per unit of the FP64-bound kernels (dadd + dmul + 2 dfma,
# counted by an ncu capture on the 64^3 x 20 workload).
FP64_FLOPS = {
    "mh_seed_kernel<3>": 238.96,           # per chain step
    "cell_weights_kernel<3>": 1815.0,      # per cell
}
# FP64 peak: the GB300's nominal FP64 rate, 1.25 TFLOP/s (FMA = 2 flops).
FP64_PEAK_TFLOPS = 1.25


def _fp64_roof(kernel, units, ms):
    f = FP64_FLOPS.get(kernel)
    if f is None or ms <= 0:
        return {"kernel": kernel, "bound": "fp64", "achieved": None, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": None, "peak_kind": "derived (nominal FP64 rate)"}
    ach = f * units / (ms / 1e3) / 1e12
    return {"kernel": kernel, "bound": "fp64", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_PEAK_TFLOPS, "fp64_flops_per_unit": f, "peak_kind": "derived (nominal FP64 rate)"}


# The transfers fold each particle's x-hat (three double-float pairs) and its
# property once, in double-float arithmetic on the FP32 pipe; per particle
# 24 + 8 B, plus the per-cell outputs amortised over 20 particles per cell:
# 2^3 corner numerators and denominators as double-float pairs (vertex
# averages), 4 coefficients and a count (least squares).
TRANSFER_BYTES_PER_PARTICLE = {"vertex_partial_kernel<3>": 32.0 + 16 * 8 / 20.0,
                               "lsq_linear_kernel<3>": 32.0 + (4 * 8 + 4) / 20.0}


def _transfer_roof(kernel, units, ms):
    hbm, kind = load_peaks()
    b = TRANSFER_BYTES_PER_PARTICLE[kernel]
    ach = b * units / (ms / 1e3) / 1e9
    return {"kernel": kernel, "bound": "fp32 issue (double-float arithmetic)", "view": "hbm",
            "algorithmic_bytes_per_particle": b, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "peak_kind": kind}


def run_next(args):
    """The rows after the hot path, each on the 64^3 x 20 workload (c2):
    f1 time interpolation, f2 property ODEs, f3 particle -> field transfers,
    f4 generation; each with its bound and the oracle timed on a sample."""
    import torch
    import oracle as O
    from paper_1612_03369_gb300 import pic as P

    wl = W.c2()
    dt = wl.dt
    mesh = P.Mesh(wl.n, wl.X, wl.U)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(reps):
            fn()
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    def cpu(fn, units, what):
        t0 = time.perf_counter()
        fn()
        el = time.perf_counter() - t0
        return {"value": units / el, "seconds": el, "cores": 1, "kind": "oracle", "sample": what}

    om = O.Mesh(wl.n, wl.X, wl.U)
    rows = {}
    # f1: time interpolation between two fields (RK4 half-step stages average them)
    parts = P.Particles(mesh, uniform_count=wl.ppc, seed=wl.pseed, n_props=3)
    N = parts.state()[0]
    steady = timed(lambda: parts.advect(dt, 4, 1), args.steps)
    mesh.set_velocity(wl.U, U_next=0.5 * wl.U)
    two = timed(lambda: parts.advect(dt, 4, 1), args.steps)
    mesh.set_velocity(wl.U)
    om2 = O.Mesh(wl.n, wl.X, wl.U)
    om2.set_velocity_next(0.5 * wl.U)
    sub = O.seed_particles(om2, uniform_count=wl.ppc, seed=wl.pseed, n_props=0)
    sub = sub.subset(np.arange(sub.n) % 2000 == 0)
    rows["f1_time_interpolation"] = {
        "value": N / (two / 1e3), "unit": "particle-steps/s", "ms_per_step": two, "steady_ms_per_step": steady,
        "bound": "alu (FP32 issue; two Q2 contractions at the c = 1/2 stages)",
        "cpu_baseline": cpu(lambda: O.advect(om2, sub, dt, 4, 1), sub.n, "%d particles, one RK4 step" % sub.n)}
    parts.close()
    # f2: property ODEs (damage + F)
    parts = P.Particles(mesh, uniform_count=wl.ppc, seed=wl.pseed, n_props=10)
    eye = np.eye(3).reshape(-1)
    for q in range(9):
        parts.set_property(1 + q, torch.full((N,), float(eye[q]), dtype=torch.float64, device="cuda"))
    odes = dict(damage=0, alpha=1.0, beta=0.5, deformation=1)
    ms = timed(lambda: parts.advect_properties(dt, 4, 1, **odes), args.steps)
    op = O.seed_particles(om, uniform_count=wl.ppc, seed=wl.pseed, n_props=10)
    op = op.subset(np.arange(op.n) % 5000 == 0)
    op.props[:, 1:10] = eye
    ode_ms = ms - steady  # the gradient and ODE kernels: the step's time beyond the plain advect + rebin
    ach = PROPS_ODE_FP32_FLOPS_PER_PARTICLE_STEP * N / (ode_ms / 1e3) / 1e12
    rows["f2_property_odes"] = {
        "value": N / (ms / 1e3), "unit": "particle-steps/s", "ms_per_step": ms,
        "roofline": {"kernel": "props_grad_kernel<3> + props_ode_kernel<3,RK4>", "bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS,
                     "fp32_flops_per_particle_step": PROPS_ODE_FP32_FLOPS_PER_PARTICLE_STEP,
                     "kernel_ms": ode_ms, "kernel_ms_how": "step with ODEs minus the plain step",
                     "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz"},
        "cpu_baseline": cpu(lambda: O.advect_properties(om, op, dt, 4, 1, damage=0, alpha=1.0, beta=0.5, defgrad=1),
                            op.n, "%d particles, one RK4 step with both ODEs" % op.n)}
    parts.close()
    # f3: transfers of one property (the store as seeded, property = x0)
    parts = P.Particles(mesh, uniform_count=wl.ppc, seed=wl.pseed, n_props=1)
    st = parts.export()
    parts.set_property(0, st["x"][0].contiguous())
    del st
    ms_v = timed(lambda: parts.vertex_average(0), args.steps)
    ms_l = timed(lambda: parts.project_linear(0), args.steps)
    ms_a = timed(lambda: parts.average(0), args.steps)
    full = O.seed_particles(om, uniform_count=wl.ppc, seed=wl.pseed, n_props=0)
    v0 = full.x[:, 0].copy()
    rows["f3_transfers"] = {
        "particles": N, "cell_average_ms": ms_a, "vertex_average_ms": ms_v, "project_linear_ms": ms_l,
        "vertex_average": {"value": N / (ms_v / 1e3), "unit": "particles/s",
                           "roofline": _transfer_roof("vertex_partial_kernel<3>", N, ms_v)},
        "project_linear": {"value": N / (ms_l / 1e3), "unit": "particles/s",
                           "roofline": _transfer_roof("lsq_linear_kernel<3>", N, ms_l)},
        "cpu_baseline": {
            "vertex_average": cpu(lambda: O.vertex_average(om, full.cell, full.xhat, v0), N, "all %d particles" % N),
            "project_linear": cpu(lambda: O.cell_lsq_linear(om, full.cell, full.xhat, v0), N, "all %d particles" % N)}}
    parts.close()
    # f4: generation with a density, and prescribed positions
    Xv = wl.X
    rho = 1.0 + 4.0 * Xv[0] * Xv[1]
    rho_d = torch.as_tensor(rho, device="cuda")
    wts = P.cell_weights(mesh, rho_d)
    ms_w = timed(lambda: P.cell_weights(mesh, rho_d), args.steps)
    ms_d = timed(lambda: P.draw_cell_counts(wts, N, 7), max(2, args.steps // 5))
    counts = P.draw_cell_counts(wts, N, 7)
    J = 8
    holder = []

    def mh():
        if holder:
            holder.pop().close()
        holder.append(P.Particles.metropolis_hastings(mesh, counts, rho_d, thinning=J, seed=3))

    ms_m = timed(mh, 3)
    holder.pop().close()
    g = np.random.default_rng(1)
    pts = torch.as_tensor(g.uniform(-0.05, 1.05, size=(3, N)), device="cuda")

    def imp():
        if holder:
            holder.pop().close()
        holder.append(P.Particles.import_points(mesh, pts)[0])

    ms_i = timed(imp, 3)
    holder.pop().close()
    w_o = O.cell_weights(om, rho)
    per_o = O.draw_cell_counts(w_o, 20000, 7).astype(np.uint32)
    pts_o = pts[:, :20000].cpu().numpy().T.copy()
    rows["f4_generation"] = {
        "particles": N, "cells": wl.ncells, "cell_weights_ms": ms_w, "draw_counts_ms": ms_d,
        "cell_weights": {"value": wl.ncells / (ms_w / 1e3), "unit": "cells/s",
                         "roofline": _fp64_roof("cell_weights_kernel<3>", wl.ncells, ms_w)},
        "metropolis_hastings_ms": ms_m, "mh_thinning": J, "import_ms": ms_i,
        "mh": {"value": N * J / (ms_m / 1e3), "unit": "chain steps/s",
               "roofline": _fp64_roof("mh_seed_kernel<3>", N * J, ms_m)},
        "import": {"value": N / (ms_i / 1e3), "unit": "points/s"},
        "cpu_baseline": {
            "cell_weights": cpu(lambda: O.cell_weights(om, rho), wl.ncells, "all %d cells" % wl.ncells),
            "draw_counts": cpu(lambda: O.draw_cell_counts(w_o, N, 7), N, "all %d draws" % N),
            "metropolis_hastings": cpu(lambda: O.seed_particles_mh(om, per_o, rho, J, 3), int(per_o.sum()) * J,
                                       "20000 particles (chain steps as unit)"),
            "import": cpu(lambda: O.import_points(om, pts_o), 20000, "20000 points")}}
    mesh.close()
    return {"metric": "rows after the hot path on 64^3 x 20 (c2 workload): time interpolation, property ODEs, "
                      "particle -> field transfers, generation",
            "n_gpus": 1, "steps": args.steps, "data": "synthetic", "dtype": "f64",
            "config": {"workload": "c2_3d_curl_64^3", "particles": N}, "rows": rows}


def roofline_object(precision, adv_avg_ms, particles, adv_bytes, hbm, peak_kind="measured", rebin_ms=None):
    """The advect kernel's HBM roofline: algorithmic bytes per particle-step x
    particles per launch / the launch's mean CUDA-event time, against the
    measured HBM copy bandwidth.  Beside it, the DRAM traffic of one launch
    (from an ncu capture of the kernel, scaled to this launch's particles) and
    the issue view of the same capture."""
    achieved = adv_bytes * particles / (adv_avg_ms / 1e3) / 1e9
    dram = ADVECT_DRAM_BYTES_PER_PARTICLE.get(precision)
    issue = ADVECT_ISSUE.get(precision)
    form = "FP64 form" if precision == 0 else "FP32-basis form"
    return {"kernel": "advect_kernel<3,RK4> (%s)" % form, "bound": "hbm", "achieved": achieved, "peak": hbm,
            "unit": "GB/s", "frac": achieved / hbm, "peak_kind": "%s HBM copy bandwidth" % peak_kind,
            "algorithmic_bytes_per_particle_step": adv_bytes, "particles_per_launch": particles,
            "avg_launch_ms": adv_avg_ms, "rebin_ms_per_step": rebin_ms,
            "traffic": dram * particles if dram else None,
            "traffic_source": "ncu dram__bytes_read+write of this kernel on the 64^3 x 20 workload, per particle, "
                              "x particles per launch" if dram else None,
            "issue_view": issue}


def _sample_particles(O, om, wl, ids):
    """Particles `ids` of the uniform-count seeding, rebuilt from the
    published generator (SplitMix64 output g*dim + j gives x-hat_j of particle
    g) and the oracle's map, without seeding the whole store in the oracle."""
    d = wl.dim
    xh = np.array([[(O.splitmix64(wl.pseed, int(g) * d + j) >> 11) * 2.0 ** -53 for j in range(d)] for g in ids])
    cell = (np.asarray(ids) // wl.ppc).astype(np.int64)
    x = np.array([om.phi(int(K), t) for K, t in zip(cell, xh)])
    props = np.zeros((len(ids), wl.n_props))
    props[:, : min(wl.n_props, d)] = x[:, : min(wl.n_props, d)]
    return O.Particles(x, xh, cell, (wl.first_id + np.asarray(ids)).astype(np.uint64), props)


def cpu_baseline(wl, seconds: float = 15.0, sample: int | None = None):
    """The oracle as it stands, single thread, on a bounded random sample of
    the workload's particles advanced one time step at a time."""
    import oracle as O

    om = O.Mesh(wl.n, wl.X, wl.U)
    rng = np.random.default_rng(0)
    n = sample or 2000
    pick = np.sort(rng.choice(wl.n_particles, min(n, wl.n_particles), replace=False))
    sub = _sample_particles(O, om, wl, pick)
    done = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        before = sub.n
        sub = O.advect(om, sub, wl.dt, wl.integrator, 1)
        done += before
    el = time.perf_counter() - t0
    return {"value": done / el, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "sample": "%d random particles of %s advanced one step at a time for %.1f s (%d particle-steps)"
                      % (len(pick), wl.name, el, done)}


# The oracle on all host cores: the sample split into one chunk per core, each
# advanced in its own process (spawned, so nothing of the GPU context is
# inherited).  The oracle is unchanged; only the particles are divided, which
# is exact because they move independently.  The field goes to the workers
# through a memory-mapped file.
_ORC_WORKER = None


def _orc_worker_init(n, X, U_path, dt, integrator):
    global _ORC_WORKER
    import oracle as O

    U = np.load(U_path, mmap_mode="r")
    _ORC_WORKER = (O, O.Mesh(n, X, np.ascontiguousarray(U)), dt, integrator)


def _orc_worker_run(task):
    x, xhat, cell, ids, props, seconds = task
    O, om, dt, integrator = _ORC_WORKER
    sub = O.Particles(x, xhat, cell, ids, props)
    done = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        before = sub.n
        sub = O.advect(om, sub, dt, integrator, 1)
        done += before
    return done, time.perf_counter() - t0


def cpu_baseline_all_cores(wl, seconds: float = 10.0, per_core: int = 2000):
    """The same sample rate with one oracle process per host core."""
    import multiprocessing as mp
    import oracle as O

    cores = os.cpu_count() or 1
    om = O.Mesh(wl.n, wl.X, wl.U)
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(wl.n_particles, min(per_core * cores, wl.n_particles), replace=False))
    sub = _sample_particles(O, om, wl, pick)
    chunks = np.array_split(np.arange(sub.n), cores)
    tasks = [(sub.x[c], sub.xhat[c], sub.cell[c], sub.id[c], sub.props[c], seconds) for c in chunks]
    ctx = mp.get_context("spawn")
    fd, U_path = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    try:
        np.save(U_path, wl.U)
        with ctx.Pool(cores, initializer=_orc_worker_init, initargs=(wl.n, wl.X, U_path, wl.dt, wl.integrator)) as pool:
            res = pool.map_async(_orc_worker_run, tasks, chunksize=1).get(timeout=seconds + 300)
    except Exception as e:  # a worker that cannot start must not hold the benchmark
        return {"unavailable": "%s: %s" % (type(e).__name__, e), "cores": cores, "kind": "oracle"}
    finally:
        os.unlink(U_path)
    done = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    return {"value": done / el, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
            "sample": "%d random particles of %s in %d processes of %d particles, each advanced one step at a time "
                      "for %.1f s" % (sub.n, wl.name, cores, len(chunks[0]), el)}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    wl = workload(args.config if args.config in ("c1", "c2", "c3") else "c3")
    import oracle as O

    om = O.Mesh(wl.n, wl.X, wl.U)
    rng = np.random.default_rng(1)
    sample = 300
    pick = np.sort(rng.choice(wl.n_particles, sample, replace=False))
    sub = _sample_particles(O, om, wl, pick)
    for _ in range(args.warmup):
        sub = O.advect(om, sub, wl.dt, wl.integrator, 1)
    done = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        before = sub.n
        sub = O.advect(om, sub, wl.dt, wl.integrator, 1)
        done += before
    el = time.perf_counter() - t0
    value = done / el
    return {
        "impl": "reference",
        "metric": "RK4 particle-steps/s (advect+locate+rebin), 3D Q2 mesh; % of HBM roofline",
        "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": {"workload": wl.name},
        "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                         "sample": "%d random particles of %s, one time step per benchmark step" % (sample, wl.name)},
        "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c3", choices=["c1", "c2", "c3", "c4", "c5", "c2p", "next"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the FP32-basis form's error measurement")
    ap.add_argument("--partition", default=None, choices=["slab", "replicas"],
                    help="one mesh split in slabs with particle exchange (the default with N > 1 GPUs; explicit at "
                         "N = 1: one slab) or N independent replicas")
    ap.add_argument("--mesh", type=int, default=None,
                    help="cells per axis instead of the configuration's (profiling only: not that configuration)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank, world, local_rank = shard.rank_env()
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if args.config in ("c4", "c2p", "next"):
        # one problem: rank 0 alone runs it
        if rank == 0:
            fn = {"c4": run_adjoint, "c2p": run_props, "next": run_next}[args.config]
            print(json.dumps(fn(args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.config == "c5":
        res = run_ensemble(args, rank, world, local_rank)
    elif args.config in ("c2", "c3") and (args.partition == "slab" or (world > 1 and args.partition is None)):
        res = run_slab(args, rank, world, local_rank)
    else:
        res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
