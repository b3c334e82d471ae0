#!/usr/bin/env python
"""Throughput of the DG RK stage: DOF-updates/s per RK stage.

Workload: isentropic vortex (beta=5, gamma=1.4, boost (1,1)) on the periodic
box [-5,5]^2 with 256^2 cells, polynomial degree k=3 (N=10 basis functions),
SSP-RK4 (5 stages), no limiter, CFL 0.2; synthetic closed-form initial data.
A step is one RK4 step (all stages, including the on-device CFL timestep)
over the whole mesh; DOF = cells x N.  The headline is the FP64 path; the
FP32 path is reported under "variants".

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun (N > 1) every rank advances its own replica of the problem
(no data-path collective): value = DOF-updates of all ranks / max time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DG DOF-updates/s per RK stage, FP32-TC vs FP64 at equal L1 err; % HBM peak"
UNIT = "DOF-updates/s"
N_CELLS_1D, K_DEG, RK_ORDER, STAGES, CFL = 256, 3, 4, 5, 0.2
N_BASIS, NV, DIM = 10, 4, 2
L2_BYTES = 129 * 2 ** 20


WORKLOADS = {
    "vortex": dict(
        name="isentropic vortex 2D, 256x256 periodic [-5,5]^2, k=3 (10 coeffs/cell/var), "
             "SSP-RK4 (5 stages), no limiter, CFL 0.2",
        dim=2, k=3, rk=4, stages=5, limiter="none", positivity=False,
        precisions=("fp64", "fp32", "fp32_tc", "mixed", "mixed_tc"), tag="vortex256_k3"),
    "vortex_tensor": dict(
        name="isentropic vortex 2D, 256x256 periodic [-5,5]^2, k=3 with the tensor-product basis Q_3 "
             "(16 coeffs/cell/var), SSP-RK4 (5 stages), no limiter, CFL 0.2",
        dim=2, k=3, rk=4, stages=5, limiter="none", positivity=False, precisions=("fp64", "fp32"),
        tag="vortex256_k3_tensor", basis="tensor"),
    "ensemble": dict(
        name="512 independent isentropic vortices (strength U(3,6)) on periodic [-5,5]^2 with "
             "sizes drawn from {32,48,64,96,128}^2 (3.4M cells), k=2 (6 coeffs/cell/var), SSP-RK3, "
             "per-problem CFL timestep, FP32, all steps in one CUDA-graph launch",
        dim=2, k=2, rk=3, stages=3, limiter="none", positivity=False, precisions=("fp32",),
        tag="ensemble512_k2", graph=True, autotune=True),
    "wave2d": dict(
        name="advected density wave 2D, 32x32 periodic [0,1]^2, k=1 (3 coeffs/cell/var), SSP-RK2, "
             "CFL 0.3, FP64; all timed steps in one CUDA-graph launch (launch-bound: time per stage "
             "of the graph replay)",
        dim=2, k=1, rk=2, stages=2, limiter="none", positivity=False, precisions=("fp64",),
        tag="wave2d32_k1", graph=True, cfl=0.3),
    "square64": dict(
        name="square advection 2D, 64x64 periodic [0,1]^2, rho 4 in a 0.5-wide square, rho 1 outside, "
             "p=2.5, v=(100,50), k=2 (6 coeffs/cell/var), SSP-RK3, characteristic TVB limiter "
             "(beta 1, Mtilde 0.5), CFL 0.2, FP64; all timed steps in one CUDA-graph launch "
             "(launch-bound: step rate of the graph replay)",
        dim=2, k=2, rk=3, stages=3, limiter="characteristic", positivity=False, precisions=("fp64",),
        tag="square64_k2", graph=True),
    "sedov3d": dict(
        name="Sedov blast 3D, 64^3 base + central 32^3 refined once (491,520 cells), k=2 "
             "(10 coeffs/cell/var), SSP-RK3, characteristic TVB limiter + positivity limiter, "
             "FP32 state with FP64 totals / positivity check",
        dim=3, k=2, rk=3, stages=3, limiter="characteristic", positivity=True,
        precisions=("fp32",), tag="sedov3d_k2", autotune=True),
    "kepler": dict(
        name="cold Keplerian disc 2D (rho 1 between r 0.5 and 2 with 0.1 ramps, background rho = p = 1e-5, "
             "v = r^-1/2 rotation, static central acceleration with eps 0.25 softening inside r 0.45), periodic "
             "[0,6]^2, 1024^2 cells, k=2 (6 coeffs/cell/var), SSP-RK3, positivity limiter only, gravity source "
             "and gravity timestep bound, gamma 5/3, CFL 0.2",
        dim=2, k=2, rk=3, stages=3, limiter="none", positivity=True, precisions=("fp64", "fp32"),
        tag="kepler1024_k2", gravity=True, gamma=5.0 / 3.0),
    "kh2d_amr": dict(
        name="Kelvin-Helmholtz 2D (rho 2|1, v_x +-0.5, p 2.5, single-mode v_y seed), periodic [0,1]^2, "
             "1024^2 base cells + one dynamic refinement level (effective 2048^2), k=3 (10 coeffs/cell/var), "
             "SSP-RK4 (5 stages), characteristic TVB limiter + positivity limiter, CFL 0.2; mesh adapted "
             "after every step (w_t 0.01, alpha 1.1, one buffer layer); a step = RK step + adaptation; "
             "timed from t = 0.003 (untimed adaptive pre-run from the initial data: the interfaces, "
             "aligned with cell faces at t = 0, carry slopes once the v_y seed has moved them)",
        dim=2, k=3, rk=4, stages=5, limiter="characteristic", positivity=True,
        precisions=("fp64", "mixed"), tag="kh1024_amr_k3", amr=True, base=1024, w_t=0.01, alpha=1.1,
        t_pre=0.003),
}


def workload_config(wk, precision, cells):
    W = WORKLOADS[wk]
    l2 = ("state larger than L2 (no flush); timed steps in one graph launch" if W.get("graph")
          else "flushed between timed steps (256 MiB write)")
    if wk in ("wave2d", "square64"):
        l2 = "L2-resident state (launch-bound workload); timed steps in one graph launch"
    if W.get("amr"):
        l2 = "state larger than L2 (no flush); steps launched one by one (the adaptation reads sizes back)"
    return {"workload": W["name"], "cells": cells, "k": W["k"], "rk_stages": W["stages"],
            "precision": precision, "l2": l2}


def mesh(n=N_CELLS_1D, half=5.0):
    from paper_1506_06140_gb300 import workloads as wl
    return wl.mesh_uniform(2, [n, n], [-half, -half], [half, half])


def make_problem(wk, precision, autotune=None):
    """Solver and initial weights (on the device) of a workload."""
    import torch
    from paper_1506_06140_gb300 import dg
    from paper_1506_06140_gb300 import workloads as wl
    W = WORKLOADS[wk]
    if wk in ("vortex", "vortex_tensor"):
        m, ic = mesh(), wl.vortex
    elif wk == "wave2d":
        m, ic = wl.mesh_uniform(2, [32, 32], [0.0, 0.0], [1.0, 1.0]), wl.wave2d
    elif wk == "square64":
        m, ic = wl.mesh_uniform(2, [64, 64], [0.0, 0.0], [1.0, 1.0]), wl.square2d
    elif wk == "ensemble":
        probs = wl.ensemble_problems()
        m = [wl.mesh_uniform(2, [n, n], [-5.0, -5.0], [5.0, 5.0]) for n, _ in probs]
        ic = None
    elif wk == "kepler":
        m, ic = wl.mesh_uniform(2, [1024, 1024], [0.0, 0.0], [6.0, 6.0]), wl.keplerian_disc
    elif wk == "kh2d_amr":
        n = W["base"]
        m, ic = wl.mesh_uniform(2, [n, n], [0.0, 0.0], [1.0, 1.0]), wl.kelvin_helmholtz
    else:
        m, ic = wl.mesh_two_level_3d(64, 16, 47), wl.sedov3d
    if autotune is None:
        autotune = W.get("autotune", False)
    s = dg.Solver(m, W["k"], W.get("gamma", 1.4), rk_order=W["rk"], cfl=W.get("cfl", CFL),
                  limiter=W["limiter"], positivity=W["positivity"], precision=precision, autotune=autotune,
                  basis=W.get("basis", "total"))
    xyz = s.quad_points().cpu().numpy()
    if W.get("gravity"):
        s.set_gravity(torch.as_tensor(wl.keplerian_accel(xyz)))
    if ic is not None:
        U = ic(xyz)  # closed-form IC at the Gauss points
    else:
        U = np.empty((s.nv, s.nq, s.n_cells))
        for p, (n, beta) in enumerate(probs):
            a, b = s.cell_offsets[p], s.cell_offsets[p + 1]
            U[:, :, a:b] = wl.vortex(xyz[:, :, a:b], beta=beta)
    W0 = s.project(torch.as_tensor(U))
    if W["limiter"] != "none" or W["positivity"]:
        s.limit(W0)
    return s, W0


# ---------------------------------------------------------------------------
# algorithmic work per cell and stage (sum-factorised contraction counts)

def shape(dim, k, basis="total"):
    N = (k + 1) * (k + 2) // 2 if dim == 2 else (k + 1) * (k + 2) * (k + 3) // 6
    if basis == "tensor":
        N = (k + 1) ** dim
    Q, QF, nv = (k + 1) ** dim, (k + 1) ** (dim - 1), dim + 2
    return N, Q, QF, nv


def kernel_flops(dim, k, basis="total", moments=False):
    """Flops of the sum-factorised kernels: (cell kernel per cell, face kernel per face).

    Per variable (FMA counts; K1 = k+1, N2 = K1 (K1+1) / 2 pairs (a,b)):
      modal->nodal   2D: N K1 + K1^3          3D: N K1 + N2 K1^2 + K1^4
      volume / dir   2D: k K1^2 + (N-K1) K1   3D: k K1^3 + (N2-K1) K1^2 + (N-N2) K1
      surface / side 2D: K1^2 + N             3D: K1^3 + N2 K1 + N
      face trace     2D: N + K1^2             3D: N + N2 K1 + K1^3
    plus Euler fluxes (18 | 27 flop per point), HLLC (90 | 100 flop per face
    point) and the stage combination (5 flop per weight).  The 2D counts hold
    for the tensor-product basis too (N = K1^2 there).  With face moments
    (3D, and 2D FP64) the face kernel contracts each face's flux once
    (2D: K1^2, 3D: K1^3 + N2 K1 per variable) and a cell side costs
    N + (number of moments)."""
    N, Q, QF, nv = shape(dim, k, basis)
    K1 = k + 1
    if dim == 2:
        m2n, vol = N * K1 + K1 ** 3, dim * (k * K1 * K1 + (N - K1) * K1)
        surf, trace, flux_pt, hllc_pt = 2 * dim * (K1 * K1 + N), N + K1 * K1, 18, 90
    else:
        N2 = K1 * (K1 + 1) // 2
        m2n = N * K1 + N2 * K1 * K1 + K1 ** 4
        vol = dim * (k * K1 ** 3 + (N2 - K1) * K1 * K1 + (N - N2) * K1)
        surf, trace, flux_pt, hllc_pt = 2 * dim * (K1 ** 3 + N2 * K1 + N), N + N2 * K1 + K1 ** 3, 27, 100
    face_mom = 0
    if moments:
        if dim == 2:
            surf, face_mom = 2 * dim * (N + K1), K1 * K1
        else:
            N2 = K1 * (K1 + 1) // 2
            surf, face_mom = 2 * dim * (N + N2), K1 ** 3 + N2 * K1
    cell = 2 * nv * (m2n + vol + surf) + flux_pt * Q + 5 * N * nv
    face = 2 * 2 * nv * trace + hllc_pt * QF + 2 * nv * face_mom
    return cell, face


def state_bytes_per_cell(dim, k, esize, basis="total"):
    N, Q, QF, nv = shape(dim, k, basis)
    return nv * N * esize


# ---------------------------------------------------------------------------

class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 10.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.skip = len(self.lines)  # samples taken before the measured region
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.th.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines[getattr(self, "skip", 0):] or self.lines[-1:]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# nominal FP64 / FP32 SIMT rates from unit counts and the maximum SM clock:
# 152 SMs x (2 FP64 | 128 FP32) FMA lanes per clock x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def dram_traffic(kernel, workload):
    """Per-launch DRAM bytes from the committed ncu summary, or None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    for ln in open(path):
        parts = ln.split()
        if len(parts) >= 3 and parts[0] == kernel and parts[1] == workload:
            try:
                return float(parts[2])
            except ValueError:
                return None
    return None


# ---------------------------------------------------------------------------

class Ranks:
    """The only cross-rank traffic of a multi-GPU run: a barrier around the
    timed region and the maximum of the ranks' times (each rank advances its
    own replica of the workload; no data-path collective)."""

    def __init__(self, world, backend="nccl", device="cuda", local_rank=0):
        import torch
        self.world, self.device = world, device
        self.dist = None
        if world > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                if backend == "nccl":
                    dist.init_process_group(backend, device_id=torch.device("cuda", local_rank))
                else:
                    dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def max(self, x):
        if not self.dist:
            return x
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return t.item()

    def sum(self, x):
        if not self.dist:
            return x
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return t.item()


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_1506_06140_gb300 import dg
    from paper_1506_06140_gb300 import workloads as wl

    torch.cuda.set_device(local_rank)
    ranks = Ranks(world, "nccl", "cuda", local_rank)
    barrier, max_over_ranks = ranks.barrier, ranks.max

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    results = {}
    for precision in args.precisions:
        s, W0 = make_problem(args.workload, precision)
        W = W0.clone()
        stream = torch.cuda.current_stream()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        graph = WORKLOADS[args.workload].get("graph", False)
        with ClockSampler(local_rank) as clk:  # sampling spans the warm-up and the timed steps
            if graph:
                # all timed steps as one graph launch; the state (> L2) is not flushed
                s.advance(W, args.warmup)
                s.advance(W, args.steps)  # records the timed graph (not timed)
                torch.cuda.synchronize()
                barrier()
                ev[0][0].record(stream)
                s.advance(W, args.steps)
                ev[0][1].record(stream)
                torch.cuda.synchronize()
                ev = ev[:1]
            else:
                # each timed step is one dg_advance of one step (a CUDA graph of
                # the step's kernels, recorded in the warm-up), L2 flushed before it
                for _ in range(args.warmup):
                    s.advance(W, 1)
                limited = WORKLOADS[args.workload]["limiter"] != "none"
                if limited:
                    s.limiter_counts(reset=True)
                torch.cuda.synchronize()
                barrier()
                for i in range(args.steps):
                    flush.zero_()  # evict the working set from L2 before each timed step
                    ev[i][0].record(stream)
                    s.advance(W, 1)
                    ev[i][1].record(stream)
                torch.cuda.synchronize()
        paths = None
        if graph and args.workload in ("wave2d", "square64"):
            # the same steps as one persistent cooperative kernel (dg_set_advance_mode)
            Wp = W.clone()
            s.set_advance_mode("persistent")
            s.advance(Wp, args.warmup)
            torch.cuda.synchronize()
            p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            p0.record(stream)
            s.advance(Wp, args.steps)
            p1.record(stream)
            torch.cuda.synchronize()
            s.set_advance_mode("graph")
            paths = {"graph_ms_per_step": ev[0][0].elapsed_time(ev[0][1]) / args.steps,
                     "persistent_ms_per_step": p0.elapsed_time(p1) / args.steps,
                     "note": "dg_advance as a CUDA graph of the stage kernels (default, timed above) "
                             "or as one persistent cooperative kernel with grid barriers"}
            del Wp
        # per-kernel durations from a separate pass of the same one-step graphs,
        # recorded with an event pair around every kernel (dg_profile_begin)
        cnt_snap = s.limiter_counts().cpu().numpy()  # limiter activity up to here
        Wp = W.clone()
        s.profile_begin()
        for _ in range(args.steps):
            if not graph:
                flush.zero_()
            s.advance(Wp, 1)
        torch.cuda.synchronize()
        prof = s.profile_end()
        del Wp
        barrier()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        ms = max_over_ranks(ms)
        assert torch.isfinite(W).all().item(), "non-finite state"
        diag = None
        if WORKLOADS[args.workload].get("gravity"):
            # total angular momentum about the disc's centre, from the mean and
            # linear weights: int_K x' m_y = |K| (x'_c w_0 + (dx/2) w_x / sqrt 3)
            cen = s.quad_points().mean(dim=1).cpu().numpy() - 3.0
            dx = 6.0 / 1024
            h = dx / 2 / math.sqrt(3.0)

            def ang(Wt):
                Wn = Wt.double().cpu().numpy()
                return float((dx * dx * (cen[0] * Wn[2, 0] + h * Wn[2, 1] - cen[1] * Wn[1, 0]
                                         - h * Wn[1, 2])).sum())
            L0, L1 = ang(W0), ang(W)
            t0, t1 = s.totals(W0).cpu().numpy(), s.totals(W).cpu().numpy()
            passes = s.n_cells * WORKLOADS[args.workload]["stages"] * (args.steps + args.warmup)
            cnt = cnt_snap
            diag = {"angular_momentum_drift_rel": abs(L1 - L0) / abs(L0),
                    "mass_drift_rel": float(abs(t1[0] - t0[0]) / abs(t0[0])),
                    "positivity_limited_fraction": float(cnt[1]) / passes,
                    "positivity_fp64_pass_fraction": float(cnt[2]) / passes,
                    "steps_since_initial_state": args.warmup + args.steps,
                    "note": "the positivity limiter does not conserve angular momentum; unlimited DG does "
                            "to rounding (GPU test)"}
        if WORKLOADS[args.workload]["limiter"] != "none":
            # limiter activity over the timed steps and conservation drift from the initial state
            cnt = cnt_snap
            passes = s.n_cells * WORKLOADS[args.workload]["stages"] * args.steps
            t0, t1 = s.totals(W0).cpu().numpy(), s.totals(W).cpu().numpy()
            diag = {"slope_limited_fraction": float(cnt[0]) / passes,
                    "positivity_limited_fraction": float(cnt[1]) / passes,
                    "positivity_fp64_pass_fraction": float(cnt[2]) / passes,
                    "steps_since_initial_state": args.warmup + args.steps,
                    "mass_drift_rel": float(abs(t1[0] - t0[0]) / abs(t0[0])),
                    "energy_drift_rel": float(abs(t1[-1] - t0[-1]) / abs(t0[-1])),
                    "momentum_abs": [float(x) for x in t1[1:-1]]}
        # end to end through the C ABI with host buffers: every step copies the
        # state in from pinned host memory, advances it one step (dg_advance:
        # the step's graph, recorded for this buffer by one untimed step) and
        # copies it back
        Wh = W0.cpu().pin_memory()
        Wd = torch.empty_like(W0)
        Wd.copy_(Wh)
        s.advance(Wd, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for i in range(args.steps):
            Wd.copy_(Wh, non_blocking=True)
            s.advance(Wd, 1)
            Wh.copy_(Wd, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = max_over_ranks(e0.elapsed_time(e1))
        tiles = None
        if WORKLOADS[args.workload].get("autotune"):
            # the fixed-tile baseline: the same graph launch with the default tiles
            sf, Wf = make_problem(args.workload, precision, autotune=False)
            sf.advance(Wf, args.warmup)
            sf.advance(Wf, args.steps)
            torch.cuda.synchronize()
            barrier()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            sf.advance(Wf, args.steps)
            f1.record(stream)
            torch.cuda.synchronize()
            tiles = {"autotuned": list(s.tiles()), "fixed": list(sf.tiles()),
                     "fixed_tile_ms": max_over_ranks(f0.elapsed_time(f1))}
            del sf, Wf
        results[precision] = dict(solver=s, ms=ms, ms_e2e=ms_e2e, prof=prof, clocks=clk.summary(),
                                  state_bytes=W.numel() * W.element_size(), n_cells=s.n_cells,
                                  tiles=tiles, diag=diag, paths=paths)
        del W, W0, Wd, Wh
    return results


def run_gpu_amr(args, rank, world, local_rank):
    """Steps of an adaptive run: one RK step, then the adaptation of the mesh
    (criterion, buffer layer, regrid where anything changed), as in the main
    loop of Sec. 4.  Both halves are timed with CUDA events on the launching
    stream; the adaptation's host round trips (sizes read back) are inside."""
    import torch
    torch.cuda.set_device(local_rank)
    ranks = Ranks(world, "nccl", "cuda", local_rank)
    wk = WORKLOADS[args.workload]
    results = {}
    for precision in args.precisions:
        s, W0 = make_problem(args.workload, precision)
        stream = torch.cuda.current_stream()

        def one_step(W, ev=None):
            cells = s.n_cells
            if ev:
                ev[0].record(stream)
            s.rk_step(W)
            if ev:
                ev[1].record(stream)
            W, changed = s.adapt(W, wk["w_t"], wk["alpha"])
            if ev:
                ev[2].record(stream)
            return W, cells, changed

        W = W0
        # adaptive pre-run to t_pre (outside the timed steps); each adaptation
        # is timed, split into steps that regridded and steps that only checked
        t, pre_steps, dt_buf = 0.0, 0, s.scalar()
        pre = {"regrid": [], "check": []}
        while t < wk.get("t_pre", 0.0):
            s.rk_step(W, 0.0, dt_buf)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            W, changed = s.adapt(W, wk["w_t"], wk["alpha"])
            a1.record(stream)
            t += dt_buf.item()  # synchronises
            pre["regrid" if changed else "check"].append((a0.elapsed_time(a1), changed, s.n_cells))
            pre_steps += 1
        with ClockSampler(local_rank) as clk:
            for _ in range(args.warmup):
                W, _, _ = one_step(W)
            s.limiter_counts(reset=True)
            t_start = s.totals(W).cpu().numpy()
            torch.cuda.synchronize()
            ranks.barrier()
            s.profile_begin()
            evs, cells, changes = [], [], []
            for _ in range(args.steps):
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                W, c, ch = one_step(W, ev)
                evs.append(ev)
                cells.append(c)
                changes.append(ch)
            torch.cuda.synchronize()
        prof = s.profile_end()
        step_ms = sum(e[0].elapsed_time(e[1]) for e in evs)
        adapt_ms = sum(e[1].elapsed_time(e[2]) for e in evs)
        ms = ranks.max(step_ms + adapt_ms)
        assert torch.isfinite(W).all().item(), "non-finite state"
        regrids = sum(1 for c in changes if c > 0)
        cnt = s.limiter_counts(reset=True).cpu().numpy()
        passes = sum(cells) * wk["stages"]
        t_end = s.totals(W).cpu().numpy()
        nbase = wk["base"] ** 2
        rg = pre["regrid"]
        diag = {"pre_run_steps": pre_steps, "t_pre": t, "pre_run_regrids": len(rg),
                "pre_run_regrid_adapt_ms_mean": sum(x[0] for x in rg) / max(len(rg), 1),
                "pre_run_regrid_base_cells_changed_mean": sum(x[1] for x in rg) / max(len(rg), 1),
                "pre_run_check_adapt_ms_mean": sum(x[0] for x in pre["check"]) / max(len(pre["check"]), 1),
                "cells_min": min(cells), "cells_max": max(cells), "cells_mean": sum(cells) / len(cells),
                "refined_base_fraction_mean": (sum(cells) / len(cells) - nbase) / (3.0 * nbase),
                "base_cells_changed_per_step": sum(changes) / len(changes),
                "regrids": regrids, "rk_step_ms": step_ms / args.steps,
                "adapt_ms": adapt_ms / args.steps, "adapt_share": adapt_ms / (step_ms + adapt_ms),
                "slope_limited_fraction": float(cnt[0]) / passes,
                "positivity_limited_fraction": float(cnt[1]) / passes,
                "mass_drift_rel_over_timed_steps": float(abs(t_end[0] - t_start[0]) / abs(t_start[0])),
                "energy_drift_rel_over_timed_steps": float(abs(t_end[-1] - t_start[-1]) / abs(t_start[-1]))}
        # end to end through the C ABI: each step's input state from pinned host
        # memory, the adapted state back to it
        Wh = torch.empty(2 * W.numel(), dtype=W.dtype).pin_memory()
        Wh[:W.numel()].copy_(W.view(-1))
        moved = 0
        torch.cuda.synchronize()
        ranks.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            n_in = W.numel()
            W.view(-1).copy_(Wh[:n_in], non_blocking=True)
            W, _, _ = one_step(W)
            assert W.numel() <= Wh.numel()
            Wh[:W.numel()].copy_(W.view(-1), non_blocking=True)
            moved += (n_in + W.numel()) * W.element_size()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = ranks.max(e0.elapsed_time(e1))
        # kernels of the adaptation: criterion + buffer + 3 scan passes per
        # step, cells + neighbours + 3 scan passes + projection + faces per regrid
        extra = 5 * args.steps + 7 * regrids
        results[precision] = dict(solver=s, ms=ms, ms_e2e=ms_e2e, prof=prof, clocks=clk.summary(),
                                  state_bytes=moved // (2 * args.steps), n_cells=sum(cells) / len(cells),
                                  tiles=None, diag=diag, extra_launches=extra)
        del W, W0, Wh
    return results


def cpu_baseline_kh(max_seconds=20.0, n_base=64):
    """The oracle on a bounded sample of the adaptive KH run: a 64^2 base grid
    (same k, RK order, limiters, adaptation after every step)."""
    from oracle import pyoracle as O
    from paper_1506_06140_gb300 import workloads as wl
    wk = WORKLOADS["kh2d_amr"]

    def make(boxes):
        return O.Oracle(2, [n_base, n_base], [0.0, 0.0], [1.0, 1.0], wk["k"], 1.4, refine_boxes=boxes,
                        rk_order=wk["rk"], cfl=CFL, limiter=O.LIM_CHARACTERISTIC, positivity=True)
    o = make([])
    W = o.limit(o.project(wl.kelvin_helmholtz(o.quad_points())))
    t0 = time.perf_counter()
    steps, dof = 0, 0
    while time.perf_counter() - t0 < max_seconds / 2 and steps < 200:
        dof += o.n_cells * N_BASIS * wk["stages"]
        W, _ = o.rk_step(W, 0.0)
        flags = o.adapt_flags(W, wk["w_t"], wk["alpha"])
        boxes = [[b % n_base, b // n_base] * 2 for b in np.nonzero(flags)[0]]
        o1 = make(boxes)
        W, o = o1.adapt_project(o, W), o1
        steps += 1
    sec = time.perf_counter() - t0
    return {"value": dof / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d adaptive steps (RK4 step + adaptation) of the KH run on a %d^2 base grid, k=3, "
                      "characteristic + positivity limiters (single-threaded FP64 C++ oracle)"
                      % (steps, n_base), "seconds": sec}


def summarize(args, results, world):
    hbm, peak_kind = peaks()
    wk = WORKLOADS[args.workload]
    dim, k, stages = wk["dim"], wk["k"], wk["stages"]
    basis = wk.get("basis", "total")
    N, _, _, nv = shape(dim, k, basis)
    lines = {}
    for precision, r in results.items():
        cells = r["n_cells"]
        dof_updates = world * cells * N * stages * args.steps
        value = dof_updates / (r["ms"] * 1e-3)
        prof = r["prof"]
        launches = sum(c for c, _ in prof.values()) + r.get("extra_launches", 0)
        # roofline of the dominant kernel of the timed region
        kind = max(prof, key=lambda kk: prof[kk][1])
        n_launch, kms = prof[kind]
        avg_s = kms / max(n_launch, 1) * 1e-3
        esize = 8 if precision in ("fp64", "mixed", "mixed_tc") else 4
        kname = {"cell": "cell_update_kernel", "face": "face_flux_kernel",
                 "limit": "limit_kernel"}.get(kind, kind)
        if precision in ("mixed", "mixed_tc") and kind in ("cell", "face"):
            kname = kind == "cell" and "cell_update_mixed_kernel" or "face_flux_mixed_kernel"
        if precision in ("fp32_tc", "mixed_tc") and kind == "cell":
            kname = "cell_tc_kernel"
        tag = "%s_%s" % (wk["tag"], precision)
        if precision == "fp64" and kind in ("cell", "face"):
            fc, ff = kernel_flops(dim, k, basis, moments=(dim == 3 or precision == "fp64"))
            fl = fc * cells if kind == "cell" else ff * dim * cells
            achieved = fl / avg_s / 1e12
            roof = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                    "peak_source": "FP64 rate from unit counts and max clock (152 SMs x 2 DFMA/clk "
                                   "x 2 flop x 2.07 GHz); measured probe 1.198",
                    "traffic": dram_traffic(kname, tag), "algorithmic_per_launch": fl,
                    "algorithmic_unit": "flop (sum-factorised count of kernel_flops)"}
            if kind == "cell":
                # the same launch against the HBM roof (3 state arrays per stage)
                byt = 3 * state_bytes_per_cell(dim, k, esize, basis) * cells
                roof["hbm"] = {"achieved": byt / avg_s / 1e9, "peak": hbm, "unit": "GB/s",
                               "frac": byt / avg_s / 1e9 / hbm, "peak_source": peak_kind,
                               "algorithmic_per_launch": byt}
        else:
            # HBM: a launch of the dominant kernel processes one stage of the mesh,
            # whose algorithmic traffic is 3 state arrays (read U_i and w^n, write U_i+1)
            byt = 3 * state_bytes_per_cell(dim, k, esize, basis) * cells
            if precision in ("mixed", "mixed_tc"):
                # FP64 state read, FP32 delta registers read and written
                byt = (state_bytes_per_cell(dim, k, 8, basis) + 2 * state_bytes_per_cell(dim, k, 4, basis)) * cells
            achieved = byt / avg_s / 1e9
            roof = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm,
                    "unit": "GB/s", "frac": achieved / hbm, "peak_source": peak_kind,
                    "traffic": dram_traffic(kname, tag), "algorithmic_per_launch": byt,
                    "algorithmic_unit": "bytes (FP64 state + 2 FP32 delta registers per stage)"
                    if precision in ("mixed", "mixed_tc") else "bytes (3 state arrays per stage)"}
        if roof["unit"] == "GB/s" or "hbm" in roof:
            # the whole stage against the HBM roof: algorithmic bytes of one
            # stage over the measured time per stage (every kernel and gap)
            byt_stage = 3 * state_bytes_per_cell(dim, k, esize, basis) * cells
            if precision in ("mixed", "mixed_tc"):
                byt_stage = (state_bytes_per_cell(dim, k, 8, basis) + 2 * state_bytes_per_cell(dim, k, 4, basis)) * cells
            t_stage = r["ms"] / args.steps / stages * 1e-3
            roof["stage"] = {"achieved": byt_stage / t_stage / 1e9, "peak": hbm, "unit": "GB/s",
                             "frac": byt_stage / t_stage / 1e9 / hbm,
                             "note": "algorithmic bytes of a stage over the time per stage of the timed steps"}
        e2e_value = dof_updates / (r["ms_e2e"] * 1e-3)
        lines[precision] = {
            "value": value, "ms_per_step": r["ms"] / args.steps, "roofline": roof,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": r["state_bytes"],
                    "d2h_bytes_per_step": r["state_bytes"]},
            "gpu_launches": launches, "clocks": r["clocks"],
            "kernel_ms": {kk: v[1] for kk, v in prof.items()},
            "cells": cells,
        }
        if r.get("diag"):
            lines[precision]["diagnostics"] = r["diag"]
        if r.get("paths"):
            lines[precision]["advance_paths"] = r["paths"]
        if r.get("tiles"):
            t = dict(r["tiles"])
            t["fixed_tile_value"] = dof_updates / (t.pop("fixed_tile_ms") * 1e-3)
            t["unit"] = "[cells per block of the cell kernel, faces per block of the face kernel]"
            lines[precision]["tiles"] = t
    return lines


def run_adjoint(args):
    """Gradient of an L2 density misfit after N frozen-dt RK3 steps of the 3D
    acoustic wave (128^3, k=2) with respect to the initial weights, by the
    per-step checkpointed adjoint, against a central finite difference."""
    import torch
    from paper_1506_06140_gb300 import dg
    from paper_1506_06140_gb300 import workloads as wl
    from paper_1506_06140_gb300.autograd import rk_steps
    torch.cuda.set_device(0)
    n, k, steps = args.size, 2, args.steps
    m = wl.mesh_uniform(3, [n] * 3, [0.0] * 3, [1.0] * 3)
    s = dg.Solver(m, k, 1.4, rk_order=3, cfl=CFL)
    W0 = s.project(torch.as_tensor(wl.acoustic3d(s.quad_points().cpu().numpy())))
    dt = s.compute_dt(W0).item()
    g = torch.Generator(device="cuda").manual_seed(1506062)
    target = W0[0] + 1e-4 * torch.randn(W0[0].shape, generator=g, device="cuda", dtype=W0.dtype)
    vol = (1.0 / n) ** 3

    def J(W):
        WN = rk_steps(W, s, steps, dt)
        return 0.5 * vol * ((WN[0] - target) ** 2).sum()

    st = torch.cuda.current_stream()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    # untimed warm-up passes: module loading and the allocator's checkpoint blocks
    for _ in range(min(args.warmup, 1)):
        Ww = W0.clone().requires_grad_(True)
        J(Ww).backward()
        del Ww
    W = W0.clone().requires_grad_(True)
    torch.cuda.synchronize()
    e[0].record(st)
    val = J(W)
    e[1].record(st)
    val.backward()
    e[2].record(st)
    torch.cuda.synchronize()
    fwd_ms, bwd_ms = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    grad = W.grad.detach()
    W.grad = None
    g2 = torch.Generator(device="cuda").manual_seed(1506063)
    v = torch.randn(W0.shape, generator=g2, device="cuda", dtype=W0.dtype)
    v /= v.norm()
    dJ = (grad * v).sum().item()
    res = {}
    with torch.no_grad():
        for rel in (1e-3, 1e-4, 1e-5):
            eps = rel * W0.abs().max().item()
            fd = (J(W0 + eps * v).item() - J(W0 - eps * v).item()) / (2 * eps)
            res["%g" % rel] = abs(fd - dJ) / abs(dJ)
    cells = s.n_cells
    value = cells * s.N * 3 * steps / (fwd_ms * 1e-3)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps,
           "warmup": min(args.warmup, 1), "ms_per_step": fwd_ms / steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "adjoint: 3D acoustic wave %d^3 periodic, k=2, SSP-RK3, %d steps "
                                  "with frozen dt, L2 density misfit, checkpoint per step" % (n, steps),
                      "cells": cells, "dt": dt},
           "adjoint": {"forward_ms_per_step": fwd_ms / steps, "backward_ms_per_step": bwd_ms / steps,
                       "checkpoint_bytes": steps * W0.numel() * W0.element_size(),
                       "max_memory_allocated_bytes": torch.cuda.max_memory_allocated(),
                       "grad_rel_err_vs_central_fd": res,
                       "fd": "central differences of J along one seeded unit direction (rng 1506063), "
                             "eps = rel * max|W0| for each rel",
                       "J": val.item()}}
    print(json.dumps(out), flush=True)
    return 0


L1_SIZES = (64, 128, 256)
L1_T_END = 2.0
L1_EQUAL_TOL = 1.05  # "equal" L1: within 5% of the FP64 error
L1_CHUNK = 100  # steps per graph launch in the L1 ladder


def l1_ladder(precisions, sizes, t_end, verbose=False, basis="total"):
    """L1 density error of the vortex against its closed form after t_end
    (fixed timestep: the CFL value of the initial state, rounded so that
    t_end is reached exactly), per precision and resolution, with the device
    time per RK stage measured by CUDA events around the steps (run as
    dg_advance_dt graphs of L1_CHUNK steps, recorded before the timed run).
    With the tensor-product basis the rows' precision reads
    "tensor_<precision>"."""
    import torch
    from paper_1506_06140_gb300 import dg
    from paper_1506_06140_gb300 import workloads as wl
    rows = []
    for precision in precisions:
        for n in sizes:
            s = dg.Solver(mesh(n), K_DEG, 1.4, rk_order=RK_ORDER, cfl=CFL, precision=precision, basis=basis)
            W = s.project(torch.as_tensor(wl.vortex(s.quad_points().cpu().numpy())))
            dt = s.compute_dt(W).item()  # the vortex translates; its CFL timestep stays put
            nsteps = int(math.ceil(t_end / dt))
            dt = t_end / nsteps
            chunks = [L1_CHUNK] * (nsteps // L1_CHUNK) + ([nsteps % L1_CHUNK] if nsteps % L1_CHUNK else [])
            W0 = W.clone()
            for c in sorted(set(chunks)):  # record the graphs (keyed by W, steps, dt)
                s.advance(W, c, dt=dt)
            W.copy_(W0)
            st = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            for c in chunks:
                s.advance(W, c, dt=dt)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            rho_ex = wl.vortex(s.l1_points().cpu().numpy(), t=t_end)[0]
            l1 = s.l1_density(W, torch.as_tensor(rho_ex)).item()
            rows.append({"precision": precision if basis == "total" else "%s_%s" % (basis, precision),
                         "n": n, "steps": nsteps, "L1": l1, "ms_per_stage": ms / (nsteps * STAGES),
                         "dof_updates_per_s": n * n * s.N * STAGES * nsteps / (ms * 1e-3)})
            if verbose:
                print(json.dumps(rows[-1]), flush=True)
            del s, W
    return rows


def equal_l1(rows, tol=L1_EQUAL_TOL):
    """For every FP64 rung of the ladder (its L1 error is the target) and
    every other precision: the coarsest resolution at which that precision's
    L1 error is within tol of the target (the cheapest run that reaches it),
    its device time per RK stage and for the whole run to t_end, and the FP64
    times over them (> 1: faster at equal error); None where no resolution of
    the ladder reaches the target."""
    ref = {r["n"]: r for r in rows if r["precision"] == "fp64"}
    out = []
    for n, r64 in sorted(ref.items()):
        run64 = r64["ms_per_stage"] * r64["steps"] * STAGES
        entry = {"fp64_n": n, "target_L1": r64["L1"], "fp64_ms_per_stage": r64["ms_per_stage"],
                 "fp64_run_ms": run64}
        for p in sorted({r["precision"] for r in rows} - {"fp64"}):
            ok = sorted((r for r in rows if r["precision"] == p and r["L1"] <= tol * r64["L1"]),
                        key=lambda r: r["n"])
            if ok:
                b = ok[0]
                run = b["ms_per_stage"] * b["steps"] * STAGES
                entry[p] = {"n": b["n"], "L1": b["L1"], "ms_per_stage": b["ms_per_stage"], "run_ms": run,
                            "stage_speedup_vs_fp64": r64["ms_per_stage"] / b["ms_per_stage"],
                            "run_speedup_vs_fp64": run64 / run}
            else:
                entry[p] = None
        out.append(entry)
    return out


def run_l1_study(args):
    """L1 density error of the vortex against its closed form after t_end,
    per precision and resolution (32^2 ... 256^2), with the device time per
    RK stage: the data for comparing precisions at equal L1 error."""
    import torch
    torch.cuda.set_device(0)
    precisions = (("fp64", "fp32", "fp32_tc", "mixed", "mixed_tc") if args.precision == "both"
                  else (args.precision,))
    rows = l1_ladder(precisions, (32,) + L1_SIZES, args.t_end, verbose=True)
    out = {"metric": "L1 density error vs closed form and DOF-updates/s per RK stage",
           "config": {"workload": "isentropic vortex k=3 SSP-RK4 CFL 0.2 to t=%g" % args.t_end},
           "rows": rows, "equal_l1": equal_l1(rows)}
    print(json.dumps(out), flush=True)
    return 0


def run_square_growth(args):
    """Square advection (64^2, v=(100,50)): L1 density error against the
    translated initial state over time for DG-2 (k=1, SSP-RK2) and DG-3 (k=2,
    SSP-RK3) with the characteristic limiter, the power law of its growth, and
    the graph-replay step rate (FP64)."""
    import torch
    from paper_1506_06140_gb300 import dg
    from paper_1506_06140_gb300 import workloads as wl
    torch.cuda.set_device(0)
    m = wl.mesh_uniform(2, [64, 64], [0.0, 0.0], [1.0, 1.0])
    chunk = 1000
    out = {"metric": "square advection: L1 density error vs time and step rate",
           "config": {"workload": WORKLOADS["square64"]["name"], "t_end": args.t_end}, "runs": []}
    for k, rk in ((1, 2), (2, 3)):
        s = dg.Solver(m, k, 1.4, rk_order=rk, cfl=CFL, limiter="characteristic", precision="fp64")
        W = s.project(torch.as_tensor(wl.square2d(s.quad_points().cpu().numpy())))
        s.limit(W)
        xyz1 = s.l1_points().cpu().numpy()
        hist = s.dt_buffer(chunk)
        s.advance(W.clone(), chunk, hist)  # records the graph
        t, steps, rows, ms = 0.0, 0, [], 0.0
        marks = [x for x in (0.01, 0.02, 0.05, 0.1, 0.2, 0.5, 1.0, 2.0, 5.0, 10.0) if x <= args.t_end]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for mark in marks:
            while t < mark:
                e0.record()
                s.advance(W, chunk, hist)
                e1.record()
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
                t += hist.sum().item()
                steps += chunk
            l1 = s.l1_density(W, torch.as_tensor(wl.square2d(xyz1, t=t)[0])).item()
            rows.append({"t": t, "steps": steps, "L1": l1})
        late = [r for r in rows if r["t"] >= 0.1]
        alpha = None
        if len(late) >= 2:
            x = np.log([r["t"] for r in late])
            y = np.log([r["L1"] for r in late])
            alpha = float(np.polyfit(x, y, 1)[0])
        run = {"k": k, "rk_order": rk, "rows": rows, "growth_exponent": alpha,
               "us_per_step": 1e3 * ms / steps, "steps_per_s": steps / (ms * 1e-3)}
        out["runs"].append(run)
        print(json.dumps(run), flush=True)
    print(json.dumps(out), flush=True)
    return 0


def run_sedov_taylor(args):
    """Sedov-Taylor blast of Sec. 5.3 at the paper's resolution: 64^3 cells in
    [0,1]^3, rho = 1, p = 1e-6, gamma = 5/3, E = 1 in the eight central
    cells, DG-2 and DG-3 with the characteristic TVB and positivity limiters
    (FP64 state, FP32 perturbation-form right-hand side), run to t = 0.05; shock front against R_0 (E t^2 / rho)^(1/5)
    with the printed R_0 ~ 1.152 (0.3477 at t = 0.05)."""
    import torch
    from paper_1506_06140_gb300 import dg
    from paper_1506_06140_gb300 import workloads as wl
    torch.cuda.set_device(0)
    n, gamma, t_end = 64, 5.0 / 3.0, 0.05
    r_exact = 1.152 * (t_end ** 2) ** 0.2
    m = wl.mesh_uniform(3, [n] * 3, [0.0] * 3, [1.0] * 3, bc=[wl.BC_TRANSMISSIVE] * 3)
    out = {"metric": "Sedov-Taylor shock radius at t = 0.05 and step rate",
           "config": {"workload": "Sedov-Taylor 3D, 64^3, rho 1, p 1e-6, gamma 5/3, E 1 in the 8 central cells, "
                                  "characteristic TVB + positivity limiters, FP64 state with the FP32 perturbation-form "
                                  "right-hand side (mixed), CFL 0.2", "t_end": t_end,
                      "analytic_radius": r_exact}, "runs": []}
    for k, rk in ((1, 2), (2, 3)):
        s = dg.Solver(m, k, gamma, rk_order=rk, cfl=CFL, limiter="characteristic", positivity=True,
                      precision="mixed")
        W = s.project(torch.as_tensor(wl.sedov3d(s.quad_points().cpu().numpy(), gamma=gamma, p0=1e-6,
                                                 energy=1.0, half_width=1.0 / n)))
        s.limit(W)
        tot0 = s.totals(W).cpu().numpy()
        chunk, t, steps, last, ms = 200, 0.0, 0, 0.0, 0.0
        hist = s.dt_buffer(chunk)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        while t + 1.5 * chunk * last < t_end:
            e0.record()
            s.advance(W, chunk, hist)
            e1.record()
            h = hist.cpu().numpy()
            ms += e0.elapsed_time(e1)
            t += h.sum()
            last = h[-1]
            steps += chunk
        graph_steps = steps
        dt_buf = s.scalar()
        while t < t_end - 1e-15:
            s.compute_dt(W, dt_buf)
            dt = min(dt_buf.item(), t_end - t)
            s.rk_step(W, dt)
            t += dt
            steps += 1
        c = s.quad_points().mean(dim=1).cpu().numpy()
        r = np.sqrt(((c - 0.5) ** 2).sum(axis=0))
        rho = W[0, 0].double().cpu().numpy()
        dr = 0.5 / n
        b = (r / dr).astype(int)
        prof = np.bincount(b, weights=rho) / np.maximum(np.bincount(b), 1)
        ip = int(np.argmax(prof))
        half = 1.0 + 0.5 * (prof[ip] - 1.0)
        o = ip + int(np.argmax(prof[ip:] < half))
        front = (o - 0.5) * dr + dr * (prof[o - 1] - half) / (prof[o - 1] - prof[o])
        tot1 = s.totals(W).cpu().numpy()
        run = {"dg": k + 1, "steps": steps, "front_radius": float(front), "peak_radius": float((ip + 0.5) * dr),
               "front_rel_err": float(front / r_exact - 1.0), "peak_compression": float(prof[ip]),
               "mass_drift_rel": float(abs(tot1[0] - tot0[0]) / tot0[0]),
               "energy_drift_rel": float(abs(tot1[-1] - tot0[-1]) / tot0[-1]),
               "status": s.status(),
               "graph_ms_per_step": ms / max(graph_steps, 1),
               "dof_updates_per_s": s.n_cells * s.N * rk * graph_steps / (ms * 1e-3) if ms > 0 else None}
        out["runs"].append(run)
        print(json.dumps(run), flush=True)
    print(json.dumps(out), flush=True)
    return 0


def host_cpu():
    """(threads available to this process, CPU model name) of the host."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu model")):
                model = ln.split(":", 1)[1].strip()
                break
    return cores, model or "unknown"


def oracle_vortex_rate(n_sample, threads, max_seconds, max_steps):
    """RK4 steps of the vortex on an n_sample^2 periodic box with the bench's
    cell size, timed on the oracle with `threads` OpenMP threads."""
    from oracle import pyoracle as O
    from paper_1506_06140_gb300 import workloads as wl
    half = 5.0 * n_sample / N_CELLS_1D
    m = mesh(n_sample, half)
    o = O.Oracle(2, m["n"], m["lo"], m["hi"], K_DEG, 1.4, rk_order=RK_ORDER, cfl=CFL)
    o.set_threads(threads)
    W = o.project(wl.vortex(o.quad_points()))
    t0 = time.perf_counter()
    steps = 0
    while True:
        W, _ = o.rk_step(W, 0.0)
        steps += 1
        if time.perf_counter() - t0 > max_seconds or steps >= max_steps:
            break
    sec = time.perf_counter() - t0
    return n_sample ** 2 * N_BASIS * STAGES * steps / sec, steps, sec


def cpu_baseline(max_seconds=10.0):
    """The oracle, as it stands, on the host cores: all cores on the bench's
    own 256^2 workload (the right-hand side in its gather form, one OpenMP
    thread per core), and one core on a 128^2 box with the same cell size."""
    cores, model = host_cpu()
    v_all, s_all, t_all = oracle_vortex_rate(N_CELLS_1D, cores, max_seconds, 400)
    v_one, s_one, t_one = oracle_vortex_rate(128, 1, max_seconds, 50)
    return {"value": v_all, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": model,
            "sample": "%d RK4 steps of the 256x256 vortex, k=3 (FP64 C++ oracle, right-hand side "
                      "cell by cell on %d OpenMP threads)" % (s_all, cores),
            "seconds": t_all,
            "single_thread": {"value": v_one, "unit": UNIT, "cores": 1,
                              "sample": "%d RK4 steps of the vortex on a 128x128 periodic box with the "
                                        "same cell size, k=3 (serial oracle)" % s_one,
                              "seconds": t_one}}


def reference_arm(args, rank, world):
    """--impl reference: the oracle timed on all host cores (rank 0 only),
    each step one RK4 step of the bench's 256^2 vortex."""
    if rank != 0:
        return 0
    from oracle import pyoracle as O
    from paper_1506_06140_gb300 import workloads as wl
    cores, model = host_cpu()
    m = mesh()
    o = O.Oracle(2, m["n"], m["lo"], m["hi"], K_DEG, 1.4, rk_order=RK_ORDER, cfl=CFL)
    o.set_threads(cores)
    W = o.project(wl.vortex(o.quad_points()))
    for _ in range(args.warmup):
        W, _ = o.rk_step(W, 0.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        W, _ = o.rk_step(W, 0.0)
    sec = time.perf_counter() - t0
    value = N_CELLS_1D ** 2 * N_BASIS * STAGES * args.steps / sec
    sample = ("each step: one RK4 step of the 256x256 vortex, k=3 (FP64 C++ oracle, right-hand side "
              "cell by cell on %d OpenMP threads)" % cores)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config("vortex", "fp64", N_CELLS_1D ** 2),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "cpu_model": model, "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-l1", action="store_true", help="vortex: skip the L1 / equal-L1 study")
    ap.add_argument("--precision", default="both",
                    choices=["both", "fp64", "fp32", "fp32_tc", "mixed", "mixed_tc"],
                    help="run one precision only (profiling); the JSON line needs both")
    ap.add_argument("--workload", default="vortex",
                    choices=sorted(WORKLOADS) + ["adjoint3d", "l1study", "square_growth", "sedov_taylor"])
    ap.add_argument("--t-end", type=float, default=2.0, help="l1study, square_growth: final time")
    ap.add_argument("--size", type=int, default=128, help="adjoint3d: cells per axis")
    args = ap.parse_args()
    if args.workload in ("adjoint3d", "l1study", "square_growth", "sedov_taylor"):
        from paper_1506_06140_gb300 import build
        build.build()
        if args.workload == "adjoint3d":
            return run_adjoint(args)
        if args.workload == "sedov_taylor":
            return run_sedov_taylor(args)
        return run_l1_study(args) if args.workload == "l1study" else run_square_growth(args)
    wprec = WORKLOADS[args.workload]["precisions"]
    args.precisions = wprec if args.precision == "both" else (args.precision,)
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    from paper_1506_06140_gb300 import build
    if rank == 0 or not os.path.exists(build.LIB):
        build.build()
    amr = WORKLOADS[args.workload].get("amr", False)
    results = (run_gpu_amr if amr else run_gpu)(args, rank, world, local_rank)
    if rank != 0:
        return 0
    lines = summarize(args, results, world)
    if args.workload != "vortex" and len(lines) > 1:
        head_p = args.precisions[0]
        head = lines[head_p]
        out = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "config": workload_config(args.workload, head_p, head["cells"]),
               "diagnostics": head.get("diagnostics")}
        out.update({kk: head[kk] for kk in ("roofline", "e2e", "gpu_launches", "clocks", "kernel_ms")})
        out["variants"] = {p: {kk: lines[p][kk] for kk in ("value", "ms_per_step", "roofline", "e2e",
                                                           "gpu_launches", "clocks", "kernel_ms")}
                           for p in args.precisions[1:]}
        for p in args.precisions[1:]:
            out["variants"][p]["diagnostics"] = lines[p].get("diagnostics")
        if args.workload == "vortex_tensor" and not args.no_l1:
            # accuracy against the paper's total-degree basis at FP64: L1 errors
            # on the ladder and the comparison at equal L1 error
            rows = l1_ladder(["fp64"], L1_SIZES, L1_T_END) + \
                l1_ladder([p for p in ("fp64", "fp32") if p in lines], L1_SIZES, L1_T_END, basis="tensor")
            at_n = {r["precision"]: r for r in rows if r["n"] == N_CELLS_1D}
            out["l1"] = at_n["tensor_fp64"]["L1"]
            for p in out["variants"]:
                out["variants"][p]["l1"] = at_n["tensor_" + p]["L1"]
            out["equal_l1"] = {"t_end": L1_T_END, "tol": L1_EQUAL_TOL,
                               "definition": "L1 density error against the closed-form vortex (Sec. 5.1) "
                                             "after t_end with a fixed timestep; \"fp64\" rows: the paper's "
                                             "total-degree basis (10 coeffs), \"tensor_*\" rows: Q_3 (16 "
                                             "coeffs); per total-degree FP64 rung the coarsest resolution "
                                             "where each tensor variant is within tol of its error, and the "
                                             "total-degree FP64 times over the variant's",
                               "ladder": rows, "comparison": equal_l1(rows)}
            out["config"]["l1"] = ("L1 density error after t=%g with a fixed timestep on the %s ladder "
                                   "(\"l1\" and variants' \"l1\": at 256^2)"
                                   % (L1_T_END, "/".join("%d^2" % n for n in L1_SIZES)))
        if amr and world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_kh()
        print(json.dumps(out), flush=True)
        return 0
    if args.workload != "vortex" or len(lines) == 1:
        prec = args.precisions[0]
        one = lines[prec]
        out = {"metric": METRIC, "value": one["value"], "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": one["ms_per_step"],
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": {"fp64": "f64", "mixed": "f32/f64", "mixed_tc": "f32/f64"}.get(prec, "f32"),
               "data": "synthetic",
               "config": workload_config(args.workload, prec, one["cells"])}
        if "tiles" in one:
            out["config"]["tiles"] = one["tiles"]
        out.update({kk: one[kk] for kk in ("roofline", "e2e", "gpu_launches", "clocks", "kernel_ms")})
        if "diagnostics" in one:
            out["diagnostics"] = one["diagnostics"]
        if "advance_paths" in one:
            out["advance_paths"] = one["advance_paths"]
        print(json.dumps(out), flush=True)
        return 0
    head = lines["fp64"]
    out = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config("vortex", "fp64", head["cells"]),
           "roofline": head["roofline"], "e2e": head["e2e"], "gpu_launches": head["gpu_launches"],
           "clocks": head["clocks"], "kernel_ms": head["kernel_ms"],
           "variants": {p: {k: lines[p][k] for k in
                            ("value", "ms_per_step", "roofline", "e2e", "gpu_launches",
                             "clocks", "kernel_ms")} for p in ("fp32", "fp32_tc", "mixed", "mixed_tc")
                         if p in lines}}
    if not args.no_l1:
        # accuracy of every variant (vortex against its closed form after
        # t = 2 on the 64^2 ... 256^2 ladder) and the comparison at equal L1 error
        rows = l1_ladder([p for p in ("fp64", "fp32", "fp32_tc", "mixed", "mixed_tc") if p in lines],
                         L1_SIZES, L1_T_END)
        at_n = {r["precision"]: r for r in rows if r["n"] == N_CELLS_1D}
        out["l1"] = at_n["fp64"]["L1"]
        for p in out["variants"]:
            out["variants"][p]["l1"] = at_n[p]["L1"]
        out["equal_l1"] = {"t_end": L1_T_END, "tol": L1_EQUAL_TOL,
                           "definition": "L1 density error against the closed-form vortex (Sec. 5.1) after "
                                         "t_end with a fixed timestep; per FP64 rung the coarsest resolution "
                                         "where each precision is within tol of the FP64 error, its device "
                                         "time per RK stage and for the run to t_end, and the FP64 times "
                                         "over them",
                           "ladder": rows, "comparison": equal_l1(rows)}
        out["config"]["l1"] = ("L1 density error after t=%g with a fixed timestep on the %s ladder "
                               "(\"l1\" and variants' \"l1\": at 256^2)"
                               % (L1_T_END, "/".join("%d^2" % n for n in L1_SIZES)))
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
