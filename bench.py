#!/usr/bin/env python
"""Benchmark of the MCD pressure-Poisson hot path on one GB300 per rank.

Workload (the metric's): the oscillating-cylinder moving-boundary problem
(2D unit box, 1024x1024 background mesh, rigid cylinder D = 0.1 oscillating
along x with KC = 5, Re = 100, fluid at rest at t = 0; Dirichlet p = 0 on
the box walls, Neumann dP/dn = -dV/dt . n on the body).  One step is one
full moving-boundary fractional step through the C ABI (mcd_flow_step):
    DP update (remask + 10 relaxation sweeps in the 5 l0 band)
    -> ALE interpolation of u, v and of the pressure guess (Appendix A)
    -> velocity and pressure MLS stencils (FP64 rows + FP32 copy)
    -> u* and the PPE source (1/dt) div u*
    -> learned warm start: the ALE pressure guess corrected by the bf16
       convolutional network (trained, untimed, on the run's first 500 steps)
       along its residual-minimising step
    -> mixed-precision Bi-CGSTAB to ||b - A p|| <= 1e-8 ||b|| (FP64 residual)
    -> projection and fluid force.
Metric: DP-unknowns (non-void DPs) solved per second.  The same steps are
also run with the plain FP64 Bi-CGSTAB from the same ALE guess
(`fp64_plain`) and with the mixed solve without the network
(`mixed_no_net`); `e2e` reads the pressure back to host memory each step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --workload spmv | tgv | poisson3d | batched | cnn | array | flow

Multi-GPU: replicas only (each rank runs its own instance; no data-path
collective; max-over-ranks timing).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DP-unknowns solved/s at rel.res 1e-8: learned+mixed vs plain FP64, same GB300"
UNIT = "DP-unknowns/s"
HBM_FALLBACK_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mcd", choices=["mcd", "reference"])
    ap.add_argument("--workload", default="cylinder", choices=["cylinder", "batched", "cnn", "array", "flow", "spmv", "tgv", "poisson3d"],
                    help="cylinder: the 1024^2 moving-cylinder step (the metric's workload); "
                         "batched: 256 independent Poisson systems of log-uniform size 32^2..512^2; "
                         "cnn: the warm-start network's inference and training step on an n^2 grid; "
                         "array: the 25-cylinder array (multiple stationary cylinders), 3x3 against "
                         "the expanded 9x9 stencil, on an n^2 grid (n = 128 is the paper's l0); "
                         "flow: full moving-boundary fractional steps (DP update, ALE interpolation, "
                         "stencils, predict, PPE, projection, fluid force) of the oscillating cylinder; "
                         "spmv: the stencil SpMV (mcd_apply_laplacian, FP32 and FP64) on an n^2 jittered "
                         "box whose rows and vectors exceed L2 (default n = 4096), and the persistent "
                         "solve at 2048^2; tgv: the periodic Taylor-Green vortex, 512^2, 200 fractional "
                         "steps, mixed against FP64, error against the closed form; poisson3d: the 128^3 "
                         "manufactured Dirichlet problem (27-point stencils), mixed against FP64")
    ap.add_argument("--profile-solve", action="store_true",
                    help="run one mixed solve of the cylinder system from p = 0 (for a profiler) "
                         "and print its iteration count")
    ap.add_argument("--trace-solve", action="store_true",
                    help="one traced mixed cylinder solve at --n: per-phase and grid-barrier stage "
                         "times from the device timestamps (medians, us)")
    ap.add_argument("--n", type=int, default=None,
                    help="background mesh cells per side (default: 1024; spmv 4096, tgv 512, poisson3d 128)")
    ap.add_argument("--bodies", default="cylinder", choices=["cylinder", "passing", "passing-sdf", "wing"],
                    help="with --workload flow: the oscillating cylinder, the two cylinders passing "
                         "each other (analytic circles, or circles given as discrete SDF grids), or the "
                         "flapping elliptic wing (a rotating SDF body)")
    ap.add_argument("--t0", type=float, default=None,
                    help="with --workload flow: start time (the flow starts at rest); default 0 for the "
                         "cylinder, 3T - 0.5 (just before the passing cylinders meet) for passing")
    ap.add_argument("--support", type=int, default=1, choices=[1, 4],
                    help="with --profile-solve --workload array: 1 = 3x3 stencil, 4 = 9x9 stencil")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--update-restart", type=int, default=0, choices=[0, 1],
                    help="with --profile-solve / --trace-solve: the mixed solve's update schedule "
                         "(0 adaptive, 1 restarting as in the flow step)")
    ap.add_argument("--barriers", type=int, default=0, choices=[0, 1, 2, 3],
                    help="with --profile-solve / --trace-solve: grid barriers per Bi-CGSTAB iteration "
                         "(0: the library default)")
    ap.add_argument("--tilings", action="store_true",
                    help="with --workload batched: time every tiling (rows x CTAs per SM) in both precisions, "
                         "one JSON line each, instead of the bench line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="time the mixed solve without the network")
    ap.add_argument("--train-steps", type=int, default=500, help="steps whose solves train the network")
    ap.add_argument("--total-steps", type=int, default=2000,
                    help="headline: length of the run over which the --steps timed steps are spread")
    ap.add_argument("--train-epochs", type=int, default=10)
    ap.add_argument("--tgv-steps", type=int, default=200, help="with --workload tgv: fractional steps per arm")
    a = ap.parse_args()
    if a.n is None:
        a.n = {"spmv": 4096, "tgv": 512, "poisson3d": 128}.get(a.workload, 1024)
    return a


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs"), "measured"
    return HBM_FALLBACK_GBS, "fallback"


def traffic_source_sha(kernel):
    """sha256[:16] of the kernel's translation unit: its .cu file and the
    csrc headers it includes."""
    csrc = os.path.join(ROOT, "paper_2404_17542_gb300", "csrc")
    files = (["krylov.cu", "krylov_common.cuh", "common.cuh"] if kernel.startswith("bicg")
             else ["stencils.cu", "common.cuh"])
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(kernel):
    """DRAM bytes per unit of work (per DP-iteration for the solve, per DP
    for the build) from the committed ncu summary profiles/traffic.txt, if
    the kernel's source is unchanged since the capture (sha256 of its
    translation unit); None otherwise."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    sha = traffic_source_sha(kernel)
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == kernel and parts[1] == sha:
            return float(parts[3])
    return None


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
class CylinderRun:
    """State of one oscillating-cylinder instance on the device."""

    def __init__(self, n, dev, mcd, inputs, tol, barriers=0, update_restart=0):
        import torch
        self.torch, self.mcd, self.inputs = torch, mcd, inputs
        self.n, self.dev, self.tol, self.barriers = n, dev, tol, barriers
        self.update_restart = update_restart
        pb = inputs.cylinder_box(n)
        self.pb, self.cyl, self.mesh = pb, pb.meta["cylinder"], pb.mesh
        N = self.mesh.N
        self.N = N
        self.dt = 0.2 * self.mesh.l0 / 1.0                 # CFL 0.2 at U = 1
        self.pos = torch.from_numpy(pb.pos.ravel().copy()).to(dev)
        self.mask = torch.from_numpy(pb.mask.copy()).to(dev)
        self.prev = torch.empty_like(self.mask)
        self.normal = torch.zeros(2 * N, dtype=torch.float64, device=dev)
        self.neu = torch.zeros(N, dtype=torch.float64, device=dev)
        self.p = torch.zeros(N, dtype=torch.float64, device=dev)
        self.dprev = torch.zeros(N, dtype=torch.float64, device=dev)   # last increment (network input)
        self.src_host = inputs.ppe_source(pb.pos, 0.0)
        self.rhs = torch.from_numpy(self.src_host.copy()).to(dev)
        c0 = self.cyl.centre(0.0)
        mcd.update_dps(self.mesh, c0, self.cyl.radius, self.cyl.body_id, self.pos, self.mask,
                       self.prev, kappa=0.2, n_relax=30, band=0.0)
        mcd.body_boundary(self.mesh, c0, self.cyl.radius, self.cyl.body_id, self.pos, self.mask,
                          acc=self.cyl.acceleration(0.0), normal=self.normal, neumann=self.neu)
        self.st = mcd.Stencils(self.mesh, self.pos, self.mask, self.normal, bc_kind=pb.bc_kind,
                               precision=mcd.MIXED)
        self.k = 0

    def snapshot(self):
        return (self.pos.clone(), self.mask.clone(), self.p.clone(), self.dprev.clone(), self.k)

    def restore(self, snap):
        pos, mask, p, dprev, k = snap
        self.pos.copy_(pos)
        self.mask.copy_(mask)
        self.p.copy_(p)
        self.dprev.copy_(dprev)
        self.k = k

    def step(self, mode, net=None):
        """One pass of the hot path; returns the solve info.  With a network
        the solve starts from its warm start and updates self.dprev."""
        mcd = self.mcd
        self.k += 1
        t = self.k * self.dt
        c = self.cyl.centre(t)
        mcd.update_dps(self.mesh, c, self.cyl.radius, self.cyl.body_id, self.pos, self.mask,
                       self.prev, kappa=0.2, n_relax=10, band=5.0 * self.mesh.l0)
        mcd.body_boundary(self.mesh, c, self.cyl.radius, self.cyl.body_id, self.pos, self.mask,
                          acc=self.cyl.acceleration(t), normal=self.normal, neumann=self.neu)
        self.st.rebuild(self.pos, self.mask, self.normal)
        _p, info = self.st.solve(self.rhs, self.neu, p=self.p, tol=self.tol, mode=mode, net=net,
                                 dprev=self.dprev if net is not None else None, barriers=self.barriers,
                                 update_restart=self.update_restart)
        return info


class FlowRun:
    """The oscillating-cylinder run of the headline (D = 0.1, KC = 5,
    Re = 100 in the unit box, fluid at rest at t = 0): full moving-boundary
    fractional steps through mcd_flow_step (mcd.AleFlow).  The PPE source is
    the step's own (1/dt) div u*, the Neumann datum -dV/dt . n with dV/dt the
    Eq. (29) difference, and every solve starts from the step-k pressure
    carried to the new DP positions by the ALE interpolation (Eq. (19),
    Appendix A).  dt = min(0.2 l0 / U, 0.2 l0^2 / nu)."""

    def __init__(self, n, dev, mcd, inputs, tol):
        import torch
        self.torch, self.mcd = torch, mcd
        cyl = inputs.Cylinder()
        pb = inputs.cylinder_box(n, cyl)
        self.cyl, self.mesh, self.N, self.n, self.dev = cyl, pb.mesh, pb.mesh.N, n, dev
        D, U = 2 * cyl.radius, 1.0
        self.nu = U * D / 100.0
        self.dt = min(0.2 * pb.mesh.l0 / U, 0.2 * pb.mesh.l0 ** 2 / self.nu)
        self.flow = mcd.AleFlow(pb.mesh, torch.from_numpy(pb.pos.ravel().copy()).to(dev),
                                torch.from_numpy(pb.mask.copy()).to(dev), self.bodies_at, self.nu, self.dt,
                                precision=mcd.MIXED, mode=mcd.MIXED, tol=tol, ale_pressure=True)
        self.dprev = torch.zeros(self.N, dtype=torch.float64, device=dev)   # last increment (network input)
        self.k = 0

    def bodies_at(self, t):
        c = self.cyl
        return [(c.body_id, c.centre(t), c.radius)], [c.velocity(t)]

    def step(self, mode, net=None, precond=None):
        """One step; the solve info (with a network the solve starts from its
        warm start and updates self.dprev; precond: the network applied at
        the restarts of the solve's refinement cycles)."""
        info = self.flow.step(mode=mode, net=net, dprev=self.dprev if net is not None else None,
                              precond=precond)
        self.k += 1
        return info["solve"]

    def snapshot(self):
        return (self.flow.snapshot(), self.dprev.clone(), self.k)

    def restore(self, snap):
        fs, dp, k = snap
        self.flow.restore(fs)
        self.dprev.copy_(dp)
        self.k = k


def train_nets(run, steps, epochs, precond=True, lr=1e-3, seed=3):
    """The networks of the learned part, trained on the first `steps` steps
    of the run (plain mixed solves, untimed).  Each step's system at its ALE
    guess gives one sample per network, target P - guess:
      warm start     features of (b, guess, the last increment);
      preconditioner features of (b, guess) without an increment (the
                     residual -> correction map it applies at the restarts
                     of a solve's refinement cycles).
    Leaves run.dprev set to the last increment.  Returns (net, precond net
    or None, info)."""
    torch, mcd = run.torch, run.mcd
    from paper_2404_17542_gb300 import inputs
    t0 = time.perf_counter()
    # the warm-start network starts as linear extrapolation in time (its
    # output equals its increment channel) and learns corrections to it
    net = mcd.Net(inputs.cnn_flatten(*inputs.cnn_weights_extrapolating(seed)))
    pre = mcd.Net(inputs.cnn_flatten(*inputs.cnn_weights(seed + 1))) if precond else None
    samples, psamples = [], []
    dprev = torch.zeros(run.N, dtype=torch.float64, device=run.dev)
    for k in range(steps):
        run.step(mcd.MIXED)
        st = run.flow.stencils(mcd.FLOW_PRESSURE)
        b = run.flow.array(mcd.FLOW_B)
        guess = run.flow.array(mcd.FLOW_GUESS)
        if k >= 2:
            samples.append(net.features(st, b, guess, dprev, run.flow.P))
            if pre is not None:
                psamples.append(pre.features(st, b, guess, None, run.flow.P))
        dprev = run.flow.P - guess
    run.dprev.copy_(dprev)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    loss = torch.zeros(1, dtype=torch.float64, device=run.dev)
    rng = np.random.default_rng(seed)
    info = {"train_steps": steps, "samples": len(samples), "epochs": epochs, "lr": lr, "data_s": round(t_data, 2)}
    t1 = time.perf_counter()
    for name, nn, S in (("warm_start", net, samples), ("precond", pre, psamples)):
        if nn is None:
            continue
        hist = []
        for ep in range(epochs):
            tot = 0.0
            for i in rng.permutation(len(S)):
                x, tg, wt = S[i]
                nn.train_step(x, tg, wt, run.n, run.n, lr, loss)
                tot += float(loss.item()) if ep in (0, epochs - 1) else 0.0
            if ep in (0, epochs - 1):
                hist.append(tot / max(1, len(S)))
        info[f"{name}_loss_first_epoch"] = hist[0] if hist else None
        info[f"{name}_loss_last_epoch"] = hist[-1] if hist else None
    torch.cuda.synchronize()
    info["train_s"] = round(time.perf_counter() - t1, 2)
    return net, pre, info


def fp64_finish_counts(infos):
    """How many solves finished in FP64 after the FP32 recursion failed, and
    why (mcd_solve_info.fallback: 1 diverged, 2 restarts exhausted, 3 alpha
    not finite or 0, 4 t.t = 0, 5 non-finite dot products, 6 iteration
    limit, 7 other)."""
    codes = [int(i["fallback"]) for i in infos]
    return {"fp64_finishes": sum(1 for c in codes if c),
            "fp64_finish_reasons": {str(c): codes.count(c) for c in sorted(set(codes)) if c}}


def flush_l2(buf):
    buf.zero_()


def timed_step(run, mode, flush_buf, net=None, host_out=None, precond=None):
    """One step bracketed by CUDA events on the current stream, after an L2
    flush (outside the events).  With host_out (pinned) the step's pressure
    is read back inside the timed region.  Returns (ms, solve info)."""
    torch = run.torch
    stream = torch.cuda.current_stream()
    flush_l2(flush_buf)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    info = run.step(mode, net, precond)
    if host_out is not None:
        host_out.copy_(run.flow.P, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), info


# Algorithmic bytes of the persistent Bi-CGSTAB solve per DP and iteration,
# FP32 recursion on 2D 9-point rows, two grid barriers per iteration (the
# kernel the step runs, bicg_persistent2): phase CA reads s, t, p, v (16 B),
# r^ and the double-float correction x, xlo (12 B) and the 9 FP32 weights
# (36 B) and writes x, xlo, r, p, v (20 B); phase B reads r, v, r^ (12 B)
# and the weights (36 B) and writes s, t (8 B): 140 B per DP-iteration.
# Halo re-reads, the phases that restart or replace the recursion and the
# true-residual updates are not counted.  (The one-barrier schedule,
# barriers = 1, moves 96 B: reads r, p, v, u, q, r^, x, xlo and the
# weights, writes r, p, v, u, q, x, xlo.)
# The stencil build reads positions and masks (17 B) and writes FP64 + FP32
# rows, Neumann weights, row scale and kind (206 B).
SOLVE_BYTES_PER_DP_ITER = 140
BUILD_BYTES_PER_DP = 206


def aggregate_ranks(ms, unknowns, world, device):
    """Whole-job figures of N replicas: the slowest rank's timed milliseconds
    (max over ranks) and the unknowns all ranks solved (sum).  Every rank
    gets both.  With one rank, no collective runs."""
    if world == 1:
        return float(ms), float(unknowns)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(unknowns)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def gpu_arm(args):
    """The headline: the oscillating cylinder at --n (1024^2).  Steps
    1..--train-steps run plain mixed solves whose systems train the network
    (untimed); --warmup learned steps follow; then --steps sample points are
    spread evenly over the rest of the --total-steps run.  At each sample
    point the same step is timed for every arm from one snapshot (learned +
    mixed, plain FP64, mixed without the network, and end to end with the
    pressure read back to host memory), after which the run continues,
    untimed, on the learned + mixed path to the next sample point."""
    import torch

    from paper_2404_17542_gb300 import build, inputs, mcd

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    mcd.lib()

    run = FlowRun(args.n, dev, mcd, inputs, args.tol)
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    host_p = torch.empty(run.N, dtype=torch.float64).pin_memory()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    net, pre, learned = None, None, None
    if not args.no_learned:
        net, pre, learned = train_nets(run, args.train_steps, args.train_epochs)
    else:
        for _ in range(args.train_steps):
            run.step(mcd.MIXED)
    for _ in range(args.warmup):
        run.step(mcd.MIXED, net)
    K = args.steps
    gap = max(1, (args.total_steps - run.k) // K)

    arms = {"main": [], "fp64": [], "no_net": [], "e2e": [], "precond": []}
    ktimes = {}
    launches = 0
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    wall0 = time.perf_counter()
    for _i in range(K):
        snap = run.snapshot()
        # the headline arm, with the kernel sampler on for this step alone
        mcd.timing_enable(1)
        l0 = mcd.launch_count()
        ms, info = timed_step(run, mcd.MIXED, flush_buf, net)
        launches += mcd.launch_count() - l0
        for kid, name in enumerate(mcd.KERNEL_NAMES):
            n_, t_ = mcd.timing_read(kid)
            if n_:
                a_ = ktimes.setdefault(name, [0, 0.0])
                a_[0] += n_
                a_[1] += t_
        mcd.timing_enable(0)
        arms["main"].append((ms, info, run.k))
        if not args.no_fp64:
            run.restore(snap)
            arms["fp64"].append(timed_step(run, mcd.FP64, flush_buf))
        if net is not None:
            run.restore(snap)
            arms["no_net"].append(timed_step(run, mcd.MIXED, flush_buf))
        if not args.no_e2e:
            run.restore(snap)
            arms["e2e"].append(timed_step(run, mcd.MIXED, flush_buf, net, host_out=host_p))
        if pre is not None:
            run.restore(snap)
            arms["precond"].append(timed_step(run, mcd.MIXED, flush_buf, net, precond=pre))
        run.restore(snap)
        for _ in range(gap):
            run.step(mcd.MIXED, net)
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()

    main = arms["main"]
    ms = sum(m for m, _i, _k in main)
    unknowns = sum(i["unknowns"] for _m, i, _k in main)
    infos = [i for _m, i, _k in main]
    ms_max, unknowns_all = aggregate_ranks(ms, unknowns, world, dev)
    value = unknowns_all / (ms_max / 1e3)

    def summary(rows):
        if not rows:
            return None
        t = sum(m for m, _i in rows)
        return {"value": sum(i["unknowns"] for _m, i in rows) / (t / 1e3), "ms_per_step": t / len(rows),
                "iters_per_step": statistics.mean(i["iters"] for _m, i in rows),
                "rel_res_max": max(i["rel_res"] for _m, i in rows),
                **fp64_finish_counts(i for _m, i in rows)}
    fp64 = summary(arms["fp64"])
    no_net = summary(arms["no_net"])
    with_pre = summary(arms["precond"])
    if with_pre is not None:
        with_pre["net_corrections_per_step"] = statistics.mean(i["net_corrections"] for _m, i in arms["precond"])
    if learned is not None:
        learned["iters_per_step"] = statistics.mean(i["iters"] for i in infos)
        learned["iters_per_step_without_net"] = no_net["iters_per_step"] if no_net else None
        learned["rel_res_guess_mean"] = statistics.mean(i["rel_res_guess"] for i in infos)
        learned["rel_res_start_mean"] = statistics.mean(i["rel_res_start"] for i in infos)
        learned["iters_gain_vs_no_net"] = (no_net["iters_per_step"] / learned["iters_per_step"]) if no_net else None
    e2e = None
    if arms["e2e"]:
        te = sum(m for m, _i in arms["e2e"])
        import ctypes
        body_bytes = 2 * ctypes.sizeof(mcd.c_body)      # the step's inputs: body states at t_k, t_k+1
        e2e = {"value": sum(i["unknowns"] for _m, i in arms["e2e"]) / (te / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": body_bytes, "d2h_bytes_per_step": run.N * 8,
               "note": "mcd_flow_step from host body states (passed by value), the step's pressure copied "
                       "to pinned host memory inside the timed region"}

    # roofline of the dominant kernel: the persistent Bi-CGSTAB solve
    peak, peak_src = measured_peaks()
    roof = None
    if ktimes:
        total = sum(v[1] for v in ktimes.values())
        name = max(ktimes, key=lambda k: ktimes[k][1])
        n_launch, t_ms = ktimes[name]
        if name == "bicg_persistent":
            iters = sum(i["iters"] for i in infos)
            algo = SOLVE_BYTES_PER_DP_ITER * run.N * iters
            unit_note = f"{SOLVE_BYTES_PER_DP_ITER} B per DP-iteration x {run.N} DPs x {iters} iterations"
        else:
            algo = BUILD_BYTES_PER_DP * run.N * n_launch
            unit_note = f"{BUILD_BYTES_PER_DP} B per DP x {run.N} DPs x {n_launch} launches"
        achieved = algo / n_launch / (t_ms / n_launch / 1e3) / 1e9
        per_unit = committed_traffic(name)
        if per_unit is not None:
            units = run.N * sum(i["iters"] for i in infos) if name == "bicg_persistent" else run.N * n_launch
            per_unit = per_unit * units / n_launch
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": per_unit,
                "kernel": ("bicg_persistent2 (two grid barriers per iteration)" if name == "bicg_persistent"
                           else name),
                "launches": n_launch, "avg_launch_ms": round(t_ms / n_launch, 3),
                "algorithmic_bytes_per_launch": algo / n_launch, "algorithmic_bytes": unit_note,
                "peak_source": f"{peak_src} hbm_gbs",
                "kernel_share": {k: round(v[1] / total, 4) for k, v in ktimes.items()}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 Krylov + f64 refinement",
            "data": "synthetic",
            "config": {"workload": f"oscillating cylinder (D=0.1, KC=5, Re=100) {args.n}x{args.n}, full "
                                   "moving-boundary fractional step (DP update, ALE, stencils, predict, "
                                   "PPE, projection, force)",
                       "mesh": [args.n, args.n], "tol": args.tol, "mode": "mixed", "dt": run.dt,
                       "ppe_source": "(1/dt) div u* of the step (Eq. (21))",
                       "learned_warm_start": net is not None,
                       "warm_start": ("step-k pressure at the new positions (ALE, Appendix A) + network "
                                      "correction" if net is not None else
                                      "step-k pressure at the new positions (ALE, Appendix A)"),
                       "schedule": f"train on steps 1-{args.train_steps}, {args.warmup} warm-up steps, "
                                   f"{K} timed steps every {gap} steps up to step {args.total_steps}",
                       "timed_steps": [k for _m, _i, k in main],
                       "l2": "flushed before each timed step (256 MB write)",
                       "parallelism": f"replicas x{world}"},
            "iters_per_step": statistics.mean(i["iters"] for i in infos),
            "updates_per_step": statistics.mean(i["refinements"] for i in infos),
            "dropped_cycles_per_step": statistics.mean(i["discarded"] for i in infos),
            **fp64_finish_counts(infos),
            "rel_res_max": max(i["rel_res"] for i in infos),
            "unknowns_per_step": unknowns / K,
            "wall_s": wall,
            "fp64_plain": fp64,
            "speedup_vs_fp64": (value / fp64["value"]) if fp64 else None,
            "mixed_no_net": no_net, "learned_with_precond": with_pre, "learned": learned,
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# the oracle on host cores (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_state(n):
    """The oracle's copy of the headline run at n x n: DPs arranged for the
    cylinder at t = 0, fluid at rest, the step-k velocity weights."""
    from oracle import mask as omask
    from oracle import mls
    from paper_2404_17542_gb300 import inputs
    cyl = inputs.Cylinder()
    pb = inputs.cylinder_box(n, cyl)
    nu = 2 * cyl.radius / 100.0
    dt = min(0.2 * pb.mesh.l0, 0.2 * pb.mesh.l0 ** 2 / nu)
    pos, m, _ = omask.update_dps_bodies(pb.mesh, pb.pos, pb.mask, [(cyl.body_id, cyl.centre(0.0), cyl.radius)],
                                        0.2, 10, 0.0)
    z = np.zeros(pb.mesh.N)
    return {"mesh": pb.mesh, "cyl": cyl, "pos": pos, "mask": m, "u": z, "v": z.copy(),
            "Wv": mls.build_weights(pb.mesh, pos, m), "t": 0.0, "nu": nu, "dt": dt}


def oracle_step(s):
    """One oracle pass of the headline's step: oracle.ale.moving_step (DP
    update, ALE, MLS weights, predict, the PPE by a direct sparse solve,
    projection, force).  Returns the unknowns (non-void DPs)."""
    from oracle import ale
    cyl, t, dt = s["cyl"], s["t"], s["dt"]
    bk = [(cyl.body_id, cyl.centre(t), cyl.radius)]
    b1 = [(cyl.body_id, cyl.centre(t + dt), cyl.radius)]
    o = ale.moving_step(s["mesh"], s["pos"], s["mask"], s["u"], s["v"], s["Wv"], bk, b1, [cyl.velocity(t)],
                        [cyl.velocity(t + dt)], dt, s["nu"])
    s.update(pos=o["pos"], mask=o["mask"], u=o["u"], v=o["v"], Wv=o["Wv"], t=t + dt)
    return int((o["mask"] != 0).sum())


ORACLE_N = 96


def _oracle_sample(n, steps):
    """One oracle instance: an untimed first step, then `steps` timed steps.
    Returns (unknowns, seconds).  Runs in a spawned worker process."""
    s = oracle_state(n)
    oracle_step(s)
    t0 = time.perf_counter()
    unknowns = 0
    for _ in range(steps):
        unknowns += oracle_step(s)
    return unknowns, time.perf_counter() - t0


def cpu_baseline(n=ORACLE_N, steps=4):
    """The oracle on every host core: one independent instance of the bounded
    sample per core (spawned processes, one BLAS thread each), throughput =
    all instances' unknowns over the slowest instance's time."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    workers = max(1, min(cores, 64))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.starmap(_oracle_sample, [(n, steps)] * workers)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    unknowns = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    single = res[0][0] / res[0][1]
    return {"value": unknowns / wall, "unit": UNIT, "cores": workers, "host_cores": cores, "kind": "oracle",
            "single_core_value": single,
            "sample": f"{workers} independent oracle instances (one per host core), each {steps} full "
                      f"moving-boundary steps (oracle.ale.moving_step: DP update, ALE, MLS weights, predict, "
                      f"direct PPE solve, projection, force) of the same cylinder run at {n}x{n} instead of "
                      "1024x1024; numpy/scipy, one BLAS thread per process"}


def reference_arm(args):
    rank, world, _local = dist_env()
    if rank != 0:
        return
    n = ORACLE_N
    s = oracle_state(n)
    for _ in range(args.warmup):
        oracle_step(s)
    t0 = time.perf_counter()
    unknowns = 0
    for _ in range(args.steps):
        unknowns += oracle_step(s)
    dt = time.perf_counter() - t0
    value = unknowns / dt
    sample = (f"each step one oracle pass of the full moving-boundary step (oracle.ale.moving_step, direct "
              f"PPE solve) of the cylinder run at {n}x{n}; single-threaded numpy/scipy")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"oscillating cylinder (D=0.1, KC=5, Re=100) {n}x{n}, full "
                                   "moving-boundary fractional step (a bounded sample of the 1024x1024 run)",
                       "mesh": [n, n], "tol": "direct solve", "mode": "oracle fp64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1,
                             "host_cores": os.cpu_count(), "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


import numpy as np  # noqa: E402  (used by the oracle legs)


TUNE_SWEEPS = 5000   # longer than any solve of the batched workload


def batched_tilings(args, bt, rhs, bnd, p, mcd):
    """Every tiling of the batched solve (tile rows x CTAs per SM, clamped by
    the kernel's occupancy) in both precisions: one whole solve each after a
    warm-up solve, L2 flushed, CUDA events; one JSON line per tiling."""
    import torch
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=p.device)
    stream = torch.cuda.current_stream()
    for mode, name in ((mcd.MIXED, "mixed"), (mcd.FP64, "fp64")):
        for rows in (1, 2, 4):
            for cps in (1, 2, 3, 4):
                bt.set_tuning(rows, cps)
                ms = []
                for _ in range(2):
                    p.zero_()
                    flush_buf.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    _p, res = bt.solve(rhs, bnd, p=p, tol=args.tol, mode=mode, graph=True)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms.append(e0.elapsed_time(e1))
                print(json.dumps({"workload": "batched", "mode": name, "rows": rows, "ctas_per_sm": cps,
                                  "ms": round(ms[-1], 1), "iters_max": int(res["iters"].max()),
                                  "iters_total": int(res["iters"].sum()),
                                  "dp_unknowns_per_s": bt.N / (ms[-1] / 1e3)}), flush=True)


def batched_arm(args):
    """One line for the batched workload: 256 degree-4 polynomial Poisson
    systems, sizes floor(exp U(ln 32, ln 512)) per side (seed 4), all solved
    by one persistent launch replayed from a CUDA graph (mixed, autotuned
    tiling), beside the same batch in FP64 and per-system plain FP64 solves
    with the single-system solver.  A "step" solves every system from p = 0."""
    import torch

    from paper_2404_17542_gb300 import build, inputs, mcd
    build.build()
    mcd.lib()
    dev = torch.device("cuda", 0)
    probs = inputs.batched_poly4(4)
    bt = mcd.Batch([pb.mesh for pb in probs], precision=mcd.MIXED)

    def d(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    pos = d(bt.pack_positions([pb.pos for pb in probs]))
    mask = d(np.concatenate([pb.mask for pb in probs]))
    rhs = d(np.concatenate([pb.rhs for pb in probs]))
    bnd = d(np.concatenate([pb.bnd for pb in probs]))
    bt.build(pos, mask)
    p = torch.zeros(bt.N, dtype=torch.float64, device=dev)
    if args.tilings:
        return batched_tilings(args, bt, rhs, bnd, p, mcd)
    # the autotuner times whole solves (the sweep budget exceeds any solve's
    # length): the first sweeps, with every system running, favour other
    # tilings than the rest of the solve, where the large systems run alone
    tune_ms = bt.autotune(rhs, bnd, p, tol=args.tol, sweeps=TUNE_SWEEPS)
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed(mode, graph, steps, **kw):
        tot, res = 0.0, None
        for _ in range(args.warmup):
            p.zero_()
            bt.solve(rhs, bnd, p=p, tol=args.tol, mode=mode, graph=graph, **kw)
        for _ in range(steps):
            p.zero_()
            flush_buf.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            _p, res = bt.solve(rhs, bnd, p=p, tol=args.tol, mode=mode, graph=graph, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / steps, res
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = mcd.launch_count()
    ms, res = timed(mcd.MIXED, True, args.steps)
    launches = (mcd.launch_count() - launches0) / max(1, args.steps + args.warmup)
    clk = clocks.stop()
    # the FP64 batch on its own autotuned tiling, then the mixed tiling again
    rows, cps = bt.tuning()
    tune_ms64 = bt.autotune(rhs, bnd, p, tol=args.tol, mode=mcd.FP64, sweeps=TUNE_SWEEPS)
    rows64, cps64 = bt.tuning()
    ms64, res64 = timed(mcd.FP64, True, max(1, args.steps // 2))
    bt.set_tuning(rows, cps)
    ms_rs, res_rs = timed(mcd.MIXED, True, max(1, args.steps // 2), update_restart=1)
    # the learned warm start: a network trained on the batch's own systems
    # (features at the zero guess, target the FP64 solution), applied to
    # every system's guess before the mixed solve
    learned = None
    if not args.no_learned:
        t0 = time.perf_counter()
        p.zero_()
        bt.solve(rhs, bnd, p=p, tol=1e-10, mode=mcd.FP64)
        net = mcd.Net(inputs.cnn_flatten(*inputs.cnn_weights(4)))
        samples = []
        for i, pb in enumerate(probs):
            o0, o1 = int(bt.offsets[i]), int(bt.offsets[i + 1])
            sti = bt.stencils(i)
            bi = sti.assemble_rhs(rhs[o0:o1].contiguous(), bnd[o0:o1].contiguous())
            zero = torch.zeros(o1 - o0, dtype=torch.float64, device=dev)
            samples.append((sti.mesh.n[0], sti.mesh.n[1]) + net.features(sti, bi, zero, None, p[o0:o1].contiguous()))
        rng = np.random.default_rng(4)
        for _ep in range(args.train_epochs):
            for j in rng.permutation(len(samples)):
                nx, ny, x, tg, wt = samples[j]
                net.train_step(x, tg, wt, nx, ny, 1e-3)
        del samples
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        ms_l, res_l = timed(mcd.MIXED, True, max(1, args.steps // 2), net=net)
        learned = {"value": bt.N / (ms_l / 1e3), "ms_per_step": ms_l, "iters_max": int(res_l["iters"].max()),
                   "iters_mean": float(res_l["iters"].mean()), "train_s": round(t_train, 1),
                   "epochs": args.train_epochs}
    # per-system plain FP64 solves with the single-system solver
    sts = [(mcd.Stencils(pb.mesh, d(pb.pos.ravel()), d(pb.mask), precision=mcd.FP64), d(pb.rhs), d(pb.bnd),
            torch.zeros(pb.mesh.N, dtype=torch.float64, device=dev)) for pb in probs]
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    its = []
    for st, r, b, pp in sts:
        pp.zero_()
        _x, info = st.solve(r, b, p=pp, tol=args.tol, mode=mcd.FP64)
        its.append(info["iters"])
    e1.record(stream)
    torch.cuda.synchronize()
    ms_each = e0.elapsed_time(e1)
    line = {"metric": METRIC, "value": bt.N / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 Krylov + f64 refinement", "data": "synthetic",
            "config": {"workload": "256 independent 2D Poisson systems, sizes log-uniform 32^2..512^2 "
                                   "(seed 4), degree-4 polynomial Dirichlet data",
                       "dps": bt.N, "tol": args.tol, "mode": "mixed (adaptive residual replacement)",
                       "graph": True,
                       "tiling": {"rows": rows, "ctas_per_sm": cps, "autotune_ms_per_sweep": tune_ms},
                       "l2": "flushed between steps (256 MB write)"},
            "iters_max": int(res["iters"].max()), "iters_mean": float(res["iters"].mean()),
            "rel_res_max": float(res["rel_res"].max()),
            "iters_total": int(res["iters"].sum()), "dropped_cycles": int(res["discarded"].sum()),
            "fp64_finishes": int((res["fallback"] != 0).sum()),
            "batched_fp64": {"value": bt.N / (ms64 / 1e3), "ms_per_step": ms64,
                             "iters_max": int(res64["iters"].max()), "iters_total": int(res64["iters"].sum()),
                             "tiling": {"rows": rows64, "ctas_per_sm": cps64, "autotune_ms_per_sweep": tune_ms64}},
            "batched_mixed_restarting": {"value": bt.N / (ms_rs / 1e3), "ms_per_step": ms_rs,
                                         "iters_total": int(res_rs["iters"].sum()),
                                         "fp64_finishes": int((res_rs["fallback"] != 0).sum())},
            "batched_learned_mixed": learned,
            "speedup_vs_batched_fp64": ms64 / ms,
            "per_system_fp64": {"value": bt.N / (ms_each / 1e3), "ms_per_step": ms_each,
                                "iters_max": int(max(its))},
            "speedup_vs_per_system_fp64": ms_each / ms,
            "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)


# FLOPs of one network inference per cell: 2 x 9 taps x (7 x 32 + 32 x 32 x 2 + 32 x 1)
CNN_FLOP_PER_CELL = 2 * 9 * (7 * 32 + 32 * 32 * 2 + 32 * 1)
# HBM bytes per cell of one layer-by-layer inference: features in (8 bf16),
# three 32-channel bf16 activations each written and read once, f32 output
CNN_LAYERED_BYTES_PER_CELL = 16 + 3 * (64 + 64) + 4


def cnn_arm(args):
    """One line for the network: inference (4 conv layers) and one training
    step (forward, loss, input and weight gradients, Adam) on an n x n grid
    of synthetic bf16 features, against the measured bf16 tensor peak."""
    import torch

    from paper_2404_17542_gb300 import build, inputs, mcd
    build.build()
    mcd.lib()
    dev = torch.device("cuda", 0)
    n = args.n
    N = n * n
    net = mcd.Net(inputs.cnn_flatten(*inputs.cnn_weights(0)))
    g = torch.Generator(device=dev).manual_seed(0)
    x = (torch.rand((N, 8), generator=g, device=dev) * 2 - 1).to(torch.bfloat16).view(torch.int16)
    y = torch.empty(N, dtype=torch.float32, device=dev)
    tg = torch.randn(N, generator=g, device=dev)
    wt = torch.ones(N, dtype=torch.float32, device=dev)
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed(f):
        for _ in range(max(3, args.warmup)):
            f()
        tot = 0.0
        for _ in range(args.steps):
            flush_buf.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            f()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / args.steps
    t_fwd = timed(lambda: net.forward(x, n, n, y))
    t_train = timed(lambda: net.train_step(x, tg, wt, n, n, 1e-4))
    flop = CNN_FLOP_PER_CELL * N
    peak = hbm = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        peaks = json.load(open(p))
        peak, hbm = peaks.get("bf16_tflops"), peaks.get("hbm_gbs")
    ach = flop / (t_fwd / 1e3) / 1e12
    layered_gbs = CNN_LAYERED_BYTES_PER_CELL * N / (t_fwd / 1e3) / 1e9
    line = {"metric": "network inference cells/s", "value": N / (t_fwd / 1e3), "unit": "cells/s",
            "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": t_fwd,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (f32 accumulate)",
            "data": "synthetic", "config": {"workload": f"4-layer 3x3 conv network, 32 channels, {n}x{n} grid",
                                            "l2": "flushed between steps (256 MB write)"},
            "train_step_ms": t_train, "train_cells_per_s": N / (t_train / 1e3),
            "roofline": {"bound": "tensor", "achieved": round(ach, 1), "peak": peak, "unit": "TFLOP/s",
                         "frac": round(ach / peak, 4) if peak else None,
                         "algorithmic": f"{CNN_FLOP_PER_CELL} FLOP per cell x {N} cells per inference"},
            # the layer-by-layer design moves every activation through HBM:
            # this is the roof that bounds it (the compulsory traffic is 20 B per cell)
            "layered_hbm": {"bytes_per_cell": CNN_LAYERED_BYTES_PER_CELL, "achieved": round(layered_gbs, 1),
                            "peak": hbm, "unit": "GB/s",
                            "frac": round(layered_gbs / hbm, 4) if hbm else None}}
    print(json.dumps(line), flush=True)


# Algorithmic bytes per DP-iteration of the persistent solve: two SpMVs read
# the S-slot rows, plus 68 (FP32) / 136 (FP64) bytes of vectors.
def solve_bytes_per_dp_iter(S, fp64):
    return 2 * S * (8 if fp64 else 4) + (136 if fp64 else 68)


def array_arm(args):
    """The multiple-stationary-cylinder experiment of Sec. 4.1 (the cost
    contrast of its Table 1): a 5 x 5 cylinder array in the square of side 2
    on an n x n mesh, gaps 12 and 2 (units of the paper's l0 = 1/64),
    Neumann cylinders, Dirichlet walls, the smooth synthetic source.  DPs
    from the multi-body DP update (10 relaxation sweeps).  For the 3x3
    stencil (cos^2 weight, r_e = 2.5 l0) and the expanded 9x9 stencil
    (least-squares MPS weight, r_e = 3.5 l0): the stencil build and PPE solves
    from p = 0 at the paper's tolerance 1e-2 and at --tol, mixed and FP64,
    each timed with CUDA events after warm-up, L2 flushed before each."""
    import torch

    from paper_2404_17542_gb300 import build, inputs, mcd
    build.build()
    mcd.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    n = args.n
    hbm = None
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        hbm = json.load(open(pk)).get("hbm_gbs")

    def d(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    def timed(f, steps):
        for _ in range(max(1, args.warmup)):
            f()
        tot, out = 0.0, None
        for _ in range(steps):
            flush_buf.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            out = f()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / steps, out

    stencils = {"3x3": dict(weight_kind=mcd.W_COS2, r_e=2.5, support=1),
                "9x9": dict(weight_kind=mcd.W_LSMPS, r_e=3.5, support=4)}
    results = []
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = mcd.launch_count()
    for gap in (12, 2):
        pb = inputs.cylinder_array_box(n, gap)
        bodies = pb.meta["bodies"]
        l0 = pb.mesh.l0
        pos, mask = d(pb.pos.ravel()), d(pb.mask)
        prev = torch.empty_like(mask)
        mcd.update_dps_bodies(pb.mesh, bodies, pos, mask, prev, n_relax=10, band=0.0)
        normal, _f = mcd.bodies_boundary(pb.mesh, bodies, pos, mask)
        m = mask.cpu().numpy()
        unknowns = int((m != 0).sum())
        rhs = d(np.where(m == -1, pb.rhs, 0.0))
        bnd = torch.zeros(pb.mesh.N, dtype=torch.float64, device=dev)
        porosity = 1.0 - math.pi * (2 * bodies[0][2]) ** 2 * len(bodies) / 16.0   # Sec. 4.1, L = 1
        for name, sp in stencils.items():
            st = mcd.Stencils(pb.mesh, pos, mask, normal, bc_kind=pb.bc_kind, weight_kind=sp["weight_kind"],
                              r_e=sp["r_e"] * l0, precision=mcd.MIXED, want_derivs=False,
                              support=sp["support"])
            if st.check()[0] != 0:
                raise RuntimeError(f"singular stencil in the {name} array system")
            ms_build, _ = timed(lambda: st.rebuild(pos, mask, normal), max(1, args.steps))
            p = torch.zeros(pb.mesh.N, dtype=torch.float64, device=dev)
            for tol in (1e-2, args.tol):
                for mode, mname in ((mcd.MIXED, "mixed"), (mcd.FP64, "fp64")):
                    def one():
                        p.zero_()
                        return st.solve(rhs, bnd, p=p, tol=tol, mode=mode)[1]
                    ms, info = timed(one, max(1, args.steps))
                    S = st.S
                    gbs = solve_bytes_per_dp_iter(S, mode == mcd.FP64) * pb.mesh.N * info["iters"] / (ms / 1e3) / 1e9
                    results.append({"gap_l0": gap, "stencil": name, "tol": tol, "mode": mname,
                                    "iters": int(info["iters"]), "rel_res": float(info["rel_res"]),
                                    "fallback": int(info.get("fallback", 0)),
                                    "solve_ms": round(ms, 3), "build_ms": round(ms_build, 3),
                                    "dp_unknowns_per_s": unknowns / (ms / 1e3),
                                    "solve_gbs": round(gbs, 1),
                                    "solve_hbm_frac": round(gbs / hbm, 4) if hbm else None})
            del st
        results_gap = [r for r in results if r["gap_l0"] == gap]
        for r in results_gap:
            r["unknowns"] = unknowns
            r["porosity"] = round(porosity, 4)
    clk = clocks.stop()
    launches = mcd.launch_count() - launches0

    def pick(gap, stencil, tol, mode):
        return next(r for r in results if r["gap_l0"] == gap and r["stencil"] == stencil and r["tol"] == tol
                    and r["mode"] == mode)
    contrast = []
    for gap in (12, 2):
        for tol in (1e-2, args.tol):
            a, b = pick(gap, "3x3", tol, "mixed"), pick(gap, "9x9", tol, "mixed")
            contrast.append({"gap_l0": gap, "tol": tol, "iters_3x3": a["iters"], "iters_9x9": b["iters"],
                             "iters_ratio": round(b["iters"] / max(1, a["iters"]), 3),
                             "time_ratio_solve": round(b["solve_ms"] / a["solve_ms"], 3),
                             "time_ratio_build_plus_solve": round((b["solve_ms"] + b["build_ms"]) /
                                                                  (a["solve_ms"] + a["build_ms"]), 3)})
    main = pick(12, "3x3", args.tol, "mixed")
    main_S = 9
    ach = solve_bytes_per_dp_iter(main_S, False) * n * n * main["iters"] / (main["solve_ms"] / 1e3) / 1e9
    line = {"metric": "PPE DP-unknowns solved/s, 25-cylinder array (Sec. 4.1)", "value": main["dp_unknowns_per_s"],
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": max(1, args.warmup),
            "ms_per_step": main["solve_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 Krylov + f64 refinement", "data": "synthetic",
            "config": {"workload": f"5x5 stationary cylinder array, side 2, {n}x{n} mesh (l0 = {2.0 / n:g}), "
                                   "gaps 12 and 2 x (1/64), Neumann cylinders, Dirichlet walls; "
                                   "value: 3x3 cos^2 stencil, gap 12, mixed, tol " + f"{args.tol:g}",
                       "l2": "flushed before every timed build and solve (256 MB write)"},
            "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(ach / hbm, 4) if hbm else None,
                         "algorithmic": f"{solve_bytes_per_dp_iter(main_S, False)} B per DP-iteration "
                                        f"x {n * n} DPs x iterations"},
            "table1_contrast": contrast, "results": results, "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)


def flow_arm(args):
    """Full moving-boundary fractional steps of the oscillating cylinder
    (D = 0.1, KC = 5, Re = 100 in the unit box, dt = 0.2 l0): per step the
    DP update, the ALE interpolation (Eq. (19), Appendix A), velocity and
    pressure stencils, predict, the mixed PPE solve (tol --tol, warm-started
    from the previous pressure), projection and the fluid force (Eqs.
    (30)-(31)).  The velocity starts at rest; --warmup steps run untimed,
    then --steps steps are timed with CUDA events (no L2 flush: the step's
    working set of about 3 GB at 1024^2 exceeds L2)."""
    import torch

    from paper_2404_17542_gb300 import build, inputs, mcd
    build.build()
    mcd.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    n = args.n
    if args.bodies == "cylinder":
        cyl = inputs.Cylinder()
        pb = inputs.cylinder_box(n, cyl)
        D, U = 2 * cyl.radius, 1.0
        nu = U * D / 100.0
        dt = 0.2 * pb.mesh.l0
        t0 = 0.0 if args.t0 is None else args.t0
        ids = [cyl.body_id]
        workload = f"oscillating cylinder (D = 0.1, KC = 5, Re = 100) {n}x{n}, full ALE steps from rest"

        def bodies_at(t):
            return [(cyl.body_id, cyl.centre(t), cyl.radius)], [cyl.velocity(t)]
    elif args.bodies == "wing":
        wing = inputs.FlappingWing()
        pb = inputs.flapping_wing_box(cfg=wing)
        D, U = wing.c, 1.0
        nu = U * D / 75.0
        dt = math.pi / 600.0
        t0 = 0.0 if args.t0 is None else args.t0
        ids = [wing.body_id]
        h = 0.5 * pb.mesh.l0
        grid_h, org = wing.sdf_grid(h)
        grid = torch.from_numpy(grid_h).to(dev)
        nx, ny = pb.mesh.n[0], pb.mesh.n[1]
        workload = (f"flapping elliptic wing (c = 1, e = 4, 16c x 16c closed box, stroke plane pi/3, "
                    f"a0 = 2.5, theta0 = pi/4, Re = 75, l0 = {pb.mesh.l0:.4g}, dt = pi/600) {nx}x{ny}, "
                    f"the wing as a {grid_h.shape[1]}x{grid_h.shape[0]} SDF grid, full ALE steps from rest "
                    f"at t0 = {t0:g}")

        def bodies_at(t):
            return ([mcd.SdfBody(wing.body_id, wing.centre(t), wing.posture(t), grid, org, h,
                                 omega=wing.omega(t))], [wing.velocity(t)])
    else:
        cfg = inputs.PassingCylinders()
        pb = inputs.passing_cylinders_box(cfg=cfg)
        D, U = cfg.D, cfg.U
        nu = U * D / 40.0
        dt = 5e-3
        t0 = 3 * cfg.T - 0.5 if args.t0 is None else args.t0
        ids = [2, 3]
        nx, ny = pb.mesh.n[0], pb.mesh.n[1]
        workload = (f"two cylinders passing each other (D = 1, 32D x 16D closed box, Re = 40, l0 = "
                    f"{pb.mesh.l0:.4g}, dt = 5e-3) {nx}x{ny}, full ALE steps from rest at t0 = {t0:g}")
        if args.bodies == "passing-sdf":
            h = 0.5 * pb.mesh.l0
            R = 0.5 * cfg.D
            m = int(round(5 * R / h)) + 1
            org = (-2.5 * R, -2.5 * R)
            grid = torch.from_numpy(inputs.sample_sdf_grid(inputs.circle_sdf(R), org, h, (m, m))).to(dev)
            workload += f"; cylinders given as {m}x{m} SDF grids (h = l0/2)"

            def bodies_at(t):
                geo, vel = cfg.bodies(t)
                return [mcd.SdfBody(bid, c, 0.0, grid, org, h) for bid, c, _R in geo], vel
        else:
            def bodies_at(t):
                return cfg.bodies(t)

    flow = mcd.AleFlow(pb.mesh, torch.from_numpy(pb.pos.ravel().copy()).to(dev),
                       torch.from_numpy(pb.mask.copy()).to(dev), bodies_at, nu, dt, t0=t0, tol=args.tol)
    for _ in range(max(1, args.warmup)):
        flow.step()
    mcd.timing_enable(1)
    launches0 = mcd.launch_count()
    clocks = ClockSampler(0)
    clocks.start()
    rows = []
    tot = 0.0
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        info = flow.step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        tot += ms
        row = {"t": round(flow.t, 6), "ms": round(ms, 3), "iters": info["solve"]["iters"],
               "unknowns": info["solve"]["unknowns"], "fallback": info["solve"]["fallback"],
               "ale_fallbacks": info["fallbacks"]}
        for bid in ids:
            F = info["forces"][bid][0]
            sfx = "" if len(ids) == 1 else f"_{bid}"
            row["cd" + sfx] = 2 * F[0] / (D * U * U)     # Eqs. (35)-(36)
            row["cl" + sfx] = 2 * F[1] / (D * U * U)
        rows.append(row)
    clk = clocks.stop()
    launches = (mcd.launch_count() - launches0) / max(1, args.steps)
    solve_ms = mcd.timing_read(mcd.K_SOLVE)[1]
    mcd.timing_enable(0)
    ms_step = tot / args.steps
    unknowns = sum(r["unknowns"] for r in rows)
    hbm = None
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        hbm = json.load(open(pk)).get("hbm_gbs")
    iters = sum(r["iters"] for r in rows)
    ach = solve_bytes_per_dp_iter(9, False) * pb.mesh.N * iters / (solve_ms / 1e3) / 1e9 if solve_ms else None
    line = {"metric": "DP-unknowns advanced/s, full moving-boundary fractional step", "value": unknowns / (tot / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": max(1, args.warmup), "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 stencils / ALE / driver, f32 Krylov + f64 refinement", "data": "synthetic",
            "config": {"workload": workload, "dt": dt, "tol": args.tol,
                       "l2": "not flushed (per-step working set above L2)"},
            "solve_share": round(solve_ms / tot, 4) if tot else None,
            "roofline": {"bound": "hbm", "achieved": round(ach, 1) if ach else None, "peak": hbm, "unit": "GB/s",
                         "frac": round(ach / hbm, 4) if (ach and hbm) else None,
                         "kernel": "bicg_persistent2<2, float>",
                         "algorithmic": f"{solve_bytes_per_dp_iter(9, False)} B per DP-iteration"},
            "steps_detail": rows, "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)


# Algorithmic bytes per DP of one stencil SpMV y = A x: the S-slot rows, x
# once, y once (neighbour reads of x are reuse, not new traffic).
def spmv_bytes_per_dp(S, fp64):
    w = 8 if fp64 else 4
    return S * w + 2 * w


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)).get("hbm_gbs"), "measured"
    return HBM_FALLBACK_GBS, "fallback"


def spmv_arm(args):
    """The matrix-free stencil SpMV (mcd_apply_laplacian, Eq. (21) rows) where
    HBM is the limit: an n x n jittered box (default 4096^2, 16.8 M DPs; FP32
    rows + vectors 738 MB, FP64 1.48 GB, both above 3x L2), Gaussian MLS
    rows.  Each dtype: --warmup untimed launches, then 10 x --steps launches
    back to back between two CUDA events (the working set does not fit in L2,
    so no flush is needed).  Then the persistent mixed and FP64 solves of the
    2048^2 manufactured problem from p = 0 (working set above L2)."""
    import torch

    from paper_2404_17542_gb300 import build, inputs, mcd
    build.build()
    mcd.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    n = args.n
    peak, peak_src = hbm_peak()
    l2 = torch.cuda.get_device_properties(0).L2_cache_size

    def d(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    pb = inputs.manufactured_box(n, 2, seed=0)
    N = pb.mesh.N
    st = mcd.Stencils(pb.mesh, d(pb.pos.ravel()), d(pb.mask), precision=mcd.MIXED)
    del pb
    g = torch.Generator(device=dev).manual_seed(0)
    reps = 10 * max(1, args.steps)
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = mcd.launch_count()
    spmv = {}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        x = torch.rand(N, generator=g, device=dev, dtype=torch.float64).to(dt)
        y = torch.empty_like(x)
        for _ in range(max(3, args.warmup)):
            st.apply(x, y)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            st.apply(x, y)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        bpd = spmv_bytes_per_dp(9, dt == torch.float64)
        gbs = bpd * N / (ms / 1e3) / 1e9
        spmv[name] = {"ms_per_launch": round(ms, 4), "bytes_per_dp": bpd,
                      "algorithmic_bytes_per_launch": bpd * N, "achieved_gbs": round(gbs, 1),
                      "frac": round(gbs / peak, 4), "dps_per_s": N / (ms / 1e3)}
        del x, y
    launches = mcd.launch_count() - launches0
    clk = clocks.stop()
    st.close()
    torch.cuda.synchronize()

    # the persistent solve where its working set leaves L2
    solve = {}
    if not args.no_fp64:
        m = 2048
        pb = inputs.manufactured_box(m, 2, seed=0)
        st = mcd.Stencils(pb.mesh, d(pb.pos.ravel()), d(pb.mask), precision=mcd.MIXED)
        rhs, bnd = d(pb.rhs), d(pb.bnd)
        p = torch.zeros(pb.mesh.N, dtype=torch.float64, device=dev)
        for mode, nm in ((mcd.MIXED, "mixed"), (mcd.FP64, "fp64")):
            p.zero_()
            st.solve(rhs, bnd, p=p, tol=args.tol, mode=mode)          # warm-up
            mcd.timing_enable(1)
            p.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _p, info = st.solve(rhs, bnd, p=p, tol=args.tol, mode=mode)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            _nl, kms = mcd.timing_read(mcd.K_SOLVE)
            mcd.timing_enable(0)
            bpi = solve_bytes_per_dp_iter(9, mode == mcd.FP64)
            ach = bpi * pb.mesh.N * info["iters"] / (kms / 1e3) / 1e9 if kms else None
            err = float(torch.linalg.norm(p - d(pb.exact)) / torch.linalg.norm(d(pb.exact)))
            solve[nm] = {"ms": round(ms, 3), "iters": info["iters"], "rel_res": info["rel_res"],
                         "us_per_iteration": round(kms * 1e3 / max(1, info["iters"]), 2),
                         "dps_per_s": info["unknowns"] / (ms / 1e3),
                         "roofline": {"achieved": round(ach, 1) if ach else None, "peak": peak,
                                      "frac": round(ach / peak, 4) if ach else None,
                                      "bytes_per_dp_iteration": bpi},
                         "err_vs_exact": err}
        solve["workload"] = (f"manufactured sin(pi x) sin(pi y), 2048x2048 jittered box, Dirichlet walls, "
                             f"from p = 0 to tol {args.tol:g}")
        st.close()
    line = {"metric": "stencil SpMV DP-rows/s (FP32 rows + vectors)", "value": spmv["f32"]["dps_per_s"],
            "unit": "DP-rows/s", "n_gpus": 1, "steps": reps, "warmup": max(3, args.warmup),
            "ms_per_step": spmv["f32"]["ms_per_launch"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (compensated sums)", "data": "synthetic",
            "config": {"workload": f"mcd_apply_laplacian on a {n}x{n} jittered box (Gaussian MLS rows, "
                                   "Dirichlet walls)", "dps": N, "l2_bytes": l2,
                       "l2": f"working set {spmv_bytes_per_dp(9, False) * N / 1e6:.0f} MB (FP32) > 3x L2"},
            "roofline": {"bound": "hbm", "achieved": spmv["f32"]["achieved_gbs"], "peak": peak, "unit": "GB/s",
                         "frac": spmv["f32"]["frac"],
                         "traffic": (committed_traffic("spmv2d_tma") * N if committed_traffic("spmv2d_tma")
                                     else None),
                         "kernel": "spmv2d_tma<float>",
                         "algorithmic": f"{spmv_bytes_per_dp(9, False)} B per DP x {N} DPs per launch",
                         "peak_source": f"{peak_src} hbm_gbs"},
            "spmv": spmv, "solve_2048": solve, "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)


def tgv_arm(args):
    """Config C2: the periodic Taylor-Green vortex (Re = 100) on an n x n
    jittered periodic cloud (default 512^2), --tgv-steps fractional steps
    (predict, PPE, projection; Eqs. (20)-(22)) at dt = 0.2 l0, each PPE solve
    warm-started from the previous pressure, DP 0 pinned to the closed form.
    Mixed and plain FP64 each run all steps from t = 0, timed with CUDA
    events over every step; the error against the closed form at the end."""
    import torch

    from paper_2404_17542_gb300 import build, inputs, mcd
    build.build()
    mcd.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    n = args.n
    pb = inputs.tgv_box(n, seed=1)
    nu = pb.meta["nu"]
    # CFL 0.2 at U = 1, capped by the explicit viscous term of Eq. (20): the
    # MLS Laplacian's spectrum reaches about -4/l0^2, so nu dt / l0^2 must
    # stay below 1/2; 0.2 keeps a margin (at 512^2 this cap decides)
    dt = min(0.2 * pb.mesh.l0, 0.2 * pb.mesh.l0 ** 2 / nu)
    nsteps = args.tgv_steps
    N = pb.mesh.N

    def d(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    st = mcd.Stencils(pb.mesh, d(pb.pos.ravel()), d(pb.mask), precision=mcd.MIXED, want_derivs=True)
    # boundary data: only DP 0 (the pinned DP) is not inner; its closed-form
    # values for every step are uploaded once, outside the timed region
    x0 = pb.pos[:, :1]
    bc = np.array([[float(v[0]) for v in inputs.tgv_fields(x0, (k + 1) * dt, nu)] for k in range(nsteps)])
    bc_dev = d(bc)
    ue, ve, pe = inputs.tgv_fields(pb.pos, nsteps * dt, nu)
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = mcd.launch_count()
    out = {}
    for mode, nm in ((mcd.MIXED, "mixed"), (mcd.FP64, "fp64")):
        if nm == "fp64" and args.no_fp64:
            continue
        u, v = d(pb.meta["u"]), d(pb.meta["v"])
        P = torch.zeros(N, dtype=torch.float64, device=dev)
        ubc, vbc, pbc = (torch.zeros(N, dtype=torch.float64, device=dev) for _ in range(3))
        iters, unknowns = [], 0
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(nsteps):
            ubc[:1].copy_(bc_dev[k, 0:1])
            vbc[:1].copy_(bc_dev[k, 1:2])
            pbc[:1].copy_(bc_dev[k, 2:3])
            us, vs, src = st.flow_predict(u, v, ubc, vbc, nu, dt)
            _p, info = st.solve(src, pbc, p=P, tol=args.tol, mode=mode)
            u, v = st.flow_project(P, pbc, us, vs, ubc, vbc, dt)
            iters.append(info["iters"])
            unknowns += info["unknowns"]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        Pm = P - P.mean()
        pex = d(pe - pe.mean())
        out[nm] = {"ms_total": round(ms, 2), "ms_per_step": round(ms / nsteps, 4),
                   "dps_per_s": unknowns / (ms / 1e3), "iters_mean": statistics.mean(iters),
                   "iters_max": max(iters),
                   "err_u": float(torch.linalg.norm(u - d(ue)) / torch.linalg.norm(d(ue))),
                   "err_v": float(torch.linalg.norm(v - d(ve)) / torch.linalg.norm(d(ve))),
                   "err_p": float(torch.linalg.norm(Pm - pex) / torch.linalg.norm(pex))}
    launches = (mcd.launch_count() - launches0) / max(1, len(out) * nsteps)
    clk = clocks.stop()
    line = {"metric": "DP-unknowns solved/s at rel.res 1e-8: learned+mixed vs plain FP64, same GB300",
            "value": out["mixed"]["dps_per_s"], "unit": UNIT, "n_gpus": 1, "steps": nsteps, "warmup": 0,
            "ms_per_step": out["mixed"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 Krylov + f64 refinement", "data": "synthetic",
            "config": {"workload": f"periodic Taylor-Green vortex, Re = 100, {n}x{n} jittered periodic cloud, "
                                   f"{nsteps} fractional steps at dt = min(0.2 l0, 0.2 l0^2/nu) = {dt:.3g} (predict, PPE, projection), "
                                   "PPE warm-started from the previous pressure, DP 0 pinned",
                       "tol": args.tol, "l2": "not flushed (one continuous run of steps)"},
            "mixed": out["mixed"], "fp64_plain": out.get("fp64"),
            "speedup_vs_fp64": (out["fp64"]["ms_total"] / out["mixed"]["ms_total"]) if "fp64" in out else None,
            "gpu_launches_per_step": launches, "clocks": clk}
    print(json.dumps(line), flush=True)


def poisson3d_arm(args):
    """Config C3: the 128^3 manufactured Poisson problem (u = sin(pi x)
    sin(pi y) sin(pi z), Dirichlet walls, one jittered DP per cell, 3x3x3
    stencils, 10-term quadratic basis).  Each step is one solve from p = 0
    (FP64 rows for the residual, FP32 rows for the recursion), mixed and
    plain FP64, L2 flushed between steps; error against the closed form."""
    import torch

    from paper_2404_17542_gb300 import build, inputs, mcd
    build.build()
    mcd.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    n = args.n
    peak, peak_src = hbm_peak()

    def d(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    pb = inputs.manufactured_box(n, 3, seed=2)
    N = pb.mesh.N
    pos, mask = d(pb.pos.ravel()), d(pb.mask)
    st = mcd.Stencils(pb.mesh, pos, mask, precision=mcd.MIXED)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st.rebuild(pos, mask)
    e1.record(stream)
    torch.cuda.synchronize()
    build_ms = e0.elapsed_time(e1)
    rhs, bnd, exact = d(pb.rhs), d(pb.bnd), d(pb.exact)
    p = torch.zeros(N, dtype=torch.float64, device=dev)
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    clocks = ClockSampler(0)
    clocks.start()
    out = {}
    launches = None
    for mode, nm in ((mcd.MIXED, "mixed"), (mcd.FP64, "fp64")):
        if nm == "fp64" and args.no_fp64:
            continue
        for _ in range(max(3, args.warmup)):
            p.zero_()
            st.solve(rhs, bnd, p=p, tol=args.tol, mode=mode)
        mcd.timing_enable(1)
        launches0 = mcd.launch_count()
        tot, infos = 0.0, []
        for _ in range(args.steps):
            p.zero_()
            flush_l2(flush_buf)
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            _p, info = st.solve(rhs, bnd, p=p, tol=args.tol, mode=mode)
            a1.record(stream)
            torch.cuda.synchronize()
            tot += a0.elapsed_time(a1)
            infos.append(info)
        if launches is None:
            launches = (mcd.launch_count() - launches0) / args.steps
        _nl, kms = mcd.timing_read(mcd.K_SOLVE)
        mcd.timing_enable(0)
        iters = sum(i["iters"] for i in infos)
        bpi = solve_bytes_per_dp_iter(27, mode == mcd.FP64)
        ach = bpi * N * iters / (kms / 1e3) / 1e9 if kms else None
        out[nm] = {"ms_per_solve": round(tot / args.steps, 3), "dps_per_s": infos[0]["unknowns"] * args.steps / (tot / 1e3),
                   "iters": infos[0]["iters"], "rel_res_max": max(i["rel_res"] for i in infos),
                   "us_per_iteration": round(kms * 1e3 / max(1, iters), 2),
                   "err_vs_exact": float(torch.linalg.norm(p - exact) / torch.linalg.norm(exact)),
                   "roofline": {"bound": "hbm", "achieved": round(ach, 1) if ach else None, "peak": peak,
                                "unit": "GB/s", "frac": round(ach / peak, 4) if ach else None,
                                "kernel": f"bicg_persistent2<3, {'double' if mode == mcd.FP64 else 'float'}>",
                                "algorithmic": f"{bpi} B per DP-iteration x {N} DPs x iterations",
                                "peak_source": f"{peak_src} hbm_gbs"}}
    clk = clocks.stop()
    line = {"metric": METRIC, "value": out["mixed"]["dps_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": out["mixed"]["ms_per_solve"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 Krylov + f64 refinement", "data": "synthetic",
            "config": {"workload": f"3D Poisson {n}^3, jittered DPs, 27-point quadratic MLS (Gaussian), "
                                   "u = sin(pi x) sin(pi y) sin(pi z), Dirichlet walls, solve from p = 0",
                       "tol": args.tol, "l2": "flushed between steps (256 MB write)"},
            "build_ms": round(build_ms, 3), "mixed": out["mixed"], "fp64_plain": out.get("fp64"),
            "speedup_vs_fp64": (out["mixed"]["dps_per_s"] / out["fp64"]["dps_per_s"]) if "fp64" in out else None,
            "roofline": out["mixed"]["roofline"], "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)


def profile_solve(args):
    """One mixed solve of the cylinder system at step 1 from p = 0 (or, with
    --workload array, of the 25-cylinder array system, gap 12, on the stencil
    --support selects)."""
    import torch

    from paper_2404_17542_gb300 import build, inputs, mcd
    build.build()
    mcd.lib()
    if args.workload == "array":
        dev = torch.device("cuda", 0)
        pb = inputs.cylinder_array_box(args.n, 12)
        bodies = pb.meta["bodies"]
        pos = torch.from_numpy(pb.pos.ravel().copy()).to(dev)
        mask = torch.from_numpy(pb.mask.copy()).to(dev)
        mcd.update_dps_bodies(pb.mesh, bodies, pos, mask, torch.empty_like(mask), n_relax=10, band=0.0)
        normal, _f = mcd.bodies_boundary(pb.mesh, bodies, pos, mask)
        wide = args.support == 4
        st = mcd.Stencils(pb.mesh, pos, mask, normal, bc_kind=pb.bc_kind,
                          weight_kind=mcd.W_LSMPS if wide else mcd.W_COS2,
                          r_e=(3.5 if wide else 2.5) * pb.mesh.l0, want_derivs=False, support=args.support)
        m = mask.cpu().numpy()
        rhs = torch.from_numpy(np.where(m == -1, pb.rhs, 0.0)).to(dev)
        bnd = torch.zeros_like(rhs)
        _p, info = st.solve(rhs, bnd, tol=args.tol, mode=mcd.MIXED, barriers=args.barriers)
        print(json.dumps({"iters": info["iters"], "fallback": info["fallback"], "dps": pb.mesh.N,
                          "rel_res": info["rel_res"], "support": args.support}), flush=True)
        return
    run = CylinderRun(args.n, torch.device("cuda", 0), mcd, inputs, args.tol, args.barriers, args.update_restart)
    info = run.step(mcd.MIXED)
    print(json.dumps({"iters": info["iters"], "fallback": info["fallback"], "dps": run.N,
                      "rel_res": info["rel_res"]}), flush=True)


def trace_solve(args):
    """Where one Bi-CGSTAB iteration's time goes: a cylinder step at --n
    (after one untimed step) with the persistent solver's %globaltimer
    stamps on.  Prints medians over the solve's first iterations: block 0's
    phase work and barrier waits, the stages of the grid barriers (block 0's
    reduction and scalar update, the latest arrival and wake-up of any
    block), and the spread of the blocks' start times in iteration 10."""
    import torch

    from paper_2404_17542_gb300 import build, inputs, mcd
    build.build()
    mcd.lib()
    if args.workload == "flow":
        # the headline's own solve: a full moving-boundary step (restarting
        # schedule, ALE pressure guess) after --warmup steps from rest
        run = FlowRun(args.n, torch.device("cuda", 0), mcd, inputs, args.tol)
        for _ in range(max(1, args.warmup)):
            run.step(mcd.MIXED)
    else:
        run = CylinderRun(args.n, torch.device("cuda", 0), mcd, inputs, args.tol, args.barriers,
                          args.update_restart)
        run.step(mcd.MIXED)
    mcd.trace_enable(True)
    mcd.timing_enable(1)
    try:
        info = run.step(mcd.MIXED)
        ph, _end, _sm, start, bar = mcd.trace_read()
        n_solve, solve_ms = mcd.timing_read(mcd.K_SOLVE)
    finally:
        mcd.trace_enable(False)
        mcd.timing_enable(0)
    ph = ph.astype(np.int64)
    bar = bar.astype(np.int64)
    # one grid barrier per iteration stamps slots 0-2 (start, phase done,
    # reduced); two barriers stamp 0-4
    one = not (ph[4:63, 3] > 0).any()
    width = 3 if one else 5
    rows = [r for r in range(4, 63) if (ph[r, :width] > 0).all() and ph[r + 1, 0] > 0]
    epochs = [e for e in range(10, 256) if (bar[e] > 0).all()]

    def med(vals):
        return round(float(np.median(vals)) / 1000.0, 3) if len(vals) else None

    if one:
        block0 = {"work": med([ph[r, 1] - ph[r, 0] for r in rows]),
                  "barrier": med([ph[r, 2] - ph[r, 1] for r in rows])}
    else:
        block0 = {"ca_work": med([ph[r, 1] - ph[r, 0] for r in rows]),
                  "ca_barrier": med([ph[r, 2] - ph[r, 1] for r in rows]),
                  "b_work": med([ph[r, 3] - ph[r, 2] for r in rows]),
                  "b_barrier": med([ph[r, 4] - ph[r, 3] for r in rows])}
    s = start[:2048].astype(np.int64)
    s = s[s > 0]
    print(json.dumps({
        "n": args.n, "iters": info["iters"], "fallback": info["fallback"],
        "barriers_per_iteration": 1 if one else 2,
        "staged_tiles": bool(int(ph[0, 7]) & 2),
        "iteration_us": med([ph[r + 1, 0] - ph[r, 0] for r in rows]),
        "iteration_us_p90": (round(float(np.percentile([ph[r + 1, 0] - ph[r, 0] for r in rows], 90)) / 1000.0, 3)
                             if rows else None),
        # the whole solve: persistent launches' time over all iterations
        # (true-residual updates and restarts included)
        "solve_us_per_iteration": round(solve_ms * 1000.0 / max(1, info["iters"]), 3),
        "solve_launches": n_solve,
        "updates": info["refinements"],
        "block0_us": block0,
        "barrier_us": {"last_arrival_to_all_partials": med([bar[e, 2] - bar[e, 6] for e in epochs]),
                       "block0_reduction": med([bar[e, 3] - bar[e, 2] for e in epochs]),
                       "scalar_update": med([bar[e, 4] - bar[e, 3] for e in epochs]),
                       "release_stores": med([bar[e, 5] - bar[e, 4] for e in epochs]),
                       "release_to_last_wake": med([bar[e, 7] - bar[e, 5] for e in epochs]),
                       "last_arrival_to_last_wake": med([bar[e, 7] - bar[e, 6] for e in epochs])},
        "start_spread_us_iteration_10": round(float(s.max() - s.min()) / 1000.0, 3) if s.size else None,
    }), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        reference_arm(args)
    elif args.profile_solve:
        profile_solve(args)
    elif args.trace_solve:
        trace_solve(args)
    elif args.workload == "batched":
        batched_arm(args)
    elif args.workload == "cnn":
        cnn_arm(args)
    elif args.workload == "array":
        array_arm(args)
    elif args.workload == "flow":
        flow_arm(args)
    elif args.workload == "spmv":
        spmv_arm(args)
    elif args.workload == "tgv":
        tgv_arm(args)
    elif args.workload == "poisson3d":
        poisson3d_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
