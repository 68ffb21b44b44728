#!/usr/bin/env python3
"""Benchmark of the short-range non-bonded hot path on one GB300 per rank.

Step: one force evaluation of the 23,500-atom solvated-chain system (62.2 A
box, rc 9 A switched from 7.5 A, Ewald alpha 0.32, 2,500-atom chain with
exclusions and scaled 1-4 pairs plus 7,000 TIP3P-shaped waters): cell-list
rebuild from the positions (wrap, column binning, z-sort, cluster bounding
boxes, exclusion map, cluster-pair list), then forces, energies and virial.
The step is replayed from a CUDA graph; the L2 cache is flushed (a 512 MiB
write) before every timed step, outside the timed interval.

Metric: pair interactions per second = unique in-cutoff, non-excluded pairs
per step / seconds per step (the pair count is the kernel's own count, taken
once before timing).  The JSON line also carries the roofline of the force
kernel (FP32 pipe; 73 algorithmic FLOP per pair), the end-to-end number
through host buffers, the adjoint and batched forms, the step with smooth
PME added, the step with tabulated radial functions, the molecular-dynamics
step (ns/day), the 1 M-atom water box, clocks, and the FP64 oracle timed on the host cores (context
only).

Multi-GPU: every rank evaluates its own replica (no data-path collective);
value = pairs of all ranks / max step time over ranks.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pair interactions/s and ms per force eval at 23.5k atoms; % FP32 roofline"
UNIT = "pairs/s"
# kernels of this library per step: binning and lists (bin + scan + staging,
# column sort, pair lists); forward (pack, force, unpack + energy/virial);
# adjoint (pack, dL/dF gather, adjoint kernel, unpack, type-pair gradients);
# nb_step (rebuild + forces in one call: binning and column sort pack, no pack kernel)
BUILD_LAUNCHES = 3
FORCE_LAUNCHES = 3
STEP_LAUNCHES = BUILD_LAUNCHES + FORCE_LAUNCHES - 1
ADJOINT_LAUNCHES = 5
# smooth PME adds spread, solve, gather (+ the FFT library's forward and
# inverse transforms, not counted as this library's kernels)
PME_LAUNCHES = 3
PME_GRID, PME_ORDER = (64, 64, 64), 4  # the paper's DHFR setting
TABLE_INTERVALS = 4096  # the paper's lookup-table size
MD_DT_PS, MD_GRAPH_STEPS = 0.004, 10  # the paper's 4 fs step with mass repartitioning
MD_WATERS = 7833  # 23,499 atoms in 61.7 A, the size of the paper's DHFR system
# MD step: kick/drift + M-SHAKE, rebuild, forces (no unpack: the second
# half reads the fixed-point sums), PME, (bonded), kick + RATTLE + energies
MD_LAUNCHES = 1 + STEP_LAUNCHES - 1 + PME_LAUNCHES + 1
FLOP_PER_PAIR = 73  # LJ + switch + Ewald real space, FMA = 2, MUFU = 1
# algorithmic DRAM bytes of one rebuild per atom: positions in (12), wrapped
# coordinates and column out and back (20 + 20), scatter slot (8), sorted
# x,y,z,q + permutation + inverse (24), cluster boxes (4 per atom), z-bin
# index (~4), the half pair lists (~67 8-byte entries per 8-atom cluster in
# water at rc 9 A: 67), exclusion-mask records (~3.5 16-byte records per
# cluster: 7), group tables and segment lengths (4), partner lookups of the
# rigid waters (2 partners: original index and inverse permutation, 16)
BUILD_BYTES_PER_ATOM = 186
WORKLOAD = ("solvated-chain system, 23,500 atoms (2,500-atom chain + 7,000 TIP3P-shaped waters), "
            "62.2 A cubic box, rc 9 A, switch 7.5 A, Ewald alpha 0.32, 1-2/1-3 excluded, 1-4 scaled")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", action="store_true", help="skip adjoint/batched/e2e/cpu legs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--pme-only", action="store_true",
                    help="time only the step with smooth PME (for profiling its kernels)")
    ap.add_argument("--tables-only", action="store_true",
                    help="time only the step with tabulated radial functions (for profiling)")
    ap.add_argument("--md-only", action="store_true", help="time only the MD leg (for profiling)")
    ap.add_argument("--md-prep-steps", type=int, default=None,
                    help="minimiser moves and 2 fs equilibration steps before the timed MD steps "
                         f"(default {MD_MIN_STEPS} each; profiling runs use fewer so that a launch list "
                         "reaches the production steps)")
    ap.add_argument("--large-only", action="store_true", help="time only the 1 M-atom leg (for profiling)")
    ap.add_argument("--adjoint-only", action="store_true", help="time only the adjoint leg (for profiling)")
    ap.add_argument("--peak", action="store_true", help="only measure the FP32 FMA peak and print it")
    return ap.parse_args()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
            os.unlink(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    from paper_0902_0827_gb300 import replicas
    return replicas.setup("nccl")


def barrier(world):
    from paper_0902_0827_gb300 import replicas
    replicas.barrier(world)


def max_over_ranks(x: float, world: int) -> float:
    from paper_0902_0827_gb300 import replicas
    return replicas.max_over_ranks(x, world, "cuda")


def graph_of(fn, dev):
    """Capture fn() (already warmed up) into a CUDA graph on a side stream."""
    import torch
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    return g


def time_steps(fn, steps, flush):
    """Mean ms of fn() over `steps` calls, L2 flushed before each (outside the events)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record()
        fn()
        ev[k][1].record()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / steps


def measure_fp32_peak(dev, iters: int = 262144, reps: int = 5):
    """FP32 FMA throughput of this GPU (nb_fp32_peak_launch: independent
    dependent-FMA chains on every SM), best of `reps` launches timed with CUDA
    events on the launching stream, with the SM clocks sampled meanwhile."""
    import torch
    from paper_0902_0827_gb300 import nb
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    for _ in range(2):
        nb.fp32_peak_launch(iters, sink)
    torch.cuda.synchronize()
    clocks = Clocks(dev.index if dev.index is not None else 0)
    clocks.start()
    best = None
    flop = 0.0
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        flop = nb.fp32_peak_launch(iters, sink)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    clk = clocks.stop()
    return {"tflops": flop / (best * 1e-3) / 1e12, "ms_per_launch": best, "flop_per_launch": flop,
            "clocks": clk, "how": "nb_fp32_peak_launch: 8 independent FMA chains x 64 warps per SM, "
                                  "best of 5 launches, CUDA events"}


def adjoint_leg(ctx, pos, q, typ, steps, flush, fwd_ms, npairs):
    """Rebuild + adjoint (dL/dx, dL/dq, type-pair gradients) of the fitting
    loss sum |F - F_target|^2 on the same system, replayed from a CUDA graph."""
    import torch
    from paper_0902_0827_gb300 import systems as S
    N = pos.shape[0]
    Ft = torch.from_numpy(S.target_forces(S.solvated_chain())).to(pos.device)
    F, _, _ = ctx.forces(pos, q, typ, virial=False)
    G = (2.0 * (F - Ft)).contiguous()
    T = ctx.n_types
    gpos = torch.empty((N, 3), dtype=torch.float32, device=pos.device)
    gq = torch.empty((N,), dtype=torch.float32, device=pos.device)
    gs = torch.empty((T, T), dtype=torch.float64, device=pos.device)
    ge = torch.empty((T, T), dtype=torch.float64, device=pos.device)
    from paper_0902_0827_gb300 import nb

    def step():
        ctx.build(pos)
        ctx._sync_stream()
        nb._check(nb.lib().nb_backward(ctx.h, nb._tptr(pos), nb._tptr(q), nb._tptr(typ), nb._tptr(G), None,
                                       nb._tptr(gpos), nb._tptr(gq), nb._tptr(gs), nb._tptr(ge)), "nb_backward")

    for _ in range(3):
        step()
    g = graph_of(step, pos.device)
    ms = time_steps(g.replay, steps, flush)
    ctx.status()
    return {"ms_per_step": ms, "pairs_per_s": npairs / (ms * 1e-3), "ratio_to_forward": ms / fwd_ms,
            "step": "cell-list rebuild + adjoint of sum|F - F_target|^2 (HVP, dL/dq, dL/dsig_ab, dL/deps_ab)",
            "gpu_launches_per_step": BUILD_LAUNCHES + ADJOINT_LAUNCHES}


def pme_leg(s, steps, flush, dev, npairs, base_ms):
    """The same step with smooth PME on (64^3 grid, fourth-order B-splines):
    rebuild + short-range forces + reciprocal space + Ewald corrections,
    replayed from a CUDA graph; and the long-range part alone."""
    import torch
    from paper_0902_0827_gb300 import nb
    ctx = nb.Nonbonded(s)
    ctx.set_pme(PME_GRID, PME_ORDER)
    pos, q, typ = nb.concat_inputs([s], device=dev)
    N = s.n_atoms
    F = torch.empty((N, 3), dtype=torch.float32, device=dev)
    E = torch.empty((1, 2), dtype=torch.float64, device=dev)
    W = torch.empty((1, 6), dtype=torch.float64, device=dev)
    E3 = torch.empty((3,), dtype=torch.float64, device=dev)
    W6 = torch.empty((6,), dtype=torch.float64, device=dev)

    def step():
        ctx.step(pos, q, typ, F=F, energy=E, virial=W)

    def lr_step():
        ctx._sync_stream()
        nb._check(nb.lib().nb_pme_forces(ctx.h, nb._tptr(pos), nb._tptr(q), nb._tptr(F), nb._tptr(E3),
                                         nb._tptr(W6)), "nb_pme_forces")

    for _ in range(3):
        step()
        lr_step()
    g = graph_of(step, dev)
    ms = time_steps(g.replay, steps, flush)
    gl = graph_of(lr_step, dev)
    lr_ms = time_steps(gl.replay, steps, flush)
    ctx.status()
    return {"grid": list(PME_GRID), "order": PME_ORDER, "ms_per_step": ms,
            "pairs_per_s": npairs / (ms * 1e-3), "added_ms_vs_short_range": ms - base_ms,
            "long_range_only_ms": lr_ms,
            "step": "cell-list rebuild + short-range forces + smooth PME + Ewald self/exclusion corrections",
            "gpu_launches_per_step": STEP_LAUNCHES + PME_LAUNCHES}


def tables_leg(s, steps, flush, dev, npairs, base_ms, base_fo_ms):
    """The same step with the radial functions interpolated from 4096-interval
    tables (the paper's lookup-table variant) instead of evaluated directly:
    rebuild + forces, and the force evaluation alone."""
    import torch
    from paper_0902_0827_gb300 import nb
    ctx = nb.Nonbonded(s)
    ctx.set_tables(TABLE_INTERVALS)
    pos, q, typ = nb.concat_inputs([s], device=dev)
    N = s.n_atoms
    F = torch.empty((N, 3), dtype=torch.float32, device=dev)
    E = torch.empty((1, 2), dtype=torch.float64, device=dev)
    W = torch.empty((1, 6), dtype=torch.float64, device=dev)

    def step():
        ctx.step(pos, q, typ, F=F, energy=E, virial=W)

    def fstep():
        ctx.forces(pos, q, typ, F=F, energy=E, virial=W)

    for _ in range(3):
        step()
    g = graph_of(step, dev)
    ms = time_steps(g.replay, steps, flush)
    ctx.build(pos)
    gf = graph_of(fstep, dev)
    fo_ms = time_steps(gf.replay, steps, flush)
    ctx.status()
    return {"intervals": TABLE_INTERVALS, "ms_per_step": ms, "pairs_per_s": npairs / (ms * 1e-3),
            "force_only_ms": fo_ms, "speedup_vs_direct": base_ms / ms, "force_only_speedup_vs_direct": base_fo_ms / fo_ms,
            "step": "cell-list rebuild + forces with tabulated radial functions (linear interpolation)",
            "gpu_launches_per_step": STEP_LAUNCHES}


MD_MIN_STEPS, MD_MIN_DISP = 500, 0.01   # capped steepest descent before the dynamics
MD_EQ_DT_PS, MD_EQ_STEPS = 0.002, 500   # 1 ps at 2 fs


def md_leg(steps, flush, dev, prep_steps=None):
    """Molecular dynamics of the DHFR-shaped solvated chain (23,500 atoms:
    2,500-atom chain with bonds, angles, dihedrals, exclusions and scaled
    1-4 pairs + 7,000 rigid waters, 62.2 A) with the paper's DHFR settings:
    PME 64^3 / order 4 every step, rc 9 A switched at 7.5 A, M-SHAKE/RATTLE,
    hydrogen mass repartitioning and a 4 fs step, Langevin thermostat
    (1/ps, 300 K).  Protocol: MD_MIN_STEPS capped steepest-descent moves
    (nb_md_minimize), 1 ps of equilibration at 2 fs (friction 5/ps), 0.2 ps
    at 4 fs, then the timed production steps: MD_GRAPH_STEPS steps captured
    in one CUDA graph, the L2 flushed before each replay, the steps inside a
    replay back to back as in a production loop."""
    import math
    import torch
    from paper_0902_0827_gb300 import nb
    from paper_0902_0827_gb300 import systems as S
    s = S.dhfr_chain_md()
    n_chain = 2500
    top = S.hmr_masses(S.md_topology(s, n_chain=n_chain))
    ctx = nb.Nonbonded(s)
    ctx.set_pme(PME_GRID, PME_ORDER)
    pos, q, typ = nb.concat_inputs([s], device=dev)
    E = torch.empty(6, dtype=torch.float64, device=dev)
    ctx.md_init(top, dt=MD_EQ_DT_PS, gamma=5.0, temperature=300.0, seed=2008)
    ctx.md_minimize(pos, q, typ, 0, MD_MIN_DISP, E)
    e_start = E.cpu().numpy().copy()
    t0 = time.time()
    n_min = MD_MIN_STEPS if prep_steps is None else prep_steps
    n_eq = MD_EQ_STEPS if prep_steps is None else prep_steps
    ctx.md_minimize(pos, q, typ, n_min, MD_MIN_DISP, E)
    torch.cuda.synchronize()
    min_s = time.time() - t0
    e_min = E.cpu().numpy().copy()
    vel = torch.from_numpy(S.initial_velocities(top, 300.0)).to(dev)
    ctx.md_step(pos, vel, q, typ, n_eq, E)
    ctx.md_init(top, dt=MD_DT_PS, gamma=1.0, temperature=300.0, seed=2009)
    ctx.md_step(pos, vel, q, typ, 50, E)
    torch.cuda.synchronize()
    ctx.status()

    def run():
        ctx.md_step(pos, vel, q, typ, MD_GRAPH_STEPS, E)

    g = graph_of(run, dev)
    reps = max(3, steps // MD_GRAPH_STEPS)
    ms = time_steps(g.replay, reps, flush)
    ms /= MD_GRAPH_STEPS
    ctx.status()
    e = E.cpu().numpy()
    # degrees of freedom: 3 per atom, less 3 constraints per rigid water
    n_dof = 3 * s.n_atoms - 3 * len(top.waters)
    temp = 2.0 * e[5] / (n_dof * 0.0019872041)
    names = ("E_LJ", "E_Coul", "E_bond", "E_angle", "E_dihedral", "E_kin")
    return {"system": f"DHFR-shaped solvated chain, {s.n_atoms} atoms ({n_chain}-atom chain + "
                      f"{len(top.waters)} waters), {float(s.box[0]):.1f} A",
            "ms_per_step": ms, "ns_per_day": MD_DT_PS * 1e-3 * 86400.0 / (ms * 1e-3), "dt_fs": MD_DT_PS * 1e3,
            "temperature_K": temp, "stable": bool(all(math.isfinite(v) for v in e) and 200.0 < temp < 400.0),
            "steps_timed": reps * MD_GRAPH_STEPS,
            "protocol": {"minimize": {"steps": n_min, "max_disp_A": MD_MIN_DISP, "seconds": min_s,
                                      "E_start": dict(zip(names[:5], map(float, e_start[:5]))),
                                      "E_after": dict(zip(names[:5], map(float, e_min[:5])))},
                         "equilibrate": {"dt_fs": MD_EQ_DT_PS * 1e3, "steps": n_eq, "gamma_per_ps": 5.0},
                         "production": {"dt_fs": MD_DT_PS * 1e3, "gamma_per_ps": 1.0, "hmr": True,
                                        "pme": {"grid": list(PME_GRID), "order": PME_ORDER}}},
            "energies_last_step": dict(zip(names, map(float, e))),
            "step": "Langevin velocity Verlet: integrate, M-SHAKE, cell-list rebuild, short-range forces, PME, "
                    "bonded terms, integrate, RATTLE",
            "paper_context": "DHFR 17.55 ms/step, 19.7 ns/day on one GTX 280 (section Performance)",
            "gpu_launches_per_step": MD_LAUNCHES + 1}


def md_water_leg(steps, flush, dev):
    """The same MD step on a 23,499-atom water box (7,833 waters, 61.7 A):
    no bonded terms."""
    import torch
    from paper_0902_0827_gb300 import nb
    from paper_0902_0827_gb300 import systems as S
    s = S.water_box(n_waters=MD_WATERS)
    top = S.hmr_masses(S.md_topology(s))
    ctx = nb.Nonbonded(s)
    ctx.set_pme(PME_GRID, PME_ORDER)
    pos, q, typ = nb.concat_inputs([s], device=dev)
    vel = torch.from_numpy(S.initial_velocities(top, 300.0)).to(dev)
    E = torch.empty(6, dtype=torch.float64, device=dev)
    ctx.md_init(top, dt=MD_EQ_DT_PS, gamma=20.0, temperature=300.0, seed=2008)
    ctx.md_minimize(pos, q, typ, 100, MD_MIN_DISP, E)
    ctx.md_step(pos, vel, q, typ, MD_EQ_STEPS, E)
    ctx.md_init(top, dt=MD_DT_PS, gamma=1.0, temperature=300.0, seed=2009)
    ctx.md_step(pos, vel, q, typ, 50, E)
    torch.cuda.synchronize()

    def run():
        ctx.md_step(pos, vel, q, typ, MD_GRAPH_STEPS, E)

    g = graph_of(run, dev)
    reps = max(3, steps // MD_GRAPH_STEPS)
    ms = time_steps(g.replay, reps, flush) / MD_GRAPH_STEPS
    ctx.status()
    e = E.cpu().numpy()
    n_dof = 3 * s.n_atoms - 3 * len(top.waters)
    return {"system": f"water box, {s.n_atoms} atoms, {float(s.box[0]):.1f} A", "ms_per_step": ms,
            "ns_per_day": MD_DT_PS * 1e-3 * 86400.0 / (ms * 1e-3), "dt_fs": MD_DT_PS * 1e3,
            "temperature_K": 2.0 * e[5] / (n_dof * 0.0019872041), "steps_timed": reps * MD_GRAPH_STEPS,
            "gpu_launches_per_step": MD_LAUNCHES}


def large_leg(steps, flush, dev):
    """The 999,999-atom water box (333,333 waters, L ~ 215 A): rebuild +
    forces every step, the rebuild alone and the force evaluation alone,
    each replayed from a CUDA graph with the L2 flushed before every step;
    the force kernel's FP32 roofline and the rebuild's algorithmic DRAM
    bandwidth (BUILD_BYTES_PER_ATOM per atom)."""
    import torch
    from paper_0902_0827_gb300 import nb
    from paper_0902_0827_gb300 import systems as S
    s = S.big_water()
    ctx = nb.Nonbonded(s)
    pos, q, typ = nb.concat_inputs([s], device=dev)
    N = s.n_atoms
    F = torch.empty((N, 3), dtype=torch.float32, device=dev)
    E = torch.empty((1, 2), dtype=torch.float64, device=dev)
    W = torch.empty((1, 6), dtype=torch.float64, device=dev)

    def step():
        ctx.step(pos, q, typ, F=F, energy=E, virial=W)

    def bstep():
        ctx.build(pos)

    def fstep():
        ctx.forces(pos, q, typ, F=F, energy=E, virial=W)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    _, npairs, _ = ctx.debug_pairs(cap=0)
    reps = max(3, steps // 5)
    ms = time_steps(graph_of(step, dev).replay, reps, flush)
    b_ms = time_steps(graph_of(bstep, dev).replay, reps, flush)
    ctx.build(pos)
    f_ms = time_steps(graph_of(fstep, dev).replay, reps, flush)
    ctx.set_profiling(True)
    ctx.profile()
    for _ in range(reps):
        flush.zero_()
        fstep()
    kms, kl = ctx.profile()
    ctx.set_profiling(False)
    ctx.status()
    k_avg = kms / max(kl, 1)
    # tile shapes on the large box (the batched leg tunes the ensemble)
    from paper_0902_0827_gb300 import autotune
    cands = [dict(group_clusters=1, blocks_per_sm=3, list_split=1), dict(group_clusters=4, blocks_per_sm=3, list_split=2),
             dict(group_clusters=8, blocks_per_sm=3, list_split=4)]
    tuned = autotune.autotune(ctx, pos, q, typ, candidates=cands, reps=3, use_cache=False)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs") if peaks else None
    b_gbs = BUILD_BYTES_PER_ATOM * N / (b_ms * 1e-3) / 1e9
    return {"n_atoms": N, "pairs_per_step": npairs, "ms_per_step": ms, "pairs_per_s": npairs / (ms * 1e-3),
            "rebuild_ms": b_ms, "force_eval_ms": f_ms, "force_kernel_ms": k_avg,
            "force_kernel_tflops": FLOP_PER_PAIR * npairs / (k_avg * 1e-3) / 1e12,
            "rebuild_algorithmic_gbs": b_gbs,
            "rebuild_roofline": {"bound": "hbm", "achieved": b_gbs, "peak": hbm, "unit": "GB/s",
                                 "frac": b_gbs / hbm if hbm else None,
                                 "bytes_per_atom": BUILD_BYTES_PER_ATOM,
                                 "peak_basis": ("fallback copy bandwidth" if peaks.get("fallback") else
                                                "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)")},
            "tuning": {"group_clusters": 1, "blocks_per_sm": 3, "list_split": 1},
            "autotune_table": tune_table(tuned),
            "step": "cell-list rebuild + forces, energies and virial (rc 9 A, Ewald real space)",
            "gpu_launches_per_step": STEP_LAUNCHES}


def batched_leg(steps, flush, dev):
    """64 water boxes (log-uniform 500..20,000 atoms): one autotuned,
    graph-captured rebuild + force step of the whole batch vs 64 sequential
    per-system contexts with plain launches."""
    import torch
    from paper_0902_0827_gb300 import autotune, nb
    from paper_0902_0827_gb300 import systems as S
    systems = S.water_ensemble()
    ctx = nb.Nonbonded(systems)
    pos, q, typ = nb.concat_inputs(systems, device=dev)
    cands = ([dict(group_clusters=1, blocks_per_sm=b, list_split=c) for b in (2, 3) for c in (1, 2, 4)]
             + [dict(group_clusters=g, blocks_per_sm=b, list_split=c) for g in (4, 8) for b in (2, 3) for c in (2, 4)])
    rec = autotune.autotune(ctx, pos, q, typ, candidates=cands, reps=3)
    N = pos.shape[0]
    F = torch.empty((N, 3), device=dev)
    E = torch.empty((len(systems), 2), dtype=torch.float64, device=dev)
    W = torch.empty((len(systems), 6), dtype=torch.float64, device=dev)

    def step():
        ctx.step(pos, q, typ, F=F, energy=E, virial=W)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    _, npairs, _ = ctx.debug_pairs(cap=0)
    g = graph_of(step, dev)
    ms = time_steps(g.replay, steps, flush)
    ctx.status()
    # sequential: one context per system, plain launches one after another
    seq = []
    for s in systems:
        c = nb.Nonbonded(s)
        p1, q1, t1 = nb.concat_inputs([s], device=dev)
        seq.append((c, p1, q1, t1))

    def seq_step():
        for c, p1, q1, t1 in seq:
            c.step(p1, q1, t1)

    for _ in range(2):
        seq_step()
    torch.cuda.synchronize()
    seq_ms = time_steps(seq_step, max(3, steps // 5), flush)
    return {"n_systems": len(systems), "n_atoms": N, "pairs_per_step": npairs, "ms_per_step": ms,
            "pairs_per_s": npairs / (ms * 1e-3), "sequential_ms_per_step": seq_ms,
            "speedup_vs_sequential": seq_ms / ms, "tuning": rec["best"],
            "autotune_table": tune_table(rec), "gpu_launches_per_step": STEP_LAUNCHES}


def measured_peaks():
    """The machine's measured HBM copy bandwidth and GEMM peaks (a JSON file
    beside this script), or the published fallback copy bandwidth."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "fallback": True}


def tune_table(rec, best_per_group: bool = True):
    """The autotuner's timings (ms per rebuild + force step), the best
    candidate of every group size first, then the overall ranking."""
    out = {}
    for t, c in rec["table"]:
        g = c.get("group_clusters", 1)
        out.setdefault(f"group{g}", {"ms": t, **c})
    return {"best_per_group_size": out, "candidates": len(rec["table"]),
            "ranking": [{"ms": t, **c} for t, c in rec["table"][:6]]}


def force_kernel_traffic():
    """DRAM bytes per force-kernel launch from the committed ncu record, or
    None when the kernel sources changed since the counters were taken."""
    import hashlib
    prof_path = os.path.join(ROOT, "profiles", "force_kernel_traffic.json")
    try:
        rec = json.load(open(prof_path))
        h = hashlib.sha256()
        for src in rec["sources"]:
            h.update(open(os.path.join(ROOT, src), "rb").read())
        if h.hexdigest() != rec["source_sha256"]:
            return None
        return rec["bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        return None


def cpu_oracle_run(system, budget_s: float = 12.0, max_reps: int = 50):
    """The FP64 oracle (cell-list traversal, OpenMP over atoms) timed on the host."""
    import oracle
    oracle.build()
    times, npairs = [], 0
    t_end = time.perf_counter() + budget_s
    for _ in range(max_reps):
        t0 = time.perf_counter()
        _, _, _, npairs = oracle.forces(system, method="cells")
        times.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end:
            break
    return times, npairs, oracle.num_threads()


def cpu_context():
    """The FP64 oracle on every configuration, for context: the all-pairs
    sum (one thread: the oracle parallelises only the cell-list traversal)
    on the 256-atom crystal, the 6,144-atom water box and the 23,500-atom
    chain, and the cell-list traversal on all cores on the chain, the
    64-box ensemble and the 999,999-atom box; one or a few evaluations each
    (about half a minute in all)."""
    import oracle
    from paper_0902_0827_gb300 import systems as S
    oracle.build()
    cores = oracle.num_threads()
    rows = []

    def run(name, systems, method, threads, reps):
        oracle.set_threads(threads)
        best, npairs = None, 0
        for _ in range(reps):
            t0 = time.perf_counter()
            npairs = sum(oracle.forces(s, method=method)[3] for s in systems)
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        rows.append({"config": name, "method": method, "threads": threads, "ms_per_eval": best * 1e3,
                     "pairs_per_s": npairs / best, "evaluations": reps})

    try:
        fcc, water, chain = S.lj_fcc(), S.water_box(k=1, n_waters=2048), S.solvated_chain()
        for name, s, reps in (("lj_fcc 256", fcc, 20), ("water_box 6,144", water, 2),
                              ("solvated_chain 23,500", chain, 1)):
            run(name, [s], "allpairs", 1, reps)
        run("solvated_chain 23,500", [chain], "cells", cores, 5)
        run("water_ensemble 64 boxes", S.water_ensemble(), "cells", cores, 1)
        run("big_water 999,999", [S.big_water()], "cells", cores, 1)
    finally:
        oracle.set_threads(cores)
    return {"kind": "oracle", "cores": cores, "rows": rows}


def reference_arm(args, world, rank):
    """--impl reference: the FP64 CPU oracle on the same workload and metric."""
    if rank != 0:
        return 0
    from paper_0902_0827_gb300 import systems as S
    s = S.solvated_chain()
    import oracle
    oracle.build()
    for _ in range(max(args.warmup, 0)):
        oracle.forces(s, method="cells")
    times = []
    npairs = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, _, _, npairs = oracle.forces(s, method="cells")
        times.append(time.perf_counter() - t0)
    per = sum(times) / len(times)
    val = npairs / per
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_atoms": s.n_atoms, "pairs_per_step": npairs},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"full force evaluation of the {s.n_atoms}-atom system per step"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return reference_arm(args, world, rank)

    import numpy as np
    import torch

    from paper_0902_0827_gb300 import nb
    from paper_0902_0827_gb300 import systems as S

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    n_sms = props.multi_processor_count
    if args.peak:
        print(json.dumps({"fp32_peak": measure_fp32_peak(dev), "n_sms": n_sms}))
        return 0
    s = S.solvated_chain()
    if args.pme_only or args.tables_only or args.md_only or args.large_only or args.adjoint_only:
        flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)
        if args.adjoint_only:
            actx = nb.Nonbonded(s)
            apos, aq, atyp = nb.concat_inputs([s], device=dev)
            actx.build(apos)
            print(json.dumps({"adjoint": adjoint_leg(actx, apos, aq, atyp, args.steps, flush, float("nan"), 0)}))
        elif args.large_only:
            print(json.dumps({"large": large_leg(args.steps, flush, dev)}))
        elif args.pme_only:
            print(json.dumps({"pme": pme_leg(s, args.steps, flush, dev, 0, 0.0)}))
        elif args.md_only:
            print(json.dumps({"md": md_leg(args.steps, flush, dev, args.md_prep_steps)}))
        else:
            print(json.dumps({"tables": tables_leg(s, args.steps, flush, dev, 0, float("nan"), float("nan"))}))
        return 0
    ctx = nb.Nonbonded(s)
    pos, q, typ = nb.concat_inputs([s], device=dev)
    N = s.n_atoms
    F = torch.empty((N, 3), dtype=torch.float32, device=dev)
    E = torch.empty((1, 2), dtype=torch.float64, device=dev)
    W = torch.empty((1, 6), dtype=torch.float64, device=dev)

    def step():
        ctx.step(pos, q, typ, F=F, energy=E, virial=W)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    ctx.status()
    _, npairs, n_ordered = ctx.debug_pairs(cap=0)
    n_tiles, n_halves = ctx.debug_fill()

    # CUDA graph of one step, captured on a side stream
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()

    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)  # 512 MiB > L2
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record()
        g.replay()
        ev[k][1].record()
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    ms = max_over_ranks(ms, world)
    ctx.status()
    value = world * npairs / (ms * 1e-3)

    # roofline of the force kernel: events on the launching stream around each launch
    ctx.set_profiling(True)
    ctx.profile()
    for _ in range(args.steps):
        flush.zero_()
        step()
    fms, fl = ctx.profile()
    ctx.set_profiling(False)
    f_avg = fms / max(fl, 1)
    sm_max = clk.get("sm_max_mhz") or 2070.0
    sm_med = clk.get("sm_mhz") or sm_max
    # nominal FP32 peak at the median SM clock sampled during the timed steps
    peak_tflops = n_sms * 128 * 2 * sm_med * 1e6 / 1e12
    peak_at_max = n_sms * 128 * 2 * sm_max * 1e6 / 1e12
    achieved = FLOP_PER_PAIR * npairs / (f_avg * 1e-3) / 1e12
    fpk = measure_fp32_peak(dev)
    traffic = force_kernel_traffic()
    # force evaluation alone, the pair lists of the last rebuild reused
    # (positions unchanged), same graph and L2 protocol
    def fstep():
        ctx.forces(pos, q, typ, F=F, energy=E, virial=W)

    ctx.build(pos)
    for _ in range(3):
        fstep()
    gf = graph_of(fstep, dev)
    fo_ms = max_over_ranks(time_steps(gf.replay, args.steps, flush), world)
    ctx.status()
    force_only = {"ms_per_eval": fo_ms, "pairs_per_s": world * npairs / (fo_ms * 1e-3),
                  "step": "pack + force kernel + unpack, lists of the last rebuild"}

    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": traffic,
                "kernel": "k_force1 (FP32 pair arithmetic, i-groups of one cluster)", "ms_per_launch": f_avg,
                "peak_basis": (f"nominal: {n_sms} SMs x 128 FP32 lanes x 2 FLOP x {sm_med:.0f} MHz "
                               f"(median SM clock sampled during the timed steps)"),
                "peak_at_max_clock": peak_at_max, "sm_max_mhz": sm_max, "sm_mhz_used": sm_med,
                "peak_measured": fpk["tflops"], "frac_measured": achieved / fpk["tflops"],
                "peak_measured_basis": fpk["how"], "peak_measured_clocks": fpk["clocks"],
                "tile_fill": npairs / (64.0 * max(n_tiles, 1)), "lane_fill": npairs / (32.0 * max(n_halves, 1)),
                "fill_basis": (f"{npairs} pairs in {n_tiles} 8x8 tiles visited, {n_halves} 4x8 tile halves "
                               "evaluated: the useful fraction of the lanes that run the pair arithmetic")}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_atoms": N, "pairs_per_step": npairs,
                   "pair_evaluations": n_ordered, "l2": "flushed before every timed step",
                   "graph": "one CUDA graph per step", "parallelism": f"replicas x{world}",
                   "tuning": ctx.tuning()},
        "ms_per_force_eval": ms,
        "force_only": force_only,
        "roofline": roofline,
        "clocks": clk,
        "gpu_launches": (STEP_LAUNCHES) * args.steps,
    }

    if not args.no_extras:
        line["adjoint"] = adjoint_leg(ctx, pos, q, typ, args.steps, flush, ms, npairs)
        line["pme"] = pme_leg(s, args.steps, flush, dev, npairs, ms)
        line["tables"] = tables_leg(s, args.steps, flush, dev, npairs, ms, fo_ms)
        line["md"] = md_leg(args.steps, flush, dev)
        line["md_water"] = md_water_leg(args.steps, flush, dev)
        line["batched"] = batched_leg(args.steps, flush, dev)
        line["large"] = large_leg(args.steps, flush, dev)
        # end to end through the public API with host buffers (pinned): the
        # step's inputs (positions, charges, types) travel in one host->device
        # copy and its results (forces, energies, virial) in one
        # device->host copy, as a caller packing its buffers would do
        nb_in = N * 12 + N * 4 + N * 4
        out_f, out_e = N * 12, (N * 12 + 7) // 8 * 8
        nb_out = out_e + 2 * 8 + 6 * 8
        h_in = torch.empty(nb_in, dtype=torch.uint8).pin_memory()
        h_out = torch.empty(nb_out, dtype=torch.uint8).pin_memory()
        h_in[:N * 12].view(torch.float32).copy_(pos.cpu().reshape(-1))
        h_in[N * 12:N * 16].view(torch.float32).copy_(q.cpu())
        h_in[N * 16:].view(torch.int32).copy_(typ.cpu())
        d_in = torch.empty(nb_in, dtype=torch.uint8, device=dev)
        d_out = torch.empty(nb_out, dtype=torch.uint8, device=dev)
        dpos = d_in[:N * 12].view(torch.float32).view(N, 3)
        dq = d_in[N * 12:N * 16].view(torch.float32)
        dt = d_in[N * 16:].view(torch.int32)
        oF = d_out[:out_f].view(torch.float32).view(N, 3)
        oE = d_out[out_e:out_e + 16].view(torch.float64).view(1, 2)
        oW = d_out[out_e + 16:].view(torch.float64).view(1, 6)

        hpos = h_in[:N * 12].view(torch.float32).view(N, 3)
        hq = h_in[N * 12:N * 16].view(torch.float32)
        ht = h_in[N * 16:].view(torch.int32)
        hF = h_out[:out_f].view(torch.float32).view(N, 3)
        hE = h_out[out_e:out_e + 16].view(torch.float64).view(1, 2)
        hW = h_out[out_e + 16:].view(torch.float64).view(1, 6)

        def e2e_copy_step():  # copy engine: one copy in, one copy out
            d_in.copy_(h_in, non_blocking=True)
            ctx.step(dpos, dq, dt, F=oF, energy=oE, virial=oW)
            h_out.copy_(d_out, non_blocking=True)

        def e2e_step():  # the kernels read the inputs and write the results in the pinned buffers
            ctx.step(hpos, hq, ht, F=hF, energy=hE, virial=hW)

        bi, bo = nb_in, nb_out
        for name, fn in (("e2e_copy_engine", e2e_copy_step), ("e2e", e2e_step)):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            # the same CUDA-graph replay as the device-side step (transfers included)
            ge = graph_of(fn, dev)
            tt = [time_steps(ge.replay, 1, flush) for _ in range(args.steps)]
            e_ms = max_over_ranks(sum(tt) / len(tt), world)
            line[name] = {"value": world * npairs / (e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": bi,
                          "d2h_bytes_per_step": bo, "ms_per_step": e_ms}
            line["gpu_launches"] += (STEP_LAUNCHES) * args.steps
        line["e2e"]["transfer"] = ("inputs read and results written by the kernels in page-locked host memory "
                                   "across the host link (no copy-engine transfer); e2e_copy_engine: one "
                                   "host-to-device and one device-to-host copy per step")
        torch.cuda.synchronize()
        line["e2e"]["results_equal_device_step"] = bool(
            torch.equal(hF, F.cpu()) and torch.equal(hE, E.cpu()) and torch.equal(hW, W.cpu()))
        ctx.status()
    if rank == 0 and not args.no_cpu and world == 1:
        times, cp, cores = cpu_oracle_run(s)
        per = sum(times) / len(times)
        line["cpu_baseline"] = {"value": cp / per, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{len(times)} full FP64 cell-list evaluations of the {N}-atom system",
                                "ms_per_eval": per * 1e3}
        line["cpu_context"] = cpu_context()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
