"""Benchmark: bead-updates/s of one dynamic-bonding call plus bonded forces.

A step is dynbond_step + dynbond_forces on a fresh snapshot of the plain
1,048,576-bead DNA-like workload (8192 strands x 64 nt, density 0.5), inputs
resident in HBM; L2 is flushed (256 MB write) between timed steps and each
step is timed with CUDA events on the library's stream.  value = beads x
steps / device time, summed over all ranks (weak scaling: every rank runs its
own independent system; there is no data-path collective).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (the paper ships no program, so the
oracle is the reference arm) on the same workload, metric and unit, on the
host cores.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "bead-updates/s of dynbond_step+dynbond_forces"
UNIT = "bead-updates/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-baseline-seconds", type=float, default=12.0)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-melt", action="store_true", help="skip the 16M-bead melting leg")
    ap.add_argument("--cell-scale", type=int, default=0,
                    help="fixed cell edge (x the creation reach) instead of autotuning, e.g. for profiler runs, "
                         "under which the autotuner's timings mean nothing")
    ap.add_argument("--cell-zdiv", type=int, default=1, help="z cells per x / y edge with --cell-scale")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, device=None) -> float:
    """The largest of the ranks' values (the slowest rank's time); x itself
    when the job has one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(beads_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Bead-updates/s of the whole job: every rank updates its own system of
    beads_per_rank beads per step (weak scaling); seconds is the slowest
    rank's time for the steps."""
    return beads_per_rank * steps * world / seconds


def workload(rank: int):
    from paper_1108_4214_gb300 import workloads as W
    s = W.config2()
    if rank:
        s = W.dna_system(s.name, 8192, 64, 0.5, 2 + 1000 * rank, W.rules_dna2())
    return s


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        loaded = [x for x in sm if mx and x > 0.5 * max(mx)] or sm
        return {"sm_mhz": float(np.median(loaded)) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


def algorithmic_bytes(stats_before, st, N, R):
    """Minimum bytes one step + forces must move (per the design notes):
    positions and slots read for the search and the breakage scan, candidate
    edges written and read, nominations per round, the angle / dihedral lists
    read by the purge and the forces, records written, and the forces."""
    c = {k: int(v) for k, v in st.items()}
    na0, nd0 = stats_before
    b = 16 * N + 16 * N  # positions + slots: candidate search / breakage scan
    b += 2 * 16 * c["candidates"] * 2  # edge list (both directions) written and read
    b += 8 * 2 * c["candidates"]  # one nomination per directed candidate (later rounds touch fewer)
    b += 16 * (na0 + nd0)  # purge reads both lists
    b += 16 * (c["angles_added"] + c["dihedrals_added"])  # appended records
    b += 16 * N + 16 * N + 16 * (c["n_angles"] + c["n_dihedrals"]) + 16 * N + 56 * R  # forces
    return b


PHASE_KERNEL = {"bead": "k_bead", "candidates": "k_candidates", "match": "k_match", "edit": "k_edit",
                "purge": "k_purge", "bond_forces": "k_bond_forces",
                "angle_dihedral_forces": "k_angle_dihedral_forces"}


def sources_sha1():
    import glob
    import hashlib
    csrc = os.path.join(ROOT, "paper_1108_4214_gb300", "csrc")
    h = hashlib.sha1()
    for f in sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")) +
                    glob.glob(os.path.join(csrc, "*.h"))):
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(phase, tuning=None):
    """DRAM bytes per launch of the phase's kernel from the committed ncu
    summary, or None if none was recorded or the kernel sources changed since."""
    kern = phase_kernel(phase, tuning) if phase in PHASE_KERNEL else None
    path = os.path.join(ROOT, "profiles", "traffic_plain-1M.txt")
    if kern is None or not os.path.exists(path):
        return None
    sha = sources_sha1()
    for line in open(path):
        parts = line.split()
        if len(parts) == 3 and parts[0] == kern and parts[2] == sha:
            return int(parts[1])
    return None


def phase_kernel(phase, tuning):
    """The kernel the roofline names for a phase (the candidate search runs the
    octant kernel when the tuned cell columns are at least twice the reach wide)."""
    if phase == "candidates" and tuning and tuning.get("octant"):
        return "k_candidates_oct"
    return PHASE_KERNEL.get(phase, phase)


def kernel_bytes(phase, N, st, na_before, nd_before):
    """Algorithmic bytes of one launch of the phase that dominates the step."""
    if phase == "bead":  # positions, the eligibility bit, the bead's cell
        return 16 * N + N // 8 + 4 * N
    if phase == "purge":  # every record read once; each hole takes one tail record (read + write)
        return 16 * (na_before + nd_before) + 2 * 16 * (st["angles_removed"] + st["dihedrals_removed"])
    if phase == "bond_forces":
        return 16 * N + 16 * N + 16 * N  # positions, slots, forces
    if phase == "angle_dihedral_forces":  # records + one force read-modify-write per role
        return 16 * (st["n_angles"] + st["n_dihedrals"]) + 2 * 16 * (3 * st["n_angles"] + 4 * st["n_dihedrals"])
    if phase == "candidates":  # the search step's bytes: positions for the search (16 B per bead), the
        # reactive beads' slots for the exclusion and maxbond tests (16 B per base, N / 2 of them), and
        # the candidate edges written and read (16 B at each end of each pair)
        return 16 * N + 16 * (N // 2) + 32 * st["candidates"]
    if phase == "cells":  # per reactive bead: position read and sorted entry written (16 B each); the cell of every bead
        return 16 * N // 2 * 2 + 8 * N
    return None


def dominant_roofline(phases, N, stats, na_before, nd_before, tuning, peak, peak_kind, traffic_ok=True):
    """Roofline of the phase with the longest device time (setup excluded):
    its algorithmic bytes per launch over its event time."""
    if not phases:
        return None
    dom = max((k for k in phases if not k.endswith("setup")), key=lambda k: phases[k])
    kb = kernel_bytes(dom, N, stats, na_before, nd_before)
    if kb is None or phases[dom] <= 0:
        return dict(kernel=phase_kernel(dom, tuning), ms_per_launch=phases[dom], bytes_per_launch=None)
    ach = kb / (phases[dom] * 1e-3) / 1e9
    return dict(bound="hbm", kernel=phase_kernel(dom, tuning), achieved=ach, peak=peak, unit="GB/s",
                frac=ach / peak, peak_source=peak_kind, bytes_per_launch=kb, ms_per_launch=phases[dom],
                traffic=recorded_traffic(dom, tuning) if traffic_ok else None)


def profiled_phases(system, snaps, warmup, steps, flush, stream, geo=None):
    """Mean per-phase device times (ms) of a context created with
    DYNBOND_FLAG_PROFILE over the timed calls (events between the phases)."""
    import torch

    from paper_1108_4214_gb300 import dynbond
    dev = snaps[0].device
    ctx = dynbond.Context(system, flags=dynbond.FLAG_PROFILE, stream=stream, params=geo)
    if not geo:
        ctx.autotune(snaps[0])
    f = torch.empty((system.n_beads, 4), dtype=torch.float32, device=dev)
    ev = torch.empty((system.n_replicas, 7), dtype=torch.float64, device=dev)
    phases = {}
    for k in range(warmup + steps):
        flush.zero_()
        ctx.step(snaps[k], k)
        ctx.forces(snaps[k], f, ev)
        if k >= warmup:
            for name, ms in ctx.phase_times().items():
                phases.setdefault(name, []).append(ms)
    ctx.close()
    return {k: float(np.mean(v)) for k, v in phases.items()}


def tuning_params(tuning):
    """Context parameters that reproduce a tuned geometry (cell edge and z
    division) without running the autotuner again."""
    if not tuning:
        return {}
    return dict(cell_scale=int(round(tuning["cell_scale"])) if float(tuning["cell_scale"]).is_integer() else 0,
                cell_zdiv=int(tuning["cell_zdiv"]))


def call(ctx, pos, k, force, ev, combined=True):
    """One step + forces: dynbond_step_forces, or the two calls in turn."""
    if combined:
        ctx.step_forces(pos, k, force, ev)
    else:
        ctx.step(pos, k)
        ctx.forces(pos, force, ev)


def time_calls(ctx, snaps, warmup, steps, flush, stream, force, ev, combined=True):
    """Device time (ms, summed) of `steps` step + forces calls after `warmup`
    untimed ones, L2 flushed before each, CUDA events on the stream."""
    import torch
    for k in range(warmup):
        call(ctx, snaps[k], k, force, ev, combined)
    torch.cuda.synchronize()
    total = 0.0
    for k in range(warmup, warmup + steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        call(ctx, snaps[k], k, force, ev, combined)
        b.record(stream)
        b.synchronize()
        total += a.elapsed_time(b)
    return total


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1108_4214_gb300 import dynbond

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", torch.cuda.current_device())
    torch.cuda.set_device(dev)
    s = workload(rank)
    N, R = s.n_beads, s.n_replicas
    K, Wm = args.steps, args.warmup
    snaps_np = s.snapshots(0, K + Wm)
    snaps = [torch.from_numpy(x).to(dev) for x in snaps_np]
    stream = torch.cuda.current_stream()
    geo = dict(cell_scale=args.cell_scale, cell_zdiv=args.cell_zdiv) if args.cell_scale > 0 else None
    ctx = dynbond.Context(s, stream=stream, params=geo)
    tuning = ctx.tuning() if geo else ctx.autotune(snaps[0])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    force = torch.empty((N, 4), dtype=torch.float32, device=dev)
    ev = torch.empty((R, 7), dtype=torch.float64, device=dev)
    for k in range(Wm):
        call(ctx, snaps[k], k, force, ev)
    ctx.sync()
    times = []
    with ClockSampler(dev.index) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(Wm, Wm + K):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            call(ctx, snaps[k], k, force, ev)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    total_ms = max_over_ranks(float(np.sum(times)), dev)
    # the same calls with the whole step as one persistent launch
    ctx_q = dynbond.Context(s, stream=stream, params=dict(geo or {}, **tuning_params(tuning)),
                            flags=dynbond.FLAG_PERSISTENT)
    persist_ms = time_calls(ctx_q, snaps, Wm, K, flush, stream, force, ev, combined=False) / K
    ctx_q.close()
    # the same work as the two calls dynbond_step, dynbond_forces in turn
    ctx_2 = dynbond.Context(s, stream=stream, params=dict(geo or {}, **tuning_params(tuning)))
    two_ms = time_calls(ctx_2, snaps, Wm, K, flush, stream, force, ev, combined=False) / K
    ctx_2.close()
    # per-phase device times from a second context that records events
    # between the phases (events inside the replayed work serialize the
    # kernels, so the headline above is timed without them)
    phases = profiled_phases(s, snaps, Wm, K, flush, stream, geo)
    # statistics of one more (untimed) call for the algorithmic byte counts
    na_before, nd_before = ctx.topology()[1].shape[0], ctx.topology()[2].shape[0]
    st = ctx.step(snaps[-1], Wm + K, stats=True)
    stats = {n: int(st[:, j].sum()) for j, n in enumerate(dynbond.STAT_NAMES)}
    ctx.forces(snaps[-1], force, ev)
    ctx.sync()
    value = whole_job_value(N, K, world, total_ms / 1e3)
    result = dict(value=value, ms=total_ms / K, N=N, R=R, phases=phases, persistent_ms=persist_ms, two_ms=two_ms,
                  stats=stats, na_before=na_before, nd_before=nd_before, clocks=clk.summary(), rank=rank,
                  world=world, name=s.name, tuning=tuning)

    # end to end through the host-buffer entry point: pinned host input, result read back
    pin_pos = torch.empty((N, 4), dtype=torch.int32).pin_memory()
    pin_f = torch.empty((N, 4), dtype=torch.float32).pin_memory()
    pin_ev = torch.empty((R, 7), dtype=torch.float64).pin_memory()
    ctx_h = dynbond.Context(s, stream=stream, params=geo)
    for k in range(min(Wm, 3)):
        pin_pos.copy_(torch.from_numpy(snaps_np[k]))
        ctx_h.run_host(pin_pos, k, pin_f, pin_ev)
    e2e_s = 0.0
    for k in range(Wm, Wm + K):
        pin_pos.copy_(torch.from_numpy(snaps_np[k]))
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx_h.run_host(pin_pos, k, pin_f, pin_ev)
        e2e_s += time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dev)
    result["e2e"] = dict(value=whole_job_value(N, K, world, e2e_s), unit=UNIT, h2d_bytes_per_step=16 * N,
                         d2h_bytes_per_step=16 * N + 56 * R)
    ctx_h.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return result


def run_batched(steps: int, warmup: int):
    """Batched vs plain on the 512-replica temperature ladder: one context
    holding every replica (one launch sequence per call, autotuned geometry)
    against one context per replica called one after another on the same
    stream.  Both time step + forces per call with CUDA events, L2 flushed
    between calls."""
    import torch

    from paper_1108_4214_gb300 import dynbond
    from paper_1108_4214_gb300 import workloads as W
    full = W.config3()
    N = full.n_beads
    snaps = full.snapshots(0, steps + warmup)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(run_call):
        for k in range(warmup):
            run_call(k)
        torch.cuda.synchronize()
        total = 0.0
        for k in range(warmup, warmup + steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run_call(k)
            b.record(stream)
            b.synchronize()
            total += a.elapsed_time(b)
        return total

    pos_all = [torch.from_numpy(x).to(dev) for x in snaps]
    ctx = dynbond.Context(full, stream=stream)
    f = torch.empty((N, 4), dtype=torch.float32, device=dev)
    ev = torch.empty((full.n_replicas, 7), dtype=torch.float64, device=dev)
    tuning = ctx.autotune(pos_all[0])

    def batched_call(k):
        call(ctx, pos_all[k], k, f, ev)
    t_b = timed(batched_call)
    ctx_q = dynbond.Context(full, stream=stream, params=tuning_params(tuning), flags=dynbond.FLAG_PERSISTENT)

    def persistent_call(k):
        ctx_q.step(pos_all[k], k)
        ctx_q.forces(pos_all[k], f, ev)
    t_q = timed(persistent_call)
    ctx_q.close()
    # one more (untimed) call for the algorithmic byte count of a call
    topo = ctx.topology()
    na0, nd0 = topo[1].shape[0], topo[2].shape[0]
    st = ctx.step(pos_all[-1], warmup + steps, stats=True)
    ctx.forces(pos_all[-1], f, ev)
    stats = {n: int(st[:, j].sum()) for j, n in enumerate(dynbond.STAT_NAMES)}
    ctx.sync()
    ctx.close()

    subs, sub_pos, sub_f, sub_ev = [], [], [], []
    for r in range(full.n_replicas):
        sub = W.sub_replicas(full, [r])
        c = dynbond.Context(sub, stream=stream, flags=dynbond.FLAG_NO_AUTOTUNE)
        sl = slice(int(full.bead_offset[r]), int(full.bead_offset[r + 1]))
        subs.append(c)
        sub_pos.append([p[sl] for p in pos_all])
        sub_f.append(f[sl])
        sub_ev.append(ev[r:r + 1])

    def plain_call(k):
        for r, c in enumerate(subs):
            call(c, sub_pos[r][k], k, sub_f[r], sub_ev[r])
    t_p = timed(plain_call)
    for c in subs:
        c.sync()
        c.close()
    vb = N * steps / (t_b / 1e3)
    vp = N * steps / (t_p / 1e3)
    alg = algorithmic_bytes((na0, nd0), stats, N, full.n_replicas)
    peak, peak_kind = peaks()
    ach = alg / (t_b / steps * 1e-3) / 1e9
    phases = profiled_phases(full, pos_all, warmup, steps, flush, stream)
    return dict(workload=full.name, replicas=full.n_replicas, beads=N, steps=steps, warmup=warmup,
                value=vb, ms_per_step=t_b / steps, plain_value=vp, plain_ms_per_step=t_p / steps,
                persistent=dict(ms_per_step=t_q / steps, value=N * steps / (t_q / 1e3),
                                note="the two calls with each step one persistent cooperative launch"),
                speedup=vb / vp, tuning=tuning, unit=UNIT,
                plain="one context per replica, called one after another on one stream",
                phases_ms=phases,
                roofline=dominant_roofline(phases, N, stats, na0, nd0, tuning, peak, peak_kind, traffic_ok=False),
                step_roofline=dict(bound="hbm", algorithmic_bytes=alg, achieved=ach, peak=peak, unit="GB/s",
                                   frac=ach / peak, peak_source=peak_kind))


def run_melt(steps: int, warmup: int):
    """The high-turnover melting workload at its full size (16,777,216 beads,
    131,072 strands x 64 nt, half of them in duplexes; form p 0.9, break p
    0.5): step + forces per call with CUDA events, L2 flushed between calls,
    per-phase times from a profiled context, roofline of the dominant phase."""
    import torch

    from paper_1108_4214_gb300 import dynbond
    from paper_1108_4214_gb300 import workloads as W
    s = W.config4()
    N, R = s.n_beads, s.n_replicas
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    snaps = [torch.from_numpy(x).to(dev) for x in s.snapshots(0, steps + warmup)]
    ctx = dynbond.Context(s, stream=stream)
    tuning = ctx.autotune(snaps[0])
    f = torch.empty((N, 4), dtype=torch.float32, device=dev)
    ev = torch.empty((R, 7), dtype=torch.float64, device=dev)
    for k in range(warmup):
        call(ctx, snaps[k], k, f, ev)
    torch.cuda.synchronize()
    total = 0.0
    for k in range(warmup, warmup + steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        call(ctx, snaps[k], k, f, ev)
        b.record(stream)
        b.synchronize()
        total += a.elapsed_time(b)
    topo = ctx.topology()
    na0, nd0 = topo[1].shape[0], topo[2].shape[0]
    st = ctx.step(snaps[-1], warmup + steps, stats=True)
    ctx.forces(snaps[-1], f, ev)
    stats = {n: int(st[:, j].sum()) for j, n in enumerate(dynbond.STAT_NAMES)}
    ctx.sync()
    ctx.close()
    phases = profiled_phases(s, snaps, warmup, steps, flush, stream)
    peak, peak_kind = peaks()
    alg = algorithmic_bytes((na0, nd0), stats, N, R)
    ach = alg / (total / steps * 1e-3) / 1e9
    return dict(workload=s.name, beads=N, steps=steps, warmup=warmup, value=N * steps / (total / 1e3), unit=UNIT,
                ms_per_step=total / steps, tuning=tuning, phases_ms=phases, stats_last_call=stats,
                roofline=dominant_roofline(phases, N, stats, na0, nd0, tuning, peak, peak_kind, traffic_ok=False),
                step_roofline=dict(bound="hbm", algorithmic_bytes=alg, achieved=ach, peak=peak, unit="GB/s",
                                   frac=ach / peak, peak_source=peak_kind))


def cpu_baseline(seconds: float):
    """The oracle as it stands, serial on one host core, on a bounded sample
    of the same workload: as many whole step + forces calls as fit in about
    `seconds` (at least one)."""
    from oracle import oracle as O
    s = workload(0)
    o = O.Oracle(s)
    snaps = s.snapshots(0, 64)
    n = 0
    t0 = time.perf_counter()
    while True:
        o.step(snaps[n], n)
        o.forces(snaps[n])
        n += 1
        if time.perf_counter() - t0 > seconds or n == len(snaps):
            break
    dt = time.perf_counter() - t0
    return dict(value=s.n_beads * n / dt, unit=UNIT, cores=1, kind="oracle",
                sample=f"{n} consecutive calls (step + forces) of the 1,048,576-bead workload, serial C++ oracle")


def reference_arm(args):
    """The oracle timed as the reference implementation: W untimed calls,
    then K timed calls of step + forces on the same workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    s = workload(0)
    o = O.Oracle(s)
    K, Wm = args.steps, args.warmup
    snaps = s.snapshots(0, K + Wm)
    for k in range(Wm):
        o.step(snaps[k], k)
        o.forces(snaps[k])
    t0 = time.perf_counter()
    for k in range(Wm, Wm + K):
        o.step(snaps[k], k)
        o.forces(snaps[k])
    dt = time.perf_counter() - t0
    v = s.n_beads * K / dt
    line = dict(impl="reference", metric=METRIC, value=v, unit=UNIT, n_gpus=args.gpus, steps=K, warmup=Wm,
                ms_per_step=1e3 * dt / K, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="int64+f64",
                data="synthetic",
                config=dict(workload=s.name, beads=s.n_beads, replicas=1, parallelism="replicas x1",
                            step="dynbond_step + dynbond_forces (the oracle's step and forces)"),
                cpu_baseline=dict(value=v, unit=UNIT, cores=1, kind="oracle",
                                  sample=f"{K} timed calls (step + forces) of the workload, serial C++ oracle"),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.steps < 1 or args.warmup < 3:
        raise SystemExit("need --steps >= 1 and --warmup >= 3")
    if args.impl == "reference":
        reference_arm(args)
        return
    import __graft_entry__  # noqa: F401  (path setup only)
    res = run_gpu(args)
    if res["rank"] != 0:
        return
    batched = None if args.no_batched or res["world"] > 1 else run_batched(10, 3)
    melt = None if args.no_melt or res["world"] > 1 else run_melt(5, 3)
    peak, peak_kind = peaks()
    ph = res["phases"]
    roof = dominant_roofline(ph, res["N"], res["stats"], res["na_before"], res["nd_before"], res["tuning"], peak,
                             peak_kind)
    alg = algorithmic_bytes((res["na_before"], res["nd_before"]), res["stats"], res["N"], res["R"])
    step_gbs = alg / (res["ms"] * 1e-3) / 1e9
    rank, world, _ = dist_env()
    cpu = cpu_baseline(args.cpu_baseline_seconds) if world == 1 else None
    kernels_per_step = 1 + 12 + 3  # argument kernel; the step's 12 kernels; bond, angle / dihedral, energy output
    line = dict(
        metric=METRIC, value=res["value"], unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=res["ms"], higher_is_better=True, scaling="weak", vs_baseline=None, dtype="int64+f32",
        data="synthetic",
        config=dict(workload=res["name"], beads=res["N"], replicas=res["R"], parallelism=f"replicas x{world}",
                    l2="flushed between timed steps (256 MB write)",
                    step="dynbond_step_forces (dynbond_step + dynbond_forces in one call)",
                    tuning=res["tuning"]),
        roofline=roof,
        step_roofline=dict(bound="hbm", algorithmic_bytes=alg, achieved=step_gbs, peak=peak, unit="GB/s",
                           frac=step_gbs / peak, peak_source=peak_kind),
        phases_ms=ph, cpu_baseline=cpu, e2e=res["e2e"], gpu_launches=kernels_per_step * args.steps,
        persistent=dict(ms_per_step=res["persistent_ms"], value=res["N"] * res["world"] / (res["persistent_ms"] * 1e-3),
                        note="the two calls with each step one persistent cooperative launch"),
        two_calls=dict(ms_per_step=res["two_ms"], value=res["N"] * res["world"] / (res["two_ms"] * 1e-3),
                       note="dynbond_step then dynbond_forces, the kernel graph of each"),
        clocks=res["clocks"], stats_last_call=res["stats"], batched=batched, melt=melt,
    )
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
