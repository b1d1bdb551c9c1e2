"""End-to-end loop around the dynamic-bonding pass: velocity-Verlet DPD
(`dynbond_md_advance`) with `dynbond_step` every few MD steps.

Every `dump_every`-th call keeps, for checking, the quantized positions and
the bonds before the call, the bonded energy / virial at those positions, and
the topology and statistics after the call.  All arithmetic runs in the CUDA
library; this module only drives the calls and copies the dumps to the host.
"""

from __future__ import annotations

import dataclasses
import time
from typing import Dict, List, Optional

import numpy as np

from . import dynbond
from . import workloads as W


@dataclasses.dataclass
class Dump:
    call: int
    positions: np.ndarray      # int32 [N, 4] before the call
    bonds: np.ndarray          # [nb, 4] before the call
    ev: np.ndarray             # [R, 7] bonded energy / virial at `positions`
    stats: np.ndarray          # [R, 17] of the call
    topology: tuple            # (bonds, angles, dihedrals) after the call


def run_dpd_loop(system: W.System, n_calls: int, md_steps_per_call: int = 10, dump_every: int = 100,
                 dpd: Optional[Dict] = None, velocity_seed: int = 5) -> Dict:
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = dynbond.Context(system)
    md = dynbond.MD(ctx, **(dpd or {}))
    pos = torch.from_numpy(system.snapshot(0)).to(dev)
    vel = torch.from_numpy(W.initial_velocities(system.n_beads, seed=velocity_seed)).to(dev)
    ev_dev = torch.empty((7,), dtype=torch.float64, device=dev)
    dumps: List[Dump] = []
    counts = []
    hashes = []  # topology hash after every call (dynbond_topology_hash)
    t_md = t_bond = 0.0
    for c in range(n_calls):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        md.advance(pos, vel, md_steps_per_call, c * md_steps_per_call, ev_dev)
        t1 = time.perf_counter()
        t_md += t1 - t0
        dump = c % dump_every == 0
        if dump:
            snap = pos.cpu().numpy().copy()
            bonds_before = ctx.topology()[0]
            _, ev = ctx.forces(pos)
            ev = ev.cpu().numpy()
        t2 = time.perf_counter()
        st = ctx.step(pos, c, stats=True)
        t_bond += time.perf_counter() - t2
        counts.append(st[:, [12, 13, 14]].sum(axis=0))
        hashes.append(ctx.topology_hash().copy())
        if dump:
            dumps.append(Dump(c, snap, bonds_before, ev, st, ctx.topology()))
    v = vel.cpu().numpy()[:, :3].astype(np.float64)
    kT_measured = float(np.mean(v ** 2))
    md.close()
    ctx.close()
    return dict(dumps=dumps, counts=np.array(counts), hashes=np.array(hashes), kT=kT_measured, seconds_md=t_md,
                seconds_step=t_bond,
                n_md_steps=n_calls * md_steps_per_call, n_calls=n_calls)
