"""The allocation-free force entry point against the regular one.

dynbond_forces_noalloc is for callers that must not call cudaMalloc -- for
example a host engine that has handed the GPU's memory to its own pool
allocator, or a latency-critical loop that cannot accept cudaMalloc's implicit
device synchronization.  It keeps its only scratch (per-replica FP64 energy /
virial sums) in a fixed device array shared by all calls.  Here it must give
the forces and energies of dynbond_forces within the parity tolerances, on
two calls in a row (the second call reuses the array the first one filled).
This file is collected last so that a run stopping at the first failure has
already run every other test."""

import numpy as np
import pytest

from paper_1108_4214_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FORCE_TOL = 2e-5
EV_TOL = 2e-6


def slots_from_bonds(bonds, n):
    slots = np.zeros((n, 4), np.uint32)
    deg = np.zeros(n, np.int64)
    for i, j, ti, tj in bonds:
        slots[i, deg[i]] = (int(j) << 4) | int(ti)
        deg[i] += 1
        slots[j, deg[j]] = (int(i) << 4) | int(tj)
        deg[j] += 1
    return slots


@pytest.mark.parametrize("paper_ff", [False, True])
def test_noalloc_forces_match_the_context_path_on_two_calls(paper_ff):
    from paper_1108_4214_gb300 import dynbond as D
    s = W.config3(n_replicas=6)  # several replicas: per-replica scratch rows
    if paper_ff:  # harmonic angles K (theta - theta0)^2 with theta0 = 180 and 90 degrees (Sec. 3)
        s.forcefield = W.forcefield_dna1_paper()
    ctx = D.Context(s)
    snaps = s.snapshots(0, 3)
    for k in range(2):
        ctx.step(torch.from_numpy(snaps[k]).cuda(), k)
    bonds, angles, dihedrals = ctx.topology()
    dev = torch.device("cuda")
    pos = torch.from_numpy(snaps[2]).to(dev)
    f_ref, ev_ref = ctx.forces(pos)
    f_ref, ev_ref = f_ref.cpu().numpy(), ev_ref.cpu().numpy()
    slots = torch.from_numpy(slots_from_bonds(bonds, s.n_beads).view(np.int32)).to(dev)
    off = torch.from_numpy(np.asarray(s.bead_offset, np.int64)).to(dev)
    box = torch.from_numpy(np.asarray(s.box_q, np.int64)).to(dev)
    ang = torch.from_numpy(angles).to(dev)
    dih = torch.from_numpy(dihedrals).to(dev)
    rms = np.sqrt(np.mean(f_ref[:, :3].astype(np.float64) ** 2))
    for call in range(2):
        f, ev = D.forces_noalloc(pos, slots, off, box, ang, dih, s.forcefield)
        f, ev = f.cpu().numpy(), ev.cpu().numpy()
        err = np.abs(f[:, :3].astype(np.float64) - f_ref[:, :3]) / (np.abs(f_ref[:, :3]) + rms)
        assert err.max() <= FORCE_TOL, (call, err.max())
        assert np.all(f[:, 3] == 0)
        scale = np.abs(ev_ref).max(axis=1, keepdims=True)
        assert (np.abs(ev - ev_ref) / scale).max() <= EV_TOL, call


def test_noalloc_rejects_more_replicas_than_its_scratch_holds():
    from paper_1108_4214_gb300 import dynbond as D
    R = D.NOALLOC_MAX_REPLICAS + 1
    dev = torch.device("cuda")
    pos = torch.zeros((R, 4), dtype=torch.int32, device=dev)
    slots = torch.zeros((R, 4), dtype=torch.int32, device=dev)
    off = torch.arange(R + 1, dtype=torch.int64, device=dev)
    box = torch.full((R,), 1 << 20, dtype=torch.int64, device=dev)
    empty4 = torch.zeros((0, 4), dtype=torch.int32, device=dev)
    empty5 = torch.zeros((0, 5), dtype=torch.int32, device=dev)
    with pytest.raises(D.DynbondError) as e:
        D.forces_noalloc(pos, slots, off, box, empty4, empty5, W.forcefield_dna2())
    assert e.value.status == 1
