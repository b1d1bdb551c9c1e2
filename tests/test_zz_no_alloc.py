"""The allocation-free force entry point.

dynbond_forces_noalloc is for callers that must not call cudaMalloc -- for
example a host engine that has handed the GPU's memory to its own pool
allocator, or a latency-critical loop that cannot accept cudaMalloc's implicit
device synchronization.  It keeps its only scratch (per-replica FP64 energy /
virial sums and an error word) in a fixed device array shared by all calls.
Its forces and energies must match the FP64 oracle within the parity bar and
the context's own force path, on two calls in a row (the second call reuses
the array the first one filled); ids outside a bead's replica must come back
as EINVAL without being dereferenced.  This file is collected last so that a
run stopping at the first failure has already run every other test."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_4214_gb300 import workloads as W

from parity import EV_TOL, FORCE_TOL, ev_error, force_error

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def D():
    from paper_1108_4214_gb300 import dynbond
    return dynbond


def slots_from_bonds(bonds, n):
    slots = np.zeros((n, 4), np.uint32)
    deg = np.zeros(n, np.int64)
    for i, j, ti, tj in bonds:
        slots[i, deg[i]] = (int(j) << 4) | int(ti)
        deg[i] += 1
        slots[j, deg[j]] = (int(i) << 4) | int(tj)
        deg[j] += 1
    return slots


def device_topology(s, bonds, angles, dihedrals, with_slots=True):
    dev = torch.device("cuda")
    sl = slots_from_bonds(bonds, s.n_beads) if with_slots else np.zeros((s.n_beads, 4), np.uint32)
    return dict(slots=torch.from_numpy(sl.view(np.int32)).to(dev),
                bead_offset=torch.from_numpy(np.asarray(s.bead_offset, np.int64)).to(dev),
                box_q=torch.from_numpy(np.asarray(s.box_q, np.int64)).to(dev),
                angles=torch.from_numpy(np.ascontiguousarray(angles, np.int32)).to(dev),
                dihedrals=torch.from_numpy(np.ascontiguousarray(dihedrals, np.int32)).to(dev))


@pytest.mark.parametrize("paper_ff", [False, True])
def test_noalloc_forces_match_the_oracle_and_the_context_path_on_two_calls(paper_ff):
    s = W.config3(n_replicas=6)  # several replicas: per-replica scratch rows
    if paper_ff:  # harmonic angles K (theta - theta0)^2 with theta0 = 180 and 90 degrees (Sec. 3)
        s.forcefield = W.forcefield_dna1_paper()
    ctx = D().Context(s)
    o = O.Oracle(s)
    snaps = s.snapshots(0, 3)
    for k in range(2):
        ctx.step(torch.from_numpy(snaps[k]).cuda(), k)
        o.step(snaps[k], k)
    topo = ctx.topology()
    for g, r in zip(topo, o.topology()):
        assert np.array_equal(g, r)
    pos = torch.from_numpy(snaps[2]).cuda()
    fr, evr = o.forces(snaps[2])
    f_ctx, ev_ctx = ctx.forces(pos)
    f_ctx, ev_ctx = f_ctx.cpu().numpy(), ev_ctx.cpu().numpy()
    t = device_topology(s, *topo)
    for call in range(2):
        f, ev = D().forces_noalloc(pos, forcefield=s.forcefield, **t)
        f, ev = f.cpu().numpy(), ev.cpu().numpy()
        assert np.all(f[:, 3] == 0)
        assert force_error(f, fr) <= FORCE_TOL, (call, force_error(f, fr))
        assert ev_error(ev, evr) <= EV_TOL, (call, ev_error(ev, evr))
        # and the context's path on the same topology, within the same bar
        assert force_error(f, f_ctx[:, :3].astype(np.float64)) <= FORCE_TOL
        assert ev_error(ev, ev_ctx) <= EV_TOL


def test_noalloc_at_its_replica_limit():
    """DYNBOND_NOALLOC_MAX_REPLICAS replicas of one 8-nt duplex each: every
    row of the scratch array in use, per-replica energies against the oracle."""
    R = D().NOALLOC_MAX_REPLICAS
    s = W.replica_batch(R, n_strands=2, n_nt=8, n_duplex=1)
    o = O.Oracle(s)
    topo = o.topology()
    snap = s.snapshot(1)
    fr, evr = o.forces(snap)
    t = device_topology(s, *topo)
    pos = torch.from_numpy(snap).cuda()
    for call in range(2):
        f, ev = D().forces_noalloc(pos, forcefield=s.forcefield, **t)
        assert force_error(f.cpu().numpy(), fr) <= FORCE_TOL, call
        assert ev_error(ev.cpu().numpy(), evr) <= EV_TOL, call


def test_noalloc_angles_without_bonds_and_an_empty_system():
    """Empty bond slots with nonempty angle and dihedral lists (bond terms
    switched off on the oracle's side), then a replica without beads."""
    s = W.config3(n_replicas=3)
    s.forcefield = W.forcefield_dna2()
    s.forcefield["bond_k"][:] = 0.0
    o = O.Oracle(s)
    topo = o.topology()
    assert len(topo[1]) and len(topo[2])
    snap = s.snapshot(0)
    fr, evr = o.forces(snap)
    t = device_topology(s, *topo, with_slots=False)
    f, ev = D().forces_noalloc(torch.from_numpy(snap).cuda(), forcefield=s.forcefield, **t)
    assert force_error(f.cpu().numpy(), fr) <= FORCE_TOL
    assert ev_error(ev.cpu().numpy(), evr) <= EV_TOL
    dev = torch.device("cuda")
    z4 = torch.zeros((0, 4), dtype=torch.int32, device=dev)
    f, ev = D().forces_noalloc(z4, z4, torch.zeros(2, dtype=torch.int64, device=dev),
                               torch.full((1,), 1 << 24, dtype=torch.int64, device=dev), z4,
                               torch.zeros((0, 5), dtype=torch.int32, device=dev), s.forcefield)
    assert f.shape == (0, 4) and not ev.cpu().numpy().any()


def test_noalloc_reports_ids_outside_their_replica():
    """A bond partner, an angle bead or a dihedral bead outside its replica,
    or a type above 15: the call returns EINVAL and never reads the bad id.
    The position buffer has spare rows past n_beads, so even an unguarded read
    would stay inside allocated memory.  The next valid call succeeds (the
    error word is cleared per call)."""
    s = W.config3(n_replicas=2)
    o = O.Oracle(s)
    bonds, angles, dihedrals = o.topology()
    N = s.n_beads
    snap = s.snapshot(0)
    dev = torch.device("cuda")
    buf = torch.zeros((N + 8, 4), dtype=torch.int32, device=dev)
    buf[:N] = torch.from_numpy(snap).to(dev)
    pos = buf[:N]
    fr, evr = o.forces(snap)
    good = device_topology(s, bonds, angles, dihedrals)
    n0 = int(s.bead_offset[1])  # first bead of replica 1
    cases = []
    sl = good["slots"].clone()
    sl[3, 0] = (N << 4) | 1  # partner past the last bead
    cases.append(dict(good, slots=sl))
    sl = good["slots"].clone()
    sl[5, 0] = (n0 + 2) << 4 | 1  # partner in the other replica
    cases.append(dict(good, slots=sl))
    a = good["angles"].clone()
    a[0, 0] = N
    cases.append(dict(good, angles=a))
    a = good["angles"].clone()
    a[1, 3] = 16
    cases.append(dict(good, angles=a))
    d = good["dihedrals"].clone()
    d[0, 3] = -1
    cases.append(dict(good, dihedrals=d))
    d = good["dihedrals"].clone()
    d[2, 4] = 99
    cases.append(dict(good, dihedrals=d))
    for k, t in enumerate(cases):
        with pytest.raises(D().DynbondError) as e:
            D().forces_noalloc(pos, forcefield=s.forcefield, **t)
        assert e.value.status == 1, k
    f, ev = D().forces_noalloc(pos, forcefield=s.forcefield, **good)
    assert force_error(f.cpu().numpy(), fr) <= FORCE_TOL
    assert ev_error(ev.cpu().numpy(), evr) <= EV_TOL


def test_noalloc_rejects_more_replicas_than_its_scratch_holds():
    R = D().NOALLOC_MAX_REPLICAS + 1
    dev = torch.device("cuda")
    pos = torch.zeros((R, 4), dtype=torch.int32, device=dev)
    slots = torch.zeros((R, 4), dtype=torch.int32, device=dev)
    off = torch.arange(R + 1, dtype=torch.int64, device=dev)
    box = torch.full((R,), 1 << 20, dtype=torch.int64, device=dev)
    empty4 = torch.zeros((0, 4), dtype=torch.int32, device=dev)
    empty5 = torch.zeros((0, 5), dtype=torch.int32, device=dev)
    with pytest.raises(D().DynbondError) as e:
        D().forces_noalloc(pos, slots, off, box, empty4, empty5, W.forcefield_dna2())
    assert e.value.status == 1
