"""Small hand-built systems for tests (inputs only)."""

import json
import os

import numpy as np

from paper_1108_4214_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def make_system(types, bonds, pos_sigma, box, rules, params=None, n_replicas=1, offsets=None, boxes=None):
    """A System with explicit beads; pos_sigma in sigma (wrapped into the box
    when snapshots are taken)."""
    types = np.asarray(types, np.int32)
    N = len(types)
    offs = np.array(offsets if offsets is not None else [0, N], np.int64)
    R = len(offs) - 1
    bq = np.array(boxes if boxes is not None else [int(round(box * W.QSCALE))] * R, np.int64)
    return W.System(
        name="hand", bead_offset=offs, box_q=bq, types=types,
        bonds=np.asarray(bonds, np.int32).reshape(-1, 4), rules=rules,
        pos0=np.asarray(pos_sigma, np.float64).reshape(N, 3), seed=11, sigma_perturb=0.0,
        form_scale=np.ones(R), break_scale=np.ones(R), rng_stream=np.arange(R, dtype=np.uint32),
        params=dict(W.default_params(11), **(params or {})),
    )


def qpos(system, pos_sigma):
    """Quantize explicit positions (sigma) for a system."""
    x = np.asarray(pos_sigma, np.float64).reshape(-1, 3)
    return W.quantize(x, system.box_q, system._rep_of_bead())


def mask_of(spec):
    if spec == "*":
        return W.ALL_BEADS
    return W.bit(*spec)


def bond_mask_of(spec):
    if spec == "*":
        return W.ALL_BONDS
    return W.bit(*spec)


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def golden_rules(entries):
    out = []
    for e in entries:
        if e["kind"] == "createangle":
            out.append(dict(kind="createangle", type=e["type"], beads=tuple(mask_of(b) for b in e["beads"]),
                            bonds=tuple(bond_mask_of(b) for b in e["bonds"])))
        elif e["kind"] == "createdihedral":
            out.append(dict(kind="createdihedral", type=e["type"], beads=tuple(mask_of(b) for b in e["beads"]),
                            bonds=tuple(bond_mask_of(b) for b in e["bonds"])))
        else:
            raise ValueError(e["kind"])
    return out


def ladder_1bead_positions(sep=0.5, spacing=0.5):
    """The 4-mer ladder of the golden fixture: strand 1 along x at y=0, strand 2
    (antiparallel) at y=sep; rung k holds beads k and 7-k."""
    p = np.zeros((8, 3))
    for k in range(4):
        p[k] = (5.0 + spacing * k, 5.0, 5.0)
        p[7 - k] = (5.0 + spacing * k, 5.0 + sep, 5.0)
    return p


# ---------------------------------------------------------------------------
# The topology hash of include/dynbond.h (dynbond_topology_hash), restated
# from its definition for exported topologies: bond ends, angles and
# dihedrals mixed with the splitmix64 finalizer and summed mod 2^64.
# ---------------------------------------------------------------------------
M64 = (1 << 64) - 1


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _chain(first, cols):
    z = _mix(np.full(len(cols[0]), first, dtype=np.uint64))
    for c in cols:
        z = _mix(z ^ np.asarray(c, dtype=np.int64).astype(np.uint64))
    return z


def topology_hash(bonds, angles, dihedrals):
    """Hash of one replica's topology (bead ids local to the replica)."""
    b = np.asarray(bonds, np.int64).reshape(-1, 4)
    u64 = lambda x: np.asarray(x, np.int64).astype(np.uint64)
    ends = np.concatenate([
        (u64(b[:, 0]) << np.uint64(32)) | (u64(b[:, 1]) << np.uint64(4)) | u64(b[:, 2]),
        (u64(b[:, 1]) << np.uint64(32)) | (u64(b[:, 0]) << np.uint64(4)) | u64(b[:, 3])])
    a = np.asarray(angles, np.int64).reshape(-1, 4)
    d = np.asarray(dihedrals, np.int64).reshape(-1, 5)
    total = 0
    with np.errstate(over="ignore"):
        for part in (_mix(ends), _chain(0xA, [a[:, k] for k in range(4)]),
                     _chain(0xD, [d[:, k] for k in range(5)])):
            total = (total + int(part.sum(dtype=np.uint64))) & M64
    return total


def half_bond_pair():
    """Two beads 1.3 sigma apart on x joined by a directional bond whose two
    stored types carry different potentials: bead 0 stores type 2 (K 100,
    r0 1.0), bead 1 stores type 3 (K 40, r0 1.2)."""
    rules = [dict(kind="createbond", btype=1, beads=(W.ALL_BEADS, W.ALL_BEADS), dist=0.5, prob=0.0)]
    s = make_system([0, 0], [[0, 1, W.BB3, W.BB5]], [[2.0, 2.0, 2.0], [3.3, 2.0, 2.0]], 10.0, rules)
    s.forcefield["bond_k"][W.BB3], s.forcefield["bond_r0"][W.BB3] = 100.0, 1.0
    s.forcefield["bond_k"][W.BB5], s.forcefield["bond_r0"][W.BB5] = 40.0, 1.2
    return s
