"""Python binding of libdynbond (include/dynbond.h): argument marshalling only.

Every step of the dynamic-bonding pass runs in the CUDA library; this module
packs rules and systems into the C structs, passes device pointers of torch
tensors and the current torch CUDA stream, and turns statuses into
exceptions.  It raises if the compiled library is missing -- there is no
fallback path.
"""

from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libdynbond.so")

STATUS = {0: "ok", 1: "EINVAL", 2: "ENOMEM", 3: "ECAPACITY", 4: "ECUDA", 5: "ETIMEOUT", 6: "ENOTCONVERGED"}
KINDS = dict(createbond=1, createdirbond=2, breakbond=3, convertbond=4, killbond=5, createangle=6,
             createdihedral=7, maxbond=8)
FLAG_NO_GRAPH, FLAG_PROFILE, FLAG_NO_AUTOTUNE, FLAG_NO_PDL, FLAG_GLOBAL_SEARCH, FLAG_STAGED_SEARCH = 1, 2, 4, 8, 16, 32
FLAG_PERSISTENT = 64
STAT_NAMES = [
    "candidates", "create_matched", "bonds_formed", "break_candidates", "break_matched", "bonds_broken",
    "bonds_killed", "bonds_converted", "angles_removed", "angles_added", "dihedrals_removed", "dihedrals_added",
    "n_bonds", "n_angles", "n_dihedrals", "create_rounds", "break_rounds",
]
EXPORTS = ["dynbond_create", "dynbond_step", "dynbond_forces", "dynbond_run_host", "dynbond_get_topology",
           "dynbond_sync", "dynbond_phase_times", "dynbond_last_error", "dynbond_status_string", "dynbond_destroy",
           "dynbond_forces_noalloc", "dynbond_autotune", "dynbond_md_create", "dynbond_md_advance",
           "dynbond_md_destroy", "dynbond_topology_hash", "dynbond_get_tuning", "dynbond_md_pair_forces",
           "dynbond_step_forces"]
NOALLOC_MAX_REPLICAS = 4096

c_i32, c_u32, c_i64, c_u64, c_dbl, c_p = (ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64,
                                          ctypes.c_double, ctypes.c_void_p)


class DynbondError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Rule(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("type", c_i32), ("type2", c_i32), ("maxn", c_i32), ("bead_mask", c_u32 * 4),
                ("bond_mask", c_u32 * 3), ("reserved", c_u32), ("dist", c_dbl), ("prob", c_dbl)]


class Params(ctypes.Structure):
    _fields_ = [("seed", c_u64), ("paircheck13", c_i32), ("paircheck14", c_i32), ("max_rounds", c_i32),
                ("prob_mode", c_i32), ("reactive_mask", c_u32), ("flags", c_i32), ("cell_scale", c_i32),
                ("block_size", c_i32), ("spin_limit", c_i32), ("cell_zdiv", c_i32),
                ("reserved", c_i32 * 4)]


class ForceField(ctypes.Structure):
    _fields_ = [("bond_k", c_dbl * 16), ("bond_r0", c_dbl * 16), ("angle_k", c_dbl * 16),
                ("dihedral_k", c_dbl * 16), ("dihedral_d", c_i32 * 16), ("angle_theta0", c_dbl * 16),
                ("angle_style", c_i32 * 16)]


class SystemDesc(ctypes.Structure):
    _fields_ = [("n_replicas", c_i32), ("reserved", c_i32), ("bead_offset", c_p), ("box_q", c_p),
                ("form_scale", c_p), ("break_scale", c_p), ("rng_stream", c_p), ("bead_type", c_p),
                ("bonds", c_p), ("n_bonds", c_i64)]


class Stats(ctypes.Structure):
    _fields_ = [(n, c_i64) for n in STAT_NAMES]


class Tuning(ctypes.Structure):
    _fields_ = [("cell_scale", c_dbl), ("bead_blocks_per_sm", c_i32), ("candidate_blocks_per_sm", c_i32),
                ("front_ms", ctypes.c_float), ("tuned", c_i32), ("cell_zdiv", c_i32),
                ("octant", c_i32), ("tiles", c_i32)]


class DPD(ctypes.Structure):
    _fields_ = [("a", c_dbl), ("gamma", c_dbl), ("kT", c_dbl), ("rc", c_dbl), ("dt", c_dbl), ("mass", c_dbl),
                ("seed", c_u64)]


class Topology(ctypes.Structure):
    _fields_ = [("n_bonds", c_i64), ("n_angles", c_i64), ("n_dihedrals", c_i64), ("bonds", c_p),
                ("angles", c_p), ("dihedrals", c_p)]


assert ctypes.sizeof(Rule) == 64 and ctypes.sizeof(Stats) == 17 * 8

_lib = None


def load() -> ctypes.CDLL:
    """Load libdynbond.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    L.dynbond_create.restype = c_i32
    L.dynbond_create.argtypes = [c_p, c_p, c_i32, c_p, c_p, c_p, ctypes.POINTER(c_p)]
    L.dynbond_step.restype = c_i32
    L.dynbond_step.argtypes = [c_p, c_p, c_u64, c_p]
    L.dynbond_forces.restype = c_i32
    L.dynbond_forces.argtypes = [c_p, c_p, c_p, c_p]
    L.dynbond_run_host.restype = c_i32
    L.dynbond_run_host.argtypes = [c_p, c_p, c_u64, c_p, c_p, c_p]
    L.dynbond_step_forces.restype = c_i32
    L.dynbond_step_forces.argtypes = [c_p, c_p, c_u64, c_p, c_p, c_p]
    L.dynbond_get_topology.restype = c_i32
    L.dynbond_get_topology.argtypes = [c_p, ctypes.POINTER(Topology)]
    L.dynbond_sync.restype = c_i32
    L.dynbond_sync.argtypes = [c_p]
    L.dynbond_phase_times.restype = c_i32
    L.dynbond_phase_times.argtypes = [c_p, c_p, c_p, c_i32, ctypes.POINTER(c_i32)]
    L.dynbond_last_error.restype = ctypes.c_char_p
    L.dynbond_last_error.argtypes = [c_p]
    L.dynbond_status_string.restype = ctypes.c_char_p
    L.dynbond_status_string.argtypes = [c_i32]
    L.dynbond_destroy.restype = None
    L.dynbond_destroy.argtypes = [c_p]
    L.dynbond_md_create.restype = c_i32
    L.dynbond_md_create.argtypes = [c_p, c_p, ctypes.POINTER(c_p)]
    L.dynbond_md_advance.restype = c_i32
    L.dynbond_md_advance.argtypes = [c_p, c_p, c_p, c_i64, c_u64, c_p]
    L.dynbond_md_pair_forces.restype = c_i32
    L.dynbond_md_pair_forces.argtypes = [c_p, c_p, c_p, c_u64, c_p]
    L.dynbond_md_destroy.restype = None
    L.dynbond_md_destroy.argtypes = [c_p]
    L.dynbond_topology_hash.restype = c_i32
    L.dynbond_topology_hash.argtypes = [c_p, c_p]
    L.dynbond_autotune.restype = c_i32
    L.dynbond_autotune.argtypes = [c_p, c_p, c_p]
    L.dynbond_get_tuning.restype = c_i32
    L.dynbond_get_tuning.argtypes = [c_p, c_p]
    L.dynbond_forces_noalloc.restype = c_i32
    L.dynbond_forces_noalloc.argtypes = [c_p, c_p, c_p, c_p, c_i32, c_i64, c_p, c_i64, c_p, c_i64, c_p, c_p, c_p, c_p]
    _lib = L
    return L


def pack_rules(rules: List[Dict]):
    arr = (Rule * max(1, len(rules)))()
    for k, r in enumerate(rules):
        a = arr[k]
        kind = r["kind"]
        a.kind = KINDS[kind]
        if kind in ("createbond", "createdirbond"):
            a.type = r["btype"]
            a.type2 = r.get("btype2", 0)
            a.bead_mask[0], a.bead_mask[1] = r["beads"]
            a.dist, a.prob = r["dist"], r["prob"]
        elif kind == "breakbond":
            a.type, a.dist, a.prob = r["btype"], r["dist"], r["prob"]
        elif kind == "convertbond":
            a.type, a.type2, a.prob = r["btype"], r["btype2"], r["prob"]
        elif kind == "killbond":
            a.type, a.dist = r["btype"], r["dist"]
        elif kind == "createangle":
            a.type = r["type"]
            for q in range(3):
                a.bead_mask[q] = r["beads"][q]
            for q in range(2):
                a.bond_mask[q] = r["bonds"][q]
        elif kind == "createdihedral":
            a.type = r["type"]
            for q in range(4):
                a.bead_mask[q] = r["beads"][q]
            for q in range(3):
                a.bond_mask[q] = r["bonds"][q]
        elif kind == "maxbond":
            a.bond_mask[0], a.bead_mask[0], a.maxn = r["bonds"], r["beads"], r["max"]
        else:
            raise ValueError(f"unknown rule kind {kind}")
    return arr


def _ptr(t) -> int:
    return t.data_ptr() if t is not None else 0


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """A dynamic-bonding context on the current CUDA device.

    `system` carries bead_offset, box_q, types, bonds, rules, params,
    forcefield and optional form_scale / break_scale / rng_stream (the
    attributes of paper_1108_4214_gb300.workloads.System)."""

    def __init__(self, system, params: Optional[Dict] = None, flags: int = 0, stream=None):
        import torch
        self.L = load()
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        prm = dict(system.params)
        prm.update(params or {})
        R = len(system.box_q)
        self.R, self.N = R, int(system.bead_offset[-1])
        keep = dict(
            off=np.ascontiguousarray(system.bead_offset, np.int64),
            box=np.ascontiguousarray(system.box_q, np.int64),
            types=np.ascontiguousarray(system.types, np.int32),
            bonds=np.ascontiguousarray(system.bonds, np.int32).reshape(-1, 4),
        )
        for name, attr, dt in (("fs", "form_scale", np.float64), ("bs", "break_scale", np.float64),
                               ("stream", "rng_stream", np.uint32)):
            v = getattr(system, attr, None)
            keep[name] = None if v is None else np.ascontiguousarray(v, dt)
        self._keep = keep
        sd = SystemDesc()
        sd.n_replicas = R
        sd.bead_offset = keep["off"].ctypes.data
        sd.box_q = keep["box"].ctypes.data
        sd.form_scale = keep["fs"].ctypes.data if keep["fs"] is not None else None
        sd.break_scale = keep["bs"].ctypes.data if keep["bs"] is not None else None
        sd.rng_stream = keep["stream"].ctypes.data if keep["stream"] is not None else None
        sd.bead_type = keep["types"].ctypes.data
        sd.bonds = keep["bonds"].ctypes.data
        sd.n_bonds = len(keep["bonds"])
        p = Params()
        p.seed = int(prm["seed"]) % (1 << 64)
        p.paircheck13, p.paircheck14 = int(prm["paircheck13"]), int(prm["paircheck14"])
        p.max_rounds, p.prob_mode = int(prm["max_rounds"]), int(prm["prob_mode"])
        p.reactive_mask = int(prm["reactive_mask"])
        p.flags = int(flags) | int(prm.get("flags", 0))
        p.cell_scale = int(prm.get("cell_scale", 0))
        p.cell_zdiv = int(prm.get("cell_zdiv", 0))
        p.spin_limit = int(prm.get("spin_limit", 0))
        ff = forcefield_struct(system.forcefield)
        rules = pack_rules(system.rules)
        h = c_p()
        st = self.L.dynbond_create(ctypes.byref(p), rules, len(system.rules), ctypes.byref(sd), ctypes.byref(ff),
                                   _stream_handle(self.stream), ctypes.byref(h))
        if st != 0:
            raise DynbondError(st, self.L.dynbond_last_error(None).decode())
        self.h = h
        self._stats = (Stats * R)()

    # -- helpers
    def _check(self, st):
        if st != 0:
            raise DynbondError(st, self.L.dynbond_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.dynbond_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the C entry points
    def step(self, pos, step: int, stats: bool = False):
        """dynbond_step on device positions pos (int32 [N, 4] CUDA tensor)."""
        assert pos.is_cuda and pos.dtype == self._torch.int32 and pos.is_contiguous()
        self._check(self.L.dynbond_step(self.h, c_p(_ptr(pos)), int(step),
                                        ctypes.byref(self._stats) if stats else None))
        if stats:
            return np.array([[getattr(s, n) for n in STAT_NAMES] for s in self._stats], np.int64)
        return None

    def forces(self, pos, force=None, ev=None):
        """dynbond_forces: returns (force float32 [N, 4], ev float64 [R, 7]) CUDA tensors."""
        torch = self._torch
        if force is None:
            force = torch.empty((self.N, 4), dtype=torch.float32, device=pos.device)
        if ev is None:
            ev = torch.empty((self.R, 7), dtype=torch.float64, device=pos.device)
        self._check(self.L.dynbond_forces(self.h, c_p(_ptr(pos)), c_p(_ptr(force)), c_p(_ptr(ev))))
        return force, ev

    def step_forces(self, pos, step: int, force=None, ev=None, stats: bool = False):
        """dynbond_step_forces: the step, then the forces at the same positions, in one call; returns
        (force, ev, stats or None)."""
        torch = self._torch
        assert pos.is_cuda and pos.dtype == torch.int32 and pos.is_contiguous()
        if force is None:
            force = torch.empty((self.N, 4), dtype=torch.float32, device=pos.device)
        if ev is None:
            ev = torch.empty((self.R, 7), dtype=torch.float64, device=pos.device)
        self._check(self.L.dynbond_step_forces(self.h, c_p(_ptr(pos)), int(step), c_p(_ptr(force)), c_p(_ptr(ev)),
                                               ctypes.byref(self._stats) if stats else None))
        st = (np.array([[getattr(s, n) for n in STAT_NAMES] for s in self._stats], np.int64) if stats else None)
        return force, ev, st

    def run_host(self, pos_host, step: int, force_host=None, ev_host=None, stats: bool = False):
        """dynbond_run_host from host buffers (numpy arrays or CPU tensors, ideally pinned)."""
        def addr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        if force_host is None:
            force_host = np.empty((self.N, 4), np.float32)
        if ev_host is None:
            ev_host = np.empty((self.R, 7), np.float64)
        self._check(self.L.dynbond_run_host(self.h, c_p(addr(pos_host)), int(step), c_p(addr(force_host)),
                                            c_p(addr(ev_host)), ctypes.byref(self._stats) if stats else None))
        st = (np.array([[getattr(s, n) for n in STAT_NAMES] for s in self._stats], np.int64) if stats else None)
        return force_host, ev_host, st

    def sync(self):
        self._check(self.L.dynbond_sync(self.h))

    def autotune(self, pos) -> Dict:
        """dynbond_autotune on device positions; returns the chosen geometry."""
        t = Tuning()
        self._check(self.L.dynbond_autotune(self.h, c_p(_ptr(pos)), ctypes.byref(t)))
        return {n: getattr(t, n) for n, _ in Tuning._fields_}

    def tuning(self) -> Dict:
        """dynbond_get_tuning: the current launch geometry (nothing is timed or launched)."""
        t = Tuning()
        self._check(self.L.dynbond_get_tuning(self.h, ctypes.byref(t)))
        return {n: getattr(t, n) for n, _ in Tuning._fields_}

    def topology_hash(self) -> np.ndarray:
        """dynbond_topology_hash: one order-independent 64-bit hash per replica."""
        h = np.zeros(self.R, np.uint64)
        self._check(self.L.dynbond_topology_hash(self.h, c_p(h.ctypes.data)))
        return h

    def topology(self):
        """(bonds [nb, 4], angles [na, 4], dihedrals [nd, 5]) canonical and sorted (numpy)."""
        t = Topology()
        self._check(self.L.dynbond_get_topology(self.h, ctypes.byref(t)))
        b = np.zeros((t.n_bonds, 4), np.int32)
        a = np.zeros((t.n_angles, 4), np.int32)
        d = np.zeros((t.n_dihedrals, 5), np.int32)
        t.bonds, t.angles, t.dihedrals = b.ctypes.data, a.ctypes.data, d.ctypes.data
        self._check(self.L.dynbond_get_topology(self.h, ctypes.byref(t)))
        return b, a, d

    def phase_times(self) -> Dict[str, float]:
        n = c_i32(0)
        ms = (ctypes.c_float * 32)()
        names = (ctypes.c_char_p * 32)()
        self._check(self.L.dynbond_phase_times(self.h, ms, names, 32, ctypes.byref(n)))
        return {names[k].decode(): float(ms[k]) for k in range(n.value)}


def forcefield_struct(f) -> ForceField:
    ff = ForceField()
    t0 = f.get("angle_theta0", np.zeros(16))
    sty = f.get("angle_style", np.zeros(16, np.int32))
    for t in range(16):
        ff.bond_k[t], ff.bond_r0[t] = float(f["bond_k"][t]), float(f["bond_r0"][t])
        ff.angle_k[t], ff.dihedral_k[t] = float(f["angle_k"][t]), float(f["dihedral_k"][t])
        ff.dihedral_d[t] = int(f["dihedral_d"][t])
        ff.angle_theta0[t], ff.angle_style[t] = float(t0[t]), int(sty[t])
    return ff


def forces_noalloc(pos, slots, bead_offset, box_q, angles, dihedrals, forcefield, force=None, ev=None, stream=None):
    """dynbond_forces_noalloc: bonded forces of a caller-supplied topology
    without any allocation inside the library.  All tensors are contiguous
    CUDA tensors on one device: pos int32 [N, 4], slots int32 [N, 4] (the
    uint32 words partner << 4 | stored type, 0 = empty), bead_offset int64
    [R+1], box_q int64 [R], angles int32 [na, 4], dihedrals int32 [nd, 5].
    Returns (force float32 [N, 4], ev float64 [R, 7]); the outputs may be
    preallocated by the caller (same shapes and dtypes).  Raises DynbondError
    with status EINVAL when a bead id or type of the topology is out of range
    (those terms are skipped by the library)."""
    import torch
    L = load()
    N, R = int(pos.shape[0]), int(box_q.shape[0])
    if force is None:
        force = torch.empty((N, 4), dtype=torch.float32, device=pos.device)
    if ev is None:
        ev = torch.empty((R, 7), dtype=torch.float64, device=pos.device)
    want = ((pos, torch.int32, (N, 4)), (slots, torch.int32, (N, 4)), (bead_offset, torch.int64, (R + 1,)),
            (box_q, torch.int64, (R,)), (angles, torch.int32, (int(angles.shape[0]), 4)),
            (dihedrals, torch.int32, (int(dihedrals.shape[0]), 5)), (force, torch.float32, (N, 4)),
            (ev, torch.float64, (R, 7)))
    for k, (t, dt, shape) in enumerate(want):
        if not (t.is_cuda and t.device == pos.device and t.dtype == dt and tuple(t.shape) == shape
                and t.is_contiguous()):
            raise ValueError(f"forces_noalloc argument {k}: need a contiguous {dt} CUDA tensor of shape {shape} "
                             f"on {pos.device}, got {t.dtype} {tuple(t.shape)} on {t.device}")
    ff = forcefield_struct(forcefield)
    st = L.dynbond_forces_noalloc(c_p(_ptr(pos)), c_p(_ptr(slots)), c_p(_ptr(bead_offset)), c_p(_ptr(box_q)), R, N,
                                  c_p(_ptr(angles)), angles.shape[0], c_p(_ptr(dihedrals)), dihedrals.shape[0],
                                  ctypes.byref(ff), c_p(_ptr(force)), c_p(_ptr(ev)), _stream_handle(stream))
    if st != 0:
        raise DynbondError(st, "dynbond_forces_noalloc failed (sizes, alignment, or a bead id / type out of range)")
    return force, ev


class MD:
    """dynbond_md_*: velocity-Verlet DPD harness around a one-replica Context."""

    def __init__(self, ctx: Context, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.01, mass=1.0, seed=12345):
        self.L = load()
        self.ctx = ctx
        p = DPD(a=a, gamma=gamma, kT=kT, rc=rc, dt=dt, mass=mass, seed=seed % (1 << 64))
        h = c_p()
        st = self.L.dynbond_md_create(ctx.h, ctypes.byref(p), ctypes.byref(h))
        if st != 0:
            raise DynbondError(st, "dynbond_md_create failed (one replica, positive rc, dt, mass)")
        self.h = h

    def advance(self, pos, vel, n_steps: int, first_step: int, ev=None):
        st = self.L.dynbond_md_advance(self.h, c_p(_ptr(pos)), c_p(_ptr(vel)), int(n_steps), int(first_step),
                                       c_p(_ptr(ev)))
        if st != 0:
            raise DynbondError(st, "dynbond_md_advance failed")

    def pair_forces(self, pos, vel, step: int, force=None):
        """dynbond_md_pair_forces: the DPD pair forces (float32 [N, 4]) at
        pos, vel for step index `step`."""
        torch = self.ctx._torch
        if force is None:
            force = torch.empty((pos.shape[0], 4), dtype=torch.float32, device=pos.device)
        st = self.L.dynbond_md_pair_forces(self.h, c_p(_ptr(pos)), c_p(_ptr(vel)), int(step), c_p(_ptr(force)))
        if st != 0:
            raise DynbondError(st, "dynbond_md_pair_forces failed")
        return force

    def close(self):
        if getattr(self, "h", None):
            self.L.dynbond_md_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
