"""CPU oracle for the dynamic-bonding pass -- TEST INFRASTRUCTURE ONLY.

ctypes wrapper around ``dynbond_oracle.cpp``, a plain serial C++ statement of
one call of the dynamic-bonding fix (Svaneborg, arXiv:1108.4214, Sec. 2 and
the Appendix steps 1-10) and of the FP64 bonded forces.  Only the tests, the
package smoke check and the benchmark's CPU-baseline / reference legs may
import this module.  It shares no code with the CUDA library: it packs its own
rule records from the neutral rule dicts of the input generator.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dynbond_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

STAT_NAMES = [
    "candidates", "create_matched", "bonds_formed", "break_candidates", "break_matched", "bonds_broken",
    "bonds_killed", "bonds_converted", "angles_removed", "angles_added", "dihedrals_removed", "dihedrals_added",
    "n_bonds", "n_angles", "n_dihedrals", "create_rounds", "break_rounds",
]

KINDS = dict(createbond=1, createdirbond=2, breakbond=3, convertbond=4, killbond=5, createangle=6,
             createdihedral=7, maxbond=8)

RULE_DTYPE = np.dtype([
    ("kind", "<i4"), ("type", "<i4"), ("type2", "<i4"), ("maxn", "<i4"),
    ("bead", "<u4", (4,)), ("bond", "<u4", (3,)), ("pad", "<u4"), ("dist", "<f8"), ("prob", "<f8"),
])
assert RULE_DTYPE.itemsize == 64


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (no CUDA involved)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = f"{LIB}.{os.getpid()}.tmp"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", SRC, "-o", tmp])
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        L.orc_new.restype = P
        L.orc_new.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, ctypes.c_int64, P, ctypes.c_int, ctypes.c_uint64,
                              ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.c_int]
        L.orc_free.argtypes = [P]
        L.orc_step.restype = ctypes.c_int
        L.orc_step.argtypes = [P, P, ctypes.c_uint64, P]
        L.orc_stat_count.restype = ctypes.c_int
        L.orc_counts.argtypes = [P, P]
        L.orc_topology.argtypes = [P, P, P, P]
        L.orc_check_rules_identity.restype = ctypes.c_int
        L.orc_check_rules_identity.argtypes = [P]
        L.orc_candidates.restype = ctypes.c_int64
        L.orc_candidates.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int64]
        L.orc_match.restype = ctypes.c_int
        L.orc_match.argtypes = [ctypes.c_int64, ctypes.c_int64, P, P, P, ctypes.c_int, P]
        L.orc_philox.argtypes = [P, P, P]
        L.orc_r2.restype = ctypes.c_int64
        L.orc_r2.argtypes = [ctypes.c_double]
        L.orc_threshold.restype = ctypes.c_uint64
        L.orc_threshold.argtypes = [ctypes.c_double]
        L.orc_forces.restype = ctypes.c_int
        L.orc_forces.argtypes = [P, P, P, P, P, P, P, P, P, P, P]
        L.orc_bond_half.argtypes = [P, ctypes.c_double, ctypes.c_double, P, P]
        L.orc_angle.argtypes = [P, P, ctypes.c_double, P, P, P]
        L.orc_angle_harmonic.argtypes = [P, P, ctypes.c_double, ctypes.c_double, P, P, P]
        L.orc_dihedral.argtypes = [P, P, P, ctypes.c_double, ctypes.c_double, P, P, P, P, P]
        L.orc_dpd_forces.argtypes = [P, P, P] + [ctypes.c_double] * 5 + [ctypes.c_uint64, ctypes.c_uint64, P]
        assert L.orc_stat_count() == len(STAT_NAMES)
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def pack_rules(rules) -> np.ndarray:
    arr = np.zeros(max(1, len(rules)), RULE_DTYPE)
    for k, r in enumerate(rules):
        kind = r["kind"]
        a = arr[k]
        a["kind"] = KINDS[kind]
        if kind in ("createbond", "createdirbond"):
            a["type"] = r["btype"]
            a["type2"] = r.get("btype2", r["btype"])
            a["bead"][0], a["bead"][1] = r["beads"]
            a["dist"], a["prob"] = r["dist"], r["prob"]
        elif kind == "breakbond":
            a["type"], a["dist"], a["prob"] = r["btype"], r["dist"], r["prob"]
        elif kind == "convertbond":
            a["type"], a["type2"], a["prob"] = r["btype"], r["btype2"], r["prob"]
        elif kind == "killbond":
            a["type"], a["dist"] = r["btype"], r["dist"]
        elif kind == "createangle":
            a["type"] = r["type"]
            for i in range(3):
                a["bead"][i] = r["beads"][i]
            for i in range(2):
                a["bond"][i] = r["bonds"][i]
        elif kind == "createdihedral":
            a["type"] = r["type"]
            for i in range(4):
                a["bead"][i] = r["beads"][i]
            for i in range(3):
                a["bond"][i] = r["bonds"][i]
        elif kind == "maxbond":
            a["bond"][0], a["bead"][0], a["maxn"] = r["bonds"], r["beads"], r["max"]
        else:
            raise ValueError(kind)
    return arr


class Oracle:
    """One system (a batch of replicas) held by the CPU oracle."""

    def __init__(self, system, use_cells: bool = True, params=None):
        L = lib()
        s = system
        R = s.n_replicas
        prm = dict(s.params)
        prm.update(params or {})
        self.R, self.N = R, s.n_beads
        self._keep = dict(
            off=np.ascontiguousarray(s.bead_offset, np.int64),
            box=np.ascontiguousarray(s.box_q, np.int64),
            fs=np.ascontiguousarray(s.form_scale if s.form_scale is not None else np.ones(R), np.float64),
            bs=np.ascontiguousarray(s.break_scale if s.break_scale is not None else np.ones(R), np.float64),
            stream=np.ascontiguousarray(s.rng_stream if s.rng_stream is not None else np.arange(R), np.uint32),
            types=np.ascontiguousarray(s.types, np.int32),
            bonds=np.ascontiguousarray(s.bonds, np.int32).reshape(-1, 4),
            rules=pack_rules(s.rules),
        )
        k = self._keep
        self.h = L.orc_new(R, _p(k["off"]), _p(k["box"]), _p(k["fs"]), _p(k["bs"]), _p(k["stream"]),
                           _p(k["types"]), _p(k["bonds"]), len(k["bonds"]), _p(k["rules"]), len(s.rules),
                           int(prm["seed"]), int(prm["paircheck13"]), int(prm["paircheck14"]),
                           int(prm["max_rounds"]), int(prm["prob_mode"]), int(prm["reactive_mask"]),
                           int(use_cells))
        if not self.h:
            raise ValueError("oracle rejected the system (bad bonds)")
        self.ff = s.forcefield

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_free(self.h)
            self.h = None

    def step(self, pos: np.ndarray, step: int) -> np.ndarray:
        pos = np.ascontiguousarray(pos, np.int32)
        st = np.zeros((self.R, len(STAT_NAMES)), np.int64)
        rc = lib().orc_step(self.h, _p(pos), int(step), _p(st))
        if rc != 0:
            raise ValueError(f"oracle step failed ({rc})")
        return st

    def counts(self):
        c = np.zeros(3, np.int64)
        lib().orc_counts(self.h, _p(c))
        return tuple(int(x) for x in c)

    def topology(self):
        nb, na, nd = self.counts()
        b = np.zeros((nb, 4), np.int32)
        a = np.zeros((na, 4), np.int32)
        d = np.zeros((nd, 5), np.int32)
        lib().orc_topology(self.h, _p(b), _p(a), _p(d))
        return b, a, d

    def check_rules_identity(self) -> bool:
        return bool(lib().orc_check_rules_identity(self.h))

    def candidates(self, pos: np.ndarray, brute: bool = False) -> np.ndarray:
        pos = np.ascontiguousarray(pos, np.int32)
        n = lib().orc_candidates(self.h, _p(pos), int(brute), None, 0)
        out = np.zeros((max(n, 1), 5), np.int32)
        lib().orc_candidates(self.h, _p(pos), int(brute), _p(out), n)
        return out[:n]

    def forces(self, pos: np.ndarray, ff=None):
        ff = ff or self.ff
        pos = np.ascontiguousarray(pos, np.int32)
        f = np.zeros((self.N, 3), np.float64)
        ev = np.zeros((self.R, 7), np.float64)
        arrs = [np.ascontiguousarray(ff[k], np.float64) for k in ("bond_k", "bond_r0", "angle_k", "dihedral_k")]
        dd = np.ascontiguousarray(ff["dihedral_d"], np.int32)
        t0 = np.ascontiguousarray(ff.get("angle_theta0", np.zeros(16)), np.float64)
        sty = np.ascontiguousarray(ff.get("angle_style", np.zeros(16)), np.int32)
        lib().orc_forces(self.h, _p(pos), *[_p(a) for a in arrs], _p(dd), _p(t0), _p(sty), _p(f), _p(ev))
        return f, ev

    def dpd_forces(self, pos: np.ndarray, vel: np.ndarray, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.01,
                   seed=12345, step=0) -> np.ndarray:
        """DPD pair forces of Sec. 3 on the oracle's current bonds (FP64,
        brute force over pairs): float64 [N, 3]."""
        pos = np.ascontiguousarray(pos, np.int32)
        vel = np.ascontiguousarray(np.asarray(vel)[:, :3], np.float64)
        f = np.zeros((self.N, 3), np.float64)
        lib().orc_dpd_forces(self.h, _p(pos), _p(vel), a, gamma, kT, rc, dt, int(seed) % (1 << 64), int(step),
                             _p(f))
        return f


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox(_p(c), _p(k), _p(o))
    return o


def r2(dist: float) -> int:
    return int(lib().orc_r2(float(dist)))


def threshold(p: float) -> int:
    return int(lib().orc_threshold(float(p)))


def match(n_beads: int, k1, a, b, max_rounds: int = 0):
    k1 = np.ascontiguousarray(k1, np.int64)
    a = np.ascontiguousarray(a, np.int32)
    b = np.ascontiguousarray(b, np.int32)
    m = np.zeros(len(k1), np.int32)
    rounds = lib().orc_match(n_beads, len(k1), _p(k1), _p(a), _p(b), max_rounds, _p(m))
    return m.astype(bool), rounds


def bond_half(rij, K, r0):
    rij = np.ascontiguousarray(rij, np.float64)
    E = np.zeros(1)
    F = np.zeros(3)
    lib().orc_bond_half(_p(rij), K, r0, _p(E), _p(F))
    return E[0], F


def angle_harmonic(ra, rc, K, theta0):
    ra = np.ascontiguousarray(ra, np.float64)
    rc = np.ascontiguousarray(rc, np.float64)
    E = np.zeros(1)
    Fa, Fc = np.zeros(3), np.zeros(3)
    lib().orc_angle_harmonic(_p(ra), _p(rc), K, theta0, _p(E), _p(Fa), _p(Fc))
    return E[0], Fa, Fc


def angle(ra, rc, K):
    ra = np.ascontiguousarray(ra, np.float64)
    rc = np.ascontiguousarray(rc, np.float64)
    E = np.zeros(1)
    Fa, Fc = np.zeros(3), np.zeros(3)
    lib().orc_angle(_p(ra), _p(rc), K, _p(E), _p(Fa), _p(Fc))
    return E[0], Fa, Fc


def dihedral(b1, b2, b3, K, d):
    b1, b2, b3 = (np.ascontiguousarray(x, np.float64) for x in (b1, b2, b3))
    E = np.zeros(1)
    F = [np.zeros(3) for _ in range(4)]
    lib().orc_dihedral(_p(b1), _p(b2), _p(b3), K, d, _p(E), *[_p(x) for x in F])
    return E[0], F
