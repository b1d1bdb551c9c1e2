"""Pins of the oracle's DPD pair forces (Sec. 3): closed forms of the
conservative and dissipative parts for a lone pair, the cutoff, the pair
exclusion below 3 bonds, Newton's third law and the statistics of the
Gaussian numbers of the random part."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_4214_gb300 import workloads as W

from helpers import make_system


def pair(sep, bonds=(), types=(0, 0), box=10.0, extra=()):
    pos = [[2.0, 3.0, 4.0], [2.0 + sep[0], 3.0 + sep[1], 4.0 + sep[2]]] + list(extra)
    return make_system(list(types) + [0] * len(extra), list(bonds), pos, box, [])


def test_conservative_force_of_a_lone_pair():
    sep = np.array([0.36, -0.48, 0.0])  # r = 0.6, w = 0.4
    s = pair(sep)
    o = O.Oracle(s)
    q = s.snapshot()
    f = o.dpd_forces(q, np.zeros((2, 3)), a=25.0, gamma=0.0, kT=0.0)
    r = (q[0, :3].astype(np.int64) - q[1, :3]) / W.QSCALE  # r_0 - r_1 on the grid
    rn = np.linalg.norm(r)
    want = 25.0 * (1.0 - rn) * r / rn
    assert np.allclose(f[0], want, rtol=1e-12, atol=1e-12) and np.allclose(f[1], -want, rtol=1e-12, atol=1e-12)


def test_dissipative_force_opposes_approach():
    s = pair([0.5, 0.0, 0.0])
    o = O.Oracle(s)
    q = s.snapshot()
    v = np.array([[0.3, 0.2, 0.0], [-0.4, 0.0, 0.1]])
    f = o.dpd_forces(q, v, a=0.0, gamma=4.5, kT=0.0)
    r = (q[0, :3].astype(np.int64) - q[1, :3]) / W.QSCALE
    rn = np.linalg.norm(r)
    w = 1.0 - rn
    want = -4.5 * w * w * (r @ (v[0] - v[1])) / rn * r / rn
    assert np.allclose(f[0], want, rtol=1e-12, atol=1e-14)
    # bead 0 sits on the -x side and moves toward bead 1: pushed back along -x
    assert f[0, 0] > 0 if r[0] > 0 else f[0, 0] < 0


def test_cutoff_is_strict_on_the_grid():
    # exactly r_c apart: d2 = (2^20)^2 is not below floor((1 * 2^20)^2)
    s = pair([1.0, 0.0, 0.0])
    o = O.Oracle(s)
    assert not o.dpd_forces(s.snapshot(), np.zeros((2, 3))).any()
    q = s.snapshot()
    q[1, 0] -= 1  # one quantum closer
    assert o.dpd_forces(q, np.zeros((2, 3)), gamma=0.0, kT=0.0)[0, 0] != 0


def test_pairs_fewer_than_three_bonds_apart_feel_nothing():
    # chain 0-1-2-3: beads 0, 1, 2 along x 0.4 apart, bead 3 folded back 0.5
    # from bead 0.  Within the cutoff: 0-1, 1-2, 2-3 (1 bond apart) and 0-2,
    # 1-3 (2 bonds apart) are excluded; only 0-3 (3 bonds apart) interacts.
    bonds = [[0, 1, 1, 1], [1, 2, 1, 1], [2, 3, 1, 1]]
    pos = [[2.0, 2, 2], [2.4, 2, 2], [2.8, 2, 2], [2.0, 2.5, 2]]
    s = make_system([0, 0, 0, 0], bonds, pos, 10.0, [])
    o = O.Oracle(s)
    q = s.snapshot()
    f = o.dpd_forces(q, np.zeros((4, 3)), gamma=0.0, kT=0.0)
    assert not f[1].any() and not f[2].any()
    assert np.allclose(f[0], -f[3]) and np.abs(f[0]).max() > 1.0


def test_newton_third_law_and_random_part_statistics():
    s = W.dna_system("dpd", 16, 16, 3.0, 31, W.rules_dna2())
    o = O.Oracle(s)
    q = s.snapshot()
    rng = np.random.default_rng(4)
    v = rng.normal(size=(s.n_beads, 3))
    f = o.dpd_forces(q, v, step=7)
    assert np.abs(f.sum(axis=0)).max() < 1e-9 * np.abs(f).max() * s.n_beads
    # random part alone on a lone pair: F / (sigma w / sqrt(dt)) is xi, a unit
    # Gaussian over steps
    sp = pair([0.5, 0.0, 0.0])
    op = O.Oracle(sp)
    qp = sp.snapshot()
    r = (qp[0, :3].astype(np.int64) - qp[1, :3]) / W.QSCALE
    rn = np.linalg.norm(r)
    scale = np.sqrt(2.0 * 1.0 * 4.5) * (1.0 - rn) / np.sqrt(0.01)
    xs = np.array([op.dpd_forces(qp, np.zeros((2, 3)), a=0.0, step=k)[0] @ (r / rn) / scale for k in range(20000)])
    assert abs(xs.mean()) < 4.0 / np.sqrt(len(xs))
    assert abs(xs.var() - 1.0) < 4.0 * np.sqrt(2.0 / len(xs))
    assert abs(np.mean(xs ** 4) - 3.0) < 0.25  # Gaussian kurtosis
