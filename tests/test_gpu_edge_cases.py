"""The hand-placed cases of the oracle's pins (Sec. 2 rule semantics,
Appendix steps 2-9) run through the CUDA path: statistics and topology must
match the oracle bit for bit after every call, forces within the parity
bar.  These are the configurations random systems almost never produce:
a distance exactly at the quantum, the half-box tie, graph distances 1-4
under paircheck13 / paircheck14, maxbond on another bond type, the last
matching rule with createdirbond, equal-distance ties, rounds against the
single nomination, breakbond's most distant partner, unlimited killbond,
convertbond retyping its angles, and nearly straight harmonic angles."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_4214_gb300 import workloads as W

from helpers import make_system
from parity import compare_forces, dynbond, run_parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HYB_RULES = [
    dict(kind="createbond", btype=1, beads=(W.bit(1), W.bit(2)), dist=1.1, prob=1.0),
    dict(kind="maxbond", bonds=W.bit(1), beads=W.bit(1, 2, 3, 4), max=1),
]


def bonds_after(system, n_calls=1, snaps=None, params=None):
    o, _ = run_parity(system, n_calls, snaps=snaps, params=params)
    return o.topology()[0].tolist(), o


@pytest.mark.parametrize("cell_scale", [0, 1, 2])
def test_distance_exactly_at_the_quantum(cell_scale):
    """d = floor(sqrt(R2)) quanta is within 1.1 sigma (inclusive), one more is not."""
    R2 = O.r2(1.1)
    d_in = int(np.floor(np.sqrt(R2)))
    for d, want in ((d_in, [[0, 1, 1, 1]]), (d_in + 1, [])):
        s = make_system([1, 2], [], np.zeros((2, 3)), 10.0, HYB_RULES)
        pos = np.zeros((2, 4), np.int32)
        pos[:, :3] = 1 << 22
        pos[1, 0] += d
        got, _ = bonds_after(s, snaps=[pos], params=dict(cell_scale=cell_scale))
        assert got == want, d


@pytest.mark.parametrize("cell_scale", [1, 2])
def test_periodic_image_and_half_box_tie(cell_scale):
    s = make_system([1, 2], [], [[0.1, 3, 3], [9.6, 3, 3]], 10.0, HYB_RULES)
    assert bonds_after(s, params=dict(cell_scale=cell_scale))[0] == [[0, 1, 1, 1]]
    # 2 dx = L exactly (a box of 2 sigma): the pair is half a box apart either way
    rules = [dict(HYB_RULES[0], dist=1.0), HYB_RULES[1]]
    s = make_system([1, 2], [], [[0.0, 0.5, 0.5], [1.0, 0.5, 0.5]], 2.0, rules)
    got, o = bonds_after(s, params=dict(cell_scale=cell_scale))
    assert got == [[0, 1, 1, 1]]


def test_complementarity_and_reactive_group():
    assert bonds_after(make_system([1, 3], [], [[1, 1, 1], [1.5, 1, 1]], 10.0, HYB_RULES))[0] == []
    s = make_system([1, 2], [], [[1, 1, 1], [1.5, 1, 1]], 10.0, HYB_RULES, params=dict(reactive_mask=W.bit(1)))
    assert bonds_after(s)[0] == []
    assert bonds_after(make_system([2, 1], [], [[1, 1, 1], [1.5, 1, 1]], 10.0, HYB_RULES))[0] == [[0, 1, 1, 1]]


@pytest.mark.parametrize("pc13,pc14,want", [(0, 0, {4}), (1, 0, {2, 4}), (0, 1, {3, 4}), (1, 1, {2, 3, 4})])
def test_graph_distance_exclusions_and_paircheck(pc13, pc14, want):
    # chain 0-1-2-3-4 of type-5 bonds; bead 0 (A) and Ts at graph distance 2, 3 and 4
    types = [1, 0, 2, 2, 2]
    chain = [[0, 1, 5, 5], [1, 2, 5, 5], [2, 3, 5, 5], [3, 4, 5, 5]]
    pos = [[1, 1, 1], [1.3, 1, 1], [1, 1.3, 1], [1, 1, 1.3], [1.3, 1.3, 1]]
    rules = [HYB_RULES[0]]
    s = make_system(types, chain, pos, 10.0, rules, params=dict(paircheck13=pc13, paircheck14=pc14))
    o = O.Oracle(s)
    assert {int(r[1]) for r in o.candidates(s.snapshot())} == want
    run_parity(s, 1)
    # graph distance 1 is never eligible, paircheck or not
    s = make_system([1, 2], [[0, 1, 5, 5]], [[1, 1, 1], [1.5, 1, 1]], 10.0, HYB_RULES,
                    params=dict(paircheck13=1, paircheck14=1))
    got, _ = bonds_after(s)
    assert got == [[0, 1, 5, 5]]


def test_maxbond_counts_only_its_own_bond_types():
    s = make_system([1, 2, 2], [[0, 2, 1, 1]], [[1, 1, 1], [1.5, 1, 1], [3, 3, 3]], 10.0, HYB_RULES)
    assert bonds_after(s)[0] == [[0, 2, 1, 1]]
    rules = [HYB_RULES[0], dict(kind="maxbond", bonds=W.bit(2), beads=W.bit(1, 2), max=1)]
    s = make_system([1, 2, 2], [[0, 2, 1, 1]], [[1, 1, 1], [1.5, 1, 1], [3, 3, 3]], 10.0, rules)
    assert bonds_after(s)[0] == [[0, 1, 1, 1], [0, 2, 1, 1]]


def test_last_matching_rule_wins_with_directional_types():
    rules = [
        dict(kind="createbond", btype=1, beads=(W.bit(1), W.bit(2)), dist=1.1, prob=1.0),
        dict(kind="createdirbond", btype=2, btype2=3, beads=(W.bit(2), W.bit(1)), dist=1.1, prob=1.0),
        dict(kind="createbond", btype=6, beads=(W.bit(1), W.bit(2)), dist=0.2, prob=1.0),
    ]
    s = make_system([1, 2], [], [[1, 1, 1], [1.5, 1, 1]], 10.0, rules)
    assert bonds_after(s)[0] == [[0, 1, 3, 2]]
    s = make_system([1, 2], [], [[1, 1, 1], [1.1, 1, 1]], 10.0, rules)
    assert bonds_after(s)[0] == [[0, 1, 6, 6]]


def test_nearest_partner_wins_and_equal_distances_go_to_the_lower_id():
    s = make_system([1, 2, 2], [], [[2, 2, 2], [2.9, 2, 2], [1.0, 2, 2]], 10.0, HYB_RULES)
    assert bonds_after(s)[0] == [[0, 1, 1, 1]]
    s = make_system([1, 2, 2], [], [[2, 2, 2], [3.0, 2, 2], [1.0, 2, 2]], 10.0, HYB_RULES)
    assert bonds_after(s)[0] == [[0, 1, 1, 1]]
    # all distances equal among four beads: the gid order decides every round
    s = make_system([1, 2, 1, 2], [], [[2, 2, 2], [2.5, 2, 2], [2.5, 2.5, 2], [2, 2.5, 2]], 10.0, HYB_RULES)
    assert bonds_after(s)[0] == [[0, 1, 1, 1], [2, 3, 1, 1]]


@pytest.mark.parametrize("max_rounds,want", [(0, [[0, 2, 1, 1], [1, 3, 1, 1]]), (1, [[0, 2, 1, 1]])])
def test_rounds_against_the_single_nomination(max_rounds, want):
    pos2 = [[2.0, 2, 2], [2.0, 3.0, 2], [2.5, 2, 2], [2.95, 2.6, 2]]
    s = make_system([1, 2, 2, 1], [], pos2, 10.0, HYB_RULES, params=dict(max_rounds=max_rounds))
    got, o = bonds_after(s)
    assert got == want


def test_breakbond_most_distant_killbond_unlimited_strict_and_directional():
    types = [1, 2, 2, 2]
    bonds = [[0, 1, 1, 1], [0, 2, 1, 1], [0, 3, 1, 1]]
    pos = [[3, 3, 3], [4.2, 3, 3], [3, 4.5, 3], [3, 3, 4.8]]
    s = make_system(types, bonds, pos, 10.0, [dict(kind="breakbond", btype=1, dist=1.1, prob=1.0)])
    assert bonds_after(s)[0] == [[0, 1, 1, 1], [0, 2, 1, 1]]
    s = make_system(types, bonds, pos, 10.0, [dict(kind="killbond", btype=1, dist=1.1)])
    assert bonds_after(s)[0] == []
    s = make_system([1, 2, 2], [[0, 1, 1, 1], [0, 2, 1, 2]], [[3, 3, 3], [4.2, 3, 3], [3, 5, 3]], 10.0,
                    [dict(kind="breakbond", btype=1, dist=1.2, prob=1.0)])
    assert bonds_after(s)[0] == [[0, 1, 1, 1], [0, 2, 1, 2]]


def test_convertbond_retypes_its_angles():
    rules = [
        dict(kind="convertbond", btype=1, btype2=3, prob=1.0),
        dict(kind="createangle", type=7, beads=(W.ALL_BEADS,) * 3, bonds=(W.bit(3), W.bit(2))),
        dict(kind="createangle", type=5, beads=(W.ALL_BEADS,) * 3, bonds=(W.bit(1), W.bit(2))),
    ]
    s = make_system([0, 0, 0], [[0, 1, 1, 1], [1, 2, 2, 2]], [[1, 1, 1], [2, 1, 1], [3, 1, 1.2]], 10.0, rules)
    got, o = bonds_after(s)
    assert got == [[0, 1, 3, 3], [1, 2, 2, 2]]
    assert o.topology()[1].tolist() == [[0, 1, 2, 7]]


@pytest.mark.parametrize("k,theta0", [(10486, np.pi), (105, np.pi), (1, np.pi), (0, np.pi), (10486, np.pi / 2),
                                      (105, np.pi / 2)])
def test_nearly_straight_harmonic_angle(k, theta0):
    """One harmonic angle bent k quanta off straight over 1 sigma (pi - theta
    = 1e-2, 1e-4, 1e-6 or exactly straight), bonds without stiffness: the GPU
    forces match the oracle's exact gradient within the parity bar."""
    rules = [dict(kind="createbond", btype=1, beads=(W.bit(7), W.bit(7)), dist=0.1, prob=0.0),
             dict(kind="createangle", type=1, beads=(W.ALL_BEADS,) * 3, bonds=(W.bit(2), W.bit(3)))]
    s = make_system([0, 0, 0], [[0, 1, 3, 2], [1, 2, 3, 2]], np.zeros((3, 3)), 20.0, rules)
    ff = W.forcefield_dna2()
    ff["bond_k"][:] = 0.0
    ff["angle_style"] = np.ones(16, np.int32)
    ff["angle_k"][1] = 20.0
    ff["angle_theta0"] = np.full(16, theta0)
    s.forcefield = ff
    o = O.Oracle(s)
    assert o.topology()[1].tolist() == [[0, 1, 2, 1]]
    X = 5 << 20
    pos = np.zeros((3, 4), np.int32)
    u = np.array([1 << 20, 37001, -21003])  # A - B, one sigma and a bit
    perp = np.array([0, 21003, 37001])      # perpendicular to u
    pos[0, :3] = X + u
    pos[1, :3] = X
    pos[2, :3] = X - u + np.rint(perp * (k / np.linalg.norm(perp))).astype(np.int64)
    ctx = dynbond().Context(s)
    fr, evr = o.forces(pos)
    # the virial of one angle is a sum of two terms of size |r| |F| that
    # nearly cancel when the angle is straight: its FP32 error is bounded
    # relative to those terms, not to the sum
    rel = (pos[[0, 2], :3].astype(np.int64) - pos[1, :3]) / W.QSCALE
    terms = float(np.linalg.norm(rel, axis=1) @ np.linalg.norm(fr[[0, 2]], axis=1)) + abs(evr[0, 0])
    compare_forces(ctx, o, pos, f"k={k}", ev_scale=[terms])
    if k == 0 and theta0 == np.pi:
        assert not fr.any()
    else:
        assert np.abs(fr).max() > 0


def test_crowded_bead_without_candidates():
    """A saturated A bead (maxbond reached) with more than
    DYNBOND_MAX_CANDIDATES complementary beads within reach: its register
    list overflows, the exact pass finds no candidate, and the bead must take
    no part in the matching; the crowd of T beads keeps bonding among the
    other A beads exactly as the oracle says."""
    rng = np.random.default_rng(12)
    n_t = 40
    crowd = 5.0 + rng.uniform(-0.6, 0.6, size=(n_t, 3))
    pos = np.concatenate([[[5.0, 5.0, 5.0], [5.0, 5.0, 5.9]], crowd, [[5.5, 5.5, 5.0], [4.5, 4.6, 5.2]]])
    types = [1, 2] + [2] * n_t + [1, 1]
    s = make_system(types, [[0, 1, 1, 1]], pos, 12.0, HYB_RULES)
    o = O.Oracle(s)
    over = [r for r in o.candidates(s.snapshot()) if 0 in (int(r[0]), int(r[1]))]
    assert not over  # bead 0 has no candidate, though more than 24 beads are within reach
    run_parity(s, 3)
