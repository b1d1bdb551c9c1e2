"""Pins of the oracle's dynamic-bonding call against hand-placed cases, the
paper's own DNA typing patterns, brute force and invariants."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_4214_gb300 import workloads as W

from helpers import golden, golden_rules, ladder_1bead_positions, make_system, qpos

HYB_RULES = [
    dict(kind="createbond", btype=1, beads=(W.bit(1), W.bit(2)), dist=1.1, prob=1.0),
    dict(kind="maxbond", bonds=W.bit(1), beads=W.bit(1, 2, 3, 4), max=1),
]


def cand_pairs(o, pos, brute=True):
    return {(int(r[0]), int(r[1])) for r in o.candidates(pos, brute=brute)}


# ---------------------------------------------------------------------------
# creation candidates (Sec. 2 and Appendix step 2)
# ---------------------------------------------------------------------------

def test_distance_threshold_is_inclusive_at_the_quantum():
    s = make_system([1, 2], [], np.zeros((2, 3)), 10.0, HYB_RULES)
    o = O.Oracle(s)
    R2 = O.r2(1.1)
    d_in = int(np.floor(np.sqrt(R2)))
    assert d_in * d_in <= R2 < (d_in + 1) ** 2
    for d, want in ((d_in, True), (d_in + 1, False)):
        pos = np.zeros((2, 4), np.int32)
        pos[:, :3] = 1 << 22
        pos[1, 0] += d
        assert (cand_pairs(o, pos) == {(0, 1)}) == want


def test_complementarity_and_reactive_group():
    s = make_system([1, 3], [], [[1, 1, 1], [1.5, 1, 1]], 10.0, HYB_RULES)
    assert cand_pairs(O.Oracle(s), s.snapshot()) == set()  # A-C is no rule pair
    s = make_system([1, 2], [], [[1, 1, 1], [1.5, 1, 1]], 10.0, HYB_RULES, params=dict(reactive_mask=W.bit(1)))
    assert cand_pairs(O.Oracle(s), s.snapshot()) == set()  # T outside the reactive group
    s = make_system([2, 1], [], [[1, 1, 1], [1.5, 1, 1]], 10.0, HYB_RULES)
    assert cand_pairs(O.Oracle(s), s.snapshot()) == {(0, 1)}  # either bead order


def test_periodic_minimum_image_and_half_box_tie():
    # across the boundary
    s = make_system([1, 2], [], [[0.1, 3, 3], [9.6, 3, 3]], 10.0, HYB_RULES)
    assert cand_pairs(O.Oracle(s), s.snapshot()) == {(0, 1)}
    # separation of exactly half the box (2 dx = L): distance L/2 either way
    s = make_system([1, 2], [], [[0.0, 0.5, 0.5], [1.0, 0.5, 0.5]], 2.0, HYB_RULES)
    o = O.Oracle(s)
    assert cand_pairs(o, s.snapshot()) == {(0, 1)}
    assert cand_pairs(o, s.snapshot(), brute=False) == {(0, 1)}
    row = o.candidates(s.snapshot())[0]
    d2 = (int(row[3]) & 0xFFFFFFFF) | (int(row[4]) << 32)
    assert d2 == (1 << 20) ** 2


def test_graph_distance_exclusions_and_paircheck():
    # chain 0-1-2-3-4 of type-5 bonds between an A (bead 0) and Ts at graph distance 2, 3, 4
    types = [1, 0, 2, 2, 2]
    bonds = [[0, 1, 5, 5], [1, 2, 5, 5], [2, 3, 5, 5], [3, 4, 5, 5]]
    pos = [[1, 1, 1], [1.3, 1, 1], [1, 1.3, 1], [1, 1, 1.3], [1.3, 1.3, 1]]
    for pc13, pc14, want in ((0, 0, {(0, 4)}), (1, 0, {(0, 2), (0, 4)}), (0, 1, {(0, 3), (0, 4)}),
                             (1, 1, {(0, 2), (0, 3), (0, 4)})):
        s = make_system(types, bonds, pos, 10.0, HYB_RULES, params=dict(paircheck13=pc13, paircheck14=pc14))
        assert cand_pairs(O.Oracle(s), s.snapshot()) == want, (pc13, pc14)
    # graph distance 1 is never eligible, paircheck or not
    s = make_system([1, 2], [[0, 1, 5, 5]], [[1, 1, 1], [1.5, 1, 1]], 10.0, HYB_RULES,
                    params=dict(paircheck13=1, paircheck14=1))
    assert cand_pairs(O.Oracle(s), s.snapshot()) == set()


def test_maxbond_discards_saturated_beads():
    # bead 0 (A) already holds one hybridization bond to bead 2
    s = make_system([1, 2, 2], [[0, 2, 1, 1]], [[1, 1, 1], [1.5, 1, 1], [3, 3, 3]], 10.0, HYB_RULES)
    assert cand_pairs(O.Oracle(s), s.snapshot()) == set()
    # a maxbond rule on another bond type does not discard it
    rules = [HYB_RULES[0], dict(kind="maxbond", bonds=W.bit(2), beads=W.bit(1, 2), max=1)]
    s = make_system([1, 2, 2], [[0, 2, 1, 1]], [[1, 1, 1], [1.5, 1, 1], [3, 3, 3]], 10.0, rules)
    assert cand_pairs(O.Oracle(s), s.snapshot()) == {(0, 1)}


def test_last_matching_rule_wins_and_directional_types():
    rules = [
        dict(kind="createbond", btype=1, beads=(W.bit(1), W.bit(2)), dist=1.1, prob=1.0),
        dict(kind="createdirbond", btype=2, btype2=3, beads=(W.bit(2), W.bit(1)), dist=1.1, prob=1.0),
        dict(kind="createbond", btype=6, beads=(W.bit(1), W.bit(2)), dist=0.2, prob=1.0),  # too short here
    ]
    s = make_system([1, 2], [], [[1, 1, 1], [1.5, 1, 1]], 10.0, rules)
    o = O.Oracle(s)
    o.step(s.snapshot(), 0)
    b, _, _ = o.topology()
    # rule 2 (createdirbond) is the last rule matching at d = 0.5: the T bead (first
    # bead type of the rule) stores 2, the A bead stores 3
    assert b.tolist() == [[0, 1, 3, 2]]
    s = make_system([1, 2], [], [[1, 1, 1], [1.1, 1, 1]], 10.0, rules)
    o = O.Oracle(s)
    o.step(s.snapshot(), 0)
    assert o.topology()[0].tolist() == [[0, 1, 6, 6]]


def test_brute_force_equals_cell_list_on_random_systems():
    for seed in range(25):
        rules = W.random_rules(seed)
        s = W.random_small_system(seed, n_beads=60, box=float(2.0 + seed % 5), n_bonds=50, rules=rules,
                                  n_replicas=1 + seed % 3,
                                  params=dict(paircheck13=seed % 2, paircheck14=(seed // 2) % 2))
        o = O.Oracle(s)
        for k in range(3):
            pos = s.snapshot(k)
            assert np.array_equal(o.candidates(pos, True), o.candidates(pos, False)), seed


def test_brute_force_equals_cell_list_on_the_2048_bead_system():
    s = W.config1()
    o = O.Oracle(s)
    pos = s.snapshot(0)
    a, b = o.candidates(pos, True), o.candidates(pos, False)
    assert len(a) > 100 and np.array_equal(a, b)


# ---------------------------------------------------------------------------
# one call with deterministic probabilities (p = 1)
# ---------------------------------------------------------------------------

def test_nearest_partner_wins_and_ties_go_to_lower_id():
    # A at 0; T at 0.9 (bead 1) and T at 1.0 (bead 2): the nearer one bonds
    s = make_system([1, 2, 2], [], [[2, 2, 2], [2.9, 2, 2], [1.0, 2, 2]], 10.0, HYB_RULES)
    o = O.Oracle(s)
    st = o.step(s.snapshot(), 0)
    assert o.topology()[0].tolist() == [[0, 1, 1, 1]]
    assert st[0][O.STAT_NAMES.index("candidates")] == 2
    # exactly equal distances: the lower id (bead 1) wins
    s = make_system([1, 2, 2], [], [[2, 2, 2], [3.0, 2, 2], [1.0, 2, 2]], 10.0, HYB_RULES)
    o = O.Oracle(s)
    o.step(s.snapshot(), 0)
    assert o.topology()[0].tolist() == [[0, 1, 1, 1]]


def test_rounds_let_a_rejected_bead_take_its_second_choice():
    # T1 - A0 - T2 - A3 on a line: A0 and T2 are closest; T1 and A3 prefer them too
    pos = [[2.0, 2, 2], [1.2, 2, 2], [2.5, 2, 2], [3.2, 2, 2]]
    types = [1, 2, 2, 1]
    # A3's nearest is T2 (0.7) but T2 takes A0 (0.5); A3's second choice T1 is too far
    s = make_system(types, [], pos, 10.0, HYB_RULES)
    o = O.Oracle(s)
    o.step(s.snapshot(), 0)
    assert o.topology()[0].tolist() == [[0, 2, 1, 1]]
    # now put T1 within reach of A3 through the box: it matches in round 2
    pos2 = [[2.0, 2, 2], [2.0, 3.0, 2], [2.5, 2, 2], [2.95, 2.6, 2]]
    s = make_system(types, [], pos2, 10.0, HYB_RULES)
    o = O.Oracle(s)
    st = o.step(s.snapshot(), 0)
    assert o.topology()[0].tolist() == [[0, 2, 1, 1], [1, 3, 1, 1]]
    assert st[0][O.STAT_NAMES.index("create_rounds")] == 2
    # the paper's single nomination (max_rounds = 1) leaves the second pair unbonded
    s = make_system(types, [], pos2, 10.0, HYB_RULES, params=dict(max_rounds=1))
    o = O.Oracle(s)
    o.step(s.snapshot(), 0)
    assert o.topology()[0].tolist() == [[0, 2, 1, 1]]


def test_breakbond_picks_most_distant_and_killbond_is_unlimited():
    # bead 0 holds three type-1 bonds of lengths 1.2, 1.5 and 1.8 (no maxbond here)
    types = [1, 2, 2, 2]
    bonds = [[0, 1, 1, 1], [0, 2, 1, 1], [0, 3, 1, 1]]
    pos = [[3, 3, 3], [4.2, 3, 3], [3, 4.5, 3], [3, 3, 4.8]]
    rules = [dict(kind="breakbond", btype=1, dist=1.1, prob=1.0)]
    s = make_system(types, bonds, pos, 10.0, rules)
    o = O.Oracle(s)
    o.step(s.snapshot(), 0)
    assert o.topology()[0].tolist() == [[0, 1, 1, 1], [0, 2, 1, 1]]  # only the longest broke
    rules = [dict(kind="killbond", btype=1, dist=1.1)]
    s = make_system(types, bonds, pos, 10.0, rules)
    o = O.Oracle(s)
    st = o.step(s.snapshot(), 0)
    assert o.topology()[0].tolist() == []  # every bond longer than 1.1 removed
    assert st[0][O.STAT_NAMES.index("bonds_killed")] == 3
    # "longer than" is strict; directional (non-symmetric) bonds are not breakbond targets
    rules = [dict(kind="breakbond", btype=1, dist=1.2, prob=1.0)]
    s = make_system([1, 2, 2], [[0, 1, 1, 1], [0, 2, 1, 2]], [[3, 3, 3], [4.2, 3, 3], [3, 5, 3]], 10.0, rules)
    o = O.Oracle(s)
    o.step(s.snapshot(), 0)
    assert o.topology()[0].tolist() == [[0, 1, 1, 1], [0, 2, 1, 2]]


def test_convertbond_retypes_interactions():
    # A - B - C with bond types 1 (A-B) and 2 (B-C); angle rule needs types (3, 2)
    rules = [
        dict(kind="convertbond", btype=1, btype2=3, prob=1.0),
        dict(kind="createangle", type=7, beads=(W.ALL_BEADS,) * 3, bonds=(W.bit(3), W.bit(2))),
        dict(kind="createangle", type=5, beads=(W.ALL_BEADS,) * 3, bonds=(W.bit(1), W.bit(2))),
    ]
    s = make_system([0, 0, 0], [[0, 1, 1, 1], [1, 2, 2, 2]], [[1, 1, 1], [2, 1, 1], [3, 1, 1]], 10.0, rules)
    o = O.Oracle(s)
    assert o.topology()[1].tolist() == [[0, 1, 2, 5]]
    st = o.step(s.snapshot(), 0)
    b, a, _ = o.topology()
    assert b.tolist() == [[0, 1, 3, 3], [1, 2, 2, 2]]
    assert a.tolist() == [[0, 1, 2, 7]]
    assert st[0][O.STAT_NAMES.index("bonds_converted")] == 1
    assert st[0][O.STAT_NAMES.index("angles_removed")] == 1 and st[0][O.STAT_NAMES.index("angles_added")] == 1


# ---------------------------------------------------------------------------
# the paper's DNA typing patterns (Sec. 3, Fig. 2) on a hand-counted ladder
# ---------------------------------------------------------------------------

def _ladder(rules_extra=(), params=None, pos=None):
    g = golden("dna1bead_ladder_4mer.json")
    rules = list(rules_extra) + golden_rules(g["rules_fig2_9_to_14"])
    s = make_system(g["types"], g["bonds"], pos if pos is not None else ladder_1bead_positions(), 20.0, rules,
                    params=params)
    return g, s


def test_dna_rule_table_types_the_ladder_as_counted_by_hand():
    g, s = _ladder()
    o = O.Oracle(s)
    _, a, d = o.topology()
    assert a.tolist() == sorted(g["expected_angles"])
    assert d.tolist() == sorted(g["expected_dihedrals"])


def test_paper_rule_set_melts_and_renatures_to_the_same_interactions():
    # Fig. 2 rules 2, 3, 5-8 (the 4-mer has no ligation) + the typing rules
    extra = [
        dict(kind="createbond", btype=1, beads=(W.bit(1), W.bit(2)), dist=0.6, prob=1.0),
        dict(kind="createbond", btype=1, beads=(W.bit(3), W.bit(4)), dist=0.6, prob=1.0),
        dict(kind="killbond", btype=1, dist=1.0),
        dict(kind="maxbond", bonds=W.bit(1), beads=W.ALL_BEADS, max=1),
        dict(kind="maxbond", bonds=W.bit(2), beads=W.ALL_BEADS, max=1),
        dict(kind="maxbond", bonds=W.bit(3), beads=W.ALL_BEADS, max=1),
    ]
    g, s = _ladder(extra, params=dict(paircheck14=1))
    o = O.Oracle(s)
    b0, a0, d0 = o.topology()
    far = qpos(s, ladder_1bead_positions(sep=1.5))
    st = o.step(far, 0)
    b1, a1, d1 = o.topology()
    assert st[0][O.STAT_NAMES.index("bonds_killed")] == 4
    assert len(d1) == 0 and sorted(set(a1[:, 3].tolist())) == [1]
    assert o.check_rules_identity()
    near = qpos(s, ladder_1bead_positions(sep=0.5))
    st = o.step(near, 1)
    assert st[0][O.STAT_NAMES.index("bonds_formed")] == 4
    b2, a2, d2 = o.topology()
    assert np.array_equal(b2, b0) and np.array_equal(a2, a0) and np.array_equal(d2, d0)


def test_two_bead_duplex_melts_and_reforms():
    # breakbond p = 1 melts every pair in one call (all pairs mutually nominate);
    # the next call re-forms each base with its old partner (nearest complement)
    rules = W.rules_dna2(p_form=1.0, p_break=1.0)
    rng = np.random.default_rng(3)
    pos, types, bonds = W._replica_strands(rng, 2, 12, 30.0, 0, n_duplex=1)
    s = W.System(name="duplex", bead_offset=np.array([0, 48]), box_q=np.array([30 * W.QSCALE]), types=types,
                 bonds=bonds, rules=rules, pos0=pos, seed=5, sigma_perturb=0.0, params=W.default_params(5))
    o = O.Oracle(s)
    b0, a0, d0 = o.topology()
    assert len(a0) == 2 * 10 + 2 * 12 and len(d0) == 2 * 11 + 12
    snap = s.snapshot(0)
    st = o.step(snap, 0)
    assert st[0][O.STAT_NAMES.index("bonds_broken")] == 12
    assert o.check_rules_identity()
    st = o.step(snap, 1)
    assert st[0][O.STAT_NAMES.index("bonds_formed")] == 12
    b2, a2, d2 = o.topology()
    assert np.array_equal(b2, b0) and np.array_equal(a2, a0) and np.array_equal(d2, d0)


# ---------------------------------------------------------------------------
# invariants over random systems and rules
# ---------------------------------------------------------------------------

def _counts(bonds, n, mask_bonds):
    c = np.zeros(n, np.int64)
    for i, j, ti, tj in bonds:
        if (mask_bonds >> ti) & 1:
            c[i] += 1
        if (mask_bonds >> tj) & 1:
            c[j] += 1
    return c


@pytest.mark.parametrize("seed", range(30))
def test_invariants_on_random_systems(seed):
    rules = W.random_rules(seed)
    s = W.random_small_system(seed, n_beads=50, box=3.0, n_bonds=45, rules=rules, n_replicas=1 + seed % 2,
                              params=dict(paircheck13=seed % 2, paircheck14=(seed // 3) % 2, max_rounds=seed % 3,
                                          prob_mode=seed % 2))
    o = O.Oracle(s)
    N = s.n_beads
    maxb = [r for r in rules if r["kind"] == "maxbond"]
    for k in range(4):
        b0 = {(int(i), int(j)): (int(ti), int(tj)) for i, j, ti, tj in o.topology()[0]}
        o.step(s.snapshot(k), k)
        bl, al, dl = o.topology()
        b1 = {(int(i), int(j)): (int(ti), int(tj)) for i, j, ti, tj in bl}
        # incremental interactions == typed set of every path of the new graph
        assert o.check_rules_identity(), (seed, k)
        # every record lies on live bonds
        for a_, b_, c_, _ in al:
            assert (min(a_, b_), max(a_, b_)) in b1 and (min(b_, c_), max(b_, c_)) in b1
        for a_, b_, c_, d_, _ in dl:
            for x, y in ((a_, b_), (b_, c_), (c_, d_)):
                assert (min(x, y), max(x, y)) in b1
        # at most one bond formed per bead; at most 4 bonds per bead
        added = [p for p in b1 if p not in b0]
        per = np.zeros(N, np.int64)
        for i, j in added:
            per[i] += 1
            per[j] += 1
        assert per.max(initial=0) <= 1
        deg = np.zeros(N, np.int64)
        for i, j in b1:
            deg[i] += 1
            deg[j] += 1
        assert deg.max(initial=0) <= 4
        # maxbond (checked by creation only, Appendix step 2): every formed bond
        # found room at both ends on the pre-call counts; without conversions the
        # counts are never newly exceeded
        has_convert = any(r["kind"] == "convertbond" for r in rules)
        for m in maxb:
            c0 = _counts([(i, j, *t) for (i, j), t in b0.items()], N, m["bonds"])
            c1 = _counts([(i, j, *t) for (i, j), t in b1.items()], N, m["bonds"])
            sel = np.array([(m["beads"] >> int(t)) & 1 for t in s.types], bool)
            for (i, j) in added:
                for x, t in ((i, b1[(i, j)][0]), (j, b1[(i, j)][1])):
                    if sel[x] and (m["bonds"] >> t) & 1:
                        assert c0[x] < m["max"]
            if not has_convert:
                assert np.all(c1[sel] <= np.maximum(c0[sel], m["max"]))
        # formed bonds stay inside one replica
        rep = np.repeat(np.arange(s.n_replicas), np.diff(s.bead_offset))
        assert all(rep[i] == rep[j] for i, j in added)
