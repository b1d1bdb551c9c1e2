"""The paper's 1-bead DNA model in the paper's own semantics on the oracle
(CPU): oligomers hybridized to templates ligate across their nicks, the
functionality limits of Fig. 2 hold after every call, and the incremental
interaction sets equal the full recomputation."""
import numpy as np

from oracle import oracle as O
from paper_1108_4214_gb300 import workloads as W


def test_oligomers_ligate_and_functionality_holds():
    s = W.dna1_oligo_system(n_motifs=16)
    o = O.Oracle(s)
    formed = 0
    for k, snap in enumerate(s.snapshots(0, 10)):
        st = o.step(snap, k)
        formed += int(st[0, O.STAT_NAMES.index("bonds_formed")])
        bonds = o.topology()[0]
        # at most one bond of each of the types 1, 2, 3 per bead (Fig. 2)
        for t in (W.HYB, W.BB3, W.BB5):
            stored = np.concatenate([bonds[bonds[:, 2] == t, 0], bonds[bonds[:, 3] == t, 1]])
            assert np.bincount(stored).max(initial=0) <= 1, (k, t)
        assert o.check_rules_identity(), k
    assert formed > 0


def test_nicked_duplexes_ligate_in_chain_direction():
    """Directional ligation in the 2-bead model (createdirbond between
    backbone beads, at most one stored bond of type 2 and one of type 3 per
    backbone bead): every nick that closes continues its strand's direction
    (the bead before the nick stores 2, the bead after it stores 3, as the
    backbone bonds of the strands do), no backbone bead ever stores two
    bonds of one direction, and the incremental interaction sets equal the
    recomputation from the rules (backbone angles and stacking dihedrals
    across the new bonds)."""
    s = W.dna2_nicked_system()
    o = O.Oracle(s)
    nb = 2 * 16
    nicks = [((2 * d + 1) * nb + 2 * m, (2 * d + 1) * nb + 2 * (m + 1)) for d in range(16) for m in (3, 7, 11)]
    for k, snap in enumerate(s.snapshots(0, 8)):
        o.step(snap, k)
        bonds = o.topology()[0]
        for t in (W.BB3, W.BB5):
            stored = np.concatenate([bonds[bonds[:, 2] == t, 0], bonds[bonds[:, 3] == t, 1]])
            assert np.bincount(stored).max(initial=0) <= 1, (k, t)
        assert o.check_rules_identity(), k
    bonds = o.topology()[0]
    have = {(int(b[0]), int(b[1])): (int(b[2]), int(b[3])) for b in bonds}
    closed = [have[nk] for nk in nicks if nk in have]
    assert len(closed) >= len(nicks) // 2, len(closed)
    assert all(c == (W.BB3, W.BB5) for c in closed), closed
