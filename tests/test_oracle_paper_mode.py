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
