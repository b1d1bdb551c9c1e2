"""Seeded synthetic inputs for the dynamic-bonding pass.

This module builds *inputs only*: bead positions on the int32 fixed-point grid
(2^-20 sigma per unit), bead types, the initial bonds with the type each
endpoint stores (Sec. 2, directional bonds), ordered rule lists in the fix
syntax of Fig. 1, per-replica probability scales and force-field tables.  It
holds none of the method's arithmetic (no distances, no matching, no typing,
no forces) and imports neither the CUDA binding nor the CPU oracle, so both
sides can be fed the same arrays.

Model (2 beads per nucleotide, the DNA-like systems of the benchmarks):
  bead types  0 = backbone, 1..4 = bases A, T, C, G (Sec. 3 numbering);
  bond types  1 = hybridization (symmetric),
              2 / 3 = directional backbone: bb_k stores 2 toward bb_{k+1},
                      bb_{k+1} stores 3 toward bb_k (the 3'/5' pair of Sec. 3),
              4 = backbone-base "sugar" bond (symmetric).
Beads of strand s occupy [2*n_nt*s, 2*n_nt*(s+1)); nucleotide k of the strand
is backbone bead 2k and base bead 2k+1.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

QBITS = 20
QSCALE = 1 << QBITS  # quantized units per sigma

BB, A, T, C, G = 0, 1, 2, 3, 4
HYB, BB3, BB5, SUGAR = 1, 2, 3, 4
COMPLEMENT = np.array([0, T, A, G, C], dtype=np.int32)

ALL_BEADS = 0xFFFF  # wildcard '*' over bead types 0..15
ALL_BONDS = 0xFFFE  # wildcard '*' over bond types 1..15


def bit(*types: int) -> int:
    m = 0
    for t in types:
        m |= 1 << t
    return m


# --------------------------------------------------------------------------
# rule lists (neutral form: plain dicts; each side packs them itself)
# --------------------------------------------------------------------------

def rules_dna2(p_form: float = 0.5, p_break: float = 0.05, backbone_maxbond: bool = False) -> List[Dict]:
    """Rule list of the 2-bead DNA-like benchmark model.

    Creation: complementary bases (A-T, C-G) within 1.1 sigma form a
    hybridization bond (createbond, Fig. 1).  Breakage: killbond above 1.3
    sigma and a stochastic breakbond with minimum distance 0.  Functionality:
    at most one hybridization bond per base (maxbond).  Interaction typing: a
    4-entry pattern table (2 createangle + 2 createdihedral rules) whose bond
    fields follow the directional conventions of Sec. 2.
    """
    rules = [
        dict(kind="createbond", btype=HYB, beads=(bit(A), bit(T)), dist=1.1, prob=p_form),
        dict(kind="createbond", btype=HYB, beads=(bit(C), bit(G)), dist=1.1, prob=p_form),
        dict(kind="killbond", btype=HYB, dist=1.3),
        dict(kind="breakbond", btype=HYB, dist=0.0, prob=p_break),
        dict(kind="maxbond", bonds=bit(HYB), beads=bit(A, T, C, G), max=1),
    ]
    if backbone_maxbond:
        rules.append(dict(kind="maxbond", bonds=bit(BB3, BB5), beads=bit(BB), max=2))
    rules += [
        # backbone stiffness at a backbone bead: B stores 2 toward A and 3 toward C
        dict(kind="createangle", type=1, beads=(bit(BB), bit(BB), bit(BB)), bonds=(bit(BB3), bit(BB5))),
        # base-pair angle at a hybridized base: B stores sugar toward its backbone A, hyb toward C
        dict(kind="createangle", type=2, beads=(bit(BB), ALL_BEADS, ALL_BEADS), bonds=(bit(SUGAR), bit(HYB))),
        # bb - base - base - bb across a base pair
        dict(kind="createdihedral", type=1, beads=(bit(BB), ALL_BEADS, ALL_BEADS, bit(BB)),
             bonds=(bit(SUGAR), bit(HYB), bit(SUGAR))),
        # base - bb - bb - base stacking along a strand
        dict(kind="createdihedral", type=2, beads=(ALL_BEADS, bit(BB), bit(BB), ALL_BEADS),
             bonds=(bit(SUGAR), bit(BB3, BB5), bit(SUGAR))),
    ]
    return rules


def rules_dna1_paper() -> List[Dict]:
    """The paper's own rule list of its 1-bead-per-nucleotide DNA model
    (Fig. 2 of Sec. 3; bead types A, T, C, G = 1..4; bond types 1 =
    hybridization, 2 / 3 = the two directions of a backbone bond):
    complementary beads within 0.6 sigma hybridize with probability 1;
    a T bead and a C bead within 0.3 sigma ligate with probability 0.1 by a
    directional backbone bond (the T end stores type 2, the C end type 3);
    hybridization bonds longer than 1 sigma are killed; every bead holds at
    most one bond of each of the types 1, 2 and 3 (the Fig. 2 maxbond lines,
    whose printed argument order is read as max, bead types, bond type); the
    typing rules 9-14 add backbone and base-pair angles and the dihedrals
    across and along base pairs.  Run it with paircheck14, one nomination per
    call and the two-uniform trial (the paper's own semantics)."""
    star = ALL_BEADS
    rules = [
        dict(kind="createbond", btype=HYB, beads=(bit(A), bit(T)), dist=0.6, prob=1.0),
        dict(kind="createbond", btype=HYB, beads=(bit(C), bit(G)), dist=0.6, prob=1.0),
        dict(kind="createdirbond", btype=BB3, btype2=BB5, beads=(bit(T), bit(C)), dist=0.3, prob=0.1),
        dict(kind="killbond", btype=HYB, dist=1.0),
        dict(kind="maxbond", bonds=bit(HYB), beads=star, max=1),
        dict(kind="maxbond", bonds=bit(BB3), beads=star, max=1),
        dict(kind="maxbond", bonds=bit(BB5), beads=star, max=1),
        dict(kind="createangle", type=1, beads=(star, star, star), bonds=(bit(BB3), bit(BB5))),
        dict(kind="createangle", type=2, beads=(star, star, star), bonds=(bit(HYB), bit(BB3, BB5))),
        dict(kind="createdihedral", type=1, beads=(star,) * 4, bonds=(bit(HYB), bit(BB3, BB5), bit(HYB))),
        dict(kind="createdihedral", type=2, beads=(star,) * 4, bonds=(bit(BB3), bit(HYB), bit(BB5))),
        dict(kind="createdihedral", type=3, beads=(star,) * 4, bonds=(bit(BB3), bit(HYB), bit(BB3))),
        dict(kind="createdihedral", type=3, beads=(star,) * 4, bonds=(bit(BB5), bit(HYB), bit(BB5))),
    ]
    return rules


def dna1_oligo_system(n_motifs: int = 64, template_nt: int = 16, oligo_nt: int = 4, seed: int = 6,
                      spacing: float = 0.5, rise: float = 0.5, nick: float = 0.25) -> "System":
    """Oligomers on templates in the paper's 1-bead model (the setting of its
    oligomer-template examples, Sec. 3): each motif is a straight template
    strand and template_nt / oligo_nt complementary oligomers lying
    anti-parallel `rise` sigma beside it, already hybridized; consecutive
    oligomers meet at a nick of `nick` sigma between a T end and a C end, so
    ligation can close it.  Motifs sit on a cubic grid 4 sigma apart with
    random orientations.  Backbone bead k stores type 2 toward bead k+1,
    which stores type 3 toward bead k."""
    rng = np.random.default_rng([seed, 61])
    n_olig = template_nt // oligo_nt
    per = 2 * template_nt
    N = n_motifs * per
    side = int(np.ceil(n_motifs ** (1.0 / 3.0)))
    box = 4.0 * side + 4.0
    pos = np.zeros((N, 3))
    types = np.zeros(N, np.int32)
    bonds = []
    for m in range(n_motifs):
        b0 = m * per
        seq = rng.integers(1, 5, size=template_nt).astype(np.int32)
        for j in range(n_olig - 1):  # template under each nick: oligo ends T (over A) and C (over G)
            seq[template_nt - oligo_nt * (j + 1)] = A
            seq[template_nt - oligo_nt * (j + 1) - 1] = G
        types[b0:b0 + template_nt] = seq
        u = _unit_vectors(rng, 1)[0]
        w = _unit_vectors(rng, 1)[0]
        v = w - np.dot(w, u) * u
        v /= np.linalg.norm(v)
        o = 2.0 + 4.0 * np.array([m % side, (m // side) % side, m // (side * side)], np.float64)
        t = np.arange(template_nt)
        pos[b0:b0 + template_nt] = o + spacing * t[:, None] * u
        bonds.append(np.stack([b0 + t[:-1], b0 + t[1:], np.full(template_nt - 1, BB3),
                               np.full(template_nt - 1, BB5)], axis=1))
        # oligomer beads: oligo j, position k (5' to 3') opposite template bead
        # template_nt - 1 - (oligo_nt * j + k)
        for j in range(n_olig):
            first = b0 + template_nt + oligo_nt * j
            for k in range(oligo_nt):
                tb = template_nt - 1 - (oligo_nt * j + k)
                shift = 0.0
                if k == 0 and j > 0:
                    shift = -0.5 * (spacing - nick)  # toward the previous oligomer's last bead
                if k == oligo_nt - 1 and j < n_olig - 1:
                    shift = 0.5 * (spacing - nick)
                pos[first + k] = o + (spacing * tb - shift) * u + rise * v
                types[first + k] = COMPLEMENT[seq[tb]]
                bonds.append(np.array([[b0 + tb, first + k, HYB, HYB]]))
            kk = np.arange(oligo_nt - 1)
            bonds.append(np.stack([first + kk, first + kk + 1, np.full(oligo_nt - 1, BB3),
                                   np.full(oligo_nt - 1, BB5)], axis=1))
    return System(
        name=f"dna1-oligo-{N}", bead_offset=np.array([0, N], np.int64),
        box_q=np.array([int(np.rint(box * QSCALE))], np.int64), types=types,
        bonds=np.concatenate(bonds).astype(np.int32), rules=rules_dna1_paper(), pos0=pos, seed=seed,
        sigma_perturb=0.05,
        params=dict(default_params(seed), paircheck14=1, max_rounds=1, prob_mode=1),
        forcefield=forcefield_dna1_paper(),
    )


def forcefield_dna1_paper() -> Dict[str, np.ndarray]:
    """Bonded parameters of the paper's 1-bead DNA model (Sec. 3): harmonic
    angles E = K (theta - theta0)^2, type 1 (along the backbone) K = 20,
    theta0 = 180 degrees, type 2 (backbone - hybridization) K = 1, theta0 =
    90 degrees; dihedrals E = K (1 + d cos phi) with K = 1, d = -1 (cis) for
    types 1 and 2 and d = +1 (trans) for type 3.  The paper's bond wells are
    garbled as printed; bonds here are harmonic, K = 100, r0 = 0.6 sigma
    (the spacing of the oligomer geometry)."""
    ff = forcefield_dna2()
    for t in (HYB, BB3, BB5):
        ff["bond_k"][t], ff["bond_r0"][t] = 100.0, 0.6
    ff["angle_style"][1:3] = 1
    ff["angle_k"][1], ff["angle_theta0"][1] = 20.0, np.pi
    ff["angle_k"][2], ff["angle_theta0"][2] = 1.0, np.pi / 2
    for t, dd in ((1, -1), (2, -1), (3, 1)):
        ff["dihedral_k"][t], ff["dihedral_d"][t] = 1.0, dd
    return ff


def forcefield_dna2() -> Dict[str, np.ndarray]:
    """Bonded force-field tables (index = type): harmonic bonds E = K (r - r0)^2
    with K = 100, r0 = 1 for bond types 1..4; cosine angles E = K (1 + cos theta)
    with K = 2 for angle types 1, 2; dihedrals E = K (1 + d cos phi) with K = 1,
    d = +1 for dihedral types 1, 2 (the dihedral form of Sec. 3)."""
    ff = dict(
        bond_k=np.zeros(16), bond_r0=np.zeros(16), angle_k=np.zeros(16),
        dihedral_k=np.zeros(16), dihedral_d=np.zeros(16, dtype=np.int32),
        angle_theta0=np.zeros(16), angle_style=np.zeros(16, dtype=np.int32),
    )
    for t in (HYB, BB3, BB5, SUGAR):
        ff["bond_k"][t] = 100.0
        ff["bond_r0"][t] = 1.0
    for t in (1, 2):
        ff["angle_k"][t] = 2.0
        ff["dihedral_k"][t] = 1.0
        ff["dihedral_d"][t] = 1
    return ff


# --------------------------------------------------------------------------
# systems
# --------------------------------------------------------------------------

@dataclasses.dataclass
class System:
    """A batch of independent replicas sharing one rule list.

    bead_offset[r]..bead_offset[r+1] are the global bead indices of replica r;
    box_q[r] its periodic box edge in quantized units (positions lie in
    [0, box_q)).  bonds rows are (i, j, type stored by i, type stored by j)
    with global indices.  pos0 holds unwrapped float64 positions in sigma from
    which every snapshot is derived.
    """
    name: str
    bead_offset: np.ndarray
    box_q: np.ndarray
    types: np.ndarray
    bonds: np.ndarray
    rules: List[Dict]
    pos0: np.ndarray
    seed: int
    sigma_perturb: float = 0.05
    form_scale: Optional[np.ndarray] = None
    break_scale: Optional[np.ndarray] = None
    rng_stream: Optional[np.ndarray] = None
    params: Dict = dataclasses.field(default_factory=dict)
    forcefield: Dict = dataclasses.field(default_factory=forcefield_dna2)

    @property
    def n_beads(self) -> int:
        return int(self.bead_offset[-1])

    @property
    def n_replicas(self) -> int:
        return len(self.box_q)

    def box_sigma(self) -> np.ndarray:
        return self.box_q.astype(np.float64) / QSCALE

    def _rep_of_bead(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_replicas), np.diff(self.bead_offset))

    def float_positions(self, k: int) -> np.ndarray:
        """Unwrapped positions of snapshot k: pos0 plus k independent Gaussian
        kicks of width sigma_perturb per component (snapshot k does not depend
        on which other snapshots were generated)."""
        x = self.pos0.copy()
        for m in range(1, k + 1):
            rng = np.random.default_rng([self.seed, 7919, m])
            x += rng.normal(0.0, self.sigma_perturb, size=x.shape)
        return x

    def snapshot(self, k: int = 0) -> np.ndarray:
        """Quantized positions of snapshot k as int32 [N, 4] = (x, y, z, 0),
        each coordinate round-half-even(x * 2^20) reduced into [0, box_q)."""
        return quantize(self.float_positions(k), self.box_q, self._rep_of_bead())

    def snapshots(self, k0: int, k1: int) -> List[np.ndarray]:
        """Snapshots k0..k1-1, generated incrementally."""
        x = self.float_positions(k0)
        out = []
        rep = self._rep_of_bead()
        for k in range(k0, k1):
            if k > k0:
                rng = np.random.default_rng([self.seed, 7919, k])
                x += rng.normal(0.0, self.sigma_perturb, size=x.shape)
            out.append(quantize(x, self.box_q, rep))
        return out


def quantize(x: np.ndarray, box_q: np.ndarray, rep: np.ndarray) -> np.ndarray:
    q = np.rint(x * QSCALE).astype(np.int64)
    L = box_q[rep][:, None]
    q = np.mod(q, L)
    out = np.zeros((x.shape[0], 4), dtype=np.int32)
    out[:, :3] = q
    return out


def _unit_vectors(rng, n):
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def _strand_bonds(first_bead: int, n_nt: int) -> np.ndarray:
    """Backbone (2 toward the next nucleotide, 3 toward the previous one) and
    sugar bonds of one strand."""
    k = np.arange(n_nt)
    bb = first_bead + 2 * k
    base = bb + 1
    sugar = np.stack([bb, base, np.full(n_nt, SUGAR), np.full(n_nt, SUGAR)], axis=1)
    bbb = np.stack([bb[:-1], bb[1:], np.full(n_nt - 1, BB3), np.full(n_nt - 1, BB5)], axis=1)
    return np.concatenate([bbb, sugar]).astype(np.int32)


def _random_walk_strands(rng, n_strands, n_nt, box):
    """Backbone random walk with step 1.0 in uniform random directions from a
    uniform random start; each base 1.0 sigma from its backbone bead in a
    uniform random direction."""
    start = rng.uniform(0.0, box, size=(n_strands, 1, 3))
    steps = _unit_vectors(rng, n_strands * n_nt).reshape(n_strands, n_nt, 3)
    steps[:, 0, :] = 0.0
    bb = start + np.cumsum(steps, axis=1)
    base = bb + _unit_vectors(rng, n_strands * n_nt).reshape(n_strands, n_nt, 3)
    pos = np.empty((n_strands, n_nt, 2, 3))
    pos[:, :, 0] = bb
    pos[:, :, 1] = base
    return pos.reshape(-1, 3)


def _replica_strands(rng, n_strands, n_nt, box, first_bead, n_duplex=0):
    """Positions, types and bonds of n_strands strands; the first 2*n_duplex
    strands are laid out as anti-parallel ladders of complementary sequences:
    backbone spacing 1.0 along the ladder axis u, the two backbones 1.8 apart
    along v, each base 0.5 toward the partner strand and 0.3 off the ladder
    plane along w (so backbone-base-base-backbone is a U, not a straight line),
    partner bases 0.8 apart, with the hybridization bonds already present."""
    nb = 2 * n_nt
    N = n_strands * nb
    seq = rng.integers(1, 5, size=(n_strands, n_nt)).astype(np.int32)
    pos = _random_walk_strands(rng, n_strands, n_nt, box).reshape(n_strands, nb, 3)
    hyb = []
    for d in range(n_duplex):
        sa, sb = 2 * d, 2 * d + 1
        seq[sb] = COMPLEMENT[seq[sa][::-1]]
        o = rng.uniform(0.0, box, size=3)
        u = _unit_vectors(rng, 1)[0]
        w = _unit_vectors(rng, 1)[0]
        v = w - np.dot(w, u) * u
        v /= np.linalg.norm(v)
        w = np.cross(u, v)
        k = np.arange(n_nt)[:, None]
        pos[sa, 0::2] = o + k * u
        pos[sa, 1::2] = o + k * u + 0.5 * v + 0.3 * w
        kb = (n_nt - 1 - np.arange(n_nt))[:, None]  # strand B's nucleotide m sits at rung n_nt-1-m
        pos[sb, 0::2] = o + kb * u + 1.8 * v
        pos[sb, 1::2] = o + kb * u + 1.3 * v + 0.3 * w
        ia = first_bead + sa * nb + 2 * np.arange(n_nt) + 1
        ib = first_bead + sb * nb + 2 * (n_nt - 1 - np.arange(n_nt)) + 1
        hyb.append(np.stack([ia, ib, np.full(n_nt, HYB), np.full(n_nt, HYB)], axis=1))
    types = np.zeros((n_strands, nb), dtype=np.int32)
    types[:, 1::2] = seq
    bonds = [_strand_bonds(first_bead + s * nb, n_nt) for s in range(n_strands)]
    if hyb:
        bonds.append(np.concatenate(hyb))
    return pos.reshape(N, 3), types.reshape(N), np.concatenate(bonds).astype(np.int32)


def dna_system(name, n_strands, n_nt, density, seed, rules, n_duplex=0, box=None, params=None):
    N = n_strands * 2 * n_nt
    if box is None:
        box = (N / density) ** (1.0 / 3.0)
    rng = np.random.default_rng(seed)
    pos, types, bonds = _replica_strands(rng, n_strands, n_nt, box, 0, n_duplex)
    return System(
        name=name,
        bead_offset=np.array([0, N], dtype=np.int64),
        box_q=np.array([int(np.rint(box * QSCALE))], dtype=np.int64),
        types=types, bonds=bonds, rules=rules, pos0=pos, seed=seed,
        params=dict(default_params(seed), **(params or {})),
    )


def rules_dna2_ligation(p_form: float = 0.5, p_break: float = 0.05, p_lig: float = 0.5,
                        lig_dist: float = 1.1) -> List[Dict]:
    """The 2-bead rules plus directional ligation of backbone ends: two
    backbone beads within lig_dist join by a directional backbone bond
    (createdirbond, types 2 / 3) with probability p_lig.  A backbone bead
    holds at most one bond of type 2 and one of type 3 (maxbond per stored
    type), so only a strand's 3' end (which stores 3 toward its neighbour)
    and a 5' end (which stores 2) can ligate, and the maxbond test picks the
    orientation that continues the chain: the 3' end stores 2, the 5' end 3.
    The new bond's backbone angles and stacking dihedrals follow from the
    pattern table of rules_dna2."""
    rules = rules_dna2(p_form=p_form, p_break=p_break)
    head = rules[:5]
    rest = rules[5:]
    return head + [
        dict(kind="maxbond", bonds=bit(BB3), beads=bit(BB), max=1),
        dict(kind="maxbond", bonds=bit(BB5), beads=bit(BB), max=1),
        dict(kind="createdirbond", btype=BB3, btype2=BB5, beads=(bit(BB), bit(BB)), dist=lig_dist, prob=p_lig),
    ] + rest


def dna2_nicked_system(n_strands: int = 64, n_nt: int = 16, n_duplex: int = 16, nick_every: int = 4,
                       density: float = 0.5, seed: int = 7, p_lig: float = 0.5) -> "System":
    """Nicked duplexes in the 2-bead model: the first 2 n_duplex strands form
    complementary anti-parallel ladders (as in the melting workload), and the
    second strand of each ladder is cut into pieces of nick_every nucleotides
    by removing the backbone bonds between them; the ends at each nick sit
    1 sigma apart along the ladder, within reach of the ligation rule
    (rules_dna2_ligation).  The other strands are random walks."""
    N = n_strands * 2 * n_nt
    box = (N / density) ** (1.0 / 3.0)
    rng = np.random.default_rng([seed, 71])
    pos, types, bonds = _replica_strands(rng, n_strands, n_nt, box, 0, n_duplex)
    nb = 2 * n_nt
    cut = set()
    for dpx in range(n_duplex):
        first = (2 * dpx + 1) * nb
        for m in range(nick_every - 1, n_nt - 1, nick_every):
            cut.add((first + 2 * m, first + 2 * (m + 1)))
    keep = np.array([(int(b[0]), int(b[1])) not in cut for b in bonds])
    assert len(bonds) - keep.sum() == len(cut)
    return System(
        name=f"nicked-{N} ({n_duplex} duplexes nicked every {nick_every} nt)",
        bead_offset=np.array([0, N], dtype=np.int64),
        box_q=np.array([int(np.rint(box * QSCALE))], dtype=np.int64),
        types=types, bonds=bonds[keep], rules=rules_dna2_ligation(p_lig=p_lig), pos0=pos, seed=seed,
        params=default_params(seed),
    )


def default_params(seed):
    return dict(seed=int(seed) * 0x9E3779B97F4A7C15 % (1 << 64), paircheck13=0, paircheck14=0,
                max_rounds=0, prob_mode=0, reactive_mask=ALL_BEADS)


# --------------------------------------------------------------------------
# the five benchmark workloads
# --------------------------------------------------------------------------

def config1() -> System:
    """64 strands x 16 nt = 2048 beads, L = 20, seed 1, no initial pairs."""
    return dna_system("plain-2048 (64 strands x 16 nt, L=20)", 64, 16, None, 1, rules_dna2(), box=20.0)


def config2() -> System:
    """8192 strands x 64 nt = 1,048,576 beads at density 0.5 (L = 128), seed 2."""
    return dna_system("plain-1M (8192 strands x 64 nt, rho=0.5, L=128)", 8192, 64, 0.5, 2, rules_dna2())


def config4() -> System:
    """131072 strands x 64 nt = 16,777,216 beads at density 0.5; half of the
    strands pre-hybridized into 32768 complementary duplexes; break p = 0.5,
    form p = 0.9; at most one hybridization bond per base and two backbone
    bonds per backbone bead."""
    return dna_system("melt-16M (131072 strands x 64 nt, 50% duplexed, rho=0.5)", 131072, 64, 0.5, 4,
                      rules_dna2(p_form=0.9, p_break=0.5, backbone_maxbond=True), n_duplex=32768)


def scaled_config4(n_strands: int, seed: int = 4) -> System:
    """The melting workload at a smaller size (same density and duplex fraction)."""
    return dna_system(f"melt-{n_strands * 128} ({n_strands} strands x 64 nt, 50% duplexed, rho=0.5)",
                      n_strands, 64, 0.5, seed, rules_dna2(p_form=0.9, p_break=0.5, backbone_maxbond=True),
                      n_duplex=n_strands // 4)


def config5() -> System:
    """32768 strands x 64 nt = 4,194,304 beads at density 0.5 (L = 203.2),
    seed 5: the end-to-end DPD loop."""
    return dna_system("dpd-4M (32768 strands x 64 nt, rho=0.5)", 32768, 64, 0.5, 5, rules_dna2())


def initial_velocities(n_beads: int, kT: float = 1.0, mass: float = 1.0, seed: int = 5) -> np.ndarray:
    """Maxwell-Boltzmann velocities float32 [N, 4] (w = 0), zero total momentum."""
    rng = np.random.default_rng([seed, 31337])
    v = rng.normal(0.0, math.sqrt(kT / mass), size=(n_beads, 3))
    v -= v.mean(axis=0)
    out = np.zeros((n_beads, 4), np.float32)
    out[:, :3] = v
    return out


def ladder_sizes(n_replicas=512, seed=3, lo=2048, hi=65536, median=8192, sigma=0.693):
    rng = np.random.default_rng([seed, 1])
    z = rng.normal(size=n_replicas)
    n = 32 * np.rint(np.exp(math.log(median) + sigma * z) / 32.0)
    return np.clip(n, lo, hi).astype(np.int64)


def config3(n_replicas: int = 512, seed: int = 3) -> System:
    """Temperature ladder of uneven replicas: bead counts log-normal (median
    8192, clipped to [2048, 65536], multiples of 32), strands of 16 nt at
    density 0.5, T_k = 0.8 + 0.4 k / (R - 1).  Formation probabilities are
    scaled by exp(2 (1/T - 1)) and breakage by exp(-2 (1/T - 1)), each capped
    at 1 by the consumer."""
    sizes = ladder_sizes(n_replicas, seed)
    rng = np.random.default_rng(seed)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pos, types, bonds, box_q = [], [], [], []
    for r, n in enumerate(sizes):
        box = (n / 0.5) ** (1.0 / 3.0)
        p, t, b = _replica_strands(rng, int(n) // 32, 16, box, int(offs[r]))
        pos.append(p)
        types.append(t)
        bonds.append(b)
        box_q.append(int(np.rint(box * QSCALE)))
    Tk = 0.8 + 0.4 * np.arange(n_replicas) / max(1, n_replicas - 1)
    return System(
        name=f"ladder-{n_replicas} (log-normal 2k-64k beads, T 0.8-1.2)",
        bead_offset=offs, box_q=np.array(box_q, dtype=np.int64),
        types=np.concatenate(types), bonds=np.concatenate(bonds), rules=rules_dna2(),
        pos0=np.concatenate(pos), seed=seed,
        form_scale=np.exp(2.0 * (1.0 / Tk - 1.0)), break_scale=np.exp(-2.0 * (1.0 / Tk - 1.0)),
        rng_stream=np.arange(n_replicas, dtype=np.uint32),
        params=default_params(seed),
    )


def replica_batch(n_replicas: int, n_strands: int = 2, n_nt: int = 8, n_duplex: int = 1, density: float = 0.5,
                  seed: int = 9) -> System:
    """n_replicas equal replicas of n_strands strands of n_nt nucleotides at
    the given bead density, the first 2 n_duplex strands of each paired into
    hybridized duplexes; the 2-bead DNA rules.  Many tiny replicas exercise
    per-replica bookkeeping at its limits."""
    rng = np.random.default_rng(seed)
    n = 2 * n_nt * n_strands
    box = (n / density) ** (1.0 / 3.0)
    pos, types, bonds = [], [], []
    for r in range(n_replicas):
        p, t, b = _replica_strands(rng, n_strands, n_nt, box, r * n, n_duplex=n_duplex)
        pos.append(p)
        types.append(t)
        bonds.append(b)
    return System(
        name=f"batch-{n_replicas}x{n}", bead_offset=np.arange(n_replicas + 1, dtype=np.int64) * n,
        box_q=np.full(n_replicas, int(np.rint(box * QSCALE)), np.int64), types=np.concatenate(types),
        bonds=np.concatenate(bonds), rules=rules_dna2(), pos0=np.concatenate(pos), seed=seed,
        rng_stream=np.arange(n_replicas, dtype=np.uint32), params=default_params(seed),
    )


def sub_replicas(sysb: System, idx) -> System:
    """The replicas idx of a batched system as a batch of their own (same
    per-replica RNG streams and probability scales)."""
    idx = list(idx)
    offs = sysb.bead_offset
    parts = [np.arange(offs[r], offs[r + 1]) for r in idx]
    sel = np.concatenate(parts)
    new_off = np.concatenate([[0], np.cumsum([len(p) for p in parts])]).astype(np.int64)
    remap = -np.ones(sysb.n_beads, dtype=np.int64)
    remap[sel] = np.arange(len(sel))
    b = sysb.bonds
    keep = (remap[b[:, 0]] >= 0)
    nb = b[keep].copy()
    nb[:, 0] = remap[nb[:, 0]]
    nb[:, 1] = remap[nb[:, 1]]
    pick = lambda a: None if a is None else np.asarray(a)[idx]
    out = dataclasses.replace(
        sysb, name=f"{sysb.name}[{len(idx)} replicas]", bead_offset=new_off, box_q=sysb.box_q[idx],
        types=sysb.types[sel], bonds=nb.astype(np.int32), pos0=sysb.pos0[sel],
        form_scale=pick(sysb.form_scale), break_scale=pick(sysb.break_scale),
        rng_stream=pick(sysb.rng_stream) if sysb.rng_stream is not None else np.asarray(idx, dtype=np.uint32),
    )
    out._sel = sel  # global indices of the parent, for perturbation parity
    return out


# --------------------------------------------------------------------------
# small systems for tests
# --------------------------------------------------------------------------

def random_small_system(seed: int, n_beads: int = 64, box: float = 4.0, n_bonds: int = 40,
                        n_types: int = 5, n_bond_types: int = 4, rules: Optional[List[Dict]] = None,
                        n_replicas: int = 1, params=None) -> System:
    """Dense random systems of a few dozen beads with random (possibly
    directional) bonds, at most 4 per bead, for brute-force property tests."""
    rng = np.random.default_rng(seed)
    pos, types, bonds, offs, boxq = [], [], [], [0], []
    for r in range(n_replicas):
        p = rng.uniform(0.0, box, size=(n_beads, 3))
        t = rng.integers(0, n_types, size=n_beads).astype(np.int32)
        deg = np.zeros(n_beads, dtype=np.int64)
        seen = set()
        bl = []
        tries = 0
        while len(bl) < n_bonds and tries < 50 * n_bonds:
            tries += 1
            i, j = rng.integers(0, n_beads, size=2)
            if i == j or (min(i, j), max(i, j)) in seen or deg[i] >= 4 or deg[j] >= 4:
                continue
            seen.add((min(i, j), max(i, j)))
            deg[i] += 1
            deg[j] += 1
            if rng.random() < 0.7:
                tt = int(rng.integers(1, n_bond_types + 1))
                bl.append((i + offs[-1], j + offs[-1], tt, tt))
            else:
                bl.append((i + offs[-1], j + offs[-1], int(rng.integers(1, n_bond_types + 1)),
                           int(rng.integers(1, n_bond_types + 1))))
        pos.append(p)
        types.append(t)
        bonds.extend(bl)
        offs.append(offs[-1] + n_beads)
        boxq.append(int(np.rint(box * QSCALE)))
    R = n_replicas
    return System(
        name=f"random-small-{seed}", bead_offset=np.array(offs, dtype=np.int64),
        box_q=np.array(boxq, dtype=np.int64), types=np.concatenate(types),
        bonds=np.array(bonds, dtype=np.int32).reshape(-1, 4), rules=rules if rules is not None else [],
        pos0=np.concatenate(pos), seed=seed, sigma_perturb=0.1,
        form_scale=np.ones(R), break_scale=np.ones(R), rng_stream=np.arange(R, dtype=np.uint32),
        params=dict(default_params(seed), **(params or {})),
    )


def random_rules(seed: int, n_types: int = 5, n_bond_types: int = 4) -> List[Dict]:
    """A random but well-formed rule list mixing every rule kind of Fig. 1."""
    rng = np.random.default_rng([seed, 99])

    def mask(nt, lo=0, p=0.5):
        m = 0
        while m == 0:
            for t in range(lo, lo + nt):
                if rng.random() < p:
                    m |= 1 << t
        return m

    bt = lambda: int(rng.integers(1, n_bond_types + 1))
    rules = []
    for _ in range(int(rng.integers(1, 4))):
        if rng.random() < 0.6:
            rules.append(dict(kind="createbond", btype=bt(), beads=(mask(n_types), mask(n_types)),
                              dist=float(rng.uniform(0.5, 1.6)), prob=float(rng.choice([0.0, 0.3, 0.7, 1.0]))))
        else:
            rules.append(dict(kind="createdirbond", btype=bt(), btype2=bt(), beads=(mask(n_types), mask(n_types)),
                              dist=float(rng.uniform(0.5, 1.6)), prob=float(rng.choice([0.3, 0.7, 1.0]))))
    for _ in range(int(rng.integers(0, 3))):
        rules.append(dict(kind="breakbond", btype=bt(), dist=float(rng.uniform(0.0, 2.5)),
                          prob=float(rng.choice([0.2, 0.6, 1.0]))))
    if rng.random() < 0.5:
        rules.append(dict(kind="convertbond", btype=bt(), btype2=bt(), prob=float(rng.choice([0.3, 1.0]))))
    if rng.random() < 0.6:
        rules.append(dict(kind="killbond", btype=bt(), dist=float(rng.uniform(1.0, 3.0))))
    for _ in range(int(rng.integers(0, 3))):
        rules.append(dict(kind="maxbond", bonds=mask(n_bond_types, 1), beads=mask(n_types),
                          max=int(rng.integers(1, 4))))
    for k in range(int(rng.integers(1, 4))):
        rules.append(dict(kind="createangle", type=k + 1, beads=(mask(n_types, p=0.7), mask(n_types, p=0.7),
                                                               mask(n_types, p=0.7)),
                          bonds=(mask(n_bond_types, 1, 0.7), mask(n_bond_types, 1, 0.7))))
    for k in range(int(rng.integers(1, 4))):
        rules.append(dict(kind="createdihedral", type=k + 1,
                          beads=tuple(mask(n_types, p=0.7) for _ in range(4)),
                          bonds=tuple(mask(n_bond_types, 1, 0.7) for _ in range(3))))
    rng.shuffle(rules)
    return rules
