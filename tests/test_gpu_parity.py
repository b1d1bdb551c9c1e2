"""GPU parity: the CUDA path through the C ABI against the CPU oracle (the
bar is stated in tests/parity.py: topology and statistics bit for bit,
forces within 1e-5 max(|f_ref|, f_rms) per component, energy / virial within
2e-6 of the largest magnitude per replica)."""

import ctypes
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_4214_gb300 import workloads as W

from helpers import golden, golden_rules, half_bond_pair, ladder_1bead_positions, make_system
from parity import compare_forces, compare_topology, dynbond, run_parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


# ---------------------------------------------------------------------------

def test_philox_oracle_matches_curand():
    """Pins the oracle's Philox4x32-10 bit for bit against cuRAND's
    Philox4_32_10: curand_init(seed, subsequence, 4m) then curand4() k times
    draws Philox on the counter (m + k as 64 bits, subsequence as 64 bits)
    with key = seed."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "native", "libcurand_philox.so")
    if not os.path.exists(path):
        import __graft_entry__
        __graft_entry__._build_test_helper()
    L = ctypes.CDLL(path)
    L.curand_philox_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
    rng = np.random.default_rng(1)
    for _ in range(12):
        seed = int(rng.integers(0, 2**63)) * 2 + 1
        sub = int(rng.integers(0, 2**62))
        m = int(rng.integers(0, 2**40))
        n = 6
        out = np.zeros((n, 4), np.uint32)
        assert L.curand_philox_draw(seed, sub, 4 * m, n, out.ctypes.data) == 0
        for k in range(n):
            c = m + k
            want = O.philox([c & 0xFFFFFFFF, c >> 32, sub & 0xFFFFFFFF, sub >> 32],
                            [seed & 0xFFFFFFFF, seed >> 32])
            assert np.array_equal(out[k], want), (seed, sub, m, k)


def test_initial_typing_of_the_papers_dna_ladder():
    g = golden("dna1bead_ladder_4mer.json")
    s = make_system(g["types"], g["bonds"], ladder_1bead_positions(), 20.0, golden_rules(g["rules_fig2_9_to_14"]))
    ctx = dynbond().Context(s)
    _, a, d = ctx.topology()
    assert a.tolist() == sorted(g["expected_angles"])
    assert d.tolist() == sorted(g["expected_dihedrals"])


@pytest.mark.parametrize("cell_scale,cell_zdiv", [(0, 0), (1, 1), (2, 1), (3, 1), (1, 4), (2, 2), (2, 4), (3, 7)])
def test_plain_2048_beads_ten_calls(cell_scale, cell_zdiv):
    """Ten calls on 2048 beads, autotuned (0) and with fixed cell edges of 1,
    2 and 3 x the creation reach along x and y (2 and 3: only the octant of
    columns on the side of the column half each bead sits in is searched)
    and 1 to 7 cells per edge along z (the cells overlapping the reach
    interval are searched)."""
    s = W.config1()
    _, worst = run_parity(s, 10, params=dict(cell_scale=cell_scale, cell_zdiv=cell_zdiv))
    print("max force / ev error", max(w[0] for w in worst), max(w[1] for w in worst))


@pytest.mark.parametrize("seed", range(40))
def test_random_systems_all_rule_kinds(seed):
    rules = W.random_rules(seed)
    s = W.random_small_system(seed, n_beads=60, box=3.0 + seed % 3, n_bonds=50, rules=rules,
                              n_replicas=1 + seed % 3,
                              params=dict(paircheck13=seed % 2, paircheck14=(seed // 2) % 2, max_rounds=seed % 3,
                                          prob_mode=(seed // 3) % 2))
    # seeds from 20 on: fixed cell geometries, 1 or 2 reaches along x / y, 1 to 5 cells per edge along z
    geo = dict(cell_scale=1 + (seed % 3 == 0), cell_zdiv=1 + seed % 5) if seed >= 20 else None
    run_parity(s, 4, params=geo)


def test_paper_exact_mode_oligomers_on_templates():
    """The paper's own 1-bead DNA rule list (Fig. 2) in the paper's own
    semantics -- paircheck14, one nomination per call, the two-uniform trial
    average -- on oligomers hybridized to templates: ligations across the
    nicks (createdirbond), kills of stretched hybridization bonds and the
    typing rules 9-14, bit-exact against the oracle for 12 calls."""
    s = W.dna1_oligo_system()
    o, worst = run_parity(s, 12)
    bonds = o.topology()[0]
    ligated = int(((bonds[:, 2] == W.BB3) & (bonds[:, 3] == W.BB5)).sum()) - 64 * (16 - 1) - 64 * 4 * 3
    assert ligated > 0, "no ligation happened"
    print("ligated", ligated, "max force / ev error", max(w[0] for w in worst), max(w[1] for w in worst))


def test_nicked_duplexes_ligate_like_the_oracle():
    """Directional ligation of backbone ends in the 2-bead model: bit-exact
    topology and statistics against the oracle while the nicks close."""
    s = W.dna2_nicked_system()
    o, _ = run_parity(s, 8)
    bonds = o.topology()[0]
    backbone = int(np.isin(bonds[:, 2], (W.BB3, W.BB5)).sum())
    assert backbone > int(np.isin(s.bonds[:, 2], (W.BB3, W.BB5)).sum()), "no nick closed"


def test_nicked_duplexes_16k_beads():
    s = W.dna2_nicked_system(n_strands=512, n_duplex=128, nick_every=8, seed=8)
    run_parity(s, 4)


def test_half_bonds_net_force_matches_the_oracle():
    """Unequal potentials on the two ends of a directional bond: the GPU's
    per-end forces (and their nonzero sum) match the oracle's closed form."""
    s = half_bond_pair()
    o = O.Oracle(s)
    ctx = dynbond().Context(s)
    snap = s.snapshot(0)
    compare_forces(ctx, o, snap, "half bonds")
    f, _ = ctx.forces(torch.from_numpy(snap).cuda())
    f = f.cpu().numpy()
    assert abs(float(f[0, 0] + f[1, 0])) > 50.0


def test_unknown_angle_style_is_rejected():
    s = W.config1()
    s.forcefield = W.forcefield_dna1_paper()
    s.forcefield["angle_style"][3] = 2
    with pytest.raises(dynbond().DynbondError) as e:
        dynbond().Context(s)
    assert e.value.status == 1 and "angle_style" in str(e.value)


def test_degenerate_systems_without_candidates_or_interactions():
    """Nothing to bin or record: beads whose types no creation rule pairs
    (empty cell lists, no candidates, no bonds, no angle or dihedral tiles in
    the force launches: zero forces and energies), and one bond without typing
    rules (bond forces only)."""
    rules = [dict(kind="createbond", btype=1, beads=(W.bit(1), W.bit(2)), dist=1.1, prob=1.0)]
    s = make_system([3, 3, 4, 4], [], [[1, 1, 1], [1.5, 1, 1], [1, 1.5, 1], [1.2, 1.2, 1.2]], 10.0, rules)
    o, _ = run_parity(s, 2, forces=False)
    f, ev = dynbond().Context(s).forces(torch.from_numpy(s.snapshot(0)).cuda())
    assert not f.any() and not ev.any()
    s2 = make_system([1, 2], [[0, 1, 1, 1]], [[1, 1, 1], [2.2, 1, 1]], 10.0, rules)
    o2, _ = run_parity(s2, 2)
    assert len(o2.topology()[1]) == 0 and len(o2.topology()[2]) == 0


def test_rounds_matching_and_single_nomination():
    pos2 = [[2.0, 2, 2], [2.0, 3.0, 2], [2.5, 2, 2], [2.95, 2.6, 2]]
    rules = [dict(kind="createbond", btype=1, beads=(W.bit(1), W.bit(2)), dist=1.1, prob=1.0),
             dict(kind="maxbond", bonds=W.bit(1), beads=W.bit(1, 2, 3, 4), max=1)]
    for mr, want in ((0, 2), (1, 1)):
        s = make_system([1, 2, 2, 1], [], pos2, 10.0, rules, params=dict(max_rounds=mr))
        o, _ = run_parity(s, 1)
        assert o.counts()[0] == want


def test_duplex_melts_and_reforms():
    rules = W.rules_dna2(p_form=1.0, p_break=1.0)
    rng = np.random.default_rng(3)
    pos, types, bonds = W._replica_strands(rng, 2, 12, 30.0, 0, n_duplex=1)
    s = W.System(name="duplex", bead_offset=np.array([0, 48]), box_q=np.array([30 * W.QSCALE]), types=types,
                 bonds=bonds, rules=rules, pos0=pos, seed=5, sigma_perturb=0.0, params=W.default_params(5))
    snap = s.snapshot(0)
    run_parity(s, 2, snaps=[snap, snap])


@pytest.mark.parametrize("cell_scale,cell_zdiv", [(0, 0), (2, 1), (2, 4)])
def test_plain_1m_beads_parity(cell_scale, cell_zdiv):
    s = W.config2()
    snaps = s.snapshots(0, 3)
    _, worst = run_parity(s, 3, snaps=snaps, params=dict(cell_scale=cell_scale, cell_zdiv=cell_zdiv))
    print("1M: max force / ev error", worst)


def test_melting_1m_beads_parity():
    s = W.scaled_config4(8192)
    snaps = s.snapshots(0, 3)
    run_parity(s, 3, snaps=snaps)


def test_batched_ladder_parity_and_replica_independence():
    full = W.config3(n_replicas=48)
    snaps = full.snapshots(0, 3)
    run_parity(full, 3, snaps=snaps)
    # the same replicas run alone (same streams and scales) reach the same bonds
    idx = [3, 17, 40]
    sub = W.sub_replicas(full, idx)
    ctx_b = dynbond().Context(full)
    ctx_s = dynbond().Context(sub)
    for k in range(3):
        ctx_b.step(torch.from_numpy(snaps[k]).cuda(), k)
        ctx_s.step(torch.from_numpy(snaps[k][sub._sel]).cuda(), k)
    bb, _, _ = ctx_b.topology()
    bs, _, _ = ctx_s.topology()
    inv = np.zeros(full.n_beads, np.int64) - 1
    inv[sub._sel] = np.arange(len(sub._sel))
    keep = inv[bb[:, 0]] >= 0
    mapped = bb[keep].copy()
    mapped[:, 0] = inv[mapped[:, 0]]
    mapped[:, 1] = inv[mapped[:, 1]]
    assert np.array_equal(mapped[np.lexsort(mapped.T[::-1])], bs)


@pytest.mark.slow
def test_batched_ladder_512_replicas_full_size():
    """The whole 512-replica temperature ladder (5,266,816 beads, uneven
    replicas of 2k-64k beads, per-replica probability scales and streams):
    statistics and topology of every replica bit for bit against the oracle
    for three calls, forces within the parity bar."""
    full = W.config3()
    snaps = full.snapshots(0, 3)
    _, worst = run_parity(full, 3, snaps=snaps)
    print("ladder-512: max force / ev error", max(w[0] for w in worst), max(w[1] for w in worst))


@pytest.mark.parametrize("flags", ["NO_GRAPH", "NO_PDL", "NO_GRAPH|NO_PDL"])
def test_graph_and_direct_launches_agree(flags):
    s = W.config1()
    D = dynbond()
    f = 0
    for name in flags.split("|"):
        f |= getattr(D, "FLAG_" + name)
    a = D.Context(s)
    b = D.Context(s, flags=f)
    for k in range(3):
        p = torch.from_numpy(s.snapshot(k)).cuda()
        assert np.array_equal(a.step(p, k, stats=True), b.step(p, k, stats=True))
    for x, y in zip(a.topology(), b.topology()):
        assert np.array_equal(x, y)


def test_dependent_launch_overlap_changes_nothing_at_scale():
    """Programmatic dependent launch lets each kernel's blocks be scheduled
    while its predecessor drains; on the 1M-bead system (multi-wave grids,
    look-back chains, the cooperative matching) every call must give the
    same topology, statistics and forces as strictly serialized launches."""
    s = W.config2()
    D = dynbond()
    a = D.Context(s, params=dict(cell_scale=1.0))
    b = D.Context(s, params=dict(cell_scale=1.0), flags=D.FLAG_NO_PDL)
    for k in range(4):
        p = torch.from_numpy(s.snapshot(k)).cuda()
        assert np.array_equal(a.step(p, k, stats=True), b.step(p, k, stats=True))
        fa, eva = a.forces(p)
        fb, evb = b.forces(p)
        torch.testing.assert_close(fa, fb, rtol=1e-5, atol=1e-4)
        # record order and atomic order differ between runs: energy and
        # virial agree to the reduction's rounding, not bit for bit
        ea, eb = eva.cpu().numpy(), evb.cpu().numpy()
        assert np.abs(ea - eb).max() <= 1e-9 * np.abs(ea).max()
    for x, y in zip(a.topology(), b.topology()):
        assert np.array_equal(x, y)


# dynbond_step_forces: the step with the bond forces on a graph branch beside
# the angle / dihedral maintenance, then the angle / dihedral forces
@pytest.mark.parametrize("cell_scale,cell_zdiv", [(0, 0), (2, 1), (1, 4)])
def test_combined_call_plain_2048(cell_scale, cell_zdiv):
    run_parity(W.config1(), 10, params=dict(cell_scale=cell_scale, cell_zdiv=cell_zdiv), combined=True)


@pytest.mark.parametrize("seed", [2, 7, 11, 19, 26, 33])
def test_combined_call_random_systems(seed):
    rules = W.random_rules(seed)
    s = W.random_small_system(seed, n_beads=60, box=3.0 + seed % 3, n_bonds=50, rules=rules,
                              n_replicas=1 + seed % 3,
                              params=dict(paircheck13=seed % 2, paircheck14=(seed // 2) % 2, max_rounds=seed % 3,
                                          prob_mode=(seed // 3) % 2))
    run_parity(s, 4, combined=True)


def test_combined_call_batches_and_1m():
    ladder = W.config3(n_replicas=48)
    run_parity(ladder, 3, snaps=ladder.snapshots(0, 3), combined=True)
    s = W.config2()
    _, worst = run_parity(s, 3, snaps=s.snapshots(0, 3), combined=True)
    print("1M combined: max force / ev error", worst)


@pytest.mark.parametrize("flag", ["PERSISTENT", "PROFILE", "NO_PDL"])
def test_combined_call_under_context_flags(flag):
    """Contexts that run each step as one persistent launch or record phase
    events take the two calls in turn inside dynbond_step_forces; without
    dependent launch the combined graph is kept.  All match the oracle."""
    run_parity(W.config1(), 4, flags=getattr(dynbond(), "FLAG_" + flag), combined=True)


def test_combined_call_equals_the_two_calls():
    """The combined call against dynbond_step then dynbond_forces on a second
    context: identical statistics and topology, forces and energy / virial to
    the rounding of the partial sums' order; the direct-launch form too."""
    s = W.config2()
    D = dynbond()
    a = D.Context(s, params=dict(cell_scale=2, cell_zdiv=2))
    b = D.Context(s, params=dict(cell_scale=2, cell_zdiv=2))
    c = D.Context(s, params=dict(cell_scale=2, cell_zdiv=2), flags=D.FLAG_NO_GRAPH)
    for k in range(3):
        p = torch.from_numpy(s.snapshot(k)).cuda()
        fa, eva, sta = a.step_forces(p, k, stats=True)
        stb = b.step(p, k, stats=True)
        fb, evb = b.forces(p)
        fc, evc, stc = c.step_forces(p, k, stats=True)
        assert np.array_equal(sta, stb) and np.array_equal(sta, stc)
        for f in (fb, fc):
            torch.testing.assert_close(fa, f, rtol=1e-5, atol=1e-4)
        for ev in (evb, evc):
            ea, eb = eva.cpu().numpy(), ev.cpu().numpy()
            assert np.abs(ea - eb).max() <= 1e-9 * np.abs(ea).max()
    for x, y, z in zip(a.topology(), b.topology(), c.topology()):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_host_buffer_entry_point_matches_device_path():
    s = W.config1()
    D = dynbond()
    a, b = D.Context(s), D.Context(s)
    for k in range(2):
        snap = s.snapshot(k)
        f_h, ev_h, st_h = a.run_host(snap, k, stats=True)
        p = torch.from_numpy(snap).cuda()
        st_d = b.step(p, k, stats=True)
        f_d, ev_d = b.forces(p)
        assert np.array_equal(st_h, st_d)
        assert np.allclose(f_h, f_d.cpu().numpy(), rtol=1e-5, atol=1e-4)
        # the two contexts hold their records in different (unordered) list
        # positions, so the FP32 partial sums group differently
        ev_d = ev_d.cpu().numpy()
        assert np.abs(ev_h - ev_d).max() <= 1e-7 * np.abs(ev_d).max()


def test_misaligned_buffers_are_rejected_before_any_launch():
    """int4 / float4 per bead: a device pointer off a 16-byte boundary is an
    argument error (nothing is launched, the context stays usable)."""
    s = W.config1()
    D = dynbond()
    ctx = D.Context(s, flags=D.FLAG_NO_AUTOTUNE)
    p = torch.from_numpy(s.snapshot(0)).cuda()
    n = p.numel()
    buf = torch.zeros(n + 4, dtype=torch.int32, device=p.device)
    buf[1:1 + n] = p.reshape(-1)
    bad = buf[1:1 + n].view(-1, 4)
    assert bad.data_ptr() % 16 == 4
    with pytest.raises(D.DynbondError) as e:
        ctx.step(bad, 0, stats=True)
    assert e.value.status == 1 and "aligned" in str(e.value)
    fbuf = torch.zeros(4 * s.n_beads + 4, dtype=torch.float32, device=p.device)
    ev = torch.zeros((s.n_replicas, 7), dtype=torch.float64, device=p.device)
    with pytest.raises(D.DynbondError) as e:
        ctx.forces(p, fbuf[1:1 + 4 * s.n_beads].view(-1, 4), ev)
    assert e.value.status == 1
    st = ctx.step(p, 0, stats=True)
    o = O.Oracle(s)
    assert np.array_equal(st, o.step(s.snapshot(0), 0))


def test_position_outside_box_is_reported_and_sticks():
    s = W.config1()
    D = dynbond()
    ctx = D.Context(s)
    snap = s.snapshot(0)
    snap[5, 1] = int(s.box_q[0])  # one past the edge
    with pytest.raises(D.DynbondError) as e:
        ctx.step(torch.from_numpy(snap).cuda(), 0, stats=True)
    assert e.value.status == 1
    with pytest.raises(D.DynbondError):
        ctx.step(torch.from_numpy(s.snapshot(0)).cuda(), 0)


def test_resume_from_exported_topology_reproduces_the_run():
    s = W.config1()
    D = dynbond()
    a = D.Context(s)
    snaps = s.snapshots(0, 6)
    for k in range(3):
        a.step(torch.from_numpy(snaps[k]).cuda(), k)
    bonds, _, _ = a.topology()
    import dataclasses
    s2 = dataclasses.replace(s, bonds=bonds)
    b = D.Context(s2)
    for x, y in zip(a.topology(), b.topology()):
        assert np.array_equal(x, y)
    for k in range(3, 6):
        p = torch.from_numpy(snaps[k]).cuda()
        assert np.array_equal(a.step(p, k, stats=True)[:, :12], b.step(p, k, stats=True)[:, :12])
    for x, y in zip(a.topology(), b.topology()):
        assert np.array_equal(x, y)


@pytest.mark.slow
def test_melting_16m_beads_full_size_two_calls():
    s = W.config4()
    snaps = s.snapshots(0, 2)
    run_parity(s, 2, snaps=snaps, forces=True)


def test_autotuned_and_fixed_geometries_give_identical_results():
    s = W.config1()
    D = dynbond()
    ctxs = [D.Context(s), D.Context(s, flags=D.FLAG_NO_AUTOTUNE), D.Context(s, params=dict(cell_scale=3))]
    for k in range(4):
        p = torch.from_numpy(s.snapshot(k)).cuda()
        sts = [c.step(p, k, stats=True) for c in ctxs]
        assert all(np.array_equal(sts[0], x) for x in sts[1:])
    tops = [c.topology() for c in ctxs]
    for t in tops[1:]:
        for x, y in zip(tops[0], t):
            assert np.array_equal(x, y)
    info = ctxs[0].autotune(torch.from_numpy(s.snapshot(4)).cuda())
    assert info["tuned"] == 1 and info["cell_scale"] in (1.0, 1.25, 1.5, 2.0, 3.0) and info["cell_zdiv"] in (1, 2, 4)
    assert ctxs[0].tuning() == info
    # a fixed geometry is reported as created: 2 x 2 columns of 2 reaches (L = 20 sigma: 7 per axis), 2 z cells per edge
    fixed = D.Context(s, params=dict(cell_scale=2, cell_zdiv=2)).tuning()
    assert fixed["tuned"] == 0 and fixed["cell_scale"] == 2.0 and fixed["cell_zdiv"] == 2 and fixed["octant"] == 1
    assert ctxs[2].tuning()["octant"] == 1 and ctxs[1].tuning()["octant"] == 0


def test_bounded_wait_gives_up_with_a_status_and_leaves_the_device_usable():
    """With every device-side wait limited to one poll, some wait (a look-back
    or the matching's grid barrier) gives up; the kernel records ETIMEOUT,
    every later kernel of the call returns at once, the host reports the
    status, and the CUDA context stays usable for new work."""
    D = dynbond()
    s = W.config2()
    pos = torch.from_numpy(s.snapshot(0)).cuda()
    status = None
    try:
        ctx = D.Context(s, params=dict(spin_limit=1), flags=D.FLAG_NO_AUTOTUNE)
        ctx.step(pos, 0, stats=True)
    except D.DynbondError as e:
        status = e.status
    assert status == 5
    if "ctx" in locals():
        with pytest.raises(D.DynbondError):
            ctx.step(pos, 1)
    assert torch.ones(1000, device="cuda").sum().item() == 1000.0
    s1 = W.config1()
    ok = D.Context(s1)
    st = ok.step(torch.from_numpy(s1.snapshot(0)).cuda(), 0, stats=True)
    assert st[0, 12] > 0


@pytest.mark.parametrize("cell_scale,cell_zdiv", [(1, 1), (2, 1), (2, 2), (1, 4), (3, 1), (2, 4)])
def test_staged_and_global_candidate_search_agree(cell_scale, cell_zdiv):
    """The candidate search over tiles of cell columns staged in shared memory
    and the per-bead search in global memory give identical statistics and
    topology (here on the 16M-bead melting recipe scaled to 1M beads: dense
    turnover, duplexes and free strands), at several cell geometries."""
    s = W.scaled_config4(8192)
    D = dynbond()
    geo = dict(cell_scale=cell_scale, cell_zdiv=cell_zdiv)
    a = D.Context(s, params=geo, flags=D.FLAG_STAGED_SEARCH)
    b = D.Context(s, params=geo, flags=D.FLAG_GLOBAL_SEARCH)
    assert a.tuning()["tiles"] == 1 and b.tuning()["tiles"] == 0
    for k in range(3):
        p = torch.from_numpy(s.snapshot(k)).cuda()
        assert np.array_equal(a.step(p, k, stats=True), b.step(p, k, stats=True)), k
    for x, y in zip(a.topology(), b.topology()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("cell_scale,cell_zdiv", [(0, 0), (1, 1), (2, 1), (1, 4)])
def test_persistent_call_matches_the_oracle(cell_scale, cell_zdiv):
    """The whole call as one persistent cooperative launch (phases separated
    by bounded grid barriers): bit-exact against the oracle on plain-2048."""
    D = dynbond()
    run_parity(W.config1(), 6, params=dict(cell_scale=cell_scale, cell_zdiv=cell_zdiv), flags=D.FLAG_PERSISTENT)


@pytest.mark.parametrize("seed", [1, 5, 8, 13, 22, 27, 31, 38])
def test_persistent_call_on_random_systems(seed):
    D = dynbond()
    rules = W.random_rules(seed)
    s = W.random_small_system(seed, n_beads=60, box=3.0 + seed % 3, n_bonds=50, rules=rules,
                              n_replicas=1 + seed % 3,
                              params=dict(paircheck13=seed % 2, paircheck14=(seed // 2) % 2, max_rounds=seed % 3,
                                          prob_mode=(seed // 3) % 2))
    run_parity(s, 4, flags=D.FLAG_PERSISTENT)


def test_persistent_call_on_batches_and_at_1m():
    """Persistent launches on 48 uneven replicas against the oracle, and on
    the 1M-bead system against the graph of one kernel per phase."""
    D = dynbond()
    full = W.config3(n_replicas=48)
    run_parity(full, 3, snaps=full.snapshots(0, 3), flags=D.FLAG_PERSISTENT)
    s = W.config2()
    a = D.Context(s, params=dict(cell_scale=2))
    b = D.Context(s, params=dict(cell_scale=2), flags=D.FLAG_PERSISTENT)
    for k in range(3):
        p = torch.from_numpy(s.snapshot(k)).cuda()
        assert np.array_equal(a.step(p, k, stats=True), b.step(p, k, stats=True)), k
    for x, y in zip(a.topology(), b.topology()):
        assert np.array_equal(x, y)


def test_persistent_call_bounded_barrier_gives_up_cleanly():
    """With every wait limited to one poll the persistent call's first grid
    barrier gives up: ETIMEOUT is reported and the CUDA context stays usable."""
    D = dynbond()
    s = W.config2()
    pos = torch.from_numpy(s.snapshot(0)).cuda()
    status = None
    try:
        ctx = D.Context(s, params=dict(spin_limit=1, cell_scale=2), flags=D.FLAG_PERSISTENT)
        ctx.step(pos, 0, stats=True)
    except D.DynbondError as e:
        status = e.status
    assert status == 5
    assert torch.ones(1000, device="cuda").sum().item() == 1000.0
