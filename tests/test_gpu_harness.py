"""The DPD loop around the dynamic-bonding pass: every dumped call is
replayed by the CPU oracle from the GPU's own quantized positions and pre-call
bonds, and must give the same statistics and post-call topology bit for bit;
the bonded energy / virial at the dumped positions must match the FP64
oracle."""

import dataclasses

import numpy as np
import pytest

from helpers import topology_hash
from oracle import oracle as O
from paper_1108_4214_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EV_TOL = 2e-6


def replay(system, res, series=None):
    """Replays every dumped call on the oracle (bit-exact statistics and
    topology) and compares the GPU's bonded energy / virial at the dumped
    positions with the FP64 oracle; `series` (a list) receives, per dump,
    (call, E_gpu, E_fp64, relative energy error, largest relative virial
    error)."""
    worst_ev = 0.0
    for d in res["dumps"]:
        s = dataclasses.replace(system, bonds=d.bonds)
        o = O.Oracle(s)
        _, evr = o.forces(d.positions)
        worst_ev = max(worst_ev, float((np.abs(d.ev - evr) / np.abs(evr).max(axis=1, keepdims=True)).max()))
        if series is not None:
            scale = np.abs(evr[0, 1:]).max()
            series.append((d.call, float(d.ev[0, 0]), float(evr[0, 0]), float(abs(d.ev[0, 0] - evr[0, 0]) / abs(evr[0, 0])),
                           float(np.abs(d.ev[0, 1:] - evr[0, 1:]).max() / scale)))
        st = o.step(d.positions, d.call)
        assert np.array_equal(st, d.stats), (d.call, st, d.stats)
        for g, r in zip(d.topology, o.topology()):
            assert np.array_equal(g, r), d.call
        # the hash logged after that call names the same topology
        assert int(res["hashes"][d.call][0]) == topology_hash(*o.topology()), d.call
    assert len(res["hashes"]) == len(res["counts"])
    assert worst_ev <= EV_TOL, worst_ev
    return worst_ev


def test_dpd_loop_small_replays_bit_exact():
    from paper_1108_4214_gb300 import harness
    s = W.dna_system("dpd-8k", 64, 64, 0.5, 15, W.rules_dna2())
    res = harness.run_dpd_loop(s, n_calls=30, md_steps_per_call=10, dump_every=6)
    assert len(res["dumps"]) == 5
    worst = replay(s, res)
    assert np.isfinite(res["kT"])
    print("kT", res["kT"], "max ev error", worst)


def test_dpd_thermostat_holds_kT_for_free_beads():
    """Free DPD beads (no bonds, no rules) at density 3 (the paper's solvent
    density, Sec. 3): after equilibration the kinetic temperature is kT = 1
    within a few per cent (velocity-Verlet DPD at dt = 0.01)."""
    from paper_1108_4214_gb300 import dynbond as D
    n, rho = 24000, 3.0
    box = (n / rho) ** (1.0 / 3.0)
    rng = np.random.default_rng(21)
    s = W.System(name="free", bead_offset=np.array([0, n]), box_q=np.array([int(round(box * W.QSCALE))]),
                 types=np.zeros(n, np.int32), bonds=np.zeros((0, 4), np.int32), rules=[],
                 pos0=rng.uniform(0, box, size=(n, 3)), seed=21, params=W.default_params(21))
    dev = torch.device("cuda")
    ctx = D.Context(s)
    md = D.MD(ctx, seed=99)
    pos = torch.from_numpy(s.snapshot(0)).to(dev)
    vel = torch.from_numpy(W.initial_velocities(n, seed=3)).to(dev)
    md.advance(pos, vel, 500, 0)
    temps = []
    for k in range(10):
        md.advance(pos, vel, 50, 500 + 50 * k)
        v = vel.cpu().numpy()[:, :3].astype(np.float64)
        temps.append(np.mean(v ** 2))
    kT = float(np.mean(temps))
    assert 0.95 < kT < 1.06, kT


@pytest.mark.slow
def test_dpd_loop_4m_beads_ten_thousand_steps():
    from paper_1108_4214_gb300 import harness
    s = W.config5()
    res = harness.run_dpd_loop(s, n_calls=1000, md_steps_per_call=10, dump_every=100)
    assert len(res["dumps"]) == 10
    series = []
    worst = replay(s, res, series)
    print("dpd-4M: kT %.4f, md %.1f s, dynbond_step %.1f s, max ev error %.3g, bonds first/last %s %s" % (
        res["kT"], res["seconds_md"], res["seconds_step"], worst, res["counts"][0], res["counts"][-1]))
    # the bonded energy and virial against FP64 along the run (one line per
    # dump): the error stays at the FP32 rounding level, it does not grow
    for call, e, er, de, dw in series:
        print("dpd-4M call %4d: E %.9e (FP64 %.9e) rel err E %.2e, virial %.2e" % (call, e, er, de, dw))
    assert max(x[3] for x in series) <= 2e-6 and max(x[4] for x in series) <= 2e-6


@pytest.mark.parametrize("step", [0, 7])
def test_dpd_pair_forces_match_the_fp64_oracle(step):
    """One evaluation of the DPD pair forces of Sec. 3 (F^C + F^D + F^R, w(r)
    = 1 - r / r_c, sigma = sqrt(2 kT gamma), pairs fewer than 3 bonds apart
    excluded) on a snapshot at the paper's solvent density 3 with random
    velocities: the GPU's FP32 forces against the oracle's FP64 brute force,
    same Gaussian numbers (Philox on pair and step)."""
    from paper_1108_4214_gb300 import dynbond as D
    from parity import FORCE_TOL, force_error
    s = W.dna_system("dpd-4k", 64, 32, 3.0, 33, W.rules_dna2(), n_duplex=16)
    ctx = D.Context(s)
    md = D.MD(ctx, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.01, seed=987654321)
    snap = s.snapshot(0)
    rng = np.random.default_rng(step)
    vel = np.zeros((s.n_beads, 4), np.float32)
    vel[:, :3] = rng.normal(size=(s.n_beads, 3))
    f = md.pair_forces(torch.from_numpy(snap).cuda(), torch.from_numpy(vel).cuda(), step).cpu().numpy()
    fr = O.Oracle(s).dpd_forces(snap, vel[:, :3].astype(np.float64), a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.01,
                                seed=987654321, step=step)
    assert np.all(f[:, 3] == 0)
    err = force_error(f, fr)
    assert err <= FORCE_TOL, err
    md.close()
    ctx.close()
