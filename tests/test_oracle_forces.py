"""Pins of the oracle's FP64 bonded forces: closed forms, finite differences of
the energy, Newton's third law, invariances and the virial's strain
derivative."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_4214_gb300 import workloads as W

from helpers import half_bond_pair, make_system


def rot(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


def test_closed_forms():
    E, F = O.bond_half([1.3, 0, 0], 100.0, 1.0)
    assert E == pytest.approx(0.5 * 100 * 0.09) and F == pytest.approx([-2 * 100 * 0.3, 0, 0])
    E, Fa, Fc = O.angle([1, 0, 0], [-2, 0, 0], 2.0)  # straight: theta = 180 deg
    assert E == pytest.approx(0.0, abs=1e-15) and np.allclose(Fa, 0) and np.allclose(Fc, 0)
    E, Fa, Fc = O.angle([1, 0, 0], [0, 3, 0], 2.0)  # right angle
    assert E == pytest.approx(2.0)
    # Fa = -K d cos / d ra = -K rc / (|ra||rc|) at 90 deg
    assert Fa == pytest.approx([0, -2.0 / 1.0, 0]) and Fc == pytest.approx([-2.0 / 3.0, 0, 0])
    # planar trans (A and D on opposite sides): phi = 180 deg, E = K (1 - d); cis: E = K (1 + d)
    trans = O.dihedral([0, -1, 0], [1, 0, 0], [0, -1, 0], 1.0, 1.0)
    cis = O.dihedral([0, -1, 0], [1, 0, 0], [0, 1, 0], 1.0, 1.0)
    assert trans[0] == pytest.approx(0.0, abs=1e-15) and cis[0] == pytest.approx(2.0)
    assert O.dihedral([0, -1, 0], [1, 0, 0], [0, 1, 0], 1.0, -1.0)[0] == pytest.approx(0.0, abs=1e-15)
    # perpendicular planes: cos phi = 0, E = K
    assert O.dihedral([0, -1, 0], [1, 0, 0], [0, 0, 1], 1.5, 1.0)[0] == pytest.approx(1.5)


def test_harmonic_angle_closed_forms():
    """E = K (theta - theta0)^2 (Sec. 3): zero at theta0; otherwise the end
    forces are tangential with magnitude 2 K |theta - theta0| / |r_end|."""
    E, Fa, Fc = O.angle_harmonic([1, 0, 0], [0, 2, 0], 1.0, np.pi / 2)  # right angle, theta0 = 90 deg
    assert E == pytest.approx(0.0, abs=1e-15) and np.allclose(Fa, 0) and np.allclose(Fc, 0)
    E, Fa, Fc = O.angle_harmonic([1, 0, 0], [-3, 0, 0], 20.0, np.pi)  # straight, theta0 = 180 deg
    assert E == pytest.approx(0.0, abs=1e-15) and np.allclose(Fa, 0) and np.allclose(Fc, 0)
    th = np.deg2rad(120.0)
    ra, rc = np.array([2.0, 0, 0]), 0.5 * np.array([np.cos(th), np.sin(th), 0])
    for K, th0 in ((20.0, np.pi), (1.0, np.pi / 2)):
        E, Fa, Fc = O.angle_harmonic(ra, rc, K, th0)
        assert E == pytest.approx(K * (th - th0) ** 2, rel=1e-12)
        assert np.linalg.norm(Fa) == pytest.approx(2 * K * abs(th - th0) / 2.0, rel=1e-12)
        assert np.linalg.norm(Fc) == pytest.approx(2 * K * abs(th - th0) / 0.5, rel=1e-12)
        assert abs(Fa @ ra) < 1e-12 and abs(Fc @ rc) < 1e-12
        # opening the angle toward theta0 lowers the energy: F_A points away from C's side when theta < theta0
        assert (np.cross(ra, Fa)[2] < 0) == (th < th0)


def _bent(delta, rng, la=1.1, lc=0.9):
    """ra, rc of an angle theta = pi - delta at the centre bead, randomly
    oriented (ra along a random unit vector, rc bent away from -ra by delta
    within a random plane)."""
    M = rot(rng)
    ra = la * np.array([1.0, 0.0, 0.0])
    rc = lc * np.array([-np.cos(delta), np.sin(delta), 0.0])
    return M @ ra, M @ rc


@pytest.mark.parametrize("delta", [1e-2, 1e-4, 1e-6])
def test_harmonic_angle_near_straight_with_theta0_180(delta):
    """The backbone angle of Sec. 3 (theta0 = 180 deg) close to straight: E =
    K (pi - theta)^2 is smooth there, |F_A| = 2 K (pi - theta) / |r_A| exactly
    (tangential), and the forces are minus the finite-difference gradient of
    the energy at pi - theta = 1e-2, 1e-4 and 1e-6 (a division by a clamped
    sin theta would shrink them by up to three orders of magnitude)."""
    rng = np.random.default_rng(int(-np.log10(delta)))
    K = 20.0
    ra, rc = _bent(delta, rng)
    E, Fa, Fc = O.angle_harmonic(ra, rc, K, np.pi)
    assert E == pytest.approx(K * delta ** 2, rel=1e-8)
    assert np.linalg.norm(Fa) == pytest.approx(2 * K * delta / 1.1, rel=1e-8)
    assert np.linalg.norm(Fc) == pytest.approx(2 * K * delta / 0.9, rel=1e-8)
    P = np.stack([ra, np.zeros(3), rc]) + 5.0

    def Eharm(x):
        x = x.reshape(3, 3)
        return O.angle_harmonic(x[0] - x[1], x[2] - x[1], K, np.pi)[0]
    g = _fd(Eharm, P.ravel(), h=1e-6).reshape(3, 3)
    F = np.stack([Fa, -(Fa + Fc), Fc])
    assert np.allclose(F, -g, rtol=1e-5, atol=1e-5 * np.abs(F).max())


@pytest.mark.parametrize("delta", [1e-2, 1e-4])
def test_harmonic_angle_near_straight_with_theta0_90(delta):
    """The backbone-hybridization angle of Sec. 3 (theta0 = 90 deg) close to
    straight: |F_A| = 2 K (theta - theta0) / |r_A| stays finite and the forces
    are minus the energy gradient (finite differences with a step well below
    the bend, where the energy is smooth)."""
    rng = np.random.default_rng(7)
    K = 1.0
    ra, rc = _bent(delta, rng)
    E, Fa, Fc = O.angle_harmonic(ra, rc, K, np.pi / 2)
    assert E == pytest.approx(K * (np.pi / 2 - delta) ** 2, rel=1e-12)
    assert np.linalg.norm(Fa) == pytest.approx(2 * K * (np.pi / 2 - delta) / 1.1, rel=1e-8)
    P = np.stack([ra, np.zeros(3), rc]) + 5.0

    def Eharm(x):
        x = x.reshape(3, 3)
        return O.angle_harmonic(x[0] - x[1], x[2] - x[1], K, np.pi / 2)[0]
    g = _fd(Eharm, P.ravel(), h=delta * 1e-3).reshape(3, 3)
    F = np.stack([Fa, -(Fa + Fc), Fc])
    assert np.allclose(F, -g, rtol=1e-5, atol=1e-6)


def test_harmonic_angle_exactly_straight_has_no_plane():
    E, Fa, Fc = O.angle_harmonic([1.0, 0, 0], [-2.0, 0, 0], 20.0, np.pi)
    assert E == 0.0 and not Fa.any() and not Fc.any()
    E, Fa, Fc = O.angle_harmonic([1.0, 0, 0], [-2.0, 0, 0], 1.0, np.pi / 2)
    assert E == pytest.approx((np.pi / 2) ** 2) and not Fa.any() and not Fc.any()


def _fd(fun, x, h=1e-6):
    g = np.zeros_like(x)
    for i in range(x.size):
        xp, xm = x.copy(), x.copy()
        xp.flat[i] += h
        xm.flat[i] -= h
        g.flat[i] = (fun(xp) - fun(xm)) / (2 * h)
    return g


@pytest.mark.parametrize("seed", range(20))
def test_finite_differences_and_newton3(seed):
    rng = np.random.default_rng(seed)
    # bond
    r = rng.normal(size=3)
    E, F = O.bond_half(r, 37.0, 0.8)
    g = _fd(lambda x: 2 * O.bond_half(x, 37.0, 0.8)[0], r)  # half energy per end
    assert np.allclose(F, -g, rtol=1e-7, atol=1e-7)
    # angle as a function of the three positions
    P = rng.normal(size=(3, 3))

    def Eang(x):
        x = x.reshape(3, 3)
        return O.angle(x[0] - x[1], x[2] - x[1], 1.7)[0]
    E, Fa, Fc = O.angle(P[0] - P[1], P[2] - P[1], 1.7)
    g = _fd(Eang, P.ravel()).reshape(3, 3)
    Fb = -(Fa + Fc)
    assert np.allclose(np.stack([Fa, Fb, Fc]), -g, rtol=1e-6, atol=1e-7)
    # harmonic angle

    def Eharm(x):
        x = x.reshape(3, 3)
        return O.angle_harmonic(x[0] - x[1], x[2] - x[1], 1.7, 1.9)[0]
    E, Fa, Fc = O.angle_harmonic(P[0] - P[1], P[2] - P[1], 1.7, 1.9)
    g = _fd(Eharm, P.ravel()).reshape(3, 3)
    assert np.allclose(np.stack([Fa, -(Fa + Fc), Fc]), -g, rtol=1e-6, atol=1e-6)
    # dihedral
    Q = rng.normal(size=(4, 3))

    def Edih(x):
        x = x.reshape(4, 3)
        return O.dihedral(x[1] - x[0], x[2] - x[1], x[3] - x[2], 0.9, -1.0)[0]
    E, Fs = O.dihedral(Q[1] - Q[0], Q[2] - Q[1], Q[3] - Q[2], 0.9, -1.0)
    g = _fd(Edih, Q.ravel()).reshape(4, 3)
    assert np.allclose(np.stack(Fs), -g, rtol=1e-6, atol=1e-7)
    assert np.allclose(np.sum(Fs, axis=0), 0, atol=1e-12)
    # rotation invariance of the energies, covariance of the forces
    M = rot(rng)
    E2, Fs2 = O.dihedral(M @ (Q[1] - Q[0]), M @ (Q[2] - Q[1]), M @ (Q[3] - Q[2]), 0.9, -1.0)
    assert E2 == pytest.approx(E, rel=1e-12)
    assert np.allclose(np.stack(Fs2), np.stack(Fs) @ M.T, atol=1e-10)


def _molecule(seed, box=40.0):
    """A random branched molecule of 12 beads in a large box, with angle and
    dihedral rules that type every path."""
    rng = np.random.default_rng(seed)
    n = 12
    parent = [-1] + [int(rng.integers(0, k)) for k in range(1, n)]
    deg = np.zeros(n, int)
    bonds = []
    for k in range(1, n):
        p = parent[k]
        if deg[p] >= 3:
            p = k - 1
        deg[p] += 1
        deg[k] += 1
        t = int(rng.integers(1, 3))
        bonds.append([p, k, t, t])
    pos = np.zeros((n, 3))
    for k in range(1, n):
        pos[k] = pos[[b[0] for b in bonds if b[1] == k][0]] + rng.normal(size=3) * 0.6
    pos += box / 2
    rules = [
        dict(kind="createangle", type=1, beads=(W.ALL_BEADS,) * 3, bonds=(W.ALL_BONDS, W.ALL_BONDS)),
        dict(kind="createdihedral", type=1, beads=(W.ALL_BEADS,) * 4, bonds=(W.bit(1), W.ALL_BONDS, W.ALL_BONDS)),
        dict(kind="createdihedral", type=2, beads=(W.ALL_BEADS,) * 4, bonds=(W.ALL_BONDS,) * 3),
    ]
    s = make_system(rng.integers(0, 5, n), bonds, pos, box, rules)
    s.forcefield = dict(bond_k=np.full(16, 30.0), bond_r0=np.full(16, 0.7), angle_k=np.full(16, 1.3),
                        dihedral_k=np.full(16, 0.8), dihedral_d=np.array([1, 1, -1] + [1] * 13, np.int32))
    return s, pos


@pytest.mark.parametrize("seed,harmonic", [(k, k % 2 == 1) for k in range(6)])
def test_system_forces_are_minus_energy_gradient(seed, harmonic):
    s, pos = _molecule(seed)
    if harmonic:  # the DNA angles of Sec. 3: K (theta - theta0)^2
        s.forcefield["angle_style"] = np.ones(16, np.int32)
        s.forcefield["angle_theta0"] = np.full(16, 1.9)
    o = O.Oracle(s)
    _, a, d = o.topology()
    assert len(a) > 5 and len(d) > 3
    q = s.snapshot()
    f, ev = o.forces(q)
    h = 64  # quanta
    for i in range(0, s.n_beads, 3):
        for c in range(3):
            qp, qm = q.copy(), q.copy()
            qp[i, c] += h
            qm[i, c] -= h
            g = (o.forces(qp)[1][0, 0] - o.forces(qm)[1][0, 0]) / (2 * h / W.QSCALE)
            assert f[i, c] == pytest.approx(-g, rel=1e-5, abs=1e-5)
    assert np.allclose(f.sum(axis=0), 0, atol=1e-9)


@pytest.mark.parametrize("seed", range(4))
def test_virial_is_minus_strain_derivative(seed):
    # under x_a -> x_a + eps x_b about the molecule's centre, dE/deps = -W_ba
    s, pos = _molecule(seed)
    o = O.Oracle(s)
    ctr = pos.mean(axis=0)
    comp = {(0, 0): 1, (1, 1): 2, (2, 2): 3, (0, 1): 4, (0, 2): 5, (1, 2): 6}
    _, ev = o.forces(s.snapshot())
    W6 = ev[0]
    Wm = np.zeros((3, 3))
    for (a_, b_), k in comp.items():
        Wm[a_, b_] = Wm[b_, a_] = W6[k]
    eps = 1e-2  # quantization noise in dE/deps is ~ 2^-21 / eps relative
    for a_ in range(3):
        for b_ in range(3):
            def energy(e):
                x = pos - ctr
                x2 = x.copy()
                x2[:, a_] += e * x[:, b_]
                from helpers import qpos
                return o.forces(qpos(s, x2 + ctr))[1][0, 0]
            dE = (energy(eps) - energy(-eps)) / (2 * eps)
            assert dE == pytest.approx(-Wm[b_, a_], rel=2e-3, abs=1e-3 * np.abs(Wm).max())


def test_translation_invariance_through_the_box():
    s, pos = _molecule(1)
    o = O.Oracle(s)
    f0, e0 = o.forces(s.snapshot())
    from helpers import qpos
    f1, e1 = o.forces(qpos(s, pos + np.array([19.75, -33.125, 5.5])))  # wraps through the boundary
    assert np.allclose(f0, f1, atol=1e-6) and np.allclose(e0, e1, rtol=1e-9, atol=1e-6)


def test_half_bonds_with_different_stored_types_give_a_net_force():
    """Each end of a directional bond feels the full force of the type it
    stores and books half the energy (Sec. 2): with unequal potentials the
    pair feels a net force (the 'active matter' remark of Sec. 2), in closed
    form (bead 1 on +x of bead 0, r the exact quantized distance)
    F0 = +2 K2 (r - r02) x^, F1 = -2 K3 (r - r03) x^."""
    s = half_bond_pair()
    o = O.Oracle(s)
    snap = s.snapshot(0)
    f, ev = o.forces(snap)
    r = (int(snap[1, 0]) - int(snap[0, 0])) / W.QSCALE
    f0 = 2.0 * 100.0 * (r - 1.0)
    f1 = -2.0 * 40.0 * (r - 1.2)
    assert np.allclose(f[0], [f0, 0.0, 0.0], rtol=1e-12, atol=1e-12)
    assert np.allclose(f[1], [f1, 0.0, 0.0], rtol=1e-12, atol=1e-12)
    assert abs(f[0, 0] + f[1, 0]) > 50.0  # no third law across a directional bond with unequal halves
    assert np.isclose(ev[0, 0], 0.5 * 100.0 * (r - 1.0) ** 2 + 0.5 * 40.0 * (r - 1.2) ** 2, rtol=1e-12)
