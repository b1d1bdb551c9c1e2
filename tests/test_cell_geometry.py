"""The two geometric facts the octant candidate search rests on, checked by
brute force over random boxes, reaches and cell counts (integer coordinates,
as on the device):

1. With columns at least twice the reach wide (2 reach nc <= L, nc >= 3), a
   coordinate in the lower half of its column (2 (x nc - c L) < L) reaches
   only its own column and the one below it, and one in the upper half only
   its own and the one above (periodically).
2. Along z, the window of cells the search forms -- cz - hz .. cz + hz with
   hz = ceil(reach nz / L), as a main run and, across the boundary, a wrapped
   run (or the whole column when it covers it) -- lists no cell twice and
   misses the cell of no coordinate within the reach.
"""
import numpy as np
import pytest


def cell(x, n, L):
    return (x * n) // L


def within(x, y, L, reach):
    d = (y - x) % L
    return min(d, L - d) <= reach


def test_octant_columns_hold_every_partner_within_reach():
    rng = np.random.default_rng(5)
    for _ in range(3000):
        reach = int(rng.integers(0, 60))
        nc = int(rng.integers(3, 14))
        L = max(2 * reach * nc, nc) + int(rng.integers(0, 50))
        x = int(rng.integers(0, L))
        c = cell(x, nc, L)
        lower = 2 * (x * nc - c * L) < L
        cols = {c, (c - 1) % nc if lower else (c + 1) % nc}
        for y in range(L):
            if within(x, y, L, reach):
                assert cell(y, nc, L) in cols, (L, nc, reach, x, y)


def z_runs(z, reach, nz, L):
    """Main run [z0, z1] and wrapped run [w0, w1] (empty if w1 < w0): the
    cells cz - hz .. cz + hz, hz = ceil(reach nz / L), periodic, or the
    whole column when they cover it."""
    hz = -(-reach * nz // L)
    cz = cell(z, nz, L)
    if 2 * hz + 1 >= nz:
        return 0, nz - 1, 0, -1
    lo, hi = cz - hz, cz + hz
    if lo < 0:
        return 0, hi, lo + nz, nz - 1
    if hi >= nz:
        return lo, nz - 1, 0, hi - nz
    return lo, hi, 0, -1


def z_runs_exact(z, reach, nz, L):
    """The staged search's runs of a whole staged column: the cells overlapping
    [z - reach, z + reach] exactly, main run [z0, z1] and wrapped run
    [w0, w1] (empty if w1 < w0)."""
    zlo, zhi = z - reach, z + reach
    w0, w1 = 0, -1
    if zlo >= 0 and zhi < L:
        z0, z1 = cell(zlo, nz, L), cell(zhi, nz, L)
    elif zlo < 0 and zhi < L:
        a, b = cell(zlo + L, nz, L), cell(zhi, nz, L)
        z0, z1 = 0, (b if a > b else nz - 1)
        if a > b:
            w0, w1 = a, nz - 1
    elif zlo >= 0 and zhi >= L:
        a, b = cell(zlo, nz, L), cell(zhi - L, nz, L)
        z0, z1 = (a if b < a else 0), nz - 1
        if b < a:
            w0, w1 = 0, b
    else:
        z0, z1 = 0, nz - 1
    return z0, z1, w0, w1


@pytest.mark.parametrize("runs", [z_runs, z_runs_exact])
def test_z_runs_cover_the_reach_interval_once(runs):
    rng = np.random.default_rng(6)
    for _ in range(3000):
        L = int(rng.integers(1, 300))
        reach = int(rng.integers(0, 160))
        nz = int(rng.integers(1, 50))
        z = int(rng.integers(0, L))
        z0, z1, w0, w1 = runs(z, reach, nz, L)
        cells = list(range(z0, z1 + 1)) + list(range(w0, w1 + 1))
        assert len(cells) == len(set(cells)) and all(0 <= c < nz for c in cells), (L, reach, nz, z)
        for y in range(L):
            if within(z, y, L, reach):
                assert cell(y, nz, L) in cells, (L, reach, nz, z, y)


# ---------------------------------------------------------------------------
# The staged search (k_candidates_tile): a tile of CT columns per axis and Z
# z cells is staged with one column around it along x and y (all columns when
# that wraps) and hz = floor(reach nz / L) + 1 cells on each side along z (the
# whole column when that covers it).  Every cell a bead of the tile can reach
# must be staged, at the local index the kernel computes, and the bead's local
# z run must lie inside the staged window.
# ---------------------------------------------------------------------------
CT, CZS_MAX = 8, 24


def xy_window(tx, nc):
    x0 = tx * CT
    Tx = min(CT, nc - x0)
    if Tx + 2 >= nc:
        return x0, Tx, 0, nc
    return x0, Tx, (x0 - 1) % nc, Tx + 2


def test_staged_columns_hold_every_partner_within_reach():
    rng = np.random.default_rng(7)
    for _ in range(3000):
        reach = int(rng.integers(1, 40))
        nc = int(rng.integers(1, 30))
        L = nc * reach + int(rng.integers(0, 3 * reach + 5))  # columns at least the reach wide
        tx = int(rng.integers(0, (nc + CT - 1) // CT))
        x0, Tx, hx0, HX = xy_window(tx, nc)
        staged = [(hx0 + k) % nc for k in range(HX)]
        assert len(set(staged)) == HX
        c = x0 + int(rng.integers(0, Tx))
        xs = [x for x in range(L) if cell(x, nc, L) == c]
        if not xs:
            continue
        x = xs[int(rng.integers(0, len(xs)))]
        for y in range(L):
            if within(x, y, L, reach):
                assert (cell(y, nc, L) - hx0) % nc < HX, (L, nc, reach, tx, x, y)


def test_staged_z_window_holds_the_bead_run():
    rng = np.random.default_rng(8)
    for _ in range(4000):
        L = int(rng.integers(2, 400))
        reach = int(rng.integers(1, 80))
        nz = int(rng.integers(1, 60))
        hz = reach * nz // L + 1
        if 2 * hz >= CZS_MAX:
            continue  # the host uses the global-memory search for this geometry
        Z = nz if nz <= CZS_MAX else min(16, CZS_MAX - 2 * hz)
        tz = int(rng.integers(0, (nz + Z - 1) // Z))
        z0 = tz * Z
        Tz = min(Z, nz - z0)
        whole = Tz + 2 * hz >= nz
        Zs, hz0 = (nz, 0) if whole else (Tz + 2 * hz, (z0 - hz) % nz)
        assert Zs <= CZS_MAX
        zs = [z for z in range(L) if z0 <= cell(z, nz, L) < z0 + Tz]
        if not zs:
            continue
        z = zs[int(rng.integers(0, len(zs)))]
        if whole:
            a0, a1, b0, b1 = z_runs_exact(z, reach, nz, L)
            local = list(range(a0, a1 + 1)) + list(range(b0, b1 + 1))
        else:
            cz = cell(z, nz, L)
            lo, hi = cell((z - reach) % L, nz, L), cell((z + reach) % L, nz, L)
            lzb = (cz - hz0) % nz
            r0, r1 = lzb - (cz - lo) % nz, lzb + (hi - cz) % nz
            assert 0 <= r0 <= r1 < Zs, (L, reach, nz, z, tz)
            local = list(range(r0, r1 + 1))
        for y in range(L):
            if within(z, y, L, reach):
                assert (cell(y, nz, L) - hz0) % nz in local, (L, reach, nz, z, y, tz)
