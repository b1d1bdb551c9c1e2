"""The two geometric facts the octant candidate search rests on, checked by
brute force over random boxes, reaches and cell counts (integer coordinates,
as on the device):

1. With columns at least twice the reach wide (2 reach nc <= L, nc >= 3), a
   coordinate in the lower half of its column (2 (x nc - c L) < L) reaches
   only its own column and the one below it, and one in the upper half only
   its own and the one above (periodically).
2. Along z, the cells overlapping the periodic interval [z - reach, z + reach]
   are the main run and, across the boundary, a wrapped run as the search
   forms them (or the whole column when those meet), without a cell listed
   twice and without missing the cell of any coordinate within the reach.
"""
import numpy as np


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
    """Main run [z0, z1] and wrapped run [w0, w1] (empty if w1 < w0)."""
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


def test_z_runs_cover_the_reach_interval_once():
    rng = np.random.default_rng(6)
    for _ in range(3000):
        L = int(rng.integers(1, 300))
        reach = int(rng.integers(0, 160))
        nz = int(rng.integers(1, 50))
        z = int(rng.integers(0, L))
        z0, z1, w0, w1 = z_runs(z, reach, nz, L)
        cells = list(range(z0, z1 + 1)) + list(range(w0, w1 + 1))
        assert len(cells) == len(set(cells)) and all(0 <= c < nz for c in cells), (L, reach, nz, z)
        for y in range(L):
            if within(z, y, L, reach):
                assert cell(y, nz, L) in cells, (L, reach, nz, z, y)
