"""Shared GPU-parity helpers: the CUDA path through the C ABI against the CPU
oracle on the same seeded inputs.

Topology (bonds with the type each end stores, angles, dihedrals) and every
per-replica statistic must match bit for bit after every call.  Bonded forces
(FP32 per term) must match the FP64 oracle per component within

    |f_gpu - f_ref| <= FORCE_TOL * max(|f_ref|, f_rms),

f_rms the root mean square of the oracle's force components over the system
(a plain relative error is undefined where f_ref is zero); the FP64-reduced
energy / virial within EV_TOL of the largest magnitude of the replica."""

import numpy as np

from oracle import oracle as O

FORCE_TOL = 1e-5
EV_TOL = 2e-6


def torch():
    import torch as t
    return t


def dynbond():
    from paper_1108_4214_gb300 import dynbond as D
    return D


def assert_same(a, b, what):
    if a.shape != b.shape or not np.array_equal(a, b):
        sa = {tuple(x) for x in a.tolist()}
        sb = {tuple(x) for x in b.tolist()}
        raise AssertionError(f"{what}: gpu {a.shape} vs oracle {b.shape}; only gpu {sorted(sa - sb)[:5]} "
                             f"only oracle {sorted(sb - sa)[:5]}")


def compare_topology(ctx, o, where):
    for name, g, r in zip(("bonds", "angles", "dihedrals"), ctx.topology(), o.topology()):
        assert_same(g, r, f"{where}: {name}")


def force_error(f, fr):
    """Largest |f - f_ref| / max(|f_ref|, f_rms) over all components."""
    f = np.asarray(f, np.float64)[:, :3]
    rms = np.sqrt(np.mean(fr ** 2))
    if rms == 0.0:
        return 0.0 if not np.any(f) else np.inf
    return float((np.abs(f - fr) / np.maximum(np.abs(fr), rms)).max())


def ev_error(ev, evr, scale=None):
    """Largest |ev - ev_ref| over a replica's 7 values, relative to the
    replica's largest magnitude (or to a given per-replica scale, e.g. the
    size of the terms when the sums cancel)."""
    if scale is None:
        scale = np.abs(evr).max(axis=1)
    scale = np.asarray(scale, np.float64).reshape(-1, 1).copy()
    err = np.abs(ev - evr)
    if np.any((scale == 0) & (err > 0).any(axis=1, keepdims=True)):
        return np.inf
    scale[scale == 0] = 1.0
    return float((err / scale).max())


def compare_forces(ctx, o, snap, where, ev_scale=None, given=None):
    """Forces and energy / virial at snap against the oracle's: computed by
    ctx.forces, or `given` as (force, ev) CUDA tensors from a combined call."""
    if given is None:
        f, ev = ctx.forces(torch().from_numpy(snap).cuda())
    else:
        f, ev = given
    f = f.cpu().numpy()
    ev = ev.cpu().numpy()
    fr, evr = o.forces(snap)
    assert np.all(f[:, 3] == 0)
    worst = force_error(f, fr)
    if not worst <= FORCE_TOL:
        bad_g = np.where(~np.isfinite(f[:, :3]).all(axis=1))[0]
        bad_r = np.where(~np.isfinite(fr).all(axis=1))[0]
        raise AssertionError(f"{where}: force error {worst:.3g} (x max(|f|, rms)); non-finite gpu rows "
                             f"{bad_g[:8].tolist()} oracle rows {bad_r[:8].tolist()}")
    evw = ev_error(ev, evr, ev_scale)
    assert evw <= EV_TOL, f"{where}: energy/virial error {evw:.3g}"
    return worst, evw


def compare_stats(st_g, st_o, where):
    if not np.array_equal(st_g, st_o):
        diff = {O.STAT_NAMES[j]: (st_g[:, j].tolist(), st_o[:, j].tolist())
                for j in range(len(O.STAT_NAMES)) if not np.array_equal(st_g[:, j], st_o[:, j])}
        raise AssertionError(f"{where}: statistics differ {diff}")


def run_parity(system, n_calls, snaps=None, params=None, flags=0, forces=True, start=0, combined=False):
    """n_calls calls on the GPU and on the oracle: statistics, topology and
    (optionally) forces compared after every call.  combined: each call is
    dynbond_step_forces (step and forces in one call) instead of the two
    calls.  Returns the oracle and the per-call (force error, energy/virial
    error)."""
    o = O.Oracle(system, params=params)
    ctx = dynbond().Context(system, params=params, flags=flags)
    compare_topology(ctx, o, "initial")
    worst = []
    for k in range(n_calls):
        snap = snaps[k] if snaps is not None else system.snapshot(k)
        pos = torch().from_numpy(snap).cuda()
        given = None
        if combined:
            f, ev, st_g = ctx.step_forces(pos, start + k, stats=True)
            given = (f, ev)
        else:
            st_g = ctx.step(pos, start + k, stats=True)
        st_o = o.step(snap, start + k)
        compare_stats(st_g, st_o, f"call {k}")
        compare_topology(ctx, o, f"call {k}")
        if forces or combined:
            worst.append(compare_forces(ctx, o, snap, f"call {k}", given=given))
    ctx.close()
    return o, worst
