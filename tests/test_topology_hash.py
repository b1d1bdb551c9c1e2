"""The topology hash restated in tests/helpers.py: order independence,
sensitivity to every field, and agreement with the GPU entry point."""
import numpy as np
import pytest

from helpers import topology_hash
from oracle import oracle as O
from paper_1108_4214_gb300 import workloads as W


def _topo(seed=1, calls=3):
    s = W.config1()
    o = O.Oracle(s)
    for k, snap in enumerate(s.snapshots(0, calls)):
        o.step(snap, k)
    return s, o


def test_hash_ignores_order_and_sees_every_field():
    _, o = _topo()
    b, a, d = o.topology()
    h = topology_hash(b, a, d)
    rng = np.random.default_rng(0)
    assert topology_hash(b[rng.permutation(len(b))], a[rng.permutation(len(a))], d[rng.permutation(len(d))]) == h
    for arr, name in ((b, "bonds"), (a, "angles"), (d, "dihedrals")):
        for col in range(arr.shape[1]):
            x = arr.copy()
            x[len(x) // 2, col] += 1
            args = dict(bonds=b, angles=a, dihedrals=d)
            args[name] = x
            assert topology_hash(**args) != h, (name, col)
    assert topology_hash(b[:-1], a, d) != h


@pytest.mark.gpu
def test_gpu_topology_hash_matches_the_definition():
    torch = pytest.importorskip("torch")
    from paper_1108_4214_gb300 import dynbond as D
    s, o = _topo()
    ctx = D.Context(s)
    for k, snap in enumerate(s.snapshots(0, 3)):
        ctx.step(torch.from_numpy(snap).cuda(), k)
    assert int(ctx.topology_hash()[0]) == topology_hash(*o.topology())
