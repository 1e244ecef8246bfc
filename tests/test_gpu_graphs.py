"""Iterations replayed from captured CUDA graphs (sip_options.graphs = 1)
give the same bits as launch-by-launch queueing, in every mode."""
import numpy as np
import pytest

from paper_1303_4538_gb300 import sip, workloads as W
from tests._gpu import GpuSystem

pytestmark = pytest.mark.gpu

MODES = [sip.SIP_MODE_F64, sip.SIP_MODE_F32_REFINED, sip.SIP_MODE_F32]


def _run(blk, mode, graphs, fn, **kw):
    g = GpuSystem(blk, mode=mode, graphs=graphs, **kw)
    out = fn(g)
    xs = [g.xs(q) for q in range(len(g.x))]
    hist = g.plan.history()
    launches = g.plan.launches()
    g.close()
    return out, xs, hist, launches


@pytest.mark.parametrize("mode", MODES)
def test_solve_bitwise_equal(mode):
    blk = W.make_block(33, 35, 18, seed=91, kind="convdiff")
    a = _run(blk, mode, 0, lambda g: g.plan.solve(1e-7 if mode == sip.SIP_MODE_F32 else 1e-9, 300))
    b = _run(blk, mode, 1, lambda g: g.plan.solve(1e-7 if mode == sip.SIP_MODE_F32 else 1e-9, 300))
    assert a[0] == b[0]
    assert all(np.array_equal(p, q) for p, q in zip(a[1], b[1]))
    assert a[2] == b[2]
    assert a[3] == b[3]


@pytest.mark.parametrize("n", [1, 16, 17, 35])
def test_iterate_counts_and_bits(n):
    blk = W.make_block(24, 20, 16, seed=92, kind="poisson")
    a = _run(blk, sip.SIP_MODE_F64, 0, lambda g: g.plan.iterate(n), sym_null=True)
    b = _run(blk, sip.SIP_MODE_F64, 1, lambda g: g.plan.iterate(n), sym_null=True)
    assert a[0] == b[0] and a[2] == b[2] and a[3] == b[3] and len(a[2]) == n
    assert np.array_equal(a[1][0], b[1][0])


def test_multiblock_with_interfaces():
    mesh = W.make_mesh([(24, 20, 16), (30, 25, 12), (16, 40, 20)], 93, "convdiff")
    f = lambda g: g.plan.solve(1e-8, 600)
    a = _run(mesh.blocks, sip.SIP_MODE_F32_REFINED, 0, f, ifaces=mesh.ifaces)
    b = _run(mesh.blocks, sip.SIP_MODE_F32_REFINED, 1, f, ifaces=mesh.ifaces)
    assert a[0] == b[0] and a[2] == b[2]
    assert all(np.array_equal(p, q) for p, q in zip(a[1], b[1]))
