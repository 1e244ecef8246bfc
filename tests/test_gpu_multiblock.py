"""Multi-block plans with x interfaces (lagged block Jacobi) against the
oracle's multi-block solve, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1303_4538_gb300 import sip, workloads as W
from tests._gpu import GpuSystem

pytestmark = pytest.mark.gpu

MESHES = [
    ([(4, 3, 3), (3, 4, 2), (5, 2, 3)], "convdiff"),
    ([(1, 3, 2), (2, 2, 3), (1, 4, 4)], "convdiff"),
    ([(40, 35, 18), (33, 40, 21), (17, 70, 9)], "convdiff"),
    ([(24, 37, 12), (30, 33, 20)], "poisson"),
]


def _oracle(mesh, iters=None, rtol=-1.0, x0=None):
    F = [oracle.factor(b.nx, b.ny, b.nz, b.coefs, 0.92) for b in mesh.blocks]
    blocks = [(b.nx, b.ny, b.nz, b.coefs, b.b) for b in mesh.blocks]
    return oracle.solve_multiblock(blocks, mesh.ifaces, F, x0=x0, rtol=rtol, max_iters=iters,
                                   symmetric=mesh.blocks[0].symmetric)


@pytest.mark.parametrize("dims,kind", MESHES)
def test_per_iteration_parity_f64(dims, kind):
    mesh = W.make_mesh(dims, 17, kind)
    g = GpuSystem(mesh.blocks, ifaces=mesh.ifaces, sym_null=mesh.blocks[0].symmetric)
    for n in (1, 3):
        for x in g.x:
            x.zero_()
        g.plan.iterate(n)
        xs, it, rel, hist = _oracle(mesh, iters=n)
        hg = g.plan.history()
        assert len(hg) == n
        assert np.abs(np.array(hg) - hist[:n]).max() <= 1e-12
        for q, x in enumerate(xs):
            got = g.xs(q)
            assert np.abs(got - x).max() <= 1e-12 * max(np.abs(x).max(), 1e-300)
    g.close()


@pytest.mark.parametrize("dims,kind", MESHES[2:])
def test_solve_matches_oracle(dims, kind):
    mesh = W.make_mesh(dims, 19, kind)
    g = GpuSystem(mesh.blocks, ifaces=mesh.ifaces, sym_null=mesh.blocks[0].symmetric)
    it, rel, conv = g.plan.solve(1e-8, 2000)
    xs, itr, relr, hist = _oracle(mesh, iters=2000, rtol=1e-8)
    assert conv and it == itr
    assert abs(rel - relr) <= 1e-12
    for q, x in enumerate(xs):
        assert np.abs(g.xs(q) - x).max() <= 1e-11 * np.abs(x).max()
    g.close()


@pytest.mark.parametrize("dims,kind", MESHES[2:])
def test_refined_solve_reaches_tolerance(dims, kind):
    mesh = W.make_mesh(dims, 23, kind)
    g = GpuSystem(mesh.blocks, ifaces=mesh.ifaces, mode=sip.SIP_MODE_F32_REFINED,
                  sym_null=mesh.blocks[0].symmetric)
    it, rel, conv = g.plan.solve(1e-8, 2000)
    assert conv and rel <= 1e-8
    # the coupled residual of the returned x, computed by the oracle
    _, _, _, hist = _oracle(mesh, iters=0, x0=[g.xs(q) for q in range(len(mesh.blocks))])
    assert hist[0] <= 1e-8 * (1 + 1e-6)
    assert abs(hist[0] - rel) <= 1e-12
    g.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("dims,kind", MESHES)
def test_refined_per_correction_parity(dims, kind):
    """FP64 refinement around m FP32 iterations on the coupled correction
    system (interface exchange after every inner iteration) against the
    oracle's float arithmetic, per correction (C13: rel 1e-5)."""
    mesh = W.make_mesh(dims, 29, kind)
    sym = mesh.blocks[0].symmetric
    F32 = [oracle.factors_f32(oracle.factor(b.nx, b.ny, b.nz, b.coefs, 0.92)) for b in mesh.blocks]
    c32 = [{k: v.astype(np.float32) for k, v in b.coefs.items()} for b in mesh.blocks]
    blocks = [(b.nx, b.ny, b.nz, b.coefs, b.b) for b in mesh.blocks]
    for m in (1, 2, 4):
        g = GpuSystem(mesh.blocks, ifaces=mesh.ifaces, mode=sip.SIP_MODE_F32_REFINED, inner=m, sym_null=sym)
        for n in (1, 3):
            for x in g.x:
                x.zero_()
            g.plan.iterate(n)
            xs, it, rel, hist = oracle.solve_refined_multiblock(blocks, mesh.ifaces, c32, F32, rtol=-1.0,
                                                                max_outer=n, m_inner=m, symmetric=sym)
            hg = np.array(g.plan.history())
            assert len(hg) == n
            assert abs(hg[0] - hist[0]) <= 1e-12
            assert np.abs(hg - hist[:n]).max() <= 1e-5 * hist[0]
            for q, x in enumerate(xs):
                assert _rel(g.xs(q), x) <= 1e-5
        g.close()


def test_interface_validation():
    blocks = [W.make_block(4, 3, 3, seed=1), W.make_block(3, 4, 2, seed=2)]
    for bad in ([(0, 0, 3, 2)], [(0, 2, 3, 2)], [(0, 1, 4, 2)], [(0, 1, 3, 3)], [(0, 1, 3, 2), (0, 1, 2, 2)],
                [(0, 1, 0, 2)]):
        with pytest.raises(sip.SipError) as e:
            GpuSystem(blocks, ifaces=bad)
        assert e.value.code == sip.SIP_ERR_INVALID_ARG


@pytest.mark.slow
def test_batched_mesh_20M_refined():
    """The 64-block ~20 M-cell mesh: refined solve to 1e-8, coupled residual
    of the returned x checked by the oracle; two FP64 iterations vs the oracle."""
    mesh = W.batched_mesh()
    assert 18_000_000 <= mesh.n <= 22_000_000 and len(mesh.blocks) == 64
    g = GpuSystem(mesh.blocks, ifaces=mesh.ifaces, mode=sip.SIP_MODE_F32_REFINED)
    it, rel, conv = g.plan.solve(1e-8, 5000)
    assert conv
    _, _, _, hist = _oracle(mesh, iters=0, x0=[g.xs(q) for q in range(64)])
    assert hist[0] <= 1e-8 * (1 + 1e-6)
    g.close()
    g = GpuSystem(mesh.blocks, ifaces=mesh.ifaces)
    g.plan.iterate(2)
    xs, _, _, hist = _oracle(mesh, iters=2)
    assert np.abs(np.array(g.plan.history()) - hist[:2]).max() <= 1e-12
    for q in (0, 31, 63):
        assert np.abs(g.xs(q) - xs[q]).max() <= 1e-12 * np.abs(xs[q]).max()
    g.close()
