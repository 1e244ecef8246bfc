"""Pins of the oracle's refined multi-block SIP (FP64 refinement around FP32
SIP iterations, the blocks exchanging the correction's interface values
after every inner iteration) against dense linear algebra on tiny meshes:
the first FP64 residual, one correction with m = 1, 2, 3 inner iterations as
the dense preconditioned iteration on the COUPLED correction system (and not
on the uncoupled one), and convergence to the dense global solution."""
import numpy as np
import pytest

import oracle
from paper_1303_4538_gb300 import workloads as W
from tests import _dense as D
from tests.test_oracle_multiblock import MESHES, dense_global

ALPHA = 0.92


def _setup(dims, kind, seed):
    mesh = W.make_mesh(dims, seed, kind)
    c32 = [{k: v.astype(np.float32) for k, v in b.coefs.items()} for b in mesh.blocks]
    c32w = [{k: v.astype(np.float64) for k, v in c.items()} for c in c32]
    # FP32 factors of the stored FP32 matrix (as the device computes them from A32)
    F32 = [oracle.factors_f32(oracle.factor(b.nx, b.ny, b.nz, c32w[q], ALPHA)) for q, b in enumerate(mesh.blocks)]
    blocks = [(b.nx, b.ny, b.nz, b.coefs, b.b) for b in mesh.blocks]
    return mesh, c32, c32w, F32, blocks


class _W:
    """The mesh with another set of coefficients (for dense_global)."""

    def __init__(self, mesh, coefs):
        self.blocks = [type("B", (), dict(nx=b.nx, ny=b.ny, nz=b.nz, n=b.n, coefs=c))()
                       for b, c in zip(mesh.blocks, coefs)]
        self.ifaces = mesh.ifaces


def _dense_M(mesh, F32):
    sizes = [b.n for b in mesh.blocks]
    off = np.concatenate([[0], np.cumsum(sizes)])
    M = np.zeros((off[-1], off[-1]))
    for q, b in enumerate(mesh.blocks):
        L, U = D.dense_LU(b.nx, b.ny, b.nz, [f.astype(np.float64) for f in F32[q]])
        M[off[q]:off[q + 1], off[q]:off[q + 1]] = L @ U
    return M


@pytest.mark.parametrize("dims,kind", MESHES)
def test_first_residual_is_global_fp64_residual(dims, kind):
    mesh, c32, c32w, F32, blocks = _setup(dims, kind, 21)
    A, off = dense_global(mesh)
    rng = np.random.default_rng(5)
    x0 = [rng.uniform(-1, 1, b.n) for b in mesh.blocks]
    xs, it, rel, hist = oracle.solve_refined_multiblock(blocks, mesh.ifaces, c32, F32, x0=x0, max_outer=0)
    bs = np.concatenate([b.b for b in mesh.blocks])
    ref = np.linalg.norm(bs - A @ np.concatenate(x0)) / np.linalg.norm(bs)
    assert it == 0
    assert abs(hist[0] - ref) <= 1e-14


@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("dims,kind", MESHES)
def test_one_correction_is_dense_iteration_on_coupled_system(dims, kind, m):
    """x1 = x0 + d_m with d_0 = 0, d_{q+1} = d_q + M^-1 (r - A32 d_q),
    r = b - A64 x0, M = blockdiag(L32_b U32_b), A32 the global matrix of the
    FP32 entries INCLUDING the interface entries (exchange after every inner
    iteration).  FP32 inner arithmetic: compared at 1e-5 of max |d|."""
    mesh, c32, c32w, F32, blocks = _setup(dims, kind, 23)
    A64, off = dense_global(mesh)
    A32g, _ = dense_global(_W(mesh, c32w))
    M = _dense_M(mesh, F32)
    rng = np.random.default_rng(6)
    x0 = [rng.uniform(-1, 1, b.n) for b in mesh.blocks]
    X0 = np.concatenate(x0)
    bs = np.concatenate([b.b for b in mesh.blocks])
    r = bs - A64 @ X0
    d = np.zeros_like(r)
    for _ in range(m):
        d = d + np.linalg.solve(M, r - A32g @ d)
    xs, it, rel, hist = oracle.solve_refined_multiblock(blocks, mesh.ifaces, c32, F32, x0=x0, rtol=-1.0,
                                                        max_outer=1, m_inner=m)
    got = np.concatenate(xs) - X0
    tol = 1e-5 * np.abs(d).max()
    assert it == 1
    assert np.abs(got - d).max() <= tol
    if m >= 2:
        # the uncoupled inner iteration (no exchange) is a different, detectably wrong answer
        Ablk = np.zeros_like(A32g)
        for q in range(len(mesh.blocks)):
            Ablk[off[q]:off[q + 1], off[q]:off[q + 1]] = A32g[off[q]:off[q + 1], off[q]:off[q + 1]]
        dw = np.zeros_like(r)
        for _ in range(m):
            dw = dw + np.linalg.solve(M, r - Ablk @ dw)
        assert np.abs(dw - d).max() > 100 * tol


@pytest.mark.parametrize("dims,kind", MESHES)
def test_converges_to_dense_global_solution(dims, kind):
    mesh, c32, c32w, F32, blocks = _setup(dims, kind, 25)
    A, off = dense_global(mesh)
    bs = np.concatenate([b.b for b in mesh.blocks])
    xs, it, rel, hist = oracle.solve_refined_multiblock(blocks, mesh.ifaces, c32, F32, rtol=1e-12,
                                                        max_outer=5000, m_inner=4)
    assert rel <= 1e-12
    assert np.all(np.diff(hist[: min(len(hist), 5)]) < 0)
    ref = np.linalg.solve(A, bs)
    assert np.abs(np.concatenate(xs) - ref).max() <= 1e-9 * np.abs(ref).max()


def test_m1_tracks_fp64_block_jacobi():
    """With one inner iteration the refined correction is the FP64 lagged
    block-Jacobi step of oracle_solve_mb up to FP32 rounding."""
    mesh, c32, c32w, F32, blocks = _setup([(4, 3, 3), (3, 4, 2), (5, 2, 3)], "convdiff", 27)
    F64 = [oracle.factor(b.nx, b.ny, b.nz, c32w[q], ALPHA) for q, b in enumerate(mesh.blocks)]
    rng = np.random.default_rng(7)
    x0 = [rng.uniform(-1, 1, b.n) for b in mesh.blocks]
    blocks32w = [(b.nx, b.ny, b.nz, c32w[q], b.b) for q, b in enumerate(mesh.blocks)]
    a = oracle.solve_multiblock(blocks32w, mesh.ifaces, F64, x0=x0, rtol=-1.0, max_iters=5)
    s = oracle.solve_refined_multiblock(blocks32w, mesh.ifaces, c32, F32, x0=x0, rtol=-1.0, max_outer=5,
                                        m_inner=1)
    for p, q in zip(a[0], s[0]):
        assert np.abs(p - q).max() <= 1e-5 * np.abs(p).max()


def test_symmetric_entries_read_from_lo_side():
    mesh, c32, c32w, F32, blocks = _setup([(3, 3, 3), (4, 3, 3)], "poisson", 29)
    rng = np.random.default_rng(8)
    x0 = [rng.uniform(-1, 1, b.n) for b in mesh.blocks]
    a = oracle.solve_refined_multiblock(blocks, mesh.ifaces, c32, F32, x0=x0, rtol=-1.0, max_outer=3, m_inner=3)
    s = oracle.solve_refined_multiblock(blocks, mesh.ifaces, c32, F32, x0=x0, rtol=-1.0, max_outer=3, m_inner=3,
                                        symmetric=True)
    assert all(np.array_equal(p, q) for p, q in zip(a[0], s[0]))
