"""Pins of the oracle's multi-block (lagged block-Jacobi) SIP against dense
linear algebra on tiny meshes: the coupled residual, one iteration as a
block-diagonal preconditioned Richardson step, and the converged solution."""
import numpy as np
import pytest

import oracle
from paper_1303_4538_gb300 import workloads as W
from tests import _dense as D

MESHES = [
    ([(4, 3, 3), (3, 4, 2), (5, 2, 3)], "convdiff"),
    ([(3, 3, 3), (4, 3, 3)], "poisson"),
    ([(1, 3, 2), (2, 2, 3), (1, 4, 4)], "convdiff"),  # nx = 1: a block touched on both x faces
]


def dense_global(mesh):
    """Global matrix: block-diagonal A_b plus the interface entries."""
    sizes = [b.n for b in mesh.blocks]
    off = np.concatenate([[0], np.cumsum(sizes)])
    A = np.zeros((off[-1], off[-1]))
    for q, b in enumerate(mesh.blocks):
        A[off[q]:off[q + 1], off[q]:off[q + 1]] = D.dense_A(b.nx, b.ny, b.nz, b.coefs)
    for lo, hi, nj, nk in mesh.ifaces:
        L, H = mesh.blocks[lo], mesh.blocks[hi]
        for k in range(nk):
            for j in range(nj):
                pl = D.idx(L.nx, L.ny, L.nx - 1, j, k)
                ph = D.idx(H.nx, H.ny, 0, j, k)
                A[off[lo] + pl, off[hi] + ph] = L.coefs["ae"][pl]
                A[off[hi] + ph, off[lo] + pl] = H.coefs["aw"][ph]
    return A, off


def _setup(dims, kind, seed):
    mesh = W.make_mesh(dims, seed, kind)
    F = [oracle.factor(b.nx, b.ny, b.nz, b.coefs, 0.92) for b in mesh.blocks]
    blocks = [(b.nx, b.ny, b.nz, b.coefs, b.b) for b in mesh.blocks]
    return mesh, F, blocks


@pytest.mark.parametrize("dims,kind", MESHES)
def test_mesh_rhs_is_global_product(dims, kind):
    mesh, F, blocks = _setup(dims, kind, 3)
    A, off = dense_global(mesh)
    xs = np.concatenate([b.xstar for b in mesh.blocks])
    bs = np.concatenate([b.b for b in mesh.blocks])
    assert np.abs(A @ xs - bs).max() <= 1e-13 * np.abs(bs).max()


@pytest.mark.parametrize("dims,kind", MESHES)
def test_first_residual_is_global_residual(dims, kind):
    mesh, F, blocks = _setup(dims, kind, 5)
    A, off = dense_global(mesh)
    rng = np.random.default_rng(2)
    x0 = [rng.uniform(-1, 1, b.n) for b in mesh.blocks]
    xs, it, rel, hist = oracle.solve_multiblock(blocks, mesh.ifaces, F, x0=x0, max_iters=0)
    bs = np.concatenate([b.b for b in mesh.blocks])
    ref = np.linalg.norm(bs - A @ np.concatenate(x0)) / np.linalg.norm(bs)
    assert it == 0
    assert abs(hist[0] - ref) <= 1e-14


@pytest.mark.parametrize("dims,kind", MESHES)
def test_iteration_is_block_jacobi_richardson(dims, kind):
    """x1 = x0 + blockdiag(L_b U_b)^-1 (b - A_global x0)."""
    mesh, F, blocks = _setup(dims, kind, 7)
    A, off = dense_global(mesh)
    M = np.zeros_like(A)
    for q, b in enumerate(mesh.blocks):
        L, U = D.dense_LU(b.nx, b.ny, b.nz, F[q])
        M[off[q]:off[q + 1], off[q]:off[q + 1]] = L @ U
    rng = np.random.default_rng(3)
    x0 = [rng.uniform(-1, 1, b.n) for b in mesh.blocks]
    xs, it, rel, hist = oracle.solve_multiblock(blocks, mesh.ifaces, F, x0=x0, rtol=-1.0, max_iters=1)
    X0 = np.concatenate(x0)
    bs = np.concatenate([b.b for b in mesh.blocks])
    ref = X0 + np.linalg.solve(M, bs - A @ X0)
    got = np.concatenate(xs)
    assert it == 1
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dims,kind", MESHES)
def test_converges_to_dense_global_solution(dims, kind):
    mesh, F, blocks = _setup(dims, kind, 9)
    A, off = dense_global(mesh)
    bs = np.concatenate([b.b for b in mesh.blocks])
    xs, it, rel, hist = oracle.solve_multiblock(blocks, mesh.ifaces, F, rtol=1e-13, max_iters=20000)
    assert rel <= 1e-13
    ref = np.linalg.solve(A, bs)
    assert np.abs(np.concatenate(xs) - ref).max() <= 1e-10 * np.abs(ref).max()


def test_symmetric_entries_read_from_lo_side():
    """sym = 1 takes hi's interface entry from lo's AE (symmetric mesh)."""
    mesh, F, blocks = _setup([(3, 3, 3), (4, 3, 3)], "poisson", 11)
    rng = np.random.default_rng(4)
    x0 = [rng.uniform(-1, 1, b.n) for b in mesh.blocks]
    a = oracle.solve_multiblock(blocks, mesh.ifaces, F, x0=x0, rtol=-1.0, max_iters=3)
    s = oracle.solve_multiblock(blocks, mesh.ifaces, F, x0=x0, rtol=-1.0, max_iters=3, symmetric=True)
    assert all(np.array_equal(p, q) for p, q in zip(a[0], s[0]))
