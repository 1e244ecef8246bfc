"""Pins of the oracle's pressure-correction coefficient assembly (the routine
celp2 of Sec. 3.1, Table 1; its system is the symmetric one of Sec. 4.1)
against facts the finite-volume discretisation fixes: the uniform-grid
closed form (the textbook 7-point Laplacian scaled by h), exact symmetry,
zero row sums away from the Dirichlet face, conservation (interior fluxes
cancel in the sum of b), and a manufactured pressure field whose discrete
gradient velocities give b = A phi."""
import numpy as np
import pytest

import oracle
from paper_1303_4538_gb300 import workloads as W

SHAPES = [(5, 4, 3), (1, 1, 6), (7, 1, 2), (3, 6, 1), (6, 5, 4)]


def _assemble(P):
    return oracle.assemble_pcorr(P.nx, P.ny, P.nz, P.dx, P.dy, P.dz, P.rho, P.g, P.ux, P.uy, P.uz,
                                 P.dirichlet_bottom)


def _grid(c, P):
    return {k: v.reshape(P.nz, P.ny, P.nx) for k, v in c.items()}


@pytest.mark.parametrize("dirichlet", [True, False])
def test_uniform_grid_closed_form(dirichlet):
    """dx = dy = dz = h, rho = g = 1: every interior face has A_nb = -h
    (S = h^2, delta = h); AP = h * (interior neighbours) + 2h on the Dirichlet
    face (half-cell distance h/2)."""
    nx, ny, nz, h = 5, 4, 3, 0.25
    P = W.pcorr_inputs(nx, ny, nz, seed=1, dirichlet_bottom=dirichlet)
    P.dx[:], P.dy[:], P.dz[:] = h, h, h
    P.rho[:] = 1.0
    P.g[:] = 1.0
    c, b = _assemble(P)
    G = _grid(c, P)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    exp = {"aw": np.where(i > 0, -h, 0.0), "ae": np.where(i < nx - 1, -h, 0.0),
           "as": np.where(j > 0, -h, 0.0), "an": np.where(j < ny - 1, -h, 0.0),
           "ab": np.where(k > 0, -h, 0.0), "at": np.where(k < nz - 1, -h, 0.0)}
    nnb = sum((exp[q] != 0).astype(int) for q in exp)
    exp["ap"] = h * nnb + (np.where(k == 0, 2 * h, 0.0) if dirichlet else 0.0)
    for q in W.COEF_NAMES:
        assert np.allclose(G[q], exp[q], rtol=1e-15, atol=0), q


@pytest.mark.parametrize("shape", SHAPES)
def test_symmetric_and_row_sums(shape):
    P = W.pcorr_inputs(*shape, seed=3)
    c, b = _assemble(P)
    G = _grid(c, P)
    # the entry of a face is the same from both of its cells, bit for bit
    assert np.array_equal(G["ae"][:, :, :-1], G["aw"][:, :, 1:])
    assert np.array_equal(G["an"][:, :-1, :], G["as"][:, 1:, :])
    assert np.array_equal(G["at"][:-1, :, :], G["ab"][1:, :, :])
    # boundary faces carry no off-diagonal entry
    assert not G["aw"][:, :, 0].any() and not G["ae"][:, :, -1].any()
    assert not G["as"][:, 0, :].any() and not G["an"][:, -1, :].any()
    assert not G["ab"][0].any() and not G["at"][-1].any()
    off = sum(G[q] for q in W.COEF_NAMES[1:])
    assert np.all(off <= 0)
    rs = G["ap"] + off
    scale = np.abs(G["ap"]).max()
    # zero row sums away from the Dirichlet face, positive on it
    if P.nz > 1:
        assert np.abs(rs[1:]).max() <= 1e-14 * scale
    assert np.all(rs[0] > 0)


@pytest.mark.parametrize("shape", SHAPES)
def test_pure_neumann_is_singular_with_constant_kernel(shape):
    P = W.pcorr_inputs(*shape, seed=4, dirichlet_bottom=False)
    c, b = _assemble(P)
    one = np.ones(P.n)
    Aone = W.apply_matrix(P.nx, P.ny, P.nz, c, one)
    assert np.abs(Aone).max() <= 1e-14 * np.abs(c["ap"]).max()


@pytest.mark.parametrize("shape", SHAPES)
def test_conservation(shape):
    """Interior face fluxes cancel in sum(b): only the open bottom face is
    left, sum(b) = sum over the bottom cells of rho_P u* S_z (walls carry no
    flow)."""
    P = W.pcorr_inputs(*shape, seed=5)
    c, b = _assemble(P)
    Sz = np.outer(P.dy, P.dx)                        # [j, i]
    rho0 = P.rho.reshape(P.nz, P.ny, P.nx)[0]
    ub = P.uz.reshape(P.nz + 1, P.ny, P.nx)[0]
    ref = float(np.sum(rho0 * ub * Sz))
    assert abs(b.sum() - ref) <= 1e-12 * max(np.abs(b).sum(), 1e-300)


@pytest.mark.parametrize("shape", SHAPES)
def test_manufactured_pressure_field(shape):
    """u* = g_f (phi_N - phi_P) / delta_f on interior faces (the velocity the
    pressure correction phi would remove), u* = g_P phi_P / (dz_0 / 2) on the
    Dirichlet face (phi = 0 beyond it), 0 on the walls: then b = A phi."""
    P = W.pcorr_inputs(*shape, seed=6)
    nx, ny, nz = shape
    rng = np.random.default_rng(9)
    phi = rng.uniform(-1, 1, P.n)
    ph = phi.reshape(nz, ny, nx)
    gg = P.g.reshape(nz, ny, nx)
    ux = np.zeros((nz, ny, nx + 1))
    uy = np.zeros((nz, ny + 1, nx))
    uz = np.zeros((nz + 1, ny, nx))
    ux[:, :, 1:nx] = 0.5 * (gg[:, :, 1:] + gg[:, :, :-1]) * (ph[:, :, 1:] - ph[:, :, :-1]) / (
        0.5 * (P.dx[1:] + P.dx[:-1]))[None, None, :]
    uy[:, 1:ny, :] = 0.5 * (gg[:, 1:, :] + gg[:, :-1, :]) * (ph[:, 1:, :] - ph[:, :-1, :]) / (
        0.5 * (P.dy[1:] + P.dy[:-1]))[None, :, None]
    uz[1:nz] = 0.5 * (gg[1:] + gg[:-1]) * (ph[1:] - ph[:-1]) / (0.5 * (P.dz[1:] + P.dz[:-1]))[:, None, None]
    uz[0] = gg[0] * ph[0] / (0.5 * P.dz[0])
    P.ux, P.uy, P.uz = ux.reshape(-1), uy.reshape(-1), uz.reshape(-1)
    c, b = _assemble(P)
    Aphi = W.apply_matrix(nx, ny, nz, c, phi)
    assert np.abs(Aphi - b).max() <= 1e-12 * np.abs(b).max()
    # and the assembled system is symmetric positive definite, solved by phi
    if P.n <= 400:
        from tests import _dense as D
        A = D.dense_A(nx, ny, nz, c)
        assert np.array_equal(A, A.T)
        assert np.linalg.eigvalsh(A).min() > 0
        assert np.abs(np.linalg.solve(A, b) - phi).max() <= 1e-10
