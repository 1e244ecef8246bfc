"""The seeded input generators (workloads.py) against the recipe they state:
finite-volume 7-point structure (off-diagonals from one conductance per
face, first-order upwind convection, AP the sum of the neighbour magnitudes
plus the Dirichlet / time terms), symmetry of the Poisson systems, zero
entries toward the outside of a block, b = A x* by an independent dense
product, the median cell Peclet number of the Peclet-10 generator, and the
size constraints of the 64-block mesh.  CPU only."""
import numpy as np
import pytest

from paper_1303_4538_gb300 import workloads as W


def _dense(blk):
    """Dense A of a block from its diagonals (natural order), built cell by cell."""
    nx, ny, nz = blk.nx, blk.ny, blk.nz
    n = blk.n
    A = np.zeros((n, n))
    c = blk.coefs
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                p = i + nx * (j + ny * k)
                A[p, p] = c["ap"][p]
                for name, di, dj, dk in (("aw", -1, 0, 0), ("ae", 1, 0, 0), ("as", 0, -1, 0),
                                         ("an", 0, 1, 0), ("ab", 0, 0, -1), ("at", 0, 0, 1)):
                    ii, jj, kk = i + di, j + dj, k + dk
                    if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                        A[p, ii + nx * (jj + ny * kk)] = c[name][p]
                    else:
                        assert c[name][p] == 0.0, (name, i, j, k)
    return A


@pytest.mark.parametrize("kind", ["poisson", "convdiff"])
@pytest.mark.parametrize("shape", [(5, 4, 3), (1, 6, 2), (7, 1, 1)])
def test_rhs_is_dense_product_and_outside_entries_are_zero(kind, shape):
    blk = W.make_block(*shape, seed=17, kind=kind)
    A = _dense(blk)
    assert np.allclose(A @ blk.xstar, blk.b, rtol=1e-14, atol=1e-14)
    assert blk.xstar.min() >= -1.0 and blk.xstar.max() <= 1.0


@pytest.mark.parametrize("kind", ["poisson", "convdiff"])
def test_diagonal_is_neighbour_sum_plus_boundary_and_time_terms(kind):
    nx, ny, nz = 6, 5, 4
    blk = W.make_block(nx, ny, nz, seed=23, kind=kind)
    c = {k: v.reshape(nz, ny, nx) for k, v in blk.coefs.items()}
    off = sum(np.abs(c[k]) for k in ("aw", "ae", "as", "an", "ab", "at"))
    extra = c["ap"] - off
    for k in ("aw", "ae", "as", "an", "ab", "at"):
        assert (c[k] <= 0).all()
    if kind == "convdiff":
        assert np.allclose(extra, 0.01, rtol=0, atol=1e-13)
    else:
        # the Dirichlet conductance U[0.5, 2] on the bottom face only
        assert np.allclose(extra[1:], 0.0, atol=1e-13)
        assert (extra[0] >= 0.5).all() and (extra[0] <= 2.0).all()


def test_poisson_is_symmetric():
    blk = W.make_block(6, 5, 4, seed=29, kind="poisson")
    A = _dense(blk)
    assert blk.symmetric
    assert np.array_equal(A, A.T)


def test_convection_entries_are_first_order_upwind_of_one_face_flux():
    """Across an x face P|E: AE(P) = -(D + max(-F, 0)) and AW(E) = -(D + max(F, 0)),
    so AE(P) - AW(E) = F and AE(P) + AW(E) = -(2 D + |F|) with D in [0.5, 2]."""
    nx, ny, nz = 6, 5, 4
    blk = W.make_block(nx, ny, nz, seed=31, kind="convdiff")
    c = {k: v.reshape(nz, ny, nx) for k, v in blk.coefs.items()}
    for up, dn, sl_p, sl_e in (("ae", "aw", np.s_[:, :, :-1], np.s_[:, :, 1:]),
                               ("an", "as", np.s_[:, :-1, :], np.s_[:, 1:, :]),
                               ("at", "ab", np.s_[:-1, :, :], np.s_[1:, :, :])):
        a, b = c[up][sl_p], c[dn][sl_e]
        F = a - b
        twoD = -(a + b) - np.abs(F)
        assert (twoD >= 1.0 - 1e-12).all() and (twoD <= 4.0 + 1e-12).all()
        # one of the two entries is the pure diffusion term -D
        assert np.allclose(np.maximum(a, b), -twoD / 2, atol=1e-12)


def test_peclet_generator_has_the_stated_median():
    blk = W.make_block(40, 40, 40, seed=4542, kind="convdiff", pe=10.0)
    c = {k: v.reshape(40, 40, 40) for k, v in blk.coefs.items()}
    a, b = c["ae"][:, :, :-1], c["aw"][:, :, 1:]
    F = a - b
    D = (-(a + b) - np.abs(F)) / 2
    pe = np.median(np.abs(F) / D)
    assert 9.5 < pe < 10.5


def test_generators_are_deterministic_per_seed():
    a = W.make_block(8, 7, 6, seed=5, kind="convdiff")
    b = W.make_block(8, 7, 6, seed=5, kind="convdiff")
    c = W.make_block(8, 7, 6, seed=6, kind="convdiff")
    for k in W.COEF_NAMES:
        assert np.array_equal(a.coefs[k], b.coefs[k])
    assert np.array_equal(a.b, b.b)
    assert not np.array_equal(a.b, c.b)


def test_batched_mesh_sizes_follow_the_recipe():
    dims, t = W.batched_mesh_dims()
    assert dims.shape == (64, 3)
    assert dims.min() >= 24 and dims.max() <= 128
    tot = int(np.prod(dims, axis=1).sum())
    assert 18_000_000 <= tot <= 22_000_000
    # the first admissible redraw: every earlier one falls outside the range
    for s in range(t):
        rng = np.random.Generator(np.random.PCG64(4541 + 1000 * s))
        d = W.random_block_dims(rng, 64, 24, 128)
        assert not 18_000_000 <= int(np.prod(d, axis=1).sum()) <= 22_000_000


def test_mesh_interfaces_couple_lo_east_to_hi_west():
    mesh = W.make_mesh([(4, 3, 2), (3, 4, 3)], seed=77, kind="convdiff")
    (lo, hi, nj, nk), = mesh.ifaces
    assert (lo, hi, nj, nk) == (0, 1, 3, 2)
    L, H = mesh.blocks
    for k in range(nk):
        for j in range(nj):
            pl = (L.nx - 1) + L.nx * (j + L.ny * k)
            ph = H.nx * (j + H.ny * k)
            assert L.coefs["ae"][pl] < 0 and H.coefs["aw"][ph] < 0
    # outside the overlap rectangle the x-face entries stay zero
    for k in range(L.nz):
        for j in range(L.ny):
            if j >= nj or k >= nk:
                assert L.coefs["ae"][(L.nx - 1) + L.nx * (j + L.ny * k)] == 0.0
