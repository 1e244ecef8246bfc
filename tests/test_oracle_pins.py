"""Pins of the CPU oracle against mathematics that does not come from the
oracle itself (dense linear algebra, textbook ILU(0), closed forms).

The SIP being pinned is Stone's method as used by the paper's solver
(arXiv:1303.4538, Sec. 1: Stone's SIP, an incomplete LU factorisation;
Sec. 4.1: factorisation once, symmetric residual of Listing 1,
single-precision relaxation).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1303_4538_gb300 import workloads as W
from tests import _dense as D

SHAPES = [(4, 3, 5), (2, 3, 2), (1, 4, 3), (3, 1, 4), (5, 4, 1), (3, 3, 3)]


def _block(shape, seed, kind="convdiff"):
    return W.make_block(*shape, seed=seed, kind=kind)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("alpha", [0.92, 0.5, 1.0])
@pytest.mark.parametrize("kind", ["convdiff", "poisson"])
def test_LU_equals_A_plus_stone_auxiliary_matrix(shape, alpha, kind):
    """L U = A + N with N Stone's auxiliary matrix: on each stencil diagonal
    N is -alpha times the sum of the two fill entries that the neighbour
    flanks, on the main diagonal +alpha times all six, on each fill diagonal
    the fill entry itself, and zero elsewhere."""
    nx, ny, nz = shape
    blk = _block(shape, 11 + sum(shape), kind)
    F = oracle.factor(nx, ny, nz, blk.coefs, alpha)
    A = D.dense_A(nx, ny, nz, blk.coefs)
    L, U = D.dense_LU(nx, ny, nz, F)
    M = L @ U
    Delta = M - A
    scale = np.abs(A).max()
    expect = np.zeros_like(A)
    for i, j, k in D.cells(nx, ny, nz):
        p = D.idx(nx, ny, i, j, k)
        c = {}
        for name, ((di, dj, dk), _) in D.FILLS.items():
            q = (i + di, j + dj, k + dk)
            c[name] = M[p, D.idx(nx, ny, *q)] if D.inside(nx, ny, nz, *q) else 0.0
            if D.inside(nx, ny, nz, *q):
                expect[p, D.idx(nx, ny, *q)] = c[name]
        for nb, (di, dj, dk) in D.OFF.items():
            q = (i + di, j + dj, k + dk)
            if not D.inside(nx, ny, nz, *q):
                continue
            flank = sum(c[name] for name, (_, pair) in D.FILLS.items() if nb in pair)
            expect[p, D.idx(nx, ny, *q)] = -alpha * flank
        expect[p, p] = alpha * sum(c.values())
    assert np.abs(Delta - expect).max() <= 1e-13 * scale


@pytest.mark.parametrize("shape", [(4, 3, 5), (3, 3, 3), (5, 4, 2)])
def test_alpha_one_annihilates_linear_fields(shape):
    """Stone's design: with alpha = 1 the auxiliary matrix N = L U - A
    vanishes on every linear field x = c0 + c1 i + c2 j + c3 k (the
    extrapolation x_fill = x_a + x_b - x_P is exact there), but not on a
    random field."""
    nx, ny, nz = shape
    blk = _block(shape, 7)
    F = oracle.factor(nx, ny, nz, blk.coefs, 1.0)
    A = D.dense_A(nx, ny, nz, blk.coefs)
    L, U = D.dense_LU(nx, ny, nz, F)
    N = L @ U - A
    g = np.array([[0.3 - 0.7 * i + 1.1 * j + 0.45 * k for i in range(nx)] for k in range(nz) for j in range(ny)])
    lin = np.array([0.3 - 0.7 * i + 1.1 * j + 0.45 * k for i, j, k in D.cells(nx, ny, nz)])
    assert np.abs(N @ lin).max() <= 1e-12 * np.abs(A).max()
    rnd = np.random.default_rng(3).uniform(-1, 1, nx * ny * nz)
    assert np.abs(N @ rnd).max() > 1e-3


@pytest.mark.parametrize("shape", [(4, 3, 5), (3, 4, 2), (2, 2, 6)])
def test_alpha_zero_is_textbook_ilu0(shape):
    """alpha = 0: SIP's factorisation is ILU(0) on the 7-point pattern."""
    nx, ny, nz = shape
    blk = _block(shape, 21)
    F = oracle.factor(nx, ny, nz, blk.coefs, 0.0)
    A = D.dense_A(nx, ny, nz, blk.coefs)
    L, U = D.dense_LU(nx, ny, nz, F)
    M_ilu = D.ilu0(A, D.pattern7(nx, ny, nz))
    assert np.abs(L @ U - M_ilu).max() <= 1e-13 * np.abs(A).max()


@pytest.mark.parametrize("shape", [(9, 1, 1), (1, 7, 1), (1, 1, 11)])
def test_single_grid_line_is_exact_lu(shape):
    """On one grid line there are no fill entries: one iteration from x = 0
    solves A x = b to rounding (the Thomas algorithm)."""
    nx, ny, nz = shape
    blk = _block(shape, 5)
    F = oracle.factor(nx, ny, nz, blk.coefs, 0.92)
    x = np.zeros(nx * ny * nz)
    oracle.iterate(nx, ny, nz, blk.coefs, F, blk.b, x)
    A = D.dense_A(nx, ny, nz, blk.coefs)
    ref = np.linalg.solve(A, blk.b)
    assert np.abs(x - ref).max() <= 1e-13 * np.abs(ref).max()


def test_golden_poisson1d_closed_form():
    path = os.path.join(os.path.dirname(__file__), "golden", "poisson1d_n8.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    xs = np.array([float(r[1]) for r in rows])
    n = xs.size
    coefs = {k: np.zeros(n) for k in W.COEF_NAMES}
    coefs["ap"][:] = 2.0
    coefs["aw"][1:] = -1.0
    coefs["ae"][:-1] = -1.0
    F = oracle.factor(n, 1, 1, coefs, 0.92)
    x = np.zeros(n)
    rn = oracle.iterate(n, 1, 1, coefs, F, np.ones(n), x)
    assert rn == pytest.approx(np.sqrt(n))
    assert np.abs(x - xs).max() <= 1e-13 * xs.max()


@pytest.mark.parametrize("shape", [(4, 3, 5), (3, 3, 3), (6, 2, 3)])
@pytest.mark.parametrize("kind", ["convdiff", "poisson"])
def test_iteration_is_preconditioned_richardson(shape, kind):
    """One SIP iteration is x + (L U)^{-1} (b - A x), by dense solves."""
    nx, ny, nz = shape
    blk = _block(shape, 31, kind)
    F = oracle.factor(nx, ny, nz, blk.coefs, 0.92)
    A = D.dense_A(nx, ny, nz, blk.coefs)
    L, U = D.dense_LU(nx, ny, nz, F)
    x0 = np.random.default_rng(1).uniform(-1, 1, nx * ny * nz)
    x = x0.copy()
    rn = oracle.iterate(nx, ny, nz, blk.coefs, F, blk.b, x)
    r = blk.b - A @ x0
    ref = x0 + np.linalg.solve(L @ U, r)
    assert rn == pytest.approx(np.linalg.norm(r), rel=1e-13)
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("shape", [(4, 3, 5), (5, 5, 4)])
@pytest.mark.parametrize("kind", ["convdiff", "poisson"])
def test_converges_to_dense_solution(shape, kind):
    nx, ny, nz = shape
    blk = _block(shape, 41, kind)
    F = oracle.factor(nx, ny, nz, blk.coefs, 0.92)
    A = D.dense_A(nx, ny, nz, blk.coefs)
    L, U = D.dense_LU(nx, ny, nz, F)
    G = np.eye(A.shape[0]) - np.linalg.solve(L @ U, A)
    assert np.abs(np.linalg.eigvals(G)).max() < 1.0
    x, it, rel, hist = oracle.solve(nx, ny, nz, blk.coefs, F, blk.b, rtol=1e-13, max_iters=5000)
    assert rel <= 1e-13 and it < 5000
    ref = np.linalg.solve(A, blk.b)
    assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()
    # manufactured solution recovered within the conditioning of A
    err = np.linalg.norm(x - blk.xstar) / np.linalg.norm(blk.xstar)
    assert err <= np.linalg.cond(A) * 1e-13 * 10


def test_manufactured_solution_8cube():
    nx = ny = nz = 8
    blk = W.make_block(nx, ny, nz, seed=4539, kind="convdiff")
    F = oracle.factor(nx, ny, nz, blk.coefs, 0.92)
    x, it, rel, _ = oracle.solve(nx, ny, nz, blk.coefs, F, blk.b, rtol=1e-10, max_iters=20000)
    assert rel <= 1e-10
    A = D.dense_A(nx, ny, nz, blk.coefs)
    err = np.linalg.norm(x - blk.xstar) / np.linalg.norm(blk.xstar)
    assert err <= np.linalg.cond(A) * 1e-10


def test_stop_rule_and_history():
    nx, ny, nz = 5, 4, 3
    blk = _block((nx, ny, nz), 51, "poisson")
    F = oracle.factor(nx, ny, nz, blk.coefs, 0.92)
    x, it, rel, hist = oracle.solve(nx, ny, nz, blk.coefs, F, blk.b, rtol=1e-6, max_iters=1000)
    assert hist.size == it + 1 and hist[-1] == rel <= 1e-6 and (hist[:-1] > 1e-6).all()
    A = D.dense_A(nx, ny, nz, blk.coefs)
    assert rel == pytest.approx(np.linalg.norm(blk.b - A @ x) / np.linalg.norm(blk.b), rel=1e-10)
    # already converged: no update, x returned unchanged
    x2, it2, rel2, _ = oracle.solve(nx, ny, nz, blk.coefs, F, blk.b, x0=x, rtol=1e-6, max_iters=10)
    assert it2 == 0 and np.array_equal(x2, x)
    # iteration cap
    _, it3, rel3, h3 = oracle.solve(nx, ny, nz, blk.coefs, F, blk.b, rtol=0.0, max_iters=7)
    assert it3 == 7 and h3.size == 8


def test_symmetric_residual_matches_general_residual():
    """Listing 1's residual, which reads only the east, north and top
    coefficients, equals the general residual for a symmetric matrix, and
    differs from it for a non-symmetric one."""
    nx, ny, nz = 6, 5, 4
    sym = W.make_block(nx, ny, nz, seed=61, kind="poisson")
    A = D.dense_A(nx, ny, nz, sym.coefs)
    assert np.array_equal(A, A.T)
    x = np.random.default_rng(2).uniform(-1, 1, nx * ny * nz)
    c = sym.coefs
    r1, n1 = oracle.residual(nx, ny, nz, c, sym.b, x)
    r2, n2 = oracle.residual_sym(nx, ny, nz, c["ap"], c["ae"], c["an"], c["at"], sym.b, x)
    assert np.abs(r1 - r2).max() <= 1e-14 * np.abs(r1).max()
    assert np.abs(r1 - (sym.b - A @ x)).max() <= 1e-13 * np.abs(r1).max()
    ns = W.make_block(nx, ny, nz, seed=61, kind="convdiff")
    c = ns.coefs
    r3, _ = oracle.residual(nx, ny, nz, c, ns.b, x)
    r4, _ = oracle.residual_sym(nx, ny, nz, c["ap"], c["ae"], c["an"], c["at"], ns.b, x)
    assert np.abs(r3 - r4).max() > 1e-3


def test_norm_matches_library():
    v = np.random.default_rng(9).standard_normal(10001) * 1e3
    assert oracle.norm2(v) == pytest.approx(np.linalg.norm(v), rel=1e-15)


def test_breakdown_detected():
    nx, ny, nz = 3, 1, 1
    coefs = {k: np.zeros(3) for k in W.COEF_NAMES}
    coefs["ap"][:] = [1.0, 1.0, 2.0]
    coefs["ae"][:2] = [1.0, -1.0]
    coefs["aw"][1:] = [1.0, -1.0]   # second pivot: 1 - 1*1/1 = 0
    with pytest.raises(oracle.BreakdownError):
        oracle.factor(nx, ny, nz, coefs, 0.92)


def test_single_precision_iteration_tracks_fp64():
    nx, ny, nz = 7, 6, 5
    blk = W.make_block(nx, ny, nz, seed=71, kind="convdiff")
    F = oracle.factor(nx, ny, nz, blk.coefs, 0.92)
    F32 = oracle.factors_f32(F)
    c32 = {k: v.astype(np.float32) for k, v in blk.coefs.items()}
    x = np.zeros(blk.n)
    x32 = np.zeros(blk.n, np.float32)
    for it in range(5):
        oracle.iterate(nx, ny, nz, blk.coefs, F, blk.b, x)
        oracle.iterate_f32(nx, ny, nz, c32, F32, blk.b.astype(np.float32), x32)
        assert np.abs(x32 - x).max() <= 1e-5 * np.abs(x).max()
    # the first float iteration from zero skips the matrix product
    y1 = np.zeros(blk.n, np.float32)
    y2 = np.zeros(blk.n, np.float32)
    oracle.iterate_f32(nx, ny, nz, c32, F32, blk.b.astype(np.float32), y1, x_is_zero=True)
    oracle.iterate_f32(nx, ny, nz, c32, F32, blk.b.astype(np.float32), y2, x_is_zero=False)
    assert np.array_equal(y1, y2)


@pytest.mark.parametrize("kind", ["convdiff", "poisson"])
def test_single_precision_solve_tracks_then_stagnates(kind):
    """The paper's FP32 relaxation follows the FP64 relres history while it is
    far above float resolution; on the fast-converging Poisson system it then
    stagnates near the float level while FP64 keeps converging."""
    nx, ny, nz = 9, 8, 7
    blk = W.make_block(nx, ny, nz, seed=73, kind=kind)
    F = oracle.factor(nx, ny, nz, blk.coefs, 0.92)
    F32 = oracle.factors_f32(F)
    c32 = {k: v.astype(np.float32) for k, v in blk.coefs.items()}
    x64, it64, rel64, h64 = oracle.solve(nx, ny, nz, blk.coefs, F, blk.b, rtol=-1.0, max_iters=200)
    x32, it32, rel32, h32 = oracle.solve_f32(nx, ny, nz, c32, F32, blk.b, rtol=-1.0, max_iters=200)
    assert it32 == 200 and len(h32) == 201
    big = h64 > 1e-4
    assert np.all(np.abs(h32[big] - h64[big]) <= 1e-4 * h64[big] + 1e-6)
    if kind == "poisson":
        assert 1e-9 < h32[-1] < 1e-6            # stagnation at the float level
        assert h64[-1] < 1e-12                   # while FP64 keeps converging
        assert np.abs(x32 - blk.xstar).max() <= 1e-5
    # stop rule: with a reachable tolerance the float solve stops like the FP64 one
    _, itA, relA, _ = oracle.solve_f32(nx, ny, nz, c32, F32, blk.b, rtol=1e-3, max_iters=200)
    assert relA <= 1e-3 and h32[itA] == relA and h32[itA - 1] > 1e-3


@pytest.mark.parametrize("m", [1, 2, 4, 8])
def test_refinement_reaches_fp64_solution(m):
    nx, ny, nz = 8, 7, 6
    blk = W.make_block(nx, ny, nz, seed=81, kind="poisson")
    F = oracle.factor(nx, ny, nz, blk.coefs, 0.92)
    c32 = {k: v.astype(np.float32) for k, v in blk.coefs.items()}
    x, outer, rel, hist = oracle.solve_refined(nx, ny, nz, blk.coefs, c32, oracle.factors_f32(F), blk.b,
                                               rtol=1e-10, max_outer=5000, m_inner=m)
    assert rel <= 1e-10
    A = D.dense_A(nx, ny, nz, blk.coefs)
    assert rel == pytest.approx(np.linalg.norm(blk.b - A @ x) / np.linalg.norm(blk.b), rel=1e-8)
    ref = np.linalg.solve(A, blk.b)
    assert np.abs(x - ref).max() <= np.linalg.cond(A) * 1e-10 * np.abs(ref).max()
