"""sip_residual_norm (||b - A x||_2, ||b||_2 on the natural layout) against the
oracle's residual, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1303_4538_gb300 import sip, workloads
from tests._gpu import GpuSystem, torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (5, 4, 3), (17, 31, 9), (64, 64, 1), (65, 64, 1), (40, 70, 21)]


def _desc(torch, blk, x, sym_null=False, coef_f32=False):
    cdt = torch.float32 if coef_f32 else torch.float64
    A = [torch.from_numpy(np.ascontiguousarray(c)).to("cuda", cdt) for c in blk.coef_list()]
    b = torch.from_numpy(blk.b).cuda()
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    coefs = list(A)
    if sym_null:
        coefs[1] = coefs[3] = coefs[5] = None
    d = sip.make_desc(blk.nx, blk.ny, blk.nz, coefs, b, xd, symmetric=blk.symmetric,
                      coef_dtype=1 if coef_f32 else 0)
    return d, (A, b, xd)


def _oracle_norms(blk, x, coef_f32=False):
    coefs = blk.coef_list()
    if coef_f32:
        coefs = [np.asarray(c, dtype=np.float32).astype(np.float64) for c in coefs]
    _, rn = oracle.residual(blk.nx, blk.ny, blk.nz, coefs, blk.b, x)
    return rn, float(np.sqrt(oracle.lib().oracle_dot_sq(blk.n, oracle._p(np.ascontiguousarray(blk.b)))))


@pytest.fixture(scope="module")
def ctx():
    torch = torch_cuda()
    c = sip.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["convdiff", "poisson"])
def test_matches_oracle(ctx, shape, kind):
    torch = torch_cuda()
    blk = workloads.make_block(*shape, seed=11, kind=kind)
    x = np.random.default_rng(5).uniform(-1, 1, blk.n)
    d, keep = _desc(torch, blk, x, sym_null=blk.symmetric)
    rn, bn = ctx.residual_norm(d)
    orn, obn = _oracle_norms(blk, x)
    assert abs(rn - orn) <= 1e-12 * orn
    assert abs(bn - obn) <= 1e-13 * obn


def test_fp32_coefficients(ctx):
    torch = torch_cuda()
    blk = workloads.make_block(33, 35, 18, seed=12, kind="convdiff")
    x = np.random.default_rng(6).uniform(-1, 1, blk.n)
    d, keep = _desc(torch, blk, x, coef_f32=True)
    rn, _ = ctx.residual_norm(d)
    orn, _ = _oracle_norms(blk, x, coef_f32=True)
    assert abs(rn - orn) <= 1e-12 * orn


def test_symmetric_general_agree(ctx):
    """A symmetric matrix read in full and in the upper-entries form (Listing 1)."""
    torch = torch_cuda()
    blk = workloads.make_block(23, 19, 12, seed=13, kind="poisson")
    x = np.random.default_rng(7).uniform(-1, 1, blk.n)
    d1, k1 = _desc(torch, blk, x, sym_null=True)
    blk.symmetric = False
    d2, k2 = _desc(torch, blk, x)
    r1, _ = ctx.residual_norm(d1)
    r2, _ = ctx.residual_norm(d2)
    assert abs(r1 - r2) <= 1e-13 * r2


def test_bitwise_reproducible(ctx):
    torch = torch_cuda()
    blk = workloads.make_block(40, 70, 21, seed=14, kind="convdiff")
    x = np.random.default_rng(8).uniform(-1, 1, blk.n)
    d, keep = _desc(torch, blk, x)
    a = ctx.residual_norm(d)
    b = ctx.residual_norm(d)
    assert a == b


def test_solution_relres_agrees_with_solver():
    """The relres a solve reports is that of the x it returns (stop rule C7)."""
    blk = workloads.make_block(24, 20, 16, seed=4539, kind="convdiff")
    g = GpuSystem(blk)
    it, rel, conv = g.plan.solve(1e-8, 200)
    d = sip.make_desc(blk.nx, blk.ny, blk.nz, g.A[0], g.b[0], g.x[0])
    rn, bn = g.ctx.residual_norm(d)
    assert abs(rn / bn - rel) <= 1e-12
    g.close()


def test_full_size_poisson_256(ctx):
    torch = torch_cuda()
    blk = workloads.poisson_256cube()
    x = np.random.default_rng(9).uniform(-1, 1, blk.n)
    d, keep = _desc(torch, blk, x, sym_null=True)
    rn, bn = ctx.residual_norm(d)
    A = blk.coef_list()
    _, orn = oracle.residual_sym(blk.nx, blk.ny, blk.nz, A[0], A[2], A[4], A[6], blk.b, x)
    assert abs(rn - orn) <= 1e-12 * orn


def test_invalid_descriptors(ctx):
    torch = torch_cuda()
    blk = workloads.make_block(5, 4, 3, seed=15, kind="convdiff")
    x = np.zeros(blk.n)
    d, keep = _desc(torch, blk, x)
    for field, val in (("nx", 0), ("coef_dtype", 3), ("x", None), ("aw", None)):
        bad = sip.sip_block_desc.from_buffer_copy(d)
        setattr(bad, field, val)
        with pytest.raises(sip.SipError) as e:
            ctx.residual_norm(bad)
        assert e.value.code == sip.SIP_ERR_INVALID_ARG
