"""sip_residual_norm_noalloc (static device scratch, no allocation) against
sip_residual_norm (per-call scratch) through the C ABI: two consecutive calls
on the same block must both agree with the allocating entry point."""
import numpy as np
import pytest

from paper_1303_4538_gb300 import sip, workloads
from tests._gpu import torch_cuda

pytestmark = pytest.mark.gpu

CASES = [((40, 70, 21), "convdiff", False), ((64, 48, 33), "poisson", False), ((33, 35, 18), "convdiff", True)]


def _desc(torch, blk, x, coef_f32):
    cdt = torch.float32 if coef_f32 else torch.float64
    A = [torch.from_numpy(np.ascontiguousarray(c)).to("cuda", cdt) for c in blk.coef_list()]
    b = torch.from_numpy(blk.b).cuda()
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    coefs = list(A)
    if blk.symmetric:
        coefs[1] = coefs[3] = coefs[5] = None
    d = sip.make_desc(blk.nx, blk.ny, blk.nz, coefs, b, xd, symmetric=blk.symmetric,
                      coef_dtype=1 if coef_f32 else 0)
    return d, (A, b, xd)


@pytest.mark.parametrize("shape,kind,coef_f32", CASES)
def test_two_calls_match_allocating_entry_point(shape, kind, coef_f32):
    torch = torch_cuda()
    ctx = sip.Context(0, torch.cuda.current_stream().cuda_stream)
    blk = workloads.make_block(*shape, seed=21, kind=kind)
    x = np.random.default_rng(22).uniform(-1, 1, blk.n)
    d, keep = _desc(torch, blk, x, coef_f32)
    rn, bn = ctx.residual_norm(d)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        ctx.residual_norm_noalloc(d, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # same kernels, chunking and summation order as sip_residual_norm: same bits
        assert got[0] == rn and got[1] == bn, (got, rn, bn)
    ctx.close()


def test_rejects_blocks_beyond_the_scratch():
    """One 4096-cell chunk beyond the limit is rejected before any launch.  The
    descriptor is backed by real arrays of its full size, so a broken size
    check would compute on valid memory instead of reading past the tensors."""
    torch = torch_cuda()
    ctx = sip.Context(0, torch.cuda.current_stream().cuda_stream)
    nx, ny, nz = 4096, 16385, 1
    n = nx * ny * nz
    assert n == sip.SIP_NOALLOC_MAX_CELLS + 4096
    a = torch.zeros(n, dtype=torch.float32, device="cuda")  # AP, AE, AN, AT (symmetric, FP32)
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    d = sip.make_desc(nx, ny, nz, [a, None, a, None, a, None, a], b, x, symmetric=True, coef_dtype=1)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(sip.SipError) as e:
        ctx.residual_norm_noalloc(d, out)
    assert e.value.code == sip.SIP_ERR_INVALID_ARG
    assert str(sip.SIP_NOALLOC_MAX_CELLS) in str(e.value)
    del a, b, x
    torch.cuda.empty_cache()
    ctx.close()


def test_rejects_bad_output_pointers():
    """A host pointer or a misaligned device pointer for the two norms is an
    argument error (nothing is launched), checked in the C library itself."""
    torch = torch_cuda()
    ctx = sip.Context(0, torch.cuda.current_stream().cuda_stream)
    blk = workloads.make_block(8, 6, 5, seed=3, kind="poisson")
    d, keep = _desc(torch, blk, np.zeros(blk.n), False)
    host = torch.zeros(2, dtype=torch.float64)
    dev = torch.zeros(4, dtype=torch.float64, device="cuda")
    for ptr in (int(host.data_ptr()), int(dev.data_ptr()) + 4):
        with pytest.raises(sip.SipError) as e:
            ctx.residual_norm_noalloc(d, ptr)
        assert e.value.code == sip.SIP_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        ctx.residual_norm_noalloc(d, host)
    ctx.close()
