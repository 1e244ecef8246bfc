"""The context's memory pool: a destroyed plan's memory stays cached for the
next plan of the same size (no new device memory is mapped), and sip_trim
returns it to the device.  Free memory is read from the CUDA driver
(cudaMemGetInfo through torch), outside the library."""
import pytest
import torch

from paper_1303_4538_gb300 import sip, workloads as W
from tests._gpu import torch_cuda

pytestmark = pytest.mark.gpu

MB = 1 << 20


def _plan(ctx, blk, A, b, x):
    d = sip.make_desc(blk.nx, blk.ny, blk.nz, [A[0], None, A[2], None, A[4], None, A[6]], b, x, symmetric=True)
    return sip.Plan(ctx, [d], sip.default_options(mode=sip.SIP_MODE_F64))


def test_pool_keeps_peak_then_trim_returns_it():
    torch_cuda()
    blk = W.poisson_256cube(160)   # FP64 plan ~ 0.6 GB + the 0.26 GB factorisation input
    A = [torch.from_numpy(c).cuda() for c in blk.coef_list()]
    b = torch.from_numpy(blk.b).cuda()
    x = torch.zeros(blk.n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    ctx = sip.Context(0, torch.cuda.current_stream().cuda_stream)
    free0 = torch.cuda.mem_get_info()[0]
    p = _plan(ctx, blk, A, b, x)
    nbytes = p.nbytes()
    p.close()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # the peak (plan + factorisation input) stays cached after the plan is gone
    assert free0 - free1 >= nbytes - 64 * MB
    # a second plan of the same size maps nothing new
    p = _plan(ctx, blk, A, b, x)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free1) <= 64 * MB
    rel = p.iterate(1)
    assert rel == pytest.approx(1.0)
    p.close()
    ctx.trim()
    free2 = torch.cuda.mem_get_info()[0]
    assert free2 >= free0 - 64 * MB
    ctx.close()
