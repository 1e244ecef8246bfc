"""A single block of more than 2^29 cells: 256 x 256 x 8193 = 536,936,448.

Record offsets (four values a cell) pass 2^31 in such a block, so this case
guards the 64-bit scaling of record addresses in the sweeps.  The block is a
stack of decoupled planes: AB = AT = 0, so the incomplete factors and every
SIP iterate of plane k depend on plane k alone (Eq. 5-9 with the k-neighbour
terms zero) and the oracle can check the whole block plane by plane.  Plane k
carries the 2-D Poisson plane P (seeded generator, Dirichlet conductances on
AP) scaled by s[k % 3] and the right-hand side b0 * c[k % 5]: fifteen
distinct plane systems, each checked against its own oracle run on every
plane that carries it, including the last planes (offsets above 2^30
cells, records above 2^32 values).  The residual norm of the whole block is
checked against the plane norms summed over the fifteen classes."""
import numpy as np
import pytest

import oracle
from paper_1303_4538_gb300 import sip, workloads as W
from tests._gpu import torch_cuda

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NX, NY, NZ = 256, 256, 8193
SCALES = (1.0, 1.25, 1.5)
RHS = (1.0, 2.0, 3.0, 4.0, 5.0)
NCLS = 15
ALPHA = 0.92


def _plane_system(cls, plane):
    s, c = SCALES[cls % 3], RHS[cls % 5]
    coefs = {k: v * s for k, v in plane.coefs.items()}
    return coefs, plane.b * c


@pytest.fixture(scope="module")
def tall():
    torch = torch_cuda()
    assert NX * NY * NZ > 2 ** 29
    plane = W.make_block(NX, NY, 1, seed=4561, kind="poisson")
    assert not plane.coefs["ab"].any() and not plane.coefs["at"].any()
    kk = torch.arange(NZ, device="cuda")
    s = torch.tensor(SCALES, dtype=torch.float64, device="cuda")[kk % 3][:, None]
    c = torch.tensor(RHS, dtype=torch.float64, device="cuda")[kk % 5][:, None]
    dev = {}
    for name in ("ap", "ae", "an"):
        dev[name] = (torch.from_numpy(plane.coefs[name]).cuda()[None, :] * s).reshape(-1)
    dev["at"] = torch.zeros(NX * NY * NZ, dtype=torch.float64, device="cuda")
    b = (torch.from_numpy(plane.b).cuda()[None, :] * c).reshape(-1)
    x = torch.zeros(NX * NY * NZ, dtype=torch.float64, device="cuda")
    counts = np.array([len(range(r, NZ, NCLS)) for r in range(NCLS)], dtype=np.float64)
    yield plane, dev, b, x, counts
    del dev, b, x
    torch.cuda.empty_cache()


def _plan(torch, dev, b, x, mode):
    ctx = sip.Context(0, torch.cuda.current_stream().cuda_stream)
    coefs = [dev["ap"], None, dev["ae"], None, dev["an"], None, dev["at"]]
    d = sip.make_desc(NX, NY, NZ, coefs, b, x, symmetric=True)
    plan = sip.Plan(ctx, [d], sip.default_options(alpha=ALPHA, mode=mode, inner_iters=4))
    return ctx, plan


def _check_planes(torch, x, expect, tol):
    """max over every plane of |x - expected| against tol * max |expected|."""
    xv = x.view(NZ, NX * NY)
    for r in range(NCLS):
        e = torch.from_numpy(expect[r]).cuda()
        err = (xv[r::NCLS] - e[None, :]).abs().max().item()
        assert err <= tol * np.abs(expect[r]).max(), (r, err)
    # the last plane by itself (cell offsets above 2^30 - its class is 8192 % 15)
    last = (NZ - 1) % NCLS
    err = (xv[NZ - 1] - torch.from_numpy(expect[last]).cuda()).abs().max().item()
    assert err <= tol * np.abs(expect[last]).max()


def test_fp64_two_iterations_every_plane(tall):
    torch = torch_cuda()
    plane, dev, b, x, counts = tall
    x.zero_()
    ctx, plan = _plan(torch, dev, b, x, sip.SIP_MODE_F64)
    expect, rn1, rn2, bn2 = [], np.zeros(NCLS), np.zeros(NCLS), np.zeros(NCLS)
    for r in range(NCLS):
        coefs, bp = _plane_system(r, plane)
        F = oracle.factor(NX, NY, 1, coefs, ALPHA)
        xp = np.zeros(NX * NY)
        rn1[r] = oracle.iterate(NX, NY, 1, coefs, F, bp, xp)
        rn2[r] = oracle.iterate(NX, NY, 1, coefs, F, bp, xp)
        bn2[r] = oracle.norm2(bp) ** 2
        expect.append(xp)
    bn = np.sqrt((counts * bn2).sum())
    rel1 = plan.iterate(1)
    rel2 = plan.iterate(1)
    plan.close()
    ctx.close()
    assert abs(rel1 - np.sqrt((counts * rn1 ** 2).sum()) / bn) <= 1e-12
    assert abs(rel2 - np.sqrt((counts * rn2 ** 2).sum()) / bn) <= 1e-12
    _check_planes(torch, x, expect, 1e-12)


def test_fp32_two_iterations_every_plane(tall):
    torch = torch_cuda()
    plane, dev, b, x, counts = tall
    x.zero_()
    ctx, plan = _plan(torch, dev, b, x, sip.SIP_MODE_F32)
    plan.iterate(2)
    plan.close()
    ctx.close()
    expect = []
    for r in range(NCLS):
        coefs, bp = _plane_system(r, plane)
        F32 = oracle.factors_f32(oracle.factor(NX, NY, 1, coefs, ALPHA))
        c32 = {k: v.astype(np.float32) for k, v in coefs.items()}
        xp, _, _, _ = oracle.solve_f32(NX, NY, 1, c32, F32, bp, rtol=-1.0, max_iters=2)
        expect.append(np.asarray(xp, dtype=np.float64))
    _check_planes(torch, x, expect, 1e-5)


def test_refined_one_correction_every_plane(tall):
    torch = torch_cuda()
    plane, dev, b, x, counts = tall
    x.zero_()
    ctx, plan = _plan(torch, dev, b, x, sip.SIP_MODE_F32_REFINED)
    rel = plan.iterate(1)
    plan.close()
    ctx.close()
    expect, h0 = [], np.zeros(NCLS)
    bn2 = np.zeros(NCLS)
    for r in range(NCLS):
        coefs, bp = _plane_system(r, plane)
        F32 = oracle.factors_f32(oracle.factor(NX, NY, 1, coefs, ALPHA))
        c32 = {k: v.astype(np.float32) for k, v in coefs.items()}
        xp, _, _, hist = oracle.solve_refined(NX, NY, 1, coefs, c32, F32, bp, rtol=0.0, max_outer=1, m_inner=4)
        expect.append(xp)
        h0[r] = hist[0]
        bn2[r] = oracle.norm2(bp) ** 2
    # relres of x = 0 is 1 in every plane
    assert np.allclose(h0, 1.0) and abs(rel - 1.0) <= 1e-12
    _check_planes(torch, x, expect, 1e-5)
