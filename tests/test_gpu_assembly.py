"""Device-side pressure-correction assembly (the routine celp2 of Sec. 3.1;
the symmetric system of Sec. 4.1) against the oracle, through the C ABI:
bit-exact coefficients and right-hand side (both evaluate the same formulas
in the same order without fused multiply-adds), then the assembled system
solved by SIP straight from the device arrays."""
import numpy as np
import pytest

import oracle
from paper_1303_4538_gb300 import sip, workloads as W
from tests._gpu import torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [(5, 4, 3), (1, 1, 6), (7, 1, 2), (3, 6, 1), (37, 29, 18), (64, 48, 40), (130, 33, 65)]


def _dev(torch, P):
    return [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (P.dx, P.dy, P.dz, P.rho, P.g, P.ux, P.uy, P.uz)]


def _assemble_gpu(torch, ctx, P, symmetric=False):
    ins = _dev(torch, P)
    outs = [torch.full((P.n,), np.nan, dtype=torch.float64, device="cuda") for _ in range(8)]
    if symmetric:
        outs[1] = outs[3] = outs[5] = None
    ctx.assemble_pcorr(P.nx, P.ny, P.nz, *ins, outs, dirichlet_bottom=P.dirichlet_bottom)
    torch.cuda.synchronize()
    return outs, ins


@pytest.mark.parametrize("dirichlet", [True, False])
@pytest.mark.parametrize("shape", SHAPES)
def test_bit_exact_against_oracle(shape, dirichlet):
    torch = torch_cuda()
    P = W.pcorr_inputs(*shape, seed=31, dirichlet_bottom=dirichlet)
    ref, bref = oracle.assemble_pcorr(*shape, P.dx, P.dy, P.dz, P.rho, P.g, P.ux, P.uy, P.uz, dirichlet)
    ctx = sip.Context(0, torch.cuda.current_stream().cuda_stream)
    outs, _ = _assemble_gpu(torch, ctx, P)
    for q, name in enumerate(W.COEF_NAMES):
        assert np.array_equal(outs[q].cpu().numpy(), ref[name]), name
    assert np.array_equal(outs[7].cpu().numpy(), bref)
    # symmetric storage: the lower entries are not written, the rest is the same
    outs_s, _ = _assemble_gpu(torch, ctx, P, symmetric=True)
    for q in (0, 2, 4, 6, 7):
        assert torch.equal(outs_s[q], outs[q])
    ctx.close()


def test_assembled_system_solved_by_sip():
    """Manufactured pressure correction phi: face velocities u* = the discrete
    gradient velocities of phi (built here on the host), so that A phi = b.
    The device assembles A and b and SIP (FP64, symmetric storage) solves
    from the device arrays; x converges to phi, and the first iterations
    follow the oracle's SIP on the oracle's assembly (1e-12)."""
    torch = torch_cuda()
    nx, ny, nz = 48, 40, 36
    P = W.pcorr_inputs(nx, ny, nz, seed=33)
    rng = np.random.default_rng(10)
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
    ctx = sip.Context(0, torch.cuda.current_stream().cuda_stream)
    outs, ins = _assemble_gpu(torch, ctx, P, symmetric=True)
    x = torch.zeros(P.n, dtype=torch.float64, device="cuda")
    desc = sip.make_desc(nx, ny, nz, outs[:7], outs[7], x, symmetric=True)
    plan = sip.Plan(ctx, [desc], sip.default_options(mode=sip.SIP_MODE_F64), keep=(outs, ins, x))
    plan.iterate(3)
    hg = plan.history()
    ref, bref = oracle.assemble_pcorr(nx, ny, nz, P.dx, P.dy, P.dz, P.rho, P.g, P.ux, P.uy, P.uz, True)
    F = oracle.factor(nx, ny, nz, ref, 0.92)
    xo, it, rel, ho = oracle.solve(nx, ny, nz, ref, F, bref, rtol=-1.0, max_iters=3)
    assert np.abs(np.array(hg) - ho[:3]).max() <= 1e-12
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-12 * np.abs(xo).max()
    x.zero_()
    it, rel, conv = plan.solve(1e-10, 20000)
    assert conv and rel <= 1e-10
    err = np.abs(x.cpu().numpy() - phi).max()
    print(f"\nassembled {nx}x{ny}x{nz} pressure correction: SIP to 1e-10 in {it} iterations, max |x - phi| {err:.2e}")
    assert err <= 2e-6   # the oracle's SIP at 1e-10 leaves 4.5e-7 on this system
    plan.close()
    ctx.close()


def test_rejects_bad_arguments():
    torch = torch_cuda()
    P = W.pcorr_inputs(4, 3, 2, seed=35)
    ctx = sip.Context(0, torch.cuda.current_stream().cuda_stream)
    ins = _dev(torch, P)
    outs = [torch.zeros(P.n, dtype=torch.float64, device="cuda") for _ in range(8)]
    d = sip.sip_pcorr_desc(0, 3, 2, 1, *[sip._ptr(t) for t in ins])
    import ctypes
    rc = sip.lib().sip_assemble_pcorr(ctx.h, ctypes.byref(d), *[ctypes.c_void_p(sip._ptr(t)) for t in outs])
    assert rc == sip.SIP_ERR_INVALID_ARG
    d = sip.sip_pcorr_desc(4, 3, 2, 1, *[sip._ptr(t) for t in ins])
    bad = [ctypes.c_void_p(sip._ptr(t)) for t in outs]
    bad[7] = ctypes.c_void_p(0)
    assert sip.lib().sip_assemble_pcorr(ctx.h, ctypes.byref(d), *bad) == sip.SIP_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        ctx.assemble_pcorr(4, 3, 2, *ins[:5], ins[6], ins[5], ins[7], outs)   # ux / uy swapped: wrong sizes
    ctx.close()
