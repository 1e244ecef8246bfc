"""Warm-started SIP as the linear solver of a time step (the paper's usage:
a few sweeps per call on factors computed once, Sec. 4.1 / Tables 1-3): each
call reads the current right-hand side and continues from the previous x."""
import numpy as np
import pytest

import oracle
from paper_1303_4538_gb300 import sip, workloads as W
from tests._gpu import GpuSystem, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [sip.SIP_MODE_F64, sip.SIP_MODE_F32_REFINED])
def test_time_steps_reuse_factors_and_warm_start(mode):
    torch = torch_cuda()
    blk = W.make_block(40, 35, 18, seed=95, kind="convdiff")
    g = GpuSystem(blk, mode=mode, inner=2)
    F = oracle.factor(blk.nx, blk.ny, blk.nz, blk.coefs, 0.92)
    F32 = oracle.factors_f32(F)
    c32 = {k: v.astype(np.float32) for k, v in blk.coefs.items()}
    rng = np.random.default_rng(96)
    xo = np.zeros(blk.n)
    for step in range(4):
        xs = blk.xstar + 0.05 * step * rng.uniform(-1, 1, blk.n)   # the solution drifts between steps
        b = W.apply_matrix(blk.nx, blk.ny, blk.nz, blk.coefs, xs)
        g.b[0].copy_(torch.from_numpy(b))
        g.plan.iterate(6)                                           # a fixed few sweeps per call
        if mode == sip.SIP_MODE_F64:
            xo, _, _, _ = oracle.solve(blk.nx, blk.ny, blk.nz, blk.coefs, F, b, x0=xo, rtol=-1.0, max_iters=6)
            assert np.abs(g.xs() - xo).max() <= 1e-12 * np.abs(xo).max()
        else:
            xo, _, _, _ = oracle.solve_refined(blk.nx, blk.ny, blk.nz, blk.coefs, c32, F32, b, x0=xo, rtol=-1.0,
                                               max_outer=6, m_inner=2)
            assert np.abs(g.xs() - xo).max() <= 1e-5 * np.abs(xo).max()
        # warm start beats a cold start with the same number of sweeps
        cold = GpuSystem(blk, mode=mode, inner=2)
        cold.b[0].copy_(torch.from_numpy(b))
        cold.plan.iterate(6)
        rw = np.linalg.norm(b - W.apply_matrix(blk.nx, blk.ny, blk.nz, blk.coefs, g.xs()))
        rc = np.linalg.norm(b - W.apply_matrix(blk.nx, blk.ny, blk.nz, blk.coefs, cold.xs()))
        cold.close()
        if step > 0:
            assert rw < rc
    assert g.plan.launches() > 0
    g.close()
