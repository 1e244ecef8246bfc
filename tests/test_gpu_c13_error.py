"""Error of the FP32-refined solver against the FP64 oracle (Sec. 4.1: the
single-precision solver variant; here FP32 coefficients, factors and sweeps
inside an FP64 refinement).

Block: 64^3 convection-diffusion with median cell Peclet 10 (the 384^3
workload's generator at a size the oracle solves in seconds), alpha 0.5.
The device solves the system whose coefficients are stored in FP32 (A32) to
a relative residual of 1e-8.  Two oracle solutions serve as references, both
from the plain FP64 oracle SIP driven to 1e-10 (alpha 0.5 stagnates near
4e-11 on this block):
  * x_A32: the stored FP32 matrix widened to FP64 (the system the device solves);
  * x_A64: the FP64 matrix the generator drew (the system a user meant).
The device's error against x_A32 is the solver's own error and must be of the
size the oracle's refined solve leaves at the same tolerance; its error
against x_A64 adds the perturbation of rounding A to FP32, which the oracle's
x_A32 shows as well.  The FP64 relative residuals of the device's x under
A64 and under the widened A32 come from the library's independent residual
norm and are checked against numpy's."""
import numpy as np
import pytest

import oracle
from paper_1303_4538_gb300 import sip, workloads as W
from tests._gpu import torch_cuda

pytestmark = pytest.mark.gpu

N = 64
ALPHA = 0.5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def refs():
    blk = W.make_block(N, N, N, seed=4544, kind="convdiff", pe=10.0)
    c32 = {k: v.astype(np.float32) for k, v in blk.coefs.items()}
    c32w = {k: v.astype(np.float64) for k, v in c32.items()}
    F64 = oracle.factor(N, N, N, blk.coefs, ALPHA)
    x64, it64, rel64, _ = oracle.solve(N, N, N, blk.coefs, F64, blk.b, rtol=1e-10, max_iters=5000)
    F32w = oracle.factor(N, N, N, c32w, ALPHA)
    x32, it32, rel32, _ = oracle.solve(N, N, N, c32w, F32w, blk.b, rtol=1e-10, max_iters=5000)
    assert rel64 <= 1e-10 and rel32 <= 1e-10
    # the oracle's own refined solve at the device's tolerance
    xr, itr, relr, _ = oracle.solve_refined(N, N, N, c32w, c32, oracle.factors_f32(F32w), blk.b, rtol=1e-8,
                                            max_outer=1000, m_inner=4)
    assert relr <= 1e-8
    return blk, c32, x64, x32, xr


def test_refined_error_against_fp64_oracle(refs):
    torch = torch_cuda()
    blk, c32, x64, x32, xr = refs
    ctx = sip.Context(0, torch.cuda.current_stream().cuda_stream)
    A32 = [torch.from_numpy(np.ascontiguousarray(c.astype(np.float32))).cuda() for c in blk.coef_list()]
    A64 = [torch.from_numpy(c).cuda() for c in blk.coef_list()]
    b = torch.from_numpy(blk.b).cuda()
    x = torch.zeros(blk.n, dtype=torch.float64, device="cuda")
    d32 = sip.make_desc(N, N, N, A32, b, x, coef_dtype=1)
    d64 = sip.make_desc(N, N, N, A64, b, x)
    plan = sip.Plan(ctx, [d32], sip.default_options(mode=sip.SIP_MODE_F32_REFINED, alpha=ALPHA),
                    keep=(A32, b, x))
    it, rel, conv = plan.solve(1e-8, 1000)
    plan.close()
    assert conv and rel <= 1e-8
    xg = x.cpu().numpy()
    e32, e64 = _rel(xg, x32), _rel(xg, x64)
    e32_oracle, e64_oracle = _rel(xr, x32), _rel(xr, x64)
    shift = _rel(x32, x64)   # what rounding A to FP32 moves the exact solution by
    print(f"\n64^3 Pe 10, alpha 0.5, FP32-refined to 1e-8 in {it} corrections:"
          f" err vs A32 oracle {e32:.2e} (oracle refined {e32_oracle:.2e}),"
          f" err vs A64 oracle {e64:.2e} (oracle refined {e64_oracle:.2e}), |x_A32 - x_A64| {shift:.2e}")
    # the solver's own error: the size the same method leaves in the oracle
    assert e32 <= 4.0 * e32_oracle + 1e-12
    # against the FP64 system: solver error plus the coefficient-rounding shift
    assert e64 <= (e32 + shift) * (1 + 1e-5)
    assert abs(e64 - e64_oracle) <= 4.0 * e32_oracle + 1e-12
    # FP64 relative residuals of the device's x under the widened A32 and under A64
    rn32, bn = ctx.residual_norm(d32)
    rn64, bn64 = ctx.residual_norm(d64)
    ctx.close()
    assert bn == pytest.approx(bn64, rel=1e-15)
    c32w = {k: v.astype(np.float64) for k, v in c32.items()}
    r32 = blk.b - W.apply_matrix(N, N, N, c32w, xg)
    r64 = blk.b - W.apply_matrix(N, N, N, blk.coefs, xg)
    assert rn32 / bn <= 1e-8 * (1 + 1e-6)
    assert rn32 == pytest.approx(np.linalg.norm(r32), rel=1e-10)
    assert rn64 == pytest.approx(np.linalg.norm(r64), rel=1e-10)
    print(f"  FP64 relres of x: A32 {rn32 / bn:.2e}, A64 {rn64 / bn:.2e}")
