"""Parity of the sm_103a SIP path (through the C ABI) with the CPU oracle.

Bars (FP64): factors within 1e-13 relative to each array's magnitude; per
iteration, x within 1e-12 relative (inf-norm) and relres within 1e-12
absolute.  The differences come only from FMA contraction and the
reciprocals on the GPU: 1/LP, stored and multiplied into UN, UE, UT, and
1/(dB dW dS) for LB, LW, LS (the oracle divides, without contraction).
"""
import numpy as np
import pytest

import oracle
from paper_1303_4538_gb300 import sip
from paper_1303_4538_gb300 import workloads as W
from tests._gpu import GpuSystem

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 9), (9, 1, 1), (1, 8, 1), (2, 3, 5), (5, 4, 3), (17, 31, 9), (33, 35, 18),
          (32, 32, 32), (40, 70, 21)]


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["convdiff", "poisson"])
def test_factors_match_oracle(shape, kind):
    blk = W.make_block(*shape, seed=100 + sum(shape), kind=kind)
    g = GpuSystem(blk)
    F = oracle.factor(*shape, blk.coefs, 0.92)
    G = g.factors()
    ref = [F[0], F[1], F[2], 1.0 / F[3], F[4], F[5], F[6]]
    for q, name in enumerate(["LB", "LW", "LS", "1/LP", "UN", "UE", "UT"]):
        scale = max(np.abs(ref[q]).max(), 1e-300)
        assert np.abs(G[q] - ref[q]).max() <= 1e-13 * scale, name
    g.close()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["convdiff", "poisson"])
def test_iterations_match_oracle(shape, kind):
    nx, ny, nz = shape
    blk = W.make_block(*shape, seed=200 + sum(shape), kind=kind)
    x0 = np.random.default_rng(7).uniform(-1, 1, blk.n)
    g = GpuSystem(blk, x0=x0)
    F = oracle.factor(nx, ny, nz, blk.coefs, 0.92)
    x = x0.copy()
    bn = oracle.norm2(blk.b)
    for it in range(6):
        rel_gpu = g.plan.iterate(1)
        rn = oracle.iterate(nx, ny, nz, blk.coefs, F, blk.b, x)
        assert abs(rel_gpu - rn / bn) <= 1e-12, it
        assert _rel(g.xs(), x) <= 1e-12, it
    g.close()


@pytest.mark.parametrize("tile", [(32, 2), (32, 4), (32, 6), (32, 8), (32, 12), (32, 8, 2), (32, 8, 4),
                                  (32, 16, 4), (32, 20, 4), (32, 32, 2), (32, 32, 4), (32, 8, 2, 4),
                                  (32, 16, 2, 6), (32, 12, 4, 3), (32, 8, 1), (32, 6, 1, 4), (32, 10, 1, 6),
                                  (32, 16, 1, 3)])
def test_tile_shapes_agree(tile):
    """(tile_j, tile_k[, rows_per_thread[, stages]]): every column-tile shape
    and prefetch depth gives the oracle's iterates (the 32 x 32 tiles factor
    with a 2-stage ring)."""
    shape = (23, 45, 37)
    blk = W.make_block(*shape, seed=31, kind="convdiff")
    g = GpuSystem(blk, tile=tile)
    F = oracle.factor(*shape, blk.coefs, 0.92)
    x = np.zeros(blk.n)
    for it in range(3):
        rel_gpu = g.plan.iterate(1)
        rn = oracle.iterate(*shape, blk.coefs, F, blk.b, x)
        assert abs(rel_gpu - rn / oracle.norm2(blk.b)) <= 1e-12
    assert _rel(g.xs(), x) <= 1e-12
    g.close()


def test_symmetric_path_and_null_lower_coefficients():
    """Listing 1's symmetric residual on the device: with aw/as/ab passed as
    NULL the plan derives them from ae/an/at and reads only four arrays."""
    shape = (21, 19, 26)
    blk = W.make_block(*shape, seed=55, kind="poisson")
    g = GpuSystem(blk, sym_null=True)
    F = oracle.factor(*shape, blk.coefs, 0.92)
    x = np.zeros(blk.n)
    for it in range(4):
        rel_gpu = g.plan.iterate(1)
        rn = oracle.iterate(*shape, blk.coefs, F, blk.b, x)
        assert abs(rel_gpu - rn / oracle.norm2(blk.b)) <= 1e-12
    assert _rel(g.xs(), x) <= 1e-12
    g.close()


@pytest.mark.parametrize("alpha", [0.0, 0.5, 1.0])
def test_alpha_values(alpha):
    shape = (12, 14, 10)
    blk = W.make_block(*shape, seed=77, kind="convdiff")
    g = GpuSystem(blk, alpha=alpha)
    F = oracle.factor(*shape, blk.coefs, alpha)
    x = np.zeros(blk.n)
    for it in range(3):
        g.plan.iterate(1)
        oracle.iterate(*shape, blk.coefs, F, blk.b, x)
    assert _rel(g.xs(), x) <= 1e-12
    g.close()


def test_solve_convdiff_32cube_matches_oracle():
    """32^3 convection-diffusion, alpha 0.92, 100 iterations or 1e-8."""
    blk = W.convdiff_32cube()
    g = GpuSystem(blk)
    F = oracle.factor(32, 32, 32, blk.coefs, 0.92)
    xr, itr, relr, hr = oracle.solve(32, 32, 32, blk.coefs, F, blk.b, rtol=1e-8, max_iters=100)
    it, rel, conv = g.plan.solve(1e-8, 100)
    assert it == itr and conv == (relr <= 1e-8)
    assert abs(rel - relr) <= 1e-12
    hist = np.array(g.plan.history())
    assert hist.size == hr.size and np.abs(hist - hr).max() <= 1e-12
    assert _rel(g.xs(), xr) <= 1e-12
    g.close()


def test_solve_poisson_to_tolerance_matches_oracle():
    shape = (20, 24, 18)
    blk = W.make_block(*shape, seed=4540, kind="poisson")
    g = GpuSystem(blk)
    F = oracle.factor(*shape, blk.coefs, 0.92)
    xr, itr, relr, hr = oracle.solve(*shape, blk.coefs, F, blk.b, rtol=1e-8, max_iters=5000)
    it, rel, conv = g.plan.solve(1e-8, 5000)
    assert conv and it == itr and abs(rel - relr) <= 1e-12
    assert _rel(g.xs(), xr) <= 1e-11
    # already converged: a second solve applies no update
    x_before = g.xs()
    it2, rel2, conv2 = g.plan.solve(1e-8, 5000)
    assert it2 == 0 and conv2 and np.array_equal(g.xs(), x_before)
    g.close()


def test_deterministic_bitwise():
    blk = W.make_block(30, 41, 27, seed=9, kind="convdiff")
    res = []
    for _ in range(2):
        g = GpuSystem(blk)
        it, rel, _ = g.plan.solve(1e-10, 40)
        res.append((it, rel, g.xs()))
        g.close()
    assert res[0][0] == res[1][0] and res[0][1] == res[1][1] and np.array_equal(res[0][2], res[1][2])


def test_full_size_poisson_256cube_one_iteration():
    """The 256^3 pressure-Poisson block in the launch configuration the
    benchmark uses: one FP64 iteration compared with the oracle everywhere."""
    blk = W.poisson_256cube()
    g = GpuSystem(blk)
    F = oracle.factor(256, 256, 256, blk.coefs, 0.92)
    x = np.zeros(blk.n)
    rel_gpu = g.plan.iterate(1)
    rn = oracle.iterate(256, 256, 256, blk.coefs, F, blk.b, x)
    assert abs(rel_gpu - rn / oracle.norm2(blk.b)) <= 1e-12
    assert _rel(g.xs(), x) <= 1e-12
    g.close()


# ------------------------------------------------------------ mixed precision
def test_refined_single_correction_matches_fp32_oracle():
    """One FP64 correction of m FP32 iterations: compare with the oracle's
    float arithmetic (C13: rel 1e-5)."""
    shape = (19, 22, 17)
    blk = W.make_block(*shape, seed=88, kind="convdiff")
    for m in (1, 2, 3):
        g = GpuSystem(blk, mode=sip.SIP_MODE_F32_REFINED, inner=m)
        F = oracle.factor(*shape, blk.coefs, 0.92)
        c32 = {k: v.astype(np.float32) for k, v in blk.coefs.items()}
        xr, outer, relr, hr = oracle.solve_refined(*shape, blk.coefs, c32, oracle.factors_f32(F), blk.b,
                                                   rtol=0.0, max_outer=1, m_inner=m)
        rel = g.plan.iterate(1)
        assert abs(rel - hr[0]) <= 1e-12
        assert _rel(g.xs(), xr) <= 1e-5
        g.close()


@pytest.mark.parametrize("kind", ["poisson", "convdiff"])
def test_refined_solve_reaches_fp64_tolerance(kind):
    shape = (24, 20, 22)
    blk = W.make_block(*shape, seed=4540, kind=kind)
    g = GpuSystem(blk, mode=sip.SIP_MODE_F32_REFINED, inner=4)
    it, rel, conv = g.plan.solve(1e-8, 2000)
    assert conv and rel <= 1e-8
    x = g.xs()
    # the oracle's own FP64 residual of the device's answer
    _, rn = oracle.residual(*shape, blk.coefs, blk.b, x)
    assert rn / oracle.norm2(blk.b) <= 1.0001e-8
    F = oracle.factor(*shape, blk.coefs, 0.92)
    xr, _, _, _ = oracle.solve(*shape, blk.coefs, F, blk.b, rtol=1e-8, max_iters=20000)
    err_ref = np.linalg.norm(xr - blk.xstar) / np.linalg.norm(blk.xstar)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 10 * max(err_ref, 1e-12)
    g.close()


def test_refined_with_fp32_coefficients():
    """A stored in FP32 (the 384^3 workload's storage) on a small block:
    refinement converges to the solution of the widened FP32 matrix."""
    shape = (18, 16, 20)
    blk = W.make_block(*shape, seed=4542, kind="convdiff", pe=10.0)
    g = GpuSystem(blk, mode=sip.SIP_MODE_F32_REFINED, inner=4, coef_f32=True)
    it, rel, conv = g.plan.solve(1e-8, 2000)
    assert conv
    c64w = {k: v.astype(np.float32).astype(np.float64) for k, v in blk.coefs.items()}
    _, rn = oracle.residual(*shape, c64w, blk.b, g.xs())
    assert rn / oracle.norm2(blk.b) <= 1.0001e-8
    g.close()


# ------------------------------------------------------------ error paths
def test_bounded_wait_times_out_without_hanging():
    blk = W.make_block(20, 70, 30, seed=3, kind="convdiff")
    with pytest.raises(sip.SipError) as e:
        GpuSystem(blk, stall=1, max_spin=2000)
    assert e.value.code == sip.SIP_ERR_DEVICE_TIMEOUT


def test_breakdown_reported():
    blk = W.make_block(3, 1, 1, seed=1, kind="convdiff")
    blk.coefs["ap"][:] = [1.0, 1.0, 2.0]
    blk.coefs["ae"][:] = [1.0, -1.0, 0.0]
    blk.coefs["aw"][:] = [0.0, 1.0, -1.0]
    with pytest.raises(sip.SipError) as e:
        GpuSystem(blk)
    assert e.value.code == sip.SIP_ERR_BREAKDOWN


def test_invalid_arguments():
    import torch
    ctx = sip.Context(0, torch.cuda.current_stream().cuda_stream)
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    d = sip.make_desc(0, 2, 2, [z] * 7, z, z)
    with pytest.raises(sip.SipError) as e:
        sip.Plan(ctx, [d])
    assert e.value.code == sip.SIP_ERR_INVALID_ARG
    d = sip.make_desc(2, 2, 2, [z, None, z, None, z, None, z], z, z, symmetric=False)
    with pytest.raises(sip.SipError):
        sip.Plan(ctx, [d])
    d = sip.make_desc(2, 2, 2, [z] * 7, z, z)
    with pytest.raises(sip.SipError):
        sip.Plan(ctx, [d], sip.default_options(alpha=1.5))
    for bad in (dict(rows_per_thread=3), dict(stages=5), dict(tile_k=7), dict(tile_j=16)):
        with pytest.raises(sip.SipError) as e:
            sip.Plan(ctx, [d], sip.default_options(**bad))
        assert e.value.code == sip.SIP_ERR_INVALID_ARG
    ctx.close()
