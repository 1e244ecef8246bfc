"""The measuring tile-shape autotuner (sip_options.autotune) and its cache
file (SIP_AUTOTUNE_CACHE): the tuned plan gives the oracle's iterates and the
same bits as its shape forced explicitly, the caller's x is untouched by the
tuning, and a cached shape is read back (and obeyed) on the next plan."""
import numpy as np
import pytest

import oracle
from paper_1303_4538_gb300 import sip, workloads as W
from tests._gpu import torch_cuda

pytestmark = pytest.mark.gpu


def _plan(torch, blk, x0=None, **kw):
    ctx = sip.Context(0, torch.cuda.current_stream().cuda_stream)
    A = [torch.from_numpy(c).cuda() for c in blk.coef_list()]
    b = torch.from_numpy(blk.b).cuda()
    x = torch.zeros(blk.n, dtype=torch.float64, device="cuda") if x0 is None else torch.from_numpy(x0.copy()).cuda()
    d = sip.make_desc(blk.nx, blk.ny, blk.nz, A, b, x)
    plan = sip.Plan(ctx, [d], sip.default_options(**kw), keep=(A, b, x))
    return ctx, plan, x


def _lines(path):
    return [l.split() for l in open(path) if l.strip() and not l.startswith("#")]


@pytest.mark.parametrize("mode", [sip.SIP_MODE_F64, sip.SIP_MODE_F32_REFINED])
def test_autotuned_plan_matches_forced_shape_and_oracle(tmp_path, monkeypatch, mode):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("SIP_AUTOTUNE_CACHE", str(cache))
    torch = torch_cuda()
    shape3 = (40, 36, 30)
    blk = W.make_block(*shape3, seed=71, kind="convdiff")
    x0 = np.random.Generator(np.random.PCG64(72)).uniform(-1, 1, blk.n)
    ctx, plan, x = _plan(torch, blk, x0=x0, mode=mode, autotune=1)
    assert np.array_equal(x.cpu().numpy(), x0)  # tuning ran on the plan's own vectors
    shape = plan.shape()
    plan.iterate(3)
    hist, xa = plan.history(), x.cpu().numpy()
    plan.close()
    ctx.close()
    q, tk, r = shape
    ctx, plan, x = _plan(torch, blk, x0=x0, mode=mode, tile_j=32, tile_k=tk, rows_per_thread=q, stages=r)
    assert plan.shape() == shape
    plan.iterate(3)
    assert plan.history() == hist
    assert np.array_equal(x.cpu().numpy(), xa)
    plan.close()
    ctx.close()
    if mode == sip.SIP_MODE_F64:
        F = oracle.factor(*shape3, blk.coefs, 0.92)
        xo = x0.copy()
        for _ in range(3):
            oracle.iterate(*shape3, blk.coefs, F, blk.b, xo)
        assert np.abs(xa - xo).max() <= 1e-12 * np.abs(xo).max()
    lines = _lines(cache)
    assert len(lines) == 1 and lines[0][1:4] == [str(q), str(tk), str(r)]


def test_cache_read_back_and_obeyed(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("SIP_AUTOTUNE_CACHE", str(cache))
    torch = torch_cuda()
    blk = W.make_block(33, 41, 27, seed=73, kind="poisson")
    ctx, plan, _ = _plan(torch, blk, autotune=1)
    first = plan.shape()
    plan.close()
    ctx.close()
    ctx, plan, _ = _plan(torch, blk, autotune=1)
    assert plan.shape() == first and len(_lines(cache)) == 1  # read, not re-tuned
    plan.close()
    ctx.close()
    # an entry edited to another valid shape is obeyed
    sig = _lines(cache)[0][0]
    cache.write_text(f"{sig} 2 4 4 0.0\n")
    ctx, plan, x = _plan(torch, blk, autotune=1)
    assert plan.shape() == (2, 4, 4) and len(_lines(cache)) == 1
    rel = plan.iterate(2)
    assert np.isfinite(rel)
    plan.close()
    ctx.close()
    # without the environment variable nothing is written
    monkeypatch.delenv("SIP_AUTOTUNE_CACHE")
    ctx, plan, _ = _plan(torch, blk, autotune=1)
    plan.close()
    ctx.close()
    assert len(_lines(cache)) == 1


def test_autotune_rejects_bad_flag():
    torch = torch_cuda()
    blk = W.make_block(8, 8, 8, seed=74, kind="poisson")
    with pytest.raises(sip.SipError) as e:
        _plan(torch, blk, autotune=2)
    assert e.value.code == sip.SIP_ERR_INVALID_ARG
