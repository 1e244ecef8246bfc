"""The serving loop (sip_server_*): requests of different sizes and kinds,
submitted together, run concurrently in slots; every result equals the same
request solved alone through a plan."""
import time

import numpy as np
import pytest

from paper_1303_4538_gb300 import sip, workloads as W
from tests._gpu import torch_cuda

pytestmark = pytest.mark.gpu


def _request(torch, q, rng):
    n = int(rng.integers(16, 49))
    kind = "poisson" if q % 2 == 0 else "convdiff"
    blk = W.make_block(n, n, n, seed=300 + q, kind=kind)
    A = [torch.from_numpy(c).cuda() for c in blk.coef_list()]
    b = torch.from_numpy(blk.b).cuda()
    x = torch.zeros(blk.n, dtype=torch.float64, device="cuda")
    coefs = list(A)
    if blk.symmetric:
        coefs[1] = coefs[3] = coefs[5] = None
    desc = sip.make_desc(blk.nx, blk.ny, blk.nz, coefs, b, x, symmetric=blk.symmetric)
    mode = sip.SIP_MODE_F64 if q % 3 else sip.SIP_MODE_F32_REFINED
    opts = sip.default_options(mode=mode)
    rtol = 1e-6 if q % 4 < 2 else 1e-8
    return dict(blk=blk, desc=desc, opts=opts, rtol=rtol, keep=(A, b, x), x=x)


def _serve(torch, reqs, budget, slots):
    ctx = sip.Context(0, torch.cuda.current_stream().cuda_stream)
    srv = sip.Server(ctx, budget, slots)
    tickets = [srv.submit(r["desc"], r["opts"], r["rtol"], 3000, keep=r["keep"]) for r in reqs]
    out = {}
    polled_twice = None
    t0 = time.time()
    seen = {"running": 0, "watch": True}
    while len(out) < len(tickets) and time.time() - t0 < 300:
        st = srv.stats()   # the counters and the watchdog age stay consistent while requests run
        seen["running"] = max(seen["running"], st["running"])
        seen["watch"] &= (st["oldest_running_ms"] > 0) == (st["running"] > 0)
        assert st["running"] <= slots and st["submitted"] == len(tickets)
        for t in tickets:
            if t not in out:
                res = srv.poll(t)
                if res is not None:
                    out[t] = res
                    if polled_twice is None:   # a finished ticket is reported once
                        with pytest.raises(sip.SipError) as e:
                            srv.poll(t)
                        polled_twice = e.value.code
        time.sleep(0.001)
    st = srv.stats()
    assert st["completed"] == len(tickets) and st["failed"] == 0 and st["queued"] == 0 and st["running"] == 0
    assert st["budget_bytes"] == budget and st["in_use_bytes"] == 0 and st["busy_ms"] > 0
    assert seen["watch"]
    srv.stop()
    assert len(out) == len(tickets) and polled_twice == sip.SIP_ERR_NOT_FOUND
    return [out[t] for t in tickets], ctx, seen["running"], st


def _alone(torch, ctx, r):
    x = torch.zeros_like(r["x"])
    d = sip.sip_block_desc.from_buffer_copy(r["desc"])
    d.x = x.data_ptr()
    plan = sip.Plan(ctx, [d], r["opts"])
    it, rel, conv = plan.solve(r["rtol"], 3000)
    plan.close()
    return it, rel, x


def test_results_equal_alone_and_in_the_mix():
    torch = torch_cuda()
    rng = np.random.default_rng(101)
    reqs = [_request(torch, q, rng) for q in range(12)]
    res, ctx, running, st = _serve(torch, reqs, 64 << 30, 4)
    assert running >= 2   # requests overlapped on the device
    assert st["peak_in_use_bytes"] <= 64 << 30
    for r, (status, it, rel) in zip(reqs, res):
        assert status in (sip.SIP_OK, sip.SIP_NOT_CONVERGED)
        assert status == sip.SIP_OK and rel <= r["rtol"]
        it1, rel1, x1 = _alone(torch, ctx, r)
        assert it1 == it and rel1 == rel
        assert torch.equal(x1, r["x"])
    ctx.close()


def test_small_budget_admits_one_at_a_time():
    torch = torch_cuda()
    rng = np.random.default_rng(102)
    reqs = [_request(torch, q, rng) for q in range(5)]
    res, ctx, running, st = _serve(torch, reqs, 1 << 20, 3)   # every request exceeds the budget: alone, in order
    assert running == 1
    for r, (status, it, rel) in zip(reqs, res):
        assert status == sip.SIP_OK and rel <= r["rtol"]
        it1, rel1, x1 = _alone(torch, ctx, r)
        assert it1 == it and torch.equal(x1, r["x"])
    ctx.close()


def test_unknown_ticket_and_bad_arguments():
    torch = torch_cuda()
    ctx = sip.Context(0, torch.cuda.current_stream().cuda_stream)
    srv = sip.Server(ctx, 1 << 30, 1)
    with pytest.raises(sip.SipError) as e:
        srv.poll(12345)
    assert e.value.code == sip.SIP_ERR_NOT_FOUND
    r = _request(torch, 1, np.random.default_rng(103))
    with pytest.raises(sip.SipError) as e:
        srv.submit(r["desc"], r["opts"], -1.0, 10)
    assert e.value.code == sip.SIP_ERR_INVALID_ARG
    t = srv.submit(r["desc"], r["opts"], 1e-6, 3000, keep=r["keep"])
    srv.stop()   # drains the queue
    ctx.close()
