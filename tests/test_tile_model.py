"""The launch model that ranks tile shapes (sip_tile_model, host only): exact
results where the replayed wavefront has a closed form, and the ranking
facts it was fitted to.  The sweeps it models are the hyperplane wavefronts
of the forward and backward substitutions (Sec. 2, Eqs. 9-10): tile (cj, ck)
may start once its producers (cj - 1, ck) and (cj, ck - 1) are far enough
ahead, and a tile of a block nx x ny x nz walks nx + njt + nkt - 2 steps."""
import pytest

from paper_1303_4538_gb300 import sip


def _cyc(dims, q, nw, ctas, fp64=False, nsm=152):
    return sip.tile_model(dims, q, nw, ctas, nsm, fp64)


def _step(q, nw, fp64=False):
    """Cycles of one step of a lone tile: the model's duration of a single
    tile divided by its step count."""
    nx, ny, nz = 50, 32, q * nw
    return _cyc([(nx, ny, nz)], q, nw, 1, fp64) / (nx + ny + nz - 2)


@pytest.mark.parametrize("q,nw", [(1, 4), (1, 12), (2, 7), (4, 2)])
@pytest.mark.parametrize("fp64", [False, True])
def test_single_tile_walks_its_steps(q, nw, fp64):
    """One tile: the duration is its step count times one step, for any nx
    and any partial tile (ny <= 32, nz <= TK)."""
    L = _step(q, nw, fp64)
    for nx, ny, nz in [(1, 1, 1), (17, 5, 1), (300, 32, q * nw), (64, 20, max(1, q * nw - 1))]:
        assert _cyc([(nx, ny, nz)], q, nw, 1, fp64) == pytest.approx((nx + ny + nz - 2) * L, rel=1e-12)


@pytest.mark.parametrize("fp64", [False, True])
def test_one_cta_runs_every_tile_in_turn(fp64):
    """With a single CTA the tiles run one after another in claim order (each
    producer has finished before its consumer is claimed): the duration is
    the sum of all tiles' walks at the lone-tile step."""
    q, nw = 1, 4
    L = _step(q, nw, fp64)
    nx, ny, nz = 40, 70, 10   # 3 x 3 tiles, ragged in j and k
    total = 0
    for cj in range(3):
        for ck in range(3):
            njt = min(32, ny - 32 * cj)
            nkt = min(4, nz - 4 * ck)
            total += nx + njt + nkt - 2
    assert _cyc([(nx, ny, nz)], q, nw, 1, fp64) == pytest.approx(total * L, rel=1e-12)
    # two blocks on one CTA: the sum over both
    nb2 = 30 + 32 + 4 - 2
    assert _cyc([(nx, ny, nz), (30, 32, 4)], q, nw, 1, fp64) == pytest.approx((total + nb2) * L, rel=1e-12)


def test_chain_of_tiles_lags_by_extent_plus_slack():
    """A column of tiles along j, one SM each: every hop adds the producer's
    32 + slack steps, the last tile then walks its own steps.  The slack is
    the same for every hop, so the duration is linear in the number of hops."""
    q, nw = 1, 4
    L = _step(q, nw)
    nx = 100
    d = [_cyc([(nx, 32 * m, 4)], q, nw, 152) for m in (1, 2, 3, 4)]
    hop = d[1] - d[0]
    assert d[2] - d[1] == pytest.approx(hop, rel=1e-12)
    assert d[3] - d[2] == pytest.approx(hop, rel=1e-12)
    assert d[0] == pytest.approx((nx + 32 + 4 - 2) * L, rel=1e-12)
    slack = hop / L - 32
    assert 0 < slack < 16


def test_fewer_ctas_never_faster():
    dims = [(96, 96, 96)]
    for q, nw in [(1, 4), (2, 4)]:
        full = _cyc(dims, q, nw, 152 * 4)
        for ctas in (152, 64, 8, 1):
            assert _cyc(dims, q, nw, ctas) >= full * (1 - 1e-12)


def test_ranking_matches_gb300_measurements():
    """Facts the fit reproduces (measured on GB300, 256^3 Poisson block,
    forward + backward sweep): one row per thread beats two at the shape
    the old two-row chooser took (32 x 14, 7 warps), in FP32 and FP64."""
    dims = [(256, 256, 256)]
    for fp64 in (False, True):
        two = _cyc(dims, 2, 7, 152, fp64)
        best_one = min(_cyc(dims, 1, nw, 152 * max(1, 4 // max(1, nw // 4)), fp64) for nw in (4, 6, 8, 12))
        assert best_one < two


@pytest.mark.parametrize("bad", [
    dict(dims=[(0, 4, 4)]), dict(q=3), dict(nw=0), dict(nw=17), dict(ctas=0), dict(nsm=0)])
def test_rejects_bad_arguments(bad):
    a = dict(dims=[(8, 8, 8)], q=1, nw=4, ctas=4, nsm=152)
    a.update(bad)
    with pytest.raises(sip.SipError):
        sip.tile_model(a["dims"], a["q"], a["nw"], a["ctas"], a["nsm"])
