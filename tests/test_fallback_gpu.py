"""The beyond-table fallback (cher_set_fallback) against the oracle with the
same fallback: a 60-degree shower with refraction tables to 61 degrees, so
that ~9 % of its bunches arrive past the tables' range and are propagated
by the ray integrals (in place in trace launches, queued and propagated by
a second kernel in hits launches).  Same tolerances as the table path: the
integrals agree with the oracle's adaptive quadrature to far below them."""
import numpy as np
import pytest

import oracle
import paper_2006_14927_gb300 as P
import workloads
from parity import FP32, FP64, compare_hits, compare_trace, context, gpu_hits, gpu_trace, host_tracks

pytestmark = pytest.mark.gpu
SEED = 41


def _scenario(theta_max):
    sc = workloads.inclined_20tev(n=4000)
    sc["H"], sc["Z"], sc["theta_max_deg"] = 400, 64, theta_max
    return sc


def _model(sc, fb, transmission=None):
    return oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"],
                        n_fine=sc["n_fine"], H=sc["H"], Z=sc["Z"],
                        theta_max_deg=sc["theta_max_deg"], t_ref=sc["t_ref"],
                        fallback_deg=fb, transmission=transmission)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("with_transmission", [False, True])
def test_fallback_trace_and_hits(prec, with_transmission):
    P.build()
    sc = _scenario(61.0)
    table = workloads.synthetic_transmission(h_obs=sc["h_obs"]) if with_transmission else None
    M = _model(sc, 80.0, table)
    M_off = _model(sc, 0.0, table)
    ctx = context(sc)
    ctx.set_fallback(80.0)
    if table is not None:
        ctx.set_transmission(table)
    tr = host_tracks(sc, prec)
    o = M.bunches(tr, SEED)
    o_off = M_off.bunches(tr, SEED)
    rescued = o_off["status"] == oracle.ST_ANGLE
    assert rescued.sum() > 5000
    assert not np.any(o["status"] == oracle.ST_ANGLE)
    g = gpu_trace(ctx, tr, sc["t_ref"], SEED, prec)
    res = compare_trace(M, o, g, prec)
    code, stats, out = gpu_hits(ctx, tr, sc["t_ref"], SEED, prec, 200_000)
    assert code == 0
    assert abs(int(stats[12]) - int(rescued.sum())) <= res["edge_status"]
    assert int(stats[13]) == 0 and int(stats[7]) == 0
    assert int(stats[8]) + int(stats[4:8].sum()) + int(stats[11]) == int(stats[3])
    rh = compare_hits(M, o, out.records(), prec)
    # the rescued bunches do cross spheres
    keys = set((((o["seg"][rescued]).astype(np.uint64) << np.uint64(32)) |
                o["j"][rescued].astype(np.uint64)).tolist())
    rec = out.records()
    assert sum(1 for k in rec["key"].tolist() if k in keys) > 10
    ctx.close()


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_bunches_past_the_fallback_limit_stay_dropped(prec):
    sc = _scenario(58.0)
    M = _model(sc, 61.0)
    ctx = context(sc)
    ctx.set_fallback(61.0)
    tr = host_tracks(sc, prec)
    o = M.bunches(tr, SEED)
    assert (o["status"] == oracle.ST_ANGLE).sum() > 500
    g = gpu_trace(ctx, tr, sc["t_ref"], SEED, prec)
    compare_trace(M, o, g, prec)
    code, stats, out = gpu_hits(ctx, tr, sc["t_ref"], SEED, prec, 200_000)
    assert code == 0
    compare_hits(M, o, out.records(), prec)
    ctx.close()


def test_fallback_queue_overflow_is_counted():
    """A queue far smaller than the bunches past the tables: the rest are
    counted as lost, and the books still balance."""
    sc = _scenario(61.0)
    ctx = context(sc)
    ctx.set_fallback(80.0, queue_records=1000)
    tr = host_tracks(sc, FP32)
    code, stats, out = gpu_hits(ctx, tr, sc["t_ref"], SEED, FP32, 200_000)
    assert code == 0
    assert int(stats[12]) == 1000 and int(stats[13]) > 1000
    assert int(stats[8]) + int(stats[4:8].sum()) + int(stats[11]) + int(stats[13]) == int(stats[3])
    ctx.close()


def test_fallback_setting_is_checked():
    sc = _scenario(61.0)
    ctx = context(sc)
    for bad in (30.0, 61.0, 86.0, -1.0, float("nan")):
        with pytest.raises(P.CherError) as e:
            ctx.set_fallback(bad)
        assert e.value.code == 1
    with pytest.raises(P.CherError):
        ctx.set_fallback(70.0, queue_records=-5)
    ctx.set_fallback(70.0)
    ctx.set_fallback(0.0)
    ctx.close()
