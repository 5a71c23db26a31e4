"""Parity of the curved atmosphere (cher_set_curved) against the oracle with
the same Earth radius: bunch counts bit-exact (the radial midpoint height
in the FP64 chain in the oracle's order, or the FP32 screen where it is
certain), and per bunch the ground point on the observation sphere,
arrival time, direction and crossings within the path's tolerances, in
both precisions; on the 60-degree shower with tables to 80 degrees, on the
vertical shower, and with the transmission draw and the wavelength-
dependent index."""
import numpy as np
import pytest

import oracle
import paper_2006_14927_gb300 as P
import workloads
from parity import (FP32, FP64, compare_hits, compare_trace, compare_yield, context, gpu_hits,
                    gpu_trace, host_tracks)

pytestmark = pytest.mark.gpu
SEED = 67
R_EARTH = 6.371e6


def _model(sc, **kw):
    return oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"],
                        n_fine=sc["n_fine"], H=sc["H"], Z=sc["Z"],
                        theta_max_deg=sc["theta_max_deg"], t_ref=sc["t_ref"],
                        earth_radius=R_EARTH, **kw)


def _scenario(which):
    if which == "inclined":
        sc = workloads.inclined_20tev(n=3000)
        sc["H"], sc["Z"], sc["theta_max_deg"] = 400, 64, 80.0
        return sc
    return workloads.vertical_1tev(n=3000)


def _ctx(sc):
    ctx = context(sc)
    ctx.set_curved(R_EARTH)
    return ctx


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("which", ["inclined", "vertical"])
def test_curved_trace_and_hits(prec, which):
    P.build()
    sc = _scenario(which)
    M = _model(sc)
    ctx = _ctx(sc)
    tr = host_tracks(sc, prec)
    o = M.bunches(tr, SEED)
    g = gpu_trace(ctx, tr, sc["t_ref"], SEED, prec)
    o_nb, o_w, _, _ = M.segment_yield(tr)
    compare_yield(o_nb, g["nb"], o_w, g["w"], prec)
    res = compare_trace(M, o, g, prec)
    assert res["n"] > 1000
    code, stats, out = gpu_hits(ctx, tr, sc["t_ref"], SEED, prec, 200_000)
    assert code == 0
    assert int(stats[3]) == int(o_nb.sum())
    assert int(stats[8]) + int(stats[4:8].sum()) == int(stats[3])
    h = compare_hits(M, o, out.records(), prec)
    assert h["n_common"] > 20
    if which == "inclined":
        # curvature matters here: the flat geometry lands elsewhere
        # (the radial heights change bunch counts: compare the first bunch of
        # the steps whose counts agree)
        ctx.set_curved(0.0)
        gf = gpu_trace(ctx, tr, sc["t_ref"], SEED, prec)
        oc = np.concatenate([[0], np.cumsum(g["nb"])])[:-1]
        of = np.concatenate([[0], np.cumsum(gf["nb"])])[:-1]
        same = np.nonzero((g["nb"] == gf["nb"]) & (g["nb"] > 0))[0]
        bc, bf = oc[same], of[same]
        ok = (g["status"][bc] == 0) & (gf["status"][bf] == 0)
        assert ok.sum() > 100
        assert np.abs(gf["pos"][bf[ok], 0] - g["pos"][bc[ok], 0]).max() > 1.0
    ctx.close()


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_curved_with_transmission_and_dispersion(prec):
    P.build()
    sc = _scenario("inclined")
    table = workloads.synthetic_transmission(h_obs=sc["h_obs"])
    kappa = workloads.synthetic_dispersion()
    M = _model(sc, transmission=table, dispersion=kappa)
    ctx = _ctx(sc)
    ctx.set_transmission(table)
    ctx.set_dispersion(kappa)
    tr = host_tracks(sc, prec)
    o = M.bunches(tr, SEED)
    g = gpu_trace(ctx, tr, sc["t_ref"], SEED, prec)
    res = compare_trace(M, o, g, prec)
    code, stats, out = gpu_hits(ctx, tr, sc["t_ref"], SEED, prec, 200_000)
    assert code == 0
    assert int(stats[8]) + int(stats[4:8].sum()) + int(stats[11]) == int(stats[3])
    assert abs(int(stats[11]) - int((o["status"] == oracle.ST_ABSORBED).sum())) <= \
        res["edge_status"]
    compare_hits(M, o, out.records(), prec)
    ctx.close()


def test_curved_settings_are_checked():
    P.build()
    sc = workloads.plain_fp64(n=10)
    ctx = P.Context(sc["atm"], sc["h_obs"], sc["telescopes"])
    for bad in (-1.0, 1.0, 5e5, 2e8, float("nan"), float("inf")):
        with pytest.raises(P.CherError) as e:
            ctx.set_curved(bad)
        assert e.value.code == 1, bad
    ctx.set_curved(R_EARTH)                           # before the tables: kept for the build
    ctx.build_refraction_tables(50, 16, 80.0, 60000.0)
    dev = P.device_tracks(host_tracks(sc, FP64), FP64, t_ref=sc["t_ref"])
    with pytest.raises(P.CherError) as e:             # the read-out is for flat layers
        ctx.density(dev, SEED, FP64)
    assert e.value.code == 1
    ctx.set_curved(0.0)
    ctx.density(dev, SEED, FP64)
    ctx.close()
