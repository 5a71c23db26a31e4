"""Parity of the atmospheric transmission draw (cher_set_transmission)
against the oracle: per bunch statuses (absorbed or arrived) and the
crossings of the survivors, both precisions, with the synthetic Rayleigh
plus aerosol table and on the inclined shower."""
import numpy as np
import pytest

import oracle
import paper_2006_14927_gb300 as P
import workloads
from parity import (FP32, FP64, compare_hits, compare_trace, context, gpu_hits, gpu_trace,
                    host_tracks)

pytestmark = pytest.mark.gpu
SEED = 77


def _model(sc, table):
    return oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"],
                        n_fine=sc["n_fine"], H=sc["H"], Z=sc["Z"],
                        theta_max_deg=sc["theta_max_deg"], t_ref=sc["t_ref"],
                        transmission=table)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("which", ["vertical", "inclined"])
def test_transmission_trace_and_hits(prec, which):
    P.build()
    if which == "vertical":
        sc = workloads.vertical_1tev(n=3000)
    else:
        sc = workloads.inclined_20tev(n=3000)
        sc["H"], sc["Z"] = 400, 64
    table = workloads.synthetic_transmission(h_obs=sc["h_obs"])
    M = _model(sc, table)
    ctx = context(sc)
    ctx.set_transmission(table)
    tr = host_tracks(sc, prec)
    o = M.bunches(tr, SEED)
    g = gpu_trace(ctx, tr, sc["t_ref"], SEED, prec)
    res = compare_trace(M, o, g, prec)
    lost_o = o["status"] == oracle.ST_ABSORBED
    lost_g = g["status"] == oracle.ST_ABSORBED
    assert lost_o.sum() > 1000
    assert abs(int(lost_o.sum()) - int(lost_g.sum())) <= res["edge_status"]
    code, stats, out = gpu_hits(ctx, tr, sc["t_ref"], SEED, prec, 200_000)
    assert code == 0
    assert abs(int(stats[11]) - int(lost_o.sum())) <= res["edge_status"]
    assert int(stats[8]) + int(stats[4:8].sum()) + int(stats[11]) == int(stats[3])
    compare_hits(M, o, out.records(), prec)
    # removing the table restores the unattenuated crossings
    ctx.set_transmission(None)
    code, stats0, _ = gpu_hits(ctx, tr, sc["t_ref"], SEED, prec, 200_000)
    assert int(stats0[11]) == 0 and int(stats0[9]) > int(stats[9])
    ctx.close()


def test_transmission_rejects_bad_tables():
    P.build()
    sc = workloads.plain_fp64(n=10)
    ctx = context(sc)
    good = workloads.synthetic_transmission()
    for bad in (dict(good, tau=good["tau"][:1]), dict(good, tau=-good["tau"]),
                dict(good, lambda_nm=(700.0, 250.0)), dict(good, height_m=(5.0, 5.0)),
                dict(good, tau=np.where(good["tau"] > 0.5, np.nan, good["tau"]))):
        with pytest.raises(P.CherError) as e:
            ctx.set_transmission(bad)
        assert e.value.code == 1
    ctx.set_transmission(good)
    ctx.set_transmission(None)
    ctx.close()
