"""Parity of the wavelength-dependent index (cher_set_dispersion) against
the oracle with the same kappa nodes: bunch counts bit-exact (the band
integral's FP64 chain in the oracle's operation order, or the FP32 screen
where it is certain), and per bunch the wavelength, direction, ground
point, time and crossings within the path's tolerances, in both
precisions; on the vertical and the inclined shower, on steps whose
Cherenkov threshold falls inside the band, and together with the
transmission draw and the beyond-table fallback."""
import math

import numpy as np
import pytest

import oracle
import paper_2006_14927_gb300 as P
import workloads
from parity import (FP32, FP64, compare_hits, compare_trace, compare_yield, context, gpu_hits,
                    gpu_trace, host_tracks)

pytestmark = pytest.mark.gpu
SEED = 59
KAPPA = workloads.synthetic_dispersion()
ME = 0.51099895000


def _model(sc, **kw):
    return oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"],
                        n_fine=sc["n_fine"], H=sc["H"], Z=sc["Z"],
                        theta_max_deg=sc["theta_max_deg"], t_ref=sc["t_ref"],
                        dispersion=KAPPA, **kw)


def _threshold_scenario(n=4000, seed=12):
    """Vertical-shower steps whose energies straddle the threshold band
    (beta n(lambda_min) = 1 to beta n(lambda_max) = 1) at their height."""
    sc = workloads.vertical_1tev(n=n, seed=seed)
    tr = sc["tracks"]
    M = oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], H=20, Z=8)
    rng = np.random.default_rng(seed)
    hm = tr["z0"] + 0.5 * tr["len"] * tr["uz"]
    eta = oracle.eta_lookup(M.eta_tab, M.h_max, hm)

    def e_th(k):
        b = 1.0 / (1.0 + eta * k)
        return ME * (1.0 / np.sqrt(1.0 - b * b) - 1.0)

    lo, hi = 0.98 * e_th(KAPPA[0]), 1.02 * e_th(KAPPA[-1])
    tr["ekin"] = lo + rng.random(n) * (hi - lo)
    tr["len"] = np.full(n, 40.0)
    return sc


def _scenario(which):
    if which == "vertical":
        return workloads.vertical_1tev(n=3000)
    if which == "inclined":
        sc = workloads.inclined_20tev(n=3000)
        sc["H"], sc["Z"] = 400, 64
        return sc
    return _threshold_scenario()


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("which", ["vertical", "inclined", "threshold"])
def test_dispersion_trace_and_hits(prec, which):
    P.build()
    sc = _scenario(which)
    M = _model(sc)
    ctx = context(sc)
    ctx.set_dispersion(KAPPA)
    tr = host_tracks(sc, prec)
    o = M.bunches(tr, SEED)
    g = gpu_trace(ctx, tr, sc["t_ref"], SEED, prec)
    o_nb, o_w, _, _ = M.segment_yield(tr)
    compare_yield(o_nb, g["nb"], o_w, g["w"], prec)
    if which == "threshold":
        cut = 0
        for i in range(len(o_nb)):
            g_ = tr["ekin"][i] / ME
            beta = math.sqrt(g_ * (2 + g_)) / (1 + g_)
            hm = tr["z0"][i] + 0.5 * tr["len"][i] * tr["uz"][i]
            eta = oracle.eta_lookup(M.eta_tab, M.h_max, hm)[0]
            cut += KAPPA[-1] < (1 / beta - 1) / eta < KAPPA[0]
        assert cut > 1000 and (o_nb > 0).sum() > 500
    res = compare_trace(M, o, g, prec)
    assert res["n"] > 1000
    code, stats, out = gpu_hits(ctx, tr, sc["t_ref"], SEED, prec, 200_000)
    assert code == 0
    assert int(stats[3]) == int(o_nb.sum())
    assert int(stats[8]) + int(stats[4:8].sum()) == int(stats[3])
    if which != "threshold":
        h = compare_hits(M, o, out.records(), prec)
        assert h["n_common"] > 50
    ctx.close()


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_dispersion_with_transmission_and_fallback(prec):
    P.build()
    sc = workloads.inclined_20tev(n=4000)
    sc["H"], sc["Z"], sc["theta_max_deg"] = 400, 64, 61.0
    table = workloads.synthetic_transmission(h_obs=sc["h_obs"])
    M = _model(sc, transmission=table, fallback_deg=80.0)
    ctx = context(sc)
    ctx.set_dispersion(KAPPA)
    ctx.set_transmission(table)
    ctx.set_fallback(80.0)
    tr = host_tracks(sc, prec)
    o = M.bunches(tr, SEED)
    g = gpu_trace(ctx, tr, sc["t_ref"], SEED, prec)
    res = compare_trace(M, o, g, prec)
    code, stats, out = gpu_hits(ctx, tr, sc["t_ref"], SEED, prec, 200_000)
    assert code == 0
    assert int(stats[12]) > 3000 and int(stats[13]) == 0
    assert int(stats[8]) + int(stats[4:8].sum()) + int(stats[11]) == int(stats[3])
    assert abs(int(stats[11]) - int((o["status"] == oracle.ST_ABSORBED).sum())) <= \
        res["edge_status"]
    compare_hits(M, o, out.records(), prec)
    ctx.close()


def test_dispersion_off_restores_the_constant_index():
    P.build()
    sc = workloads.vertical_1tev(n=2000)
    ctx = context(sc)
    tr = host_tracks(sc, FP32)
    _, s0, out0 = gpu_hits(ctx, tr, sc["t_ref"], SEED, FP32, 200_000)
    ctx.set_dispersion(KAPPA)
    _, s1, out1 = gpu_hits(ctx, tr, sc["t_ref"], SEED, FP32, 200_000)
    ctx.set_dispersion(None)
    _, s2, out2 = gpu_hits(ctx, tr, sc["t_ref"], SEED, FP32, 200_000)
    assert np.array_equal(s0, s2) and not np.array_equal(s0, s1)
    r0, r2 = out0.records(), out2.records()
    assert np.array_equal(r0["key"], r2["key"]) and np.array_equal(r0["x"], r2["x"])
    ctx.close()


def test_dispersion_settings_are_checked():
    P.build()
    sc = workloads.plain_fp64(n=10)
    ctx = P.Context(sc["atm"], sc["h_obs"], sc["telescopes"])
    with pytest.raises(P.CherError) as e:
        ctx.set_dispersion(KAPPA)                      # tables not built yet
    assert e.value.code == 4
    ctx.build_refraction_tables(50, 16, 70.0, 60000.0)
    for bad in ([1.0], [1.0] * 10, [1.0, 1.01], [1.0, 0.0], [1.0, float("nan")],
                [1.0, -0.5], [100.0, 50.0]):
        with pytest.raises(P.CherError) as e:
            ctx.set_dispersion(bad)
        assert e.value.code == 1, bad
    ctx.set_dispersion(KAPPA)
    import torch
    dev = P.device_tracks(host_tracks(sc, FP64), FP64, t_ref=sc["t_ref"])
    with pytest.raises(P.CherError) as e:             # the read-out is for a constant index
        ctx.density(dev, SEED, FP64)
    assert e.value.code == 1
    ctx.set_dispersion(None)
    ctx.density(dev, SEED, FP64)
    torch.cuda.synchronize()
    ctx.close()
