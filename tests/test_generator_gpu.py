"""The device step generator (cher_generate_steps) against the oracle's
generator, step by step, and the generated steps through the hot path.

Tolerances from the arithmetic: the device evaluates each step in FP32 (a
chain of ~10 operations on values up to ~1e5 m: 1e-6 relative, 1 cm
absolute) and inverts an FP32 copy of the depth CDF with an FP32 deviate,
so the depth t moves by up to ~2.5e-7 / f(t) (f the normalised Greisen
density), which moves the height by 8000 m * dt / t; positions and times
follow the height along the axis.  Shower indices and reference times are
exact; energies, lengths and directions to 1e-6.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2006_14927_gb300 as P
import workloads
from parity import FP32, FP64, compare_hits, compare_trace, context, gpu_hits, gpu_trace

pytestmark = pytest.mark.gpu

H_OBS = 2200.0
SHOWERS = [dict(e0_mev=1.0e6, zenith=0.35, azimuth=2.0, core_x=40.0, core_y=-15.0, n=30000),
           dict(e0_mev=5.0e4, zenith=0.0, azimuth=0.0, core_x=0.0, core_y=0.0, n=10000),
           dict(e0_mev=2.0e7, zenith=1.0, azimuth=-0.7, core_x=-300.0, core_y=250.0, n=20000)]
SEED = 0x5EED


def _ctx():
    sc = workloads.vertical_1tev(n=10)
    return sc, context(sc)


def _greisen_pdf(t, e0, cz):
    y = math.log(e0 / 85.0)
    t_g = 1030.0 * math.exp(-H_OBS / 8000.0) / cz / 36.7
    grid = np.linspace(0.0, t_g, 200001)
    def g(x):
        x = np.maximum(x, 1e-300)
        return np.exp(x * (1.0 - 1.5 * np.log(3.0 * x / (x + 2.0 * y))))
    gg = g(grid)
    norm = np.sum(0.5 * (gg[1:] + gg[:-1]) * np.diff(grid))
    return g(t) / norm


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_generated_steps_match_the_oracle(prec):
    P.build()
    sc, ctx = _ctx()
    dev = ctx.generate_steps(SHOWERS, SEED, prec)
    got = {k: v.cpu().numpy().astype(np.float64) if v.dtype.is_floating_point else v.cpu().numpy()
           for k, v in dev.items()}
    o = oracle.generate_steps(SHOWERS, H_OBS, SEED)
    assert np.array_equal(got["shower"].astype(np.uint32), o["shower"])
    np.testing.assert_allclose(got["t_ref"], o["t_ref"], rtol=1e-15, atol=0)
    np.testing.assert_allclose(got["ekin"], o["ekin"], rtol=1e-6)
    np.testing.assert_allclose(got["len"], o["len"], rtol=0, atol=2e-5)
    for k in ("ux", "uy", "uz"):
        np.testing.assert_allclose(got[k], o[k], rtol=0, atol=1e-6)
    off = 0
    for s in SHOWERS:
        sl = slice(off, off + s["n"])
        off += s["n"]
        cz = math.cos(s["zenith"])
        sz = math.sin(s["zenith"])
        axis = np.array([sz * math.cos(s["azimuth"]), sz * math.sin(s["azimuth"]), -cz])
        pos = np.stack([o["x0"][sl], o["y0"][sl], o["z0"][sl]], 1)
        along = (pos - np.array([s["core_x"], s["core_y"], H_OBS])) @ axis
        h = H_OBS - along * cz
        t = 1030.0 * np.exp(-h / 8000.0) / cz / 36.7
        dt = 2.5e-7 / np.maximum(_greisen_pdf(t, s["e0_mev"], cz), 1e-30)
        dh = 8000.0 * dt / t
        clamped = h > 29998.0
        tol = np.where(clamped, 1.0, dh / cz) + 0.01 + 1e-6 * np.abs(pos).max()
        for k in ("x0", "y0", "z0"):
            d = np.abs(got[k][sl] - o[k][sl])
            assert np.all(d <= tol), (k, d.max(), np.argmax(d - tol))
        dtime = np.abs(got["t0"][sl] - o["t0"][sl])
        assert np.all(dtime <= tol / 0.299792458 + 0.01), dtime.max()
        # most steps sit far from the tails: the typical error is small
        assert np.median(np.abs(got["z0"][sl] - o["z0"][sl])) < 0.02
    ctx.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_generated_steps_through_the_hot_path(prec):
    """The device-generated steps feed cher_generate_propagate directly; the
    result is what the oracle gives for the same steps (downloaded)."""
    sc, ctx = _ctx()
    sh = [dict(e0_mev=3.0e5, zenith=0.2, azimuth=1.0, core_x=10.0, core_y=20.0, n=3000)]
    dev = ctx.generate_steps(sh, SEED, prec)
    tr = {k: v.cpu().numpy().astype(np.float64) for k, v in dev.items()
          if k not in ("shower", "t_ref")}
    tr["shower"] = dev["shower"].cpu().numpy().astype(np.uint32)
    t_ref = dev["t_ref"].cpu().numpy()
    M = oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"],
                     n_fine=sc["n_fine"], H=sc["H"], Z=sc["Z"],
                     theta_max_deg=sc["theta_max_deg"], t_ref=t_ref)
    o = M.bunches(tr, 11)
    g = gpu_trace(ctx, tr, t_ref, 11, prec)
    compare_trace(M, o, g, prec)
    out = ctx.alloc_hits(100_000, prec)
    ctx.generate_propagate(dev, 11, prec, out)
    code, stats = ctx.sync_status(out)
    assert code == 0 and int(stats[3]) == len(o["status"])
    compare_hits(M, o, out.records(), prec)
    ctx.close()


def test_generator_rejects_bad_showers():
    sc, ctx = _ctx()
    bad = [dict(SHOWERS[0], e0_mev=80.0), dict(SHOWERS[0], zenith=1.6),
           dict(SHOWERS[0], n=-1), dict(SHOWERS[0], core_x=float("nan"))]
    for s in bad:
        with pytest.raises(P.CherError) as e:
            ctx.generate_steps([s], SEED, FP32)
        assert e.value.code == 1
    empty = ctx.generate_steps([dict(SHOWERS[0], n=0)], SEED, FP32)
    assert empty["x0"].numel() == 0
    ctx.close()


def test_back_to_back_calls_keep_their_tables():
    """The per-call tables go up asynchronously from one pinned staging: calls
    queued back to back on a stream, with different shower lists and no
    synchronisation in between, give what each gives alone."""
    import torch
    sc, ctx = _ctx()
    lists = [SHOWERS, [SHOWERS[2], SHOWERS[0]], [dict(SHOWERS[1], n=5000)], SHOWERS[:1]]
    alone = []
    for sh in lists:
        d = ctx.generate_steps(sh, SEED, FP32)
        torch.cuda.synchronize()
        alone.append({k: v.clone() for k, v in d.items()})
    queued = [ctx.generate_steps(sh, SEED, FP32) for sh in lists]
    torch.cuda.synchronize()
    for a, q in zip(alone, queued):
        for k in a:
            assert torch.equal(a[k], q[k]), k
    ctx.close()


def test_reused_outputs_match_fresh_ones():
    """`out=` writes an earlier call's arrays again: the same steps as a fresh
    call; a mismatched dict is refused before anything is launched."""
    import torch
    sc, ctx = _ctx()
    fresh = ctx.generate_steps(SHOWERS, SEED, FP32)
    buf = ctx.generate_steps(SHOWERS, SEED + 1, FP32)
    again = ctx.generate_steps(SHOWERS, SEED, FP32, out=buf)
    torch.cuda.synchronize()
    assert again is buf
    for k in fresh:
        assert torch.equal(fresh[k], again[k]), k
    with pytest.raises(ValueError):
        ctx.generate_steps(SHOWERS[:2], SEED, FP32, out=buf)
    with pytest.raises(ValueError):
        ctx.generate_steps(SHOWERS, SEED, FP64, out=buf)
    ctx.close()
