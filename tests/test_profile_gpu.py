"""Parity of the longitudinal production profile (CERLDE) computed in the
fused launch against the oracle.

FP64 path: every bin to 1e-9 relative (the sums are atomic, so their
order varies; edge heights come from the layer formula's inverse on the
device and from bisection in the oracle).

FP32 path, allowance per bin derived from the arithmetic: the step's photon
count keeps the FP32 yield's rounding (1e-4 relative, as the photons per
bunch); the depth T(h) is an FP32 exponential (relative error ~1e-6, taken
as 1e-5), so a step whose shallowest or deepest point lies within that of a
bin edge may fall wholly on either side; and an edge height is an FP32
logarithm times the layer's scale height (error ~1 cm, taken as 3 cm), so a
step crossing an edge may move 3 cm / (its height span) of its photons.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2006_14927_gb300 as P
import workloads
from parity import FP32, FP64, context, host_tracks, oracle_model

pytestmark = pytest.mark.gpu


def _gpu_profile(ctx, sc, tr, prec, bin_gcm2, n_bins, axis_cos=None, seed=5, cap=20000,
                 profile=None):
    import torch
    dev = P.device_tracks(tr, prec, t_ref=sc["t_ref"])
    out = ctx.alloc_hits(cap, prec)
    rows = max(len(sc["t_ref"]), 1)
    if profile is None:
        profile = torch.zeros((rows, n_bins), dtype=torch.float64, device="cuda")
    ctx.generate_propagate(dev, seed, prec, out, profile=profile, bin_gcm2=bin_gcm2,
                           axis_cos=axis_cos)
    code, stats = ctx.sync_status(out)
    assert code == 0
    return profile, stats, out


def _allowance(M, sc, tr, bin_gcm2, n_bins, axis_cos, P_o):
    nb, w, _, _ = M.segment_yield(tr)
    N = nb * w
    rows = P_o.shape[0]
    allow = 1e-4 * P_o
    sh = tr["shower"].astype(np.int64)
    z1 = tr["z0"] + tr["len"] * tr["uz"]
    lo = np.minimum(tr["z0"], z1)
    hi = np.maximum(tr["z0"], z1)
    em = np.nonzero(nb > 0)[0]
    Xt = oracle.thickness(sc["atm"], hi[em])
    Xb = oracle.thickness(sc["atm"], lo[em])
    for q, i in enumerate(em):
        s = sh[i]
        if s >= rows:
            continue
        cz = axis_cos[s] if axis_cos is not None else 1.0
        a, b = Xt[q] / cz / bin_gcm2, Xb[q] / cz / bin_gcm2
        ka, kb = int(math.floor(a)), int(math.floor(b))
        span = hi[i] - lo[i]
        # ends within 1e-5 relative of an edge: anything may move
        for x in (a, b):
            e = round(x)
            if abs(x - e) <= 1e-5 * x + 1e-9:
                for k in (e - 1, e):
                    if 0 <= k < n_bins:
                        allow[s, k] += N[i]
        # crossed edges: 3 cm of height per edge
        if kb > ka:
            f = N[i] * min(1.0, 0.03 / span) if span > 0 else N[i]
            for k in range(max(ka, 0), min(kb, n_bins - 1) + 1):
                allow[s, k] += 2 * f
    return allow


def _compare(M, sc, tr, prec, got, bin_gcm2, n_bins, axis_cos=None):
    P_o = M.profile(tr, bin_gcm2, n_bins, axis_cos=axis_cos)
    got = got.cpu().numpy()
    assert got.shape == P_o.shape
    assert P_o.sum() > 0
    if prec == FP64:
        np.testing.assert_allclose(got, P_o, rtol=1e-9, atol=1e-9 * P_o.max())
    else:
        allow = _allowance(M, sc, tr, bin_gcm2, n_bins, axis_cos, P_o)
        bad = np.abs(got - P_o) > allow + 1e-9 * P_o.max()
        assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], P_o[bad][:5])
        # the allowance is not the whole bin
        assert (allow < 0.05 * np.maximum(P_o, 1e-300))[P_o > 1e-3 * P_o.max()].mean() > 0.9


@pytest.fixture(scope="module")
def vertical():
    P.build()
    sc = workloads.vertical_1tev(n=20000)
    return sc, oracle_model(sc), context(sc)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("n_bins", [120, 45])
def test_profile_vertical(vertical, prec, n_bins):
    sc, M, ctx = vertical
    tr = host_tracks(sc, prec)
    got, _, _ = _gpu_profile(ctx, sc, tr, prec, 10.0, n_bins)
    _compare(M, sc, tr, prec, got, 10.0, n_bins)


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_profile_batched_slant(prec):
    sc = workloads.batched_256(total=12000, n_showers=8)
    M = oracle_model(sc)
    ctx = context(sc)
    tr = host_tracks(sc, prec)
    cz = np.cos(sc["axis_zenith_rad"])
    got, _, _ = _gpu_profile(ctx, sc, tr, prec, 20.0, 80, axis_cos=cz)
    _compare(M, sc, tr, prec, got, 20.0, 80, axis_cos=cz)
    ctx.close()


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_profile_inclined(prec):
    sc = workloads.inclined_20tev(n=20000)
    sc["H"], sc["Z"] = 400, 64
    M = oracle_model(sc)
    ctx = context(sc)
    tr = host_tracks(sc, prec)
    cz = np.cos(sc["axis_zenith_rad"])
    got, _, _ = _gpu_profile(ctx, sc, tr, prec, 10.0, 200, axis_cos=cz)
    _compare(M, sc, tr, prec, got, 10.0, 200, axis_cos=cz)
    ctx.close()


def test_profile_adds_and_leaves_the_crossings_alone(vertical):
    sc, M, ctx = vertical
    tr = host_tracks(sc, FP32)
    prof, st1, out1 = _gpu_profile(ctx, sc, tr, FP32, 10.0, 120)
    first = prof.clone()
    prof, st2, out2 = _gpu_profile(ctx, sc, tr, FP32, 10.0, 120, profile=prof)
    np.testing.assert_allclose(prof.cpu().numpy(), 2 * first.cpu().numpy(), rtol=1e-12,
                               atol=1e-12 * float(first.max()))
    dev = P.device_tracks(tr, FP32, t_ref=sc["t_ref"])
    out3 = ctx.alloc_hits(20000, FP32)
    ctx.generate_propagate(dev, 5, FP32, out3)
    code, st3 = ctx.sync_status(out3)
    assert np.array_equal(st1, st3) and np.array_equal(st2, st3)
    assert np.array_equal(out1.count.cpu().numpy(), out3.count.cpu().numpy())


def test_profile_rejects_bad_arguments(vertical):
    import torch
    sc, M, ctx = vertical
    tr = host_tracks(sc, FP32, slice(0, 100))
    dev = P.device_tracks(tr, FP32, t_ref=sc["t_ref"])
    out = ctx.alloc_hits(100, FP32)
    cases = [((1, 0), 10.0), ((1, 10), 0.0), ((1, 10), -1.0), ((1, 10), float("nan")),
             ((1, 10), float("inf")), ((1, 70000), 10.0)]
    for shape, width in cases:
        prof = torch.zeros(shape, dtype=torch.float64, device="cuda")
        with pytest.raises(P.CherError) as e:
            ctx.generate_propagate(dev, 5, FP32, out, profile=prof, bin_gcm2=width)
        assert e.value.code == 1                      # CHER_EINVAL
    torch.cuda.synchronize()


def test_profile_full_size_conserves_photons():
    """2e6 steps in the benchmark's launch shape: with bins covering every
    depth, the profile's total is the photons of the launch's own yield."""
    import torch
    sc = workloads.vertical_1tev()
    ctx = context(sc)
    ctx.set_launch(512, 2)
    dev = P.device_tracks(sc["tracks"], FP32, t_ref=sc["t_ref"])
    nb, w = ctx.segment_yield(dev, FP32)
    N = float((nb.to(torch.float64) * w).sum())
    out = ctx.alloc_hits(600_000, FP32)
    prof = torch.zeros((1, 130), dtype=torch.float64, device="cuda")
    ctx.generate_propagate(dev, 11, FP32, out, profile=prof, bin_gcm2=10.0)
    code, st = ctx.sync_status(out)
    assert code == 0
    assert float(prof.sum()) == pytest.approx(N, rel=1e-5)
    p = prof[0].cpu().numpy()
    assert p[-1] == 0.0 and p.argmax() > 20
    ctx.close()
