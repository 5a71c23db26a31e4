"""cher_generate_propagate_noalloc against cher_generate_propagate.

The no-alloc entry point serves callers that must not allocate device memory
while they run the hot path (device memory held entirely by another
allocator; real-time loops that forbid allocation after start-up).  It runs
the same kernel with its tile counter in a fixed array compiled into the
library, so its records must equal the regular entry point's, on two calls in
a row (the second call finds the first call's counter in the array and must
clear it).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import paper_2006_14927_gb300 as P
import workloads
from parity import FP32, FP64, context, host_tracks

pytestmark = pytest.mark.gpu

SEED = 0xC0FFEE


def _run(ctx, dev, prec, cap, noalloc):
    out = ctx.alloc_hits(cap, prec)
    t = ctx.tracks_struct(dev)
    o = out.struct()
    fn = P.lib().cher_generate_propagate_noalloc if noalloc else P.lib().cher_generate_propagate
    import torch
    code = fn(ctx._h, ctypes.byref(t), ctypes.c_uint64(SEED), int(prec), ctypes.byref(o),
              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0, code
    code, stats = ctx.sync_status(out)
    assert code == 0, code
    return stats, out.records()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_noalloc_matches_regular_entry_point(prec):
    P.build()
    sc = workloads.vertical_1tev(n=30_011)
    ctx = context(sc)
    tr = host_tracks(sc, prec)
    dev = P.device_tracks(tr, prec, t_ref=sc["t_ref"])
    ref_stats, ref = _run(ctx, dev, prec, 100_000, noalloc=False)
    assert ref_stats[9] > 0
    for _ in range(2):                      # two calls in a row
        stats, rec = _run(ctx, dev, prec, 100_000, noalloc=True)
        assert np.array_equal(stats, ref_stats)
        assert np.array_equal(rec["tel"], ref["tel"])
        assert np.array_equal(rec["key"], ref["key"])
        tol = 0.0 if prec == FP64 else 0.0   # same kernel, same arithmetic
        for k in ("x", "y", "cx", "cy", "t", "zem", "w", "lam"):
            np.testing.assert_allclose(rec[k], ref[k], rtol=0, atol=tol)
    ctx.close()


@pytest.mark.parametrize("feature", ["dispersion", "curved", "both"])
def test_noalloc_with_the_index_and_geometry_options(feature):
    """The 128-step instantiations of the wavelength-dependent index and the
    curved atmosphere through the allocation-free entry point (their larger
    shared-memory tiles and forced tile size come from the same launch
    preparation)."""
    P.build()
    sc = workloads.inclined_20tev(n=20_011)
    sc["H"], sc["Z"], sc["theta_max_deg"] = 200, 32, 80.0
    ctx = context(sc)
    if feature in ("dispersion", "both"):
        ctx.set_dispersion(workloads.synthetic_dispersion())
    if feature in ("curved", "both"):
        ctx.set_curved(6.371e6)
    prec = FP32
    dev = P.device_tracks(host_tracks(sc, prec), prec, t_ref=sc["t_ref"])
    ref_stats, ref = _run(ctx, dev, prec, 200_000, noalloc=False)
    assert ref_stats[9] > 0
    stats, rec = _run(ctx, dev, prec, 200_000, noalloc=True)
    assert np.array_equal(stats, ref_stats)
    assert np.array_equal(rec["key"], ref["key"])
    for k in ("x", "y", "t", "lam"):
        np.testing.assert_array_equal(rec[k], ref[k])
    ctx.close()


def test_noalloc_refuses_oversized_input():
    P.build()
    sc = workloads.plain_fp64(n=10)
    ctx = context(sc)
    dev = P.device_tracks(host_tracks(sc, FP32), FP32, t_ref=sc["t_ref"])
    t = ctx.tracks_struct(dev)
    t.n = (1 << 40) + 1                     # refused before any launch
    out = ctx.alloc_hits(4, FP32)
    o = out.struct()
    code = P.lib().cher_generate_propagate_noalloc(ctx._h, ctypes.byref(t), 0, FP32,
                                                   ctypes.byref(o), None)
    assert code == 5                        # CHER_ERANGE
    ctx.close()


def test_noalloc_refuses_an_active_fallback():
    """With the beyond-table fallback active the regular entry point queues
    the bunches past the tables' zenith range in memory the context
    allocates and integrates them; the allocation-free call cannot, so it
    refuses the context (CHER_EINVAL) before anything is launched, and
    serves it again once the fallback is switched off."""
    import torch
    P.build()
    sc = workloads.inclined_20tev(n=20_011)
    sc["H"], sc["Z"], sc["theta_max_deg"] = 200, 32, 61.0
    ctx = context(sc)
    prec = FP32
    dev = P.device_tracks(host_tracks(sc, prec), prec, t_ref=sc["t_ref"])
    ctx.set_fallback(80.0)
    ref_stats, _ = _run(ctx, dev, prec, 200_000, noalloc=False)
    assert ref_stats[12] > 0                # the fallback propagated some bunches
    out = ctx.alloc_hits(200_000, prec)
    out.stats.fill_(7)                      # a launch would clear these
    out.count.fill_(7)
    t = ctx.tracks_struct(dev)
    o = out.struct()
    code = P.lib().cher_generate_propagate_noalloc(
        ctx._h, ctypes.byref(t), ctypes.c_uint64(SEED), int(prec), ctypes.byref(o),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 1                        # CHER_EINVAL
    torch.cuda.synchronize()
    assert bool((out.stats == 7).all()) and bool((out.count == 7).all())
    ctx.set_fallback(0.0)                   # off: served again, same as the regular call
    ref_stats, ref = _run(ctx, dev, prec, 200_000, noalloc=False)
    stats, rec = _run(ctx, dev, prec, 200_000, noalloc=True)
    assert np.array_equal(stats, ref_stats)
    assert np.array_equal(rec["key"], ref["key"])
    ctx.close()
