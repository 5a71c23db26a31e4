"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Sizes: the small workloads in full, reduced versions of the shower workloads
that still span many tiles and end in a ragged tile, and the 2e6-step
vertical 1 TeV shower at full size in the launch configuration the benchmark
times, where the oracle checks every bunch count and a sample of steps bunch
by bunch.
"""
import numpy as np
import pytest

import oracle
import paper_2006_14927_gb300 as P
import workloads
from parity import (FP32, FP64, borderline_status, compare_hits, compare_trace, compare_yield,
                    context, gpu_hits, gpu_trace, host_tracks, oracle_model, sphere_distance,
                    trace_blocks)

pytestmark = pytest.mark.gpu

SEED = 0x5EED_1234_ABCD
# the largest errors of the full-size run (read by a script that runs it)
MEASURED = {}


@pytest.fixture(scope="module", autouse=True)
def _built():
    P.build()


def _reduced(sc, n, stride=None):
    """The first n steps of a scenario (or every stride-th one)."""
    sl = slice(0, n) if stride is None else slice(0, n * stride, stride)
    sc = dict(sc)
    sc["tracks"] = {k: np.asarray(v)[sl] for k, v in sc["tracks"].items()}
    return sc


def _full_compare(sc, prec, seed=SEED, cap=200_000):
    M = oracle_model(sc)
    ctx = context(sc)
    tr = host_tracks(sc, prec)
    o = M.bunches(tr, seed)
    nb_o, w_o, _, _ = M.segment_yield(tr)
    g = gpu_trace(ctx, tr, sc["t_ref"], seed, prec)
    compare_yield(nb_o, g["nb"], w_o, g["w"], prec)
    rt = compare_trace(M, o, g, prec)
    code, stats, out = gpu_hits(ctx, tr, sc["t_ref"], seed, prec, cap)
    assert code == 0
    rec = out.records()
    rh = compare_hits(M, o, rec, prec)
    # the counters add up (conservation of bunches)
    assert stats[P.STAT_NAMES.index("bunches")] == nb_o.sum()
    assert stats[3] == stats[4] + stats[5] + stats[6] + stats[7] + stats[8]
    assert stats[9] == len(rec["tel"])
    assert stats[0] == len(nb_o)
    ctx.close()
    return rt, rh, stats


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_plain_fp64_workload(prec):
    rt, rh, stats = _full_compare(workloads.plain_fp64(), prec)
    assert rt["edge_status"] + rt["edge_hit"] < 0.01 * rt["n"]
    assert rh["n_common"] > 0


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_vertical_shower_reduced(prec):
    sc = _reduced(workloads.vertical_1tev(n=20_011), 20_011)
    rt, rh, stats = _full_compare(sc, prec)
    assert rt["n"] > 100_000
    assert rh["n_common"] > 100
    assert rt["edge_status"] + rt["edge_hit"] < 0.01 * rt["n"]


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_inclined_shower_large_tables(prec):
    sc = workloads.inclined_20tev(n=6_007)
    rt, rh, stats = _full_compare(sc, prec)
    assert rt["n"] > 10_000


def test_batched_showers_reduced():
    sc = workloads.batched_256(total=60_000)
    rt, rh, stats = _full_compare(sc, FP32)
    assert rt["n"] > 50_000


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_refraction_table_edges(prec):
    """Bunches in the refraction tables' last height row (emitted within the
    top 400 m below h_max) and last zenith column (steps at 66-70.5 degrees,
    the tables reaching 70), and some just past both (emitted above h_max,
    arriving beyond the zenith range): the lookups clamped into the last
    cell, the drops counted."""
    import math
    sc = workloads.plain_fp64(n=1_500)
    n = 1_500
    rng = np.random.default_rng(31)
    tr = {k: np.array(v, dtype=float) for k, v in sc["tracks"].items()}
    top = np.arange(n) < n // 2
    h_max = sc["h_max"]
    tr["z0"] = np.where(top, rng.uniform(h_max - 400.0, h_max + 30.0, n),
                        rng.uniform(3000.0, 5000.0, n))
    zen = np.where(top, rng.uniform(0.0, math.radians(5.0), n),
                   rng.uniform(math.radians(66.0), math.radians(70.5), n))
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    tr["ux"], tr["uy"], tr["uz"] = np.sin(zen) * np.cos(ph), np.sin(zen) * np.sin(ph), -np.cos(zen)
    # (near h_max the threshold is above 1 GeV)
    tr["ekin"] = np.where(top, np.exp(rng.uniform(math.log(5e3), math.log(5e4), n)),
                          np.exp(rng.uniform(math.log(200.0), math.log(2000.0), n)))
    tr["t0"] = (workloads.H_START - tr["z0"]) / workloads.C_LIGHT
    sc["tracks"] = tr
    rt, rh, stats = _full_compare(sc, prec)
    assert rt["n"] > 10_000
    assert stats[6] > 0                     # emitted above h_max
    assert stats[7] > 0                     # beyond the tables' zenith range
    assert rt["edge_status"] + rt["edge_hit"] < 0.02 * rt["n"]


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_dense_overlapping_spheres(prec):
    """Large, overlapping and stacked spheres around the core of a reduced
    vertical shower: most bunches cross one sphere or more, so nearly every
    window holds crossings, lanes hold several, and the per-warp crossing
    queue fills, wraps and is flushed many times per tile."""
    sc = _reduced(workloads.vertical_1tev(n=3_001), 3_001)
    sc["telescopes"] = np.array([
        (0.0, 0.0, 0.0, 150.0),        # at the core
        (120.0, 0.0, 0.0, 150.0),      # overlapping the first
        (0.0, 0.0, 200.0, 100.0),      # above the first (centre 200 m up)
        (-60.0, 80.0, 40.0, 60.0),     # inside the first's reach
        (300.0, 300.0, 0.0, 12.0),     # a small one off to the side
    ])
    rt, rh, stats = _full_compare(sc, prec, cap=400_000)
    n_cross = int(stats[9])
    assert n_cross > int(stats[8])          # more crossings than bunches on the ground
    assert rh["n_common"] > 0.99 * n_cross
    assert rt["edge_status"] + rt["edge_hit"] < 0.02 * rt["n"]


def test_launch_shapes_agree():
    """Persistent and one-CTA-per-tile launches, every block size and the
    builds for 9 and 10 CTAs per SM: the same records (order inside a
    telescope aside)."""
    sc = _reduced(workloads.vertical_1tev(n=5_000), 5_000)
    ctx = context(sc)
    tr = host_tracks(sc, FP32)
    ref = None
    for launch in [(256, 3), (128, 0), (512, 1), (256, 8), (128, 5), (128, 9), (128, 10)]:
        code, stats, out = gpu_hits(ctx, tr, sc["t_ref"], SEED, FP32, 50_000, launch=launch)
        assert code == 0
        rec = out.records()
        if ref is None:
            ref = (rec, stats)
            continue
        assert np.array_equal(stats, ref[1])
        for k in rec:
            assert np.array_equal(rec[k], ref[0][k]), k


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_many_tiles_per_persistent_cta(prec):
    """A persistent launch where every CTA works through ~10 tiles (shared
    memory reused tile after tile) gives exactly the records of one CTA per
    tile, where nothing is reused."""
    sc = _reduced(workloads.vertical_1tev(n=200_003), 200_003)
    ctx = context(sc)
    tr = host_tracks(sc, prec)
    recs = []
    for launch in [(128, 0), (128, 1), (256, 1)]:
        code, stats, out = gpu_hits(ctx, tr, sc["t_ref"], SEED, prec, 400_000, launch=launch)
        assert code == 0
        recs.append((out.records(), stats))
    for rec, stats in recs[1:]:
        assert np.array_equal(stats, recs[0][1])
        for k in rec:
            assert np.array_equal(rec[k], recs[0][0][k]), k
    ctx.close()


def test_track_base_splits_reproduce():
    """Two calls over halves with track_base give the records of one call."""
    sc = _reduced(workloads.vertical_1tev(n=3_000), 3_000)
    ctx = context(sc)
    tr = host_tracks(sc, FP32)
    _, st, out = gpu_hits(ctx, tr, sc["t_ref"], SEED, FP32, 50_000)
    whole = out.records()
    parts = []
    for lo, hi in [(0, 1234), (1234, 3000)]:
        sub = {k: v[lo:hi] for k, v in tr.items()}
        _, _, o = gpu_hits(ctx, sub, sc["t_ref"], SEED, FP32, 50_000, track_base=lo)
        parts.append(o.records())
    cat = {k: np.concatenate([p[k] for p in parts]) for k in whole}
    order = np.lexsort((cat["key"], cat["tel"]))
    for k in whole:
        assert np.array_equal(cat[k][order], whole[k]), k


def test_edge_cases():
    sc = workloads.plain_fp64(n=300)
    ctx = context(sc)
    # empty input: nothing launched, counters cleared
    tr0 = host_tracks(sc, FP32, slice(0, 0))
    code, stats, out = gpu_hits(ctx, tr0, sc["t_ref"], SEED, FP32, 16)
    assert code == 0 and stats.sum() == 0 and out.count.sum().item() == 0
    # a single step, and every step below threshold
    tr1 = host_tracks(sc, FP32, slice(0, 1))
    code, stats, _ = gpu_hits(ctx, tr1, sc["t_ref"], SEED, FP32, 16)
    assert code == 0 and stats[0] == 1
    low = host_tracks(sc, FP32)
    low["ekin"] = np.full(len(low["ekin"]), 5.0)
    code, stats, out = gpu_hits(ctx, low, sc["t_ref"], SEED, FP32, 16)
    assert code == 0 and stats[1] == 0 and stats[3] == 0
    # invalid fields are counted, not propagated
    bad = host_tracks(sc, FP32)
    bad["len"][::7] = np.nan
    bad["ekin"][3::11] = -1.0
    bad["x0"][5::13] = np.inf
    bad["uy"][2::17] = np.nan
    code, stats, _ = gpu_hits(ctx, bad, sc["t_ref"], SEED, FP32, 4096)
    n_bad = np.sum(~np.isfinite(bad["len"]) | (bad["ekin"] <= 0) | ~np.isfinite(bad["x0"])
                   | ~np.isfinite(bad["uy"]))
    assert stats[2] == n_bad
    # capacity overflow: counted, never written past the buffer
    full = host_tracks(workloads.plain_fp64(n=1000), FP32)
    code, stats, out = gpu_hits(ctx, full, sc["t_ref"], SEED, FP32, 2)
    cnt = out.count.cpu().numpy()
    if cnt.max() > 2:
        assert code == 6
        assert stats[10] == np.maximum(cnt - 2, 0).sum()
    # a NULL track list is rejected before any launch
    assert P.lib().cher_generate_propagate(ctx._h, None, 0, 1, None, None) == 1
    ctx.close()


def test_full_size_vertical_shower_sampled():
    """2e6 steps (the benchmark's workload and launch shape): every bunch
    count against the oracle, and every crossing of 400 sampled steps."""
    sc = workloads.vertical_1tev()
    M = oracle_model(sc)
    ctx = context(sc)
    tr = host_tracks(sc, FP32)
    import torch
    dev = P.device_tracks(tr, FP32, t_ref=sc["t_ref"])
    nb_g, w_g = ctx.segment_yield(dev, FP32)
    nb_o, w_o, _, _ = M.segment_yield(tr)
    dw_max = compare_yield(nb_o, nb_g.cpu().numpy(), w_o, w_g.cpu().numpy(), FP32)
    out = ctx.alloc_hits(2_000_000, FP32)
    ctx.generate_propagate(dev, SEED, FP32, out)
    code, stats = ctx.sync_status(out)
    assert code == 0
    assert stats[3] == nb_o.sum()
    rec = out.records()
    assert stats[9] == len(rec["tel"])
    rng = np.random.default_rng(17)
    sample = np.sort(rng.choice(len(nb_o), 400, replace=False))
    sub = {k: v[sample] for k, v in tr.items()}
    # the oracle must see the same global step indices: run it per step
    o_all = []
    for i in sample:
        one = {k: v[i:i + 1] for k, v in tr.items()}
        o_all.append(M.bunches(one, SEED, track_base=int(i)))
    keys = set()
    for i, o in zip(sample, o_all):
        j = o["j"]
        keys |= set(((np.uint64(i) << np.uint64(32)) | j.astype(np.uint64)).tolist())
    sel = np.array([k in keys for k in rec["key"].tolist()], bool)
    grec = {k: v[sel] for k, v in rec.items()}
    got = 0
    for i, o in zip(sample, o_all):
        kk = set(((np.uint64(i) << np.uint64(32)) | o["j"].astype(np.uint64)).tolist())
        m = np.array([k in kk for k in grec["key"].tolist()], bool)
        r = compare_hits(M, o, {k: v[m] for k, v in grec.items()}, FP32, track_base=int(i))
        got += r["n_common"]
    assert got > 0
    torch.cuda.synchronize()
    tb = trace_blocks(M, ctx, tr, sc["t_ref"], SEED, FP32, rng)
    assert tb["n"] > 100_000
    MEASURED["vertical_1tev"] = dict(tb, max_dw_yield_all_steps=dw_max)
    ctx.close()


def test_graph_capture_replays_the_call():
    """A captured graph of the whole call gives the direct call's records,
    launch after launch."""
    sc = workloads.batched_256(total=20_000)
    ctx = context(sc)
    tr = host_tracks(sc, FP32)
    _, st_ref, out = gpu_hits(ctx, tr, sc["t_ref"], SEED, FP32, 50_000)
    ref = out.records()
    import torch
    dev = P.device_tracks(tr, FP32, t_ref=sc["t_ref"])
    out2 = ctx.alloc_hits(50_000, FP32)
    g = ctx.graph(dev, SEED, FP32, out2)
    for _ in range(3):
        out2.count.zero_()
        g.launch()
        code, st = ctx.sync_status(out2)
        assert code == 0
        assert np.array_equal(st, st_ref)
        rec = out2.records()
        for k in ref:
            assert np.array_equal(rec[k], ref[k]), k
    g.close()
    torch.cuda.synchronize()
    ctx.close()


def test_fp32_yield_screen_exact_at_integer_and_threshold_edges():
    """The FP32 path screens the yield in single precision and falls back to
    the FP64 chain when the bunch count is not certain.  Horizontal steps (the
    midpoint height then does not depend on the length) whose N/B lies within
    1e-12 .. 1e-6 of an integer, and steps at the Cherenkov threshold to
    1e-7, must give the oracle's bunch counts."""
    import math
    sc = workloads.plain_fp64(n=10)
    M = oracle_model(sc)
    ctx = context(sc)
    rng = np.random.default_rng(23)
    K = 2 * math.pi * 7.2973525693e-3 * (1e9 / 300.0 - 1e9 / 600.0)
    rows = []
    for _ in range(400):
        z = float(rng.uniform(0.0, 59000.0))
        e = float(np.exp(rng.uniform(math.log(25.0), math.log(5e4))))
        probe = dict(x0=[0.0], y0=[0.0], z0=[z], t0=[0.0], len=[1.0], ekin=[e],
                     ux=[1.0], uy=[0.0], uz=[0.0])
        _, _, s2, _ = M.segment_yield({k: np.array(v) for k, v in probe.items()})
        if not s2[0] > 0:
            continue
        for m in (1, 2, 7, 40, 173):
            for d in (-1e-6, -1e-9, -1e-12, 0.0, 1e-12, 1e-9, 1e-6):
                L = m * 5.0 / (K * s2[0]) * (1.0 + d)
                rows.append((z, e, L))
    # threshold: n at the height from the table, E_t from beta n = 1
    for z in np.linspace(0.0, 50000.0, 60):
        eta = oracle.eta_lookup(M.eta_tab, M.h_max, z)[0]
        n = 1.0 + eta
        e_t = 0.51099895 * (n / math.sqrt(n * n - 1.0) - 1.0)
        for d in (-1e-7, -1e-9, 0.0, 1e-9, 1e-7, 1e-5):
            rows.append((float(z), e_t * (1.0 + d), 7.5))
    rows = np.array(rows)
    n = len(rows)
    tr = dict(x0=np.zeros(n), y0=np.zeros(n), z0=rows[:, 0], t0=np.zeros(n), len=rows[:, 2],
              ekin=rows[:, 1], ux=np.ones(n), uy=np.zeros(n), uz=np.zeros(n),
              shower=np.zeros(n, np.uint32))
    nb_o, w_o, _, _ = M.segment_yield(tr)
    dev = P.device_tracks(tr, FP32, t_ref=sc["t_ref"])
    nb_g, w_g = ctx.segment_yield(dev, FP32)
    compare_yield(nb_o, nb_g.cpu().numpy(), w_o, w_g.cpu().numpy(), FP32)
    # and the fused kernel generates exactly that many bunches
    code, stats, _ = gpu_hits(ctx, tr, sc["t_ref"], SEED, FP32, 16)
    assert int(stats[3]) == int(nb_o.sum())
    ctx.close()


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_overflow_writes_nothing_past_the_buffers(prec):
    """Capacity overflow with canary words: every record buffer sits inside a
    larger allocation filled with a canary pattern.  After a launch whose
    telescopes overflow, the slots past each telescope's stored count and
    the words after the last telescope still hold the canary, and every
    stored record is a crossing of its own telescope in the oracle (a write
    past telescope k's capacity would land in telescope k + 1's slots with a
    key that does not cross k + 1)."""
    import torch
    sc = _reduced(workloads.vertical_1tev(n=4_001), 4_001)
    M = oracle_model(sc)
    ctx = context(sc)
    tr = host_tracks(sc, prec)
    o = M.bunches(tr, SEED)
    orec = oracle.hit_records(o)
    dist = sphere_distance(M, o)
    tol = 0.05 if prec == FP32 else 1e-6
    near = np.any(np.abs(dist) < tol, axis=1) | borderline_status(M, o, prec)
    seg_key = (o["seg"].astype(np.uint64) << np.uint64(32)) | o["j"].astype(np.uint64)
    near_keys = set(seg_key[near].tolist())
    crossing = set(zip(orec["tel"].tolist(), orec["key"].tolist()))
    # a capacity between the telescopes' counts: some overflow, some do not
    _, _, full = gpu_hits(ctx, tr, sc["t_ref"], SEED, prec, 100_000)
    c_full = np.sort(full.count.cpu().numpy())
    n_tel, tail = ctx.n_tel, 4096
    cap = int(max(1, c_full[n_tel // 2]))
    dt = torch.float32 if prec == FP32 else torch.float64
    CAN = -12345.0
    big = {k: torch.full((n_tel * cap + tail, 4), CAN, dtype=dt, device="cuda")
           for k in ("pos", "tim")}
    bigkey = torch.full((n_tel * cap + tail,), -7, dtype=torch.int64, device="cuda")
    out = P.HitBuffers(pos=big["pos"][:n_tel * cap].view(n_tel, cap, 4),
                       tim=big["tim"][:n_tel * cap].view(n_tel, cap, 4),
                       key=bigkey[:n_tel * cap].view(n_tel, cap),
                       count=torch.zeros(n_tel, dtype=torch.int64, device="cuda"),
                       stats=torch.zeros(P.NSTATS, dtype=torch.int64, device="cuda"),
                       cap=cap, precision=prec)
    dev = P.device_tracks(tr, prec, t_ref=sc["t_ref"])
    ctx.generate_propagate(dev, SEED, prec, out)
    code, stats = ctx.sync_status(out)
    cnt = out.count.cpu().numpy()
    assert code == 6 and stats[10] == np.maximum(cnt - cap, 0).sum() > 0
    assert (cnt > cap).sum() >= 3 and (cnt < cap).sum() >= 3   # both kinds present
    pos = big["pos"].cpu().numpy()
    tim = big["tim"].cpu().numpy()
    key = bigkey.cpu().numpy()
    assert np.all(pos[n_tel * cap:] == CAN) and np.all(tim[n_tel * cap:] == CAN)
    assert np.all(key[n_tel * cap:] == -7)
    for k in range(n_tel):
        stored = int(min(cnt[k], cap))
        sl = slice(k * cap + stored, (k + 1) * cap)
        assert np.all(pos[sl] == CAN) and np.all(tim[sl] == CAN) and np.all(key[sl] == -7)
        for r in range(k * cap, k * cap + stored):
            kk = int(key[r]) & 0xFFFFFFFFFFFFFFFF
            assert (k, kk) in crossing or kk in near_keys, (k, hex(kk))
    ctx.close()


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_library_refuses_steps_past_its_bunch_limit(prec):
    """The per-tile bunch scan runs in 32-bit integers, so the library counts
    a step of 2^22 bunches or more as invalid (stats[INVALID]) and emits
    nothing for it.  The oracle has no such limit: it gives that step
    ceil(N / B) bunches; every other step still matches it exactly."""
    sc = workloads.plain_fp64(n=300)
    ctx = context(sc)
    M = oracle_model(sc)
    tr = host_tracks(sc, prec)
    tr["len"][17] = 3.0e6                   # ~1.3e8 photons: past 2^22 bunches
    tr["z0"][17] = 1.0e4 + 1.5e6 * 1e-6     # midpoint at 10 km
    tr["uz"][17] = -1e-6 if prec == FP64 else float(np.float32(-1e-6))
    tr["ekin"][17] = 1000.0
    nb_o, w_o, _, valid_o = M.segment_yield(tr)
    assert valid_o[17] and nb_o[17] >= 2 ** 22
    dev = P.device_tracks(tr, prec, t_ref=sc["t_ref"])
    nb_g, w_g = ctx.segment_yield(dev, prec)
    nb_g = nb_g.cpu().numpy()
    assert nb_g[17] == 0
    keep = np.arange(len(nb_o)) != 17
    compare_yield(nb_o[keep], nb_g[keep], w_o[keep], w_g.cpu().numpy()[keep], prec)
    code, stats, _ = gpu_hits(ctx, tr, sc["t_ref"], SEED, prec, 4096)
    assert code == 0
    assert stats[2] == 1 and stats[3] == nb_o[keep].sum()
    ctx.close()
