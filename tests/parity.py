"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and
the oracle on the same seeded inputs, compare element by element.

Tolerances (the FP64 path against the FP64 oracle; the FP32-bulk path with
the stated accuracy targets):

* bunch counts nb: bit-exact on both paths (the FP64 path evaluates the
  yield in FP64 in the oracle's operation order; the FP32 path screens it in
  FP32 with a rounding-error bound and falls back to that FP64 chain
  whenever the count is not certain);
* FP64 path: relative 1e-9 of max(|value|, scale), scale 1 km for ground
  coordinates and 1 us for times (the sizes of the terms they are formed
  from), 1e-9 for direction cosines;
* FP32 path: 5 cm in ground position, 0.1 ns in arrival time, 1e-5 in
  direction cosines, 1e-5 relative in photons per bunch (the yield is
  screened in FP32 and kept only where the Cherenkov-threshold cancellation
  costs at most a factor ~10: a few ulp of n - 1 times A / num <= 11, about
  4e-6; nearer the threshold the FP64 chain gives them), 1e-6 relative in
  wavelength (24-bit deviate against the oracle's 32-bit one, < 3e-8, plus
  the FP32 inversion's few ulp);
* statuses and telescope crossings: exact, after leaving out the bunches
  whose oracle value lies within the path's precision of a decision
  boundary (5 cm of a sphere surface or of h_obs / h_max, 1e-5 of the
  largest sin^2 zenith, 1e-6 of horizontal travel, 2e-5 between the
  transmission draw u3 and its survival probability for FP32 -- the FP32
  probability is an FP32 exponential of an FP32-interpolated depth; 1e-6 m /
  1e-12 for FP64).  The number left out is reported and must stay far below
  1 %.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
import paper_2006_14927_gb300 as P

FP32 = P.CHER_FP32_BULK
FP64 = P.CHER_FP64

TOL = {
    FP64: dict(pos_rel=1e-9, pos_scale=1e3, t_rel=1e-9, t_scale=1e3, dir=1e-9, rel=1e-12,
               edge_m=1e-6, edge_q=1e-12, edge_pz=1e-12, edge_tr=1e-12),
    FP32: dict(pos_abs=0.05, t_abs=0.1, dir=1e-5, rel=1e-5, edge_m=0.05, edge_q=1e-5,
               edge_pz=1e-6, edge_tr=2e-5),
}


def oracle_model(sc: dict) -> oracle.Model:
    return oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"],
                        n_fine=sc["n_fine"], H=sc["H"], Z=sc["Z"],
                        theta_max_deg=sc["theta_max_deg"], bunch_size=sc["bunch_size"],
                        lambda1_nm=sc["lambda1_nm"], lambda2_nm=sc["lambda2_nm"],
                        t_ref=sc["t_ref"])


def context(sc: dict) -> P.Context:
    ctx = P.Context(sc["atm"], sc["h_obs"], sc["telescopes"], bunch_size=sc["bunch_size"],
                    lambda_min_nm=sc["lambda1_nm"], lambda_max_nm=sc["lambda2_nm"],
                    n_fine=sc["n_fine"])
    ctx.build_refraction_tables(sc["H"], sc["Z"], sc["theta_max_deg"], sc["h_max"])
    return ctx


def host_tracks(sc: dict, precision: int, sl=slice(None)) -> dict:
    """The tracks as both sides see them: for the FP32 path the directions
    are rounded to float first, and the oracle gets those same values."""
    tr = {k: np.asarray(v[sl]) for k, v in sc["tracks"].items()}
    if precision == FP32:
        for k in ("ux", "uy", "uz"):
            tr[k] = tr[k].astype(np.float32).astype(np.float64)
    return tr


def gpu_trace(ctx: P.Context, tr: dict, t_ref, seed: int, precision: int, track_base=0):
    import torch
    dev = P.device_tracks(tr, precision, t_ref=t_ref)
    nb, w = ctx.segment_yield(dev, precision)
    off = torch.zeros(len(tr["x0"]) + 1, dtype=torch.int64, device="cuda")
    off[1:] = torch.cumsum(nb.to(torch.int64), 0)
    out = ctx.trace_bunches(dev, seed, precision, off, track_base=track_base)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["nb"] = nb.cpu().numpy()
    res["w"] = w.cpu().numpy()
    return res


def gpu_hits(ctx: P.Context, tr: dict, t_ref, seed: int, precision: int, cap: int,
             track_base=0, launch=None):
    dev = P.device_tracks(tr, precision, t_ref=t_ref)
    if launch is not None:
        ctx.set_launch(*launch)
    out = ctx.alloc_hits(cap, precision)
    ctx.generate_propagate(dev, seed, precision, out, track_base=track_base)
    code, stats = ctx.sync_status(out)
    return code, stats, out


def _eta_interp(M: oracle.Model, h):
    grid = np.arange(M.n_fine) * (M.h_max / (M.n_fine - 1))
    return np.interp(h, grid, M.eta_tab)


def bunch_kappa(M: oracle.Model, o: dict):
    """The (n - 1) scale at each bunch's wavelength (1 for a constant index)."""
    kap = getattr(M, "dispersion", None)
    if kap is None:
        return 1.0
    kap = np.asarray(kap, float)
    u = np.linspace(1.0 / M.lambda1_nm, 1.0 / M.lambda2_nm, kap.size)
    return np.interp(1.0 / o["lam"], u[::-1], kap[::-1])


def borderline_status(M: oracle.Model, o: dict, precision: int) -> np.ndarray:
    """Bunches whose oracle drop decision is within the path's precision."""
    t = TOL[precision]
    he = o["he"]
    kap = bunch_kappa(M, o)
    ratio = (1 + kap * _eta_interp(M, he)) / (1 + kap * _eta_interp(M, M.h_obs))
    R = getattr(M, "earth_radius", 0.0)
    if R > 0.0:
        # curved: the local vertical at the emission point (he is radial)
        rho2 = o["xe"] ** 2 + o["ye"] ** 2
        zc = np.sqrt(np.maximum((R + he) ** 2 - rho2, 0.0))
        rv = np.stack([o["xe"], o["ye"], zc], 1) / (R + he)[:, None]
        pv = np.stack([o["px"], o["py"], o["pz"]], 1)
        ce = np.sum(pv * rv, 1)
        se2 = np.sum(np.cross(pv, rv) ** 2, 1)
        near = np.abs(ce) < t["edge_pz"]
        q = se2 * ((R + he) / (R + M.h_obs)) ** 2 * ratio ** 2
    else:
        near = np.abs(o["pz"]) < t["edge_pz"]
        q = (o["px"] ** 2 + o["py"] ** 2) * ratio ** 2
    near |= np.abs(he - M.h_obs) < t["edge_m"]
    near |= np.abs(he - M.h_max) < t["edge_m"]
    q_max = math.sin(M.theta_max_rad) ** 2
    near |= np.abs(q - q_max) < t["edge_q"]
    if "tr_margin" in o:       # the transmission draw u3 < P
        near |= np.abs(np.nan_to_num(o["tr_margin"], nan=1.0)) < t["edge_tr"]
    return near


def sphere_distance(M: oracle.Model, o: dict) -> np.ndarray:
    """Distance from each ground-reaching bunch's arrival line to each sphere
    centre minus the radius, (n_bunch, n_tel); +inf for dropped bunches."""
    g = o["status"] == oracle.ST_GROUND
    T = M.telescopes
    out = np.full((len(g), T.shape[0]), np.inf)
    if not g.any():
        return out
    zg = o["Zg"][g] if "Zg" in o else np.zeros(g.sum())
    P0 = np.stack([o["X"][g], o["Y"][g], zg], 1)
    D = np.stack([o["cx"][g], o["cy"][g], o["cz"][g]], 1)
    for k, (tx, ty, tz, tr) in enumerate(T):
        d = np.array([tx, ty, tz])[None, :] - P0
        out[g, k] = np.linalg.norm(np.cross(d, D), axis=1) - tr
    return out


def compare_yield(o_nb, g_nb, o_w, g_w, precision=FP64):
    """Bunch counts bit-exact; photons per bunch to 1e-15 (FP64) or 1e-5
    relative plus 1e-6 photons (FP32: the yield is screened in FP32 and its
    photon count keeps FP32 rounding, amplified at most ~10 times by the
    threshold cancellation).  Returns the largest relative photon error."""
    assert np.array_equal(o_nb, g_nb), f"{np.sum(o_nb != g_nb)} bunch counts differ"
    if precision == FP64:
        np.testing.assert_allclose(g_w, o_w, rtol=1e-15, atol=0)
    else:
        np.testing.assert_allclose(g_w, o_w, rtol=TOL[FP32]["rel"], atol=1e-6)
    m = o_w > 0
    return float(np.max(np.abs(g_w[m] - o_w[m]) / o_w[m], initial=0.0))


def compare_trace(M: oracle.Model, o: dict, g: dict, precision: int) -> dict:
    """Per-bunch comparison; returns the largest errors and the count left out."""
    t = TOL[precision]
    n = len(o["status"])
    assert len(g["status"]) == n
    edge = borderline_status(M, o, precision)
    st_o, st_g = o["status"], g["status"]
    bad = (st_o != st_g) & ~edge
    assert not bad.any(), f"{bad.sum()} statuses differ off the boundaries, first at {np.argmax(bad)}"
    both = (st_o == oracle.ST_GROUND) & (st_g == oracle.ST_GROUND)
    pos, tim = g["pos"].astype(np.float64), g["tim"].astype(np.float64)
    dX = np.abs(pos[both, 0] - o["X"][both])
    dY = np.abs(pos[both, 1] - o["Y"][both])
    dcx = np.abs(pos[both, 2] - o["cx"][both])
    dcy = np.abs(pos[both, 3] - o["cy"][both])
    dt = np.abs(tim[both, 0] - o["t"][both])
    # emission height, photons and wavelength exist for every bunch
    dz = np.abs(tim[:, 1] - o["he"])
    dw = np.abs(tim[:, 2] - o["w"]) / o["w"]
    dl = np.abs(tim[:, 3] - o["lam"]) / o["lam"]
    if precision == FP64:
        sX = np.maximum(np.abs(o["X"][both]), t["pos_scale"])
        sY = np.maximum(np.abs(o["Y"][both]), t["pos_scale"])
        st = np.maximum(np.abs(o["t"][both]), t["t_scale"])
        assert np.all(dX <= t["pos_rel"] * sX), dX.max()
        assert np.all(dY <= t["pos_rel"] * sY), dY.max()
        assert np.all(dt <= t["t_rel"] * st), dt.max()
        assert np.all(dz <= 1e-9 * np.maximum(np.abs(o["he"]), 1e3)), dz.max()
    else:
        assert np.all(dX <= t["pos_abs"]), dX.max()
        assert np.all(dY <= t["pos_abs"]), dY.max()
        assert np.all(dt <= t["t_abs"]), dt.max()
        assert np.all(dz <= t["pos_abs"]), dz.max()
    assert np.all(dcx <= t["dir"]) and np.all(dcy <= t["dir"]), (dcx.max(), dcy.max())
    assert np.all(dw <= t["rel"] + 1e-6 / o["w"]), dw.max()
    if getattr(M, "dispersion", None) is None:
        lam_tol = 1e-6 if precision == FP32 else 1e-14
    else:
        # a wavelength-dependent index inverts each step's spectrum through a
        # quadratic per piece: near the Cherenkov threshold the density falls
        # to zero at the cut and the inversion amplifies rounding (seen: 4.5e-6
        # in FP32, 2e-14 in FP64).  2e-5 of the wavelength moves kappa by
        # ~1e-6 and n by ~2e-10, far below what the cone, Snell and time
        # tolerances above can see; FP64 keeps 1e-12, inside its 1e-9 bar.
        lam_tol = 2e-5 if precision == FP32 else 1e-12
    assert np.all(dl <= lam_tol), dl.max()
    # crossings per bunch
    dist = sphere_distance(M, o)
    hit_edge = np.any(np.abs(dist) < t["edge_m"], axis=1)
    ok = both & ~hit_edge
    assert np.array_equal(g["nhit"][ok], np.minimum(o["nhit"][ok], 32))
    first_o = np.where(o["nhit"] > 0, o["hit_tel"][:, 0], -1)
    assert np.array_equal(g["first_hit"][ok], first_o[ok])
    return dict(n=n, edge_status=int(edge.sum()), edge_hit=int((both & hit_edge).sum()),
                max_dX=float(max(dX.max(initial=0), dY.max(initial=0))),
                max_dt=float(dt.max(initial=0)),
                max_ddir=float(max(dcx.max(initial=0), dcy.max(initial=0))),
                max_dw=float(dw.max(initial=0)), max_dlam=float(dl.max(initial=0)))


def trace_blocks(M: oracle.Model, ctx: P.Context, tracks: dict, t_ref, seed: int, precision: int,
                 rng, n_blocks: int = 12, block: int = 2000) -> dict:
    """Every bunch of n_blocks runs of `block` consecutive steps, at random
    places of a (large) step list, traced on the device and by the oracle
    with the steps' own global indices (track_base = the run's first step):
    the largest errors over all of them and the bunches compared."""
    n = len(tracks["x0"])
    starts = np.sort(rng.choice(max(n - block, 1), n_blocks, replace=False))
    agg = dict(n=0, edge_status=0, edge_hit=0, max_dX=0.0, max_dt=0.0, max_ddir=0.0,
               max_dw=0.0, max_dlam=0.0)
    for s0 in starts.tolist():
        sub = {k: np.asarray(v)[s0:s0 + block] for k, v in tracks.items()}
        if precision == FP32:
            for k in ("ux", "uy", "uz"):
                sub[k] = sub[k].astype(np.float32).astype(np.float64)
        o = M.bunches(sub, seed, track_base=int(s0))
        g = gpu_trace(ctx, sub, t_ref, seed, precision, track_base=int(s0))
        r = compare_trace(M, o, g, precision)
        for k in agg:
            agg[k] = agg[k] + r[k] if k in ("n", "edge_status", "edge_hit") else max(agg[k], r[k])
    return agg


def compare_hits(M: oracle.Model, o: dict, grec: dict, precision: int, track_base=0,
                 restrict_keys=None) -> dict:
    """Compare hit records (sorted by telescope and key)."""
    t = TOL[precision]
    orec = oracle.hit_records(o, track_base)
    dist = sphere_distance(M, o)
    edge_b = np.any(np.abs(dist) < t["edge_m"], axis=1) | borderline_status(M, o, precision)
    seg_key = ((o["seg"] + track_base).astype(np.uint64) << np.uint64(32)) | \
        o["j"].astype(np.uint64)
    edge_keys = set(seg_key[edge_b].tolist())
    gk = list(zip(grec["tel"].tolist(), grec["key"].tolist()))
    ok_ = list(zip(orec["tel"].tolist(), orec["key"].tolist()))
    if restrict_keys is not None:
        gk = [p for p in gk if p[1] in restrict_keys]
    sg, so = set(gk), set(ok_)
    assert len(sg) == len(gk), "duplicate records in a telescope buffer"
    diff = {p for p in sg ^ so if p[1] not in edge_keys}
    assert not diff, f"{len(diff)} crossings differ, e.g. {sorted(diff)[:3]}"
    common = sorted(sg & so)
    gi = {p: i for i, p in enumerate(zip(grec["tel"].tolist(), grec["key"].tolist()))}
    oi = {p: i for i, p in enumerate(ok_)}
    ig = np.array([gi[p] for p in common], dtype=np.int64)
    io = np.array([oi[p] for p in common], dtype=np.int64)
    res = dict(n_common=len(common), n_edge=len((sg ^ so) - diff))
    if len(common) == 0:
        return res
    dx = np.abs(grec["x"][ig] - orec["x"][io])
    dy = np.abs(grec["y"][ig] - orec["y"][io])
    dt_ = np.abs(grec["t"][ig] - orec["t"][io])
    dcx = np.abs(grec["cx"][ig] - orec["cx"][io])
    dw = np.abs(grec["w"][ig] - orec["w"][io]) / orec["w"][io]
    if precision == FP64:
        assert dx.max() <= 1e-9 * t["pos_scale"] and dy.max() <= 1e-9 * t["pos_scale"]
        assert dt_.max() <= 1e-9 * t["t_scale"]
    else:
        assert dx.max() <= t["pos_abs"] and dy.max() <= t["pos_abs"], (dx.max(), dy.max())
        assert dt_.max() <= t["t_abs"], dt_.max()
    assert dcx.max() <= t["dir"]
    assert dw.max() <= t["rel"]
    res.update(max_dxy=float(max(dx.max(), dy.max())), max_dt=float(dt_.max()))
    return res
