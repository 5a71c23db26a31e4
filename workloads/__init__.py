"""Seeded synthetic workloads: shower-shaped sets of e+- track segments.

These stand in for CORSIKA/EGS4 output and for the paper's workload of 2500
gamma-ray showers of a CTA production (paper section 5.2), neither of which
exists outside a CORSIKA installation.  The module draws inputs only: it holds
none of the arithmetic of the photon-bunch method, and both the CUDA path and
the CPU oracle read what it returns.

Every generator uses ``numpy.random.Generator(PCG64(seed))``.  The five
workloads:

* ``plain_fp64``   1000 segments, start heights U(5, 25) km, directions within
  2 degrees of vertical, E_kin log-uniform 30 MeV - 1 GeV, length U(1, 20) m,
  one sphere of radius 12 m at the origin, tables 1000 x 64 up to 70 deg.
* ``vertical_1tev`` one 1 TeV vertical gamma-like shower, 2e6 segments with
  heights from a Greisen longitudinal profile (maximum near 8-9 km), energies
  log-uniform 20 MeV - 5 GeV, angular spread Gaussian of 3 deg * (50 MeV/E),
  lateral offsets exponential with scale 50 m; 19 spheres of radius U(6, 12) m
  on a hexagonal grid of pitch 120 m.
* ``batched_256``  256 showers, E0 log-uniform 10 GeV - 10 TeV, segment count
  proportional to E0 clamped to [1e3, 1e7], 2e8 in total; zenith U(0, 40 deg);
  cores uniform over 2 x 2 km; 100 spheres (60 x 6 m, 35 x 12 m, 5 x 23 m)
  scattered without overlap over 2 x 2 km.
* ``adjoint_300gev`` 1e5 segments of a 300 GeV vertical shower, 19 spheres.
* ``inclined_20tev`` 1e8 segments of a 20 TeV shower at 60 deg zenith, tables
  4000 x 256 up to 75 deg, the 100 spheres of ``batched_256``.

Depth-to-height mapping of the synthetic showers uses an isothermal
atmosphere X(h) = 1030 g/cm^2 exp(-h / 8 km); it only places the segments
and is unrelated to the layered atmosphere the method propagates through.
"""
from __future__ import annotations

import math

import numpy as np

C_LIGHT = 0.299792458          # m/ns, to stamp segment start times
X0_RAD = 36.7                  # radiation length of air, g/cm^2
E_CRIT = 85.0                  # critical energy of air, MeV
X_SEA = 1030.0                 # isothermal sea-level depth, g/cm^2
H_SCALE = 8000.0               # isothermal scale height, m
H_START = 30000.0              # height at which the synthetic clock starts, m


def us_standard_atmosphere(n0_minus_1: float = 2.83e-4) -> dict:
    """Five-layer exponential thickness profile T(h) = a_i + b_i exp(-h/c_i).

    Layers 1-4 use the US-standard (Linsley) parameters as published for
    CORSIKA (c in m).  Layer 5 (above 100 km) is written in the same
    exponential form with a_5 chosen so that T is continuous at 100 km; no
    workload propagates light above 75 km, so it never enters a result.
    """
    a = [-186.555305, -94.919, 0.61289, 0.0, 0.0]
    b = [1222.6562, 1144.9069, 1305.5948, 540.1778, 1.0]
    c = [9941.8638, 8781.5355, 6361.4304, 7721.7016, 1.0e7]
    t4_top = a[3] + b[3] * math.exp(-100000.0 / c[3])
    a[4] = t4_top - b[4] * math.exp(-100000.0 / c[4])
    h_top = -c[4] * math.log(-a[4] / b[4])      # where layer 5 reaches T = 0
    return dict(h_bound=[0.0, 4000.0, 10000.0, 40000.0, 100000.0, h_top],
                a=a, b=b, c=c, n0_minus_1=n0_minus_1)


def hex_telescopes(rng, n: int = 19, pitch: float = 120.0, r_lo: float = 6.0,
                   r_hi: float = 12.0) -> np.ndarray:
    """Centre plus hexagonal rings of spacing `pitch`; radii U(r_lo, r_hi)."""
    pts = [(0.0, 0.0)]
    ring = 1
    while len(pts) < n:
        corners = [(ring * pitch * math.cos(math.pi / 3 * k),
                    ring * pitch * math.sin(math.pi / 3 * k)) for k in range(6)]
        for k in range(6):
            x0, y0 = corners[k]
            x1, y1 = corners[(k + 1) % 6]
            for s in range(ring):
                f = s / ring
                pts.append((x0 + f * (x1 - x0), y0 + f * (y1 - y0)))
        ring += 1
    pts = np.array(pts[:n])
    r = rng.uniform(r_lo, r_hi, n)
    return np.column_stack([pts[:, 0], pts[:, 1], np.zeros(n), r])


def scattered_telescopes(rng, counts=(60, 35, 5), radii=(6.0, 12.0, 23.0),
                         half: float = 1000.0, gap: float = 2.0) -> np.ndarray:
    """Spheres placed uniformly over [-half, half]^2 with no two overlapping."""
    out = []
    for cnt, r in sorted(zip(counts, radii), key=lambda p: -p[1]):
        placed = 0
        while placed < cnt:
            x, y = rng.uniform(-half, half, 2)
            if all(math.hypot(x - q[0], y - q[1]) > r + q[3] + gap for q in out):
                out.append((x, y, 0.0, r))
                placed += 1
    return np.array(out)


def _log_uniform(rng, lo, hi, n):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), n))


def _greisen_sampler(e0_mev: float, t_max: float, npts: int = 4096):
    """Inverse-CDF table of the Greisen profile N(t) in t = X/X0 on (0, t_max]."""
    y = math.log(e0_mev / E_CRIT)
    t = np.linspace(t_max / npts, t_max, npts)
    s = 3.0 * t / (t + 2.0 * y)
    pdf = np.exp(t * (1.0 - 1.5 * np.log(s))) / math.sqrt(y)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(t))])
    cdf /= cdf[-1]
    return t, cdf


def _depth_to_height(x_vert):
    return H_SCALE * np.log(X_SEA / np.maximum(x_vert, 1e-6))


def shower_segments(rng, n: int, e0_mev: float, zenith: float, azimuth: float,
                    core_x: float, core_y: float, h_obs: float,
                    e_lo: float = 20.0, e_hi: float = 5000.0):
    """Segments of one shower along an axis of the given zenith and azimuth.

    Returns a dict of float64 arrays plus the reference time t_ref at which
    the axis reaches the observation level.
    """
    cz = math.cos(zenith)
    axis = np.array([math.sin(zenith) * math.cos(azimuth),
                     math.sin(zenith) * math.sin(azimuth), -cz])
    # transverse basis of the axis
    b1 = np.cross(axis, [0.0, 0.0, 1.0]) if abs(axis[2]) < 0.999999 else np.array([1.0, 0, 0])
    b1 /= np.linalg.norm(b1)
    b2 = np.cross(axis, b1)
    x_ground = X_SEA * math.exp(-h_obs / H_SCALE) / cz        # slant depth at ground
    tg, cdf = _greisen_sampler(e0_mev, x_ground / X0_RAD)
    t = np.interp(rng.uniform(0.0, 1.0, n), cdf, tg)
    h = _depth_to_height(t * X0_RAD * cz)
    h = np.minimum(h, H_START - 1.0)
    s = (h - h_obs) / cz                                       # distance up the axis
    r = rng.exponential(50.0, n)
    psi = rng.uniform(0.0, 2.0 * math.pi, n)
    lat = (r * np.cos(psi))[:, None] * b1 + (r * np.sin(psi))[:, None] * b2
    pos = np.array([core_x, core_y, h_obs]) - s[:, None] * axis + lat
    ekin = _log_uniform(rng, e_lo, e_hi, n)
    sig = math.radians(3.0) * (50.0 / ekin)
    tx = rng.normal(0.0, 1.0, n) * sig
    ty = rng.normal(0.0, 1.0, n) * sig
    d = axis + tx[:, None] * b1 + ty[:, None] * b2
    d /= np.linalg.norm(d, axis=1)[:, None]
    s_ref = (H_START - h_obs) / cz
    return dict(x0=pos[:, 0], y0=pos[:, 1], z0=pos[:, 2],
                t0=(s_ref - s) / C_LIGHT,
                len=rng.uniform(1.0, 20.0, n), ekin=ekin,
                ux=d[:, 0], uy=d[:, 1], uz=d[:, 2]), s_ref / C_LIGHT


def _scenario(name, tracks, telescopes, t_ref, seed, h_obs=2200.0, H=1000, Z=64,
              theta_max_deg=70.0, h_max=60000.0):
    n = len(tracks["x0"])
    if "shower" not in tracks:
        tracks["shower"] = np.zeros(n, np.uint32)
    n_sh = len(np.atleast_1d(t_ref))
    return dict(name=name, axis_zenith_rad=np.zeros(n_sh), tracks=tracks, telescopes=np.asarray(telescopes, float),
                t_ref=np.atleast_1d(np.asarray(t_ref, float)),
                atm=us_standard_atmosphere(), h_obs=h_obs, h_max=h_max, n_fine=10000,
                H=H, Z=Z, theta_max_deg=theta_max_deg, bunch_size=5.0,
                lambda1_nm=300.0, lambda2_nm=600.0, seed=seed)


def synthetic_transmission(h_obs: float = 2200.0, h_max: float = 60000.0, n_lambda: int = 16,
                           n_height: int = 121, tau_rayleigh: float = 0.36,
                           tau_aerosol: float = 0.10) -> dict:
    """A stand-in for an external transmission profile: vertical optical
    depth between height h and h_obs, Rayleigh scattering (lambda^-4, scale
    height 8.4 km, tau_rayleigh at 400 nm from sea level) plus aerosols
    (lambda^-1.3, scale height 1.2 km, tau_aerosol at 400 nm from sea
    level), on a uniform (lambda, h) grid over 250-700 nm and [h_obs, h_max]."""
    lam = np.linspace(250.0, 700.0, n_lambda)
    h = np.linspace(h_obs, h_max, n_height)
    ray = tau_rayleigh * (lam / 400.0) ** -4.0
    aer = tau_aerosol * (lam / 400.0) ** -1.3
    col_r = np.exp(-h_obs / 8400.0) - np.exp(-h / 8400.0)
    col_a = np.exp(-h_obs / 1200.0) - np.exp(-h / 1200.0)
    tau = ray[:, None] * col_r[None, :] + aer[:, None] * col_a[None, :]
    return dict(tau=tau, lambda_nm=(float(lam[0]), float(lam[-1])),
                height_m=(float(h[0]), float(h[-1])))


def synthetic_dispersion(k: int = 9, lambda1_nm: float = 300.0, lambda2_nm: float = 600.0,
                         lambda_ref_nm: float = 400.0) -> np.ndarray:
    """A stand-in for a measured dispersion curve of air: kappa(lambda) =
    (n(lambda) - 1) / (n(lambda_ref) - 1) from Edlen's 1966 formula for
    standard air, (n - 1) 1e8 = 8342.13 + 2406030 / (130 - s^2) +
    15997 / (38.9 - s^2) with s the vacuum wavenumber in 1/um, at k nodes
    uniform in 1/lambda from 1/lambda1 (node 0, the short end) to 1/lambda2.
    About +3 % at 300 nm and -2 % at 600 nm against 400 nm."""
    def edlen(lam_nm):
        s2 = (1000.0 / lam_nm) ** 2
        return 8342.13 + 2406030.0 / (130.0 - s2) + 15997.0 / (38.9 - s2)
    u = np.linspace(1.0 / lambda1_nm, 1.0 / lambda2_nm, k)
    return edlen(1.0 / u) / edlen(lambda_ref_nm)


def plain_fp64(n: int = 1000, seed: int = 1) -> dict:
    rng = np.random.Generator(np.random.PCG64(seed))
    z0 = rng.uniform(5000.0, 25000.0, n)
    ct = rng.uniform(math.cos(math.radians(2.0)), 1.0, n)
    st = np.sqrt(1.0 - ct * ct)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    tracks = dict(x0=rng.uniform(-50.0, 50.0, n), y0=rng.uniform(-50.0, 50.0, n), z0=z0,
                  t0=(H_START - z0) / C_LIGHT,
                  len=rng.uniform(1.0, 20.0, n), ekin=_log_uniform(rng, 30.0, 1000.0, n),
                  ux=st * np.cos(ph), uy=st * np.sin(ph), uz=-ct)
    return _scenario("plain_fp64", tracks, [[0.0, 0.0, 0.0, 12.0]],
                     (H_START - 2200.0) / C_LIGHT, seed)


def vertical_1tev(n: int = 2_000_000, seed: int = 2, e0_mev: float = 1.0e6) -> dict:
    rng = np.random.Generator(np.random.PCG64(seed))
    tel = hex_telescopes(rng)
    tracks, t_ref = shower_segments(rng, n, e0_mev, 0.0, 0.0, 0.0, 0.0, 2200.0)
    return _scenario("vertical_1tev", tracks, tel, t_ref, seed)


def adjoint_300gev(n: int = 100_000, seed: int = 4) -> dict:
    sc = vertical_1tev(n, seed, e0_mev=3.0e5)
    sc["name"] = "adjoint_300gev"
    return sc


def _shower_counts(e0, total, lo=1000, hi=10_000_000):
    """Counts proportional to e0, clamped to [lo, hi], summing to `total`."""
    k_lo, k_hi = 0.0, float(total) / e0.min() * 10
    for _ in range(200):
        k = 0.5 * (k_lo + k_hi)
        s = np.clip(np.round(k * e0), lo, hi).sum()
        if s < total:
            k_lo = k
        else:
            k_hi = k
    cnt = np.clip(np.round(k_hi * e0), lo, hi).astype(np.int64)
    cnt[np.argmax(cnt)] += total - cnt.sum()       # exact total
    return cnt


def batched_256(total: int = 200_000_000, n_showers: int = 256, seed: int = 3) -> dict:
    rng = np.random.Generator(np.random.PCG64(seed))
    tel = scattered_telescopes(rng)
    e0 = _log_uniform(rng, 1.0e4, 1.0e7, n_showers)
    zen = np.radians(rng.uniform(0.0, 40.0, n_showers))
    az = rng.uniform(0.0, 2.0 * math.pi, n_showers)
    cx = rng.uniform(-1000.0, 1000.0, n_showers)
    cy = rng.uniform(-1000.0, 1000.0, n_showers)
    lo = max(1, min(1000, total // (4 * n_showers)))
    cnt = _shower_counts(e0, total, lo=lo, hi=max(lo, min(10_000_000, total)))
    keys = ("x0", "y0", "z0", "t0", "len", "ekin", "ux", "uy", "uz")
    tracks = {k: np.empty(total) for k in keys}
    tracks["shower"] = np.empty(total, np.uint32)
    t_ref = np.empty(n_showers)
    o = 0
    for s in range(n_showers):
        seg, t_ref[s] = shower_segments(rng, int(cnt[s]), float(e0[s]), float(zen[s]),
                                        float(az[s]), float(cx[s]), float(cy[s]), 2200.0)
        m = int(cnt[s])
        for k in keys:
            tracks[k][o:o + m] = seg[k]
        tracks["shower"][o:o + m] = s
        o += m
    sc = _scenario("batched_256", tracks, tel, t_ref, seed)
    sc["shower_counts"] = cnt
    sc["primary_energy_mev"] = e0
    sc["axis_zenith_rad"] = zen
    return sc


def inclined_20tev(n: int = 100_000_000, seed: int = 5) -> dict:
    rng = np.random.Generator(np.random.PCG64(seed))
    tel = scattered_telescopes(np.random.Generator(np.random.PCG64(3)))
    tracks, t_ref = shower_segments(rng, n, 2.0e7, math.radians(60.0), 0.0, 0.0, 0.0, 2200.0)
    sc = _scenario("inclined_20tev", tracks, tel, t_ref, seed, H=4000, Z=256,
                   theta_max_deg=75.0)
    sc["axis_zenith_rad"] = np.array([math.radians(60.0)])
    return sc


WORKLOADS = {
    "plain_fp64": plain_fp64,
    "vertical_1tev": vertical_1tev,
    "batched_256": batched_256,
    "adjoint_300gev": adjoint_300gev,
    "inclined_20tev": inclined_20tev,
}
