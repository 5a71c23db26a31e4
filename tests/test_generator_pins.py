"""Pins of the oracle's parameterised shower-step generator.

Each sampled quantity is checked against the distribution the generator
states, through a route of its own: the depths against the Greisen profile
integrated here with scipy's adaptive quadrature (Kolmogorov-Smirnov), the
lateral offsets recovered geometrically from the positions (exponential,
mean 50 m, uniform azimuth), the energies (log-uniform), the angles to the
axis scaled by their stated width (Rayleigh), the start times from the
distance along the axis, the lengths (uniform); plus convergence of the
tabulated inverse CDF.
"""
import math

import numpy as np
import pytest

import oracle

scipy_integrate = pytest.importorskip("scipy.integrate")
scipy_stats = pytest.importorskip("scipy.stats")

H_OBS = 2200.0
E_C, X0, X_SEA, H = 85.0, 36.7, 1030.0, 8000.0


@pytest.fixture(scope="module")
def gen():
    sh = [dict(e0_mev=1.0e6, zenith=0.35, azimuth=2.0, core_x=40.0, core_y=-15.0, n=60000),
          dict(e0_mev=5.0e4, zenith=0.0, azimuth=0.0, core_x=0.0, core_y=0.0, n=20000)]
    return sh, oracle.generate_steps(sh, H_OBS, 1234)


def _axis(s):
    sz = math.sin(s["zenith"])
    return np.array([sz * math.cos(s["azimuth"]), sz * math.sin(s["azimuth"]),
                     -math.cos(s["zenith"])])


def _slice(sh, k):
    a = sum(s["n"] for s in sh[:k])
    return slice(a, a + sh[k]["n"])


@pytest.mark.parametrize("k", [0, 1])
def test_depth_follows_the_greisen_profile(gen, k):
    sh, o = gen
    s, sl = sh[k], _slice(sh, k)
    cz = math.cos(s["zenith"])
    y = math.log(s["e0_mev"] / E_C)
    t_g = X_SEA * math.exp(-H_OBS / H) / cz / X0
    prof = lambda t: math.exp(t * (1.0 - 1.5 * math.log(3.0 * t / (t + 2.0 * y)))) if t > 0 else 1.0
    tot = scipy_integrate.quad(prof, 0.0, t_g, limit=200)[0]
    # the depth of each step from its height (isothermal slant depth)
    t = X_SEA * np.exp(-o["z0"][sl] / H) / cz / X0
    # heights clamped at 29999 m are the shallowest tail: leave them out of
    # the comparison by restricting both CDFs to t >= t_cut
    t_cut = X_SEA * math.exp(-29999.0 / H) / cz / X0 * 1.0001
    t = np.sort(t[t >= t_cut])
    F0 = scipy_integrate.quad(prof, 0.0, t_cut, limit=200)[0] / tot
    probe = np.quantile(t, np.linspace(0.01, 0.99, 40))
    emp = np.searchsorted(t, probe, side="right") / t.size
    ref = np.array([(scipy_integrate.quad(prof, 0.0, q, limit=200)[0] / tot - F0) / (1 - F0)
                    for q in probe])
    assert np.max(np.abs(emp - ref)) < 1.63 / math.sqrt(t.size) * 1.5


@pytest.mark.parametrize("k", [0, 1])
def test_lateral_offsets_are_exponential_and_isotropic(gen, k):
    sh, o = gen
    s, sl = sh[k], _slice(sh, k)
    ax = _axis(s)
    core = np.array([s["core_x"], s["core_y"], H_OBS])
    d = np.stack([o["x0"][sl], o["y0"][sl], o["z0"][sl]], 1) - core
    along = d @ ax
    lat = d - along[:, None] * ax
    r = np.linalg.norm(lat, axis=1)
    assert scipy_stats.kstest(r, "expon", args=(0.0, 50.0)).pvalue > 1e-3
    # azimuth in a fixed transverse basis
    b1 = np.cross(ax, [0.0, 0.0, 1.0])
    b1 = b1 / np.linalg.norm(b1) if np.linalg.norm(b1) > 1e-12 else np.array([1.0, 0, 0])
    b2 = np.cross(ax, b1)
    psi = np.mod(np.arctan2(lat @ b2, lat @ b1), 2 * math.pi)
    assert scipy_stats.kstest(psi, "uniform", args=(0.0, 2 * math.pi)).pvalue > 1e-3
    # start time = distance to the 30 km plane along the axis, at c
    s_ref = (30000.0 - H_OBS) / math.cos(s["zenith"])
    np.testing.assert_allclose(o["t0"][sl] * 0.299792458, s_ref + along, rtol=0, atol=1e-6)
    assert np.allclose(o["t_ref"][k] * 0.299792458, s_ref, rtol=1e-14)
    assert np.all(o["shower"][sl] == k)


def test_energies_lengths_and_directions(gen):
    sh, o = gen
    e = o["ekin"]
    assert e.min() >= 20.0 and e.max() <= 5000.0
    assert scipy_stats.kstest(np.log(e), "uniform",
                              args=(math.log(20.0), math.log(250.0))).pvalue > 1e-3
    assert scipy_stats.kstest(o["len"], "uniform", args=(1.0, 19.0)).pvalue > 1e-3
    u = np.stack([o["ux"], o["uy"], o["uz"]], 1)
    np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, rtol=0, atol=1e-14)
    # angle to the axis over its width: Rayleigh(1) in the small-angle limit
    sl = _slice(sh, 0)
    ang = np.arccos(np.clip(u[sl] @ _axis(sh[0]), -1, 1))
    sig = math.radians(3.0) * 50.0 / e[sl]
    sel = sig < math.radians(0.5)
    assert scipy_stats.kstest(ang[sel] / np.arctan(sig[sel]), "rayleigh").pvalue > 1e-3


def test_inverse_cdf_table_converges(gen):
    sh, o = gen
    o2 = oracle.generate_steps(sh, H_OBS, 1234, n_cdf=8192)
    dz = np.abs(o2["z0"] - o["z0"])
    assert np.median(dz) < 0.05 and dz.max() < 20.0
    for k in ("ekin", "len", "ux"):
        assert np.array_equal(o2[k], o[k])


def test_bad_showers_are_refused():
    with pytest.raises(ValueError):
        oracle.generate_steps([dict(e0_mev=50.0, zenith=0.0, azimuth=0.0, core_x=0.0,
                                    core_y=0.0, n=10)], H_OBS, 1)
    with pytest.raises(ValueError):
        oracle.generate_steps([dict(e0_mev=1e5, zenith=1.6, azimuth=0.0, core_x=0.0,
                                    core_y=0.0, n=10)], H_OBS, 1)
