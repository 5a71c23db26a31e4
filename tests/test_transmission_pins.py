"""Pins of the oracle's atmospheric transmission draw.

A bunch that reaches the observation level survives when its fourth
Philox deviate is below exp(-tau / cos(theta_obs)), tau interpolated in a
(wavelength, height) table.  Checked without retyping the oracle: a zero
table changes nothing; only ground-level bunches can be lost and nothing
else about a bunch changes; doubling the table only removes survivors; the
survival fraction, overall, per zenith band and per wavelength band,
follows Beer-Lambert within binomial errors (a linear law, a cosine instead
of a secant or a swapped table axis fails); the draw is independent of the
emission point; and a table that is a plane in (lambda, h) gives the same
decisions on any grid (bilinear interpolation of a plane is exact, so an
indexing or weight error shows).
"""
import numpy as np
import pytest

import oracle
import workloads

SEED = 31


def _model(sc, transmission=None):
    return oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"], H=200,
                        Z=32, theta_max_deg=sc["theta_max_deg"], t_ref=sc["t_ref"],
                        transmission=transmission)


def _table(tau, lam=(250.0, 700.0), h=(2200.0, 60000.0)):
    return dict(tau=np.asarray(tau, float), lambda_nm=lam, height_m=h)


@pytest.fixture(scope="module")
def base():
    sc = workloads.vertical_1tev(n=2500)
    o = _model(sc).bunches(sc["tracks"], SEED)
    return sc, o


def test_zero_table_changes_nothing(base):
    sc, o0 = base
    o1 = _model(sc, _table(np.zeros((4, 5)))).bunches(sc["tracks"], SEED)
    for k in ("status", "X", "Y", "t", "cx", "cy", "lam", "he", "nhit"):
        assert np.array_equal(o0[k], o1[k]), k


def test_only_ground_bunches_are_lost(base):
    sc, o0 = base
    o1 = _model(sc, workloads.synthetic_transmission()).bunches(sc["tracks"], SEED)
    g = o0["status"] == oracle.ST_GROUND
    assert np.array_equal(o1["status"][~g], o0["status"][~g])
    assert set(np.unique(o1["status"][g])) <= {oracle.ST_GROUND, oracle.ST_ABSORBED}
    lost = o1["status"] == oracle.ST_ABSORBED
    assert 0.05 < lost.sum() / g.sum() < 0.95
    kept = o1["status"] == oracle.ST_GROUND
    for k in ("X", "Y", "t", "cx", "cy", "cz"):           # survivors arrive unchanged
        assert np.array_equal(o0[k][kept], o1[k][kept]), k
    for k in ("lam", "he", "w"):
        assert np.array_equal(o0[k], o1[k]), k
    assert np.all(o1["nhit"][lost] == 0)
    assert np.array_equal(o1["nhit"][kept], o0["nhit"][kept])


def test_more_optical_depth_only_removes_survivors(base):
    sc, _ = base
    tr = workloads.synthetic_transmission()
    o1 = _model(sc, tr).bunches(sc["tracks"], SEED)
    tr2 = dict(tr, tau=2.0 * tr["tau"])
    o2 = _model(sc, tr2).bunches(sc["tracks"], SEED)
    s1 = o1["status"] == oracle.ST_GROUND
    s2 = o2["status"] == oracle.ST_GROUND
    assert np.all(s1[s2])
    assert s2.sum() < s1.sum()


def _binomial_ok(surv, p, n_sigma=4.5):
    n = surv.size
    exp = p.sum()
    sd = np.sqrt((p * (1 - p)).sum())
    return abs(surv.sum() - exp) <= n_sigma * sd + 1, (surv.sum(), exp, sd)


@pytest.fixture(scope="module")
def inclined():
    sc = workloads.inclined_20tev(n=1500)
    sc["theta_max_deg"] = 75.0
    o = _model(sc).bunches(sc["tracks"], SEED)
    return sc, o


@pytest.mark.parametrize("tau0", [0.1, 0.7])
@pytest.mark.parametrize("which", ["base", "inclined"])
def test_survival_follows_beer_lambert_per_zenith_band(request, which, tau0):
    sc, o0 = request.getfixturevalue(which)
    o1 = _model(sc, _table(np.full((3, 3), tau0))).bunches(sc["tracks"], SEED)
    g = o0["status"] == oracle.ST_GROUND
    cos_obs = -o0["cz"][g]
    surv = o1["status"][g] == oracle.ST_GROUND
    p = np.exp(-tau0 / cos_obs)
    ok, info = _binomial_ok(surv, p)
    assert ok, info
    edges = np.quantile(cos_obs, [0, 0.25, 0.5, 0.75, 1.0])
    for a, b in zip(edges[:-1], edges[1:]):
        sel = (cos_obs >= a) & (cos_obs <= b)
        ok, info = _binomial_ok(surv[sel], p[sel])
        assert ok, (a, b, info)
    # the 60 degree shower's photons tell the secant from a cosine
    if which == "inclined":
        c = np.exp(-tau0 * cos_obs)
        assert abs(c.sum() - p.sum()) > 8 * np.sqrt((p * (1 - p)).sum())
    # at this depth a linear law 1 - tau/cos would predict a visibly
    # different fraction
    if tau0 > 0.5:
        lin = np.clip(1.0 - tau0 / cos_obs, 0, 1)
        assert abs(lin.sum() - p.sum()) > 6 * np.sqrt((p * (1 - p)).sum())


def test_survival_follows_the_wavelength_axis(base):
    sc, o0 = base
    lam_nodes = np.linspace(250.0, 700.0, 10)
    tau = np.repeat((0.4 * (lam_nodes / 400.0) ** -4.0)[:, None], 4, axis=1)
    o1 = _model(sc, _table(tau)).bunches(sc["tracks"], SEED)
    g = o0["status"] == oracle.ST_GROUND
    lam = o0["lam"][g]
    t = np.interp(lam, lam_nodes, tau[:, 0])
    p = np.exp(-t / -o0["cz"][g])
    surv = o1["status"][g] == oracle.ST_GROUND
    for a, b in ((300, 350), (350, 420), (420, 520), (520, 600)):
        sel = (lam >= a) & (lam < b)
        ok, info = _binomial_ok(surv[sel], p[sel])
        assert ok, (a, b, info)
    # the short wavelengths are lost far more often
    assert surv[lam < 340].mean() < surv[lam > 500].mean() - 0.2


def test_draw_is_independent_of_the_emission_point(base):
    sc, o0 = base
    o1 = _model(sc, _table(np.full((2, 2), 0.5))).bunches(sc["tracks"], SEED)
    g = o0["status"] == oracle.ST_GROUND
    seg = o0["seg"][g]
    # position of the emission inside its step, in [0, 1)
    z0 = sc["tracks"]["z0"][seg]
    L = sc["tracks"]["len"][seg] * sc["tracks"]["uz"][seg]
    f = np.where(np.abs(L) > 1e-9, (o0["he"][g] - z0) / np.where(np.abs(L) > 1e-9, L, 1), 0.5)
    surv = (o1["status"][g] == oracle.ST_GROUND).astype(float)
    r = np.corrcoef(f, surv)[0, 1]
    assert abs(r) < 5.0 / np.sqrt(surv.size)


def test_plane_table_is_grid_independent(base):
    sc, o0 = base
    def plane(nl, nh):
        lam = np.linspace(250.0, 700.0, nl)
        h = np.linspace(2200.0, 60000.0, nh)
        return _table(0.05 + 6e-4 * (700.0 - lam)[:, None] + 8e-6 * (60000.0 - h)[None, :])
    a = _model(sc, plane(2, 2)).bunches(sc["tracks"], SEED)
    b = _model(sc, plane(17, 53)).bunches(sc["tracks"], SEED)
    assert np.array_equal(a["status"], b["status"])
    g = o0["status"] == oracle.ST_GROUND
    lost = (a["status"][g] == oracle.ST_ABSORBED).mean()
    assert 0.1 < lost < 0.9
