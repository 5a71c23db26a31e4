"""Pins of the oracle's wavelength-dependent index of refraction.

n(h, lambda) - 1 = eta(h) kappa(lambda), kappa linear in 1/lambda between
nodes.  Checked against what does not come from the oracle's own formulas:
the per-step yield against numerical quadrature of the Frank-Tamm
integrand (1 - 1/(beta n)^2)_+ over the band, steps whose threshold falls
inside the band included; a constant kappa = c against the constant-index
path of an atmosphere whose n - 1 is scaled by c, bunch by bunch; every
bunch's wavenumber against the quadrature of its spectrum (the fraction of
the step's photons at shorter wavelengths is its Philox deviate); the
Cherenkov angle and Snell's invariant with the bunch's own index; the
tables interpolated in kappa against the ray integrals themselves; and no
bunch at a wavelength where beta n <= 1.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
import workloads

SEED = 53
ME = 0.51099895000
ALPHA = 7.2973525693e-3
KAPPA = workloads.synthetic_dispersion()


def _model(sc, dispersion=KAPPA, atm=None, H=200, Z=32):
    return oracle.Model(atm or sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"],
                        H=H, Z=Z, theta_max_deg=sc["theta_max_deg"], t_ref=sc["t_ref"],
                        dispersion=dispersion)


def _nodes(M):
    """Node wavenumbers (1/m) in ascending order, kappa at them."""
    k = np.asarray(M.dispersion, float)
    u = np.linspace(1e9 / M.lambda1_nm, 1e9 / M.lambda2_nm, k.size)
    return u[::-1], k[::-1]


def _step_beta_eta(M, tr, i):
    g = tr["ekin"][i] / ME
    beta = math.sqrt(g * (2 + g)) / (1 + g)
    hm = tr["z0"][i] + 0.5 * tr["len"][i] * tr["uz"][i]
    eta = oracle.eta_lookup(M.eta_tab, M.h_max, hm)[0]
    return beta, eta


def _density(u, beta, eta, un, kn):
    n = 1.0 + eta * np.interp(u, un, kn)
    return max(0.0, 1.0 - 1.0 / (beta * n) ** 2)


def _band_integral(M, beta, eta, lo=None, hi=None):
    un, kn = _nodes(M)
    lo = un[0] if lo is None else lo
    hi = un[-1] if hi is None else hi
    pts = [u for u in un if lo < u < hi]
    # the threshold, where beta n = 1, is a kink
    kth = (1.0 / beta - 1.0) / eta
    for a, b, ka, kb in zip(un[:-1], un[1:], kn[:-1], kn[1:]):
        if (ka - kth) * (kb - kth) < 0:
            pts.append(a + (kth - ka) / (kb - ka) * (b - a))
    v, _ = integrate.quad(_density, lo, hi, args=(beta, eta, un, kn), points=sorted(pts) or None,
                          epsabs=0.0, epsrel=1e-12, limit=200)
    return v


def _near_threshold_tracks(n=60, h=5000.0):
    """Steps at one height with energies across the band's threshold range."""
    e = np.linspace(26.5, 27.8, n)
    z = np.full(n, h)
    return dict(x0=np.zeros(n), y0=np.zeros(n), z0=z, t0=np.zeros(n), len=np.full(n, 50.0),
                ekin=e, ux=np.full(n, 0.1), uy=np.zeros(n), uz=np.full(n, -math.sqrt(0.99)),
                shower=np.zeros(n, np.uint32))


@pytest.fixture(scope="module")
def vertical():
    return workloads.vertical_1tev(n=1500)


def test_yield_is_the_band_integral(vertical):
    sc = vertical
    M = _model(sc)
    for tr, idx in ((sc["tracks"], range(0, 1500, 25)), (_near_threshold_tracks(), range(60))):
        nb, w, _, valid = M.segment_yield(tr)
        crossing = 0
        for i in idx:
            beta, eta = _step_beta_eta(M, tr, i)
            ref = tr["len"][i] * 2 * math.pi * ALPHA * _band_integral(M, beta, eta)
            N = nb[i] * w[i]
            if ref == 0.0:
                assert nb[i] == 0
                continue
            # (abs: the quadrature of 1 - 1/(beta n)^2 itself cancels near threshold)
            assert N == pytest.approx(ref, rel=1e-9, abs=1e-9), i
            assert nb[i] == math.ceil(N / 5.0 - 1e-9) or nb[i] == math.ceil(N / 5.0)
            kth = (1.0 / beta - 1.0) / eta
            crossing += KAPPA[-1] < kth < KAPPA[0]
        if tr is not sc["tracks"]:
            assert crossing >= 10          # the threshold fell inside the band
            assert (nb == 0).sum() >= 5    # and below it for the whole band


def test_constant_kappa_is_a_scaled_constant_index(vertical):
    sc = vertical
    c = 1.013
    Md = _model(sc, dispersion=np.full(5, c))
    Ms = _model(sc, dispersion=None, atm=dict(sc["atm"], n0_minus_1=sc["atm"]["n0_minus_1"] * c))
    od = Md.bunches(sc["tracks"], SEED)
    os_ = Ms.bunches(sc["tracks"], SEED)
    assert np.array_equal(od["nb"], os_["nb"])
    assert np.array_equal(od["status"], os_["status"])
    np.testing.assert_allclose(od["lam"], os_["lam"], rtol=1e-11)
    for k in ("px", "py", "pz", "cx", "cy", "cz"):
        np.testing.assert_allclose(od[k], os_[k], rtol=0, atol=1e-11, err_msg=k)
    np.testing.assert_allclose(od["X"], os_["X"], rtol=0, atol=1e-7)
    np.testing.assert_allclose(od["Y"], os_["Y"], rtol=0, atol=1e-7)
    np.testing.assert_allclose(od["t"], os_["t"], rtol=0, atol=1e-7)
    assert np.array_equal(od["nhit"], os_["nhit"])


def _bunches(sc, M, tr, variant=0):
    o = M.bunches(tr, SEED, variant=variant)
    return o


def test_wavelength_inverts_the_spectrum(vertical):
    sc = vertical
    M = _model(sc)
    tr = _near_threshold_tracks(n=40)
    for src in (sc["tracks"], tr):
        o = M.bunches(src, SEED)
        steps = np.unique(o["seg"])[:: max(1, len(np.unique(o["seg"])) // 12)]
        checked = 0
        for i in steps:
            beta, eta = _step_beta_eta(M, src, i)
            total = _band_integral(M, beta, eta)
            sel = np.nonzero(o["seg"] == i)[0][:6]
            words = oracle.philox_stream(SEED, int(i), int(o["j"][sel[0]]), len(sel))
            for b, wd in zip(sel, words):
                u2 = (float(wd[2]) + 0.5) / 4294967296.0
                u = 1e9 / o["lam"][b]
                short = _band_integral(M, beta, eta, lo=u)      # 1/lambda above the bunch's
                assert short / total == pytest.approx(u2, abs=2e-9), (i, b)
                checked += 1
        assert checked >= 30, checked


def test_angle_snell_and_threshold(vertical):
    sc = vertical
    M = _model(sc)
    un, kn = _nodes(M)
    tr = sc["tracks"]
    o = M.bunches(tr, SEED)
    i = o["seg"]
    g = tr["ekin"][i] / ME
    beta = np.sqrt(g * (2 + g)) / (1 + g)
    hm = tr["z0"][i] + 0.5 * tr["len"][i] * tr["uz"][i]
    eta_m = np.array([oracle.eta_lookup(M.eta_tab, M.h_max, h)[0] for h in hm[:4000]])
    kap = np.interp(1e9 / o["lam"], un, kn)
    sl = slice(0, 4000)
    cos_ref = 1.0 / (beta[sl] * (1 + eta_m * kap[sl]))
    cos_got = o["px"][sl] * tr["ux"][i[sl]] + o["py"][sl] * tr["uy"][i[sl]] + \
        o["pz"][sl] * tr["uz"][i[sl]]
    np.testing.assert_allclose(cos_got, cos_ref, rtol=0, atol=2e-12)
    assert np.all(beta[sl] * (1 + eta_m * kap[sl]) > 1.0)
    # Snell with the bunch's index, emission point to the ground
    gnd = np.nonzero(o["status"][sl] == oracle.ST_GROUND)[0]
    assert gnd.size > 1000
    eta_e = np.array([oracle.eta_lookup(M.eta_tab, M.h_max, h)[0] for h in o["he"][gnd]])
    eta_o = oracle.eta_lookup(M.eta_tab, M.h_max, M.h_obs)[0]
    s_em = np.hypot(o["px"][gnd], o["py"][gnd])
    s_obs = np.hypot(o["cx"][gnd], o["cy"][gnd])
    np.testing.assert_allclose((1 + kap[gnd] * eta_o) * s_obs, (1 + kap[gnd] * eta_e) * s_em,
                               rtol=1e-13)
    # the spectrum leans to the short end where n is larger: more than the
    # 1/lambda^2 share (one half of the photons below 400 nm) falls there
    assert (o["lam"] < 400.0).mean() > 0.5


def test_kappa_tables_match_the_ray_integrals(vertical):
    """(T) with the kappa-interpolated tables against (B) with the exact
    n = 1 + kappa eta(h), at random heights, zeniths and kappas in the band:
    the constant-index bound (2 mm, 10 ps) holds."""
    sc = vertical
    M = _model(sc, H=1000, Z=64)
    rng = np.random.default_rng(8)
    worst_x = worst_t = 0.0
    for _ in range(150):
        th = math.radians(rng.uniform(0, 68))
        ph = rng.uniform(0, 6.28)
        p = (math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), -math.cos(th))
        he = rng.uniform(2300, 59000)
        kap = rng.uniform(KAPPA[-1], KAPPA[0])
        sT, rT = M.propagate_photon(0.0, 0.0, he, 0.0, *p, variant=0, kappa=kap)
        sB, rB = M.propagate_photon(0.0, 0.0, he, 0.0, *p, variant=1, kappa=kap)
        assert sT == sB == oracle.ST_GROUND
        worst_x = max(worst_x, abs(rT[0] - rB[0]), abs(rT[1] - rB[1]))
        worst_t = max(worst_t, abs(rT[2] - rB[2]))
    assert worst_x < 2e-3
    assert worst_t < 1e-2
    # the kappa interpolation matters: the band's ends differ by far more
    _, r_hi = M.propagate_photon(0.0, 0.0, 30000.0, 0.0, 0.6, 0.0, -0.8, variant=1,
                                 kappa=KAPPA[0])
    _, r_lo = M.propagate_photon(0.0, 0.0, 30000.0, 0.0, 0.6, 0.0, -0.8, variant=1,
                                 kappa=KAPPA[-1])
    assert abs(r_hi[0] - r_lo[0]) > 0.05


def test_dispersion_settings_are_checked(vertical):
    sc = vertical
    for bad in ([1.0], [1.0] * 10, [1.0, 1.01], [1.0, 0.0], [1.0, -0.5]):
        with pytest.raises(ValueError):
            _model(sc, dispersion=bad)
