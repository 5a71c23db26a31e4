"""Pins of the FP64 oracle to what the paper and the physics fix.

None of these compare the oracle with itself: each checks it against a
published value (Philox known answers), a closed form (Cherenkov threshold,
Frank-Tamm in the textbook form, straight rays when n = 1, piecewise-constant
slabs, the vertical optical path from the thickness profile), a conservation
law (photons, bunches), or a distribution (the 1/lambda^2 spectrum, uniform
azimuth).  A dropped term, a wrong sign or a transposed operand in any step
of the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALPHA = 7.2973525693e-3          # CODATA 2018
ME = 0.51099895                  # MeV
C = 0.299792458                  # m/ns


def _atm():
    return workloads.us_standard_atmosphere()


def _model(**kw):
    args = dict(atm=_atm(), h_obs=2200.0, telescopes=np.array([[0.0, 0.0, 0.0, 12.0]]),
                H=200, Z=32)
    args.update(kw)
    return oracle.Model(**args)


def _slab_atm(rho1, rho2, hb, n0m1=2.83e-4):
    """Two slabs of (almost exactly) constant density: rho1 below hb, rho2 above.

    A scale height of 1e15 m makes exp(-h/c) constant to 1e-10 over 100 km.
    """
    c = 1.0e15
    bnd = [0.0, hb, 2.0e5, 3.0e5, 4.0e5, 5.0e5]
    b = [rho1 * c, rho2 * c, rho2 * c, rho2 * c, rho2 * c]
    return dict(h_bound=bnd, a=[0.0] * 5, b=b, c=[c] * 5, n0_minus_1=n0m1)


# --------------------------------------------------------------------------
# Philox4x32-10: published known answers, uniformity
# --------------------------------------------------------------------------
def test_philox_known_answers():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        got = oracle.philox4x32_10(v[0:4], v[4:6])
        assert got.tolist() == v[6:10]


def test_philox_uniform_chi2():
    w = oracle.philox_stream(seed=987654321, track=42, j0=0, n=250_000).ravel()
    counts = np.bincount(w >> np.uint32(24), minlength=256)     # top byte
    exp = len(w) / 256.0
    chi2 = ((counts - exp) ** 2 / exp).sum()
    # 255 degrees of freedom: mean 255, sd 22.6; 6 sd band
    assert 120 < chi2 < 390
    bits = np.unpackbits(w.view(np.uint8)).mean()
    assert abs(bits - 0.5) < 5e-4


# --------------------------------------------------------------------------
# Atmosphere tables (fast interpolation, paper section 3.3.2)
# --------------------------------------------------------------------------
def test_eta_sea_level_and_table_nodes():
    atm = _atm()
    assert oracle.eta_exact(atm, 0.0)[0] == pytest.approx(2.83e-4, rel=1e-15)
    M = _model()
    h = np.arange(0, M.n_fine) * (M.h_max / (M.n_fine - 1))
    sel = h[::97]
    # at the nodes the lookup returns the node value
    got = oracle.eta_lookup(M.eta_tab, M.h_max, sel)
    assert np.allclose(got, oracle.eta_exact(atm, sel), rtol=1e-14, atol=0)


def test_eta_table_accuracy_10000_points():
    """10000 uniform points interpolate n-1 to ~1e-7 inside a layer (the paper's
    'excellent agreement' with on-demand interpolation)."""
    atm = _atm()
    M = _model()
    rng = np.random.default_rng(0)
    hs = rng.uniform(0, M.h_max, 3000)
    dh = M.h_max / (M.n_fine - 1)
    # cells that straddle a layer boundary see the density jump: skip them
    keep = np.ones_like(hs, bool)
    for b in atm["h_bound"][1:5]:
        keep &= np.abs(hs - b) > 2 * dh
    hs = hs[keep]
    got = oracle.eta_lookup(M.eta_tab, M.h_max, hs)
    ref = oracle.eta_exact(atm, hs)
    assert np.max(np.abs(got / ref - 1)) < 2e-7


def test_density_is_derivative_of_thickness():
    atm = _atm()
    for h in [100.0, 3000.0, 7000.0, 25000.0, 55000.0]:
        d = 1e-3
        fd = -(oracle.thickness(atm, h + d)[0] - oracle.thickness(atm, h - d)[0]) / (2 * d)
        assert oracle.rho(atm, h)[0] == pytest.approx(fd, rel=1e-7)


# --------------------------------------------------------------------------
# a1: Cherenkov threshold and Frank-Tamm yield (CERENK)
# --------------------------------------------------------------------------
def _yield_one(M, z0, ekin, length=10.0):
    tr = dict(z0=np.array([z0 + 0.5 * length]), len=np.array([length]),
              ekin=np.array([ekin]), uz=np.array([-1.0]))
    nb, w, s2, valid = M.segment_yield(tr)
    return nb[0], w[0], s2[0], valid[0]


def test_cherenkov_threshold():
    """Emission starts where beta n = 1: gamma_t = n / sqrt(n^2 - 1).
    At sea level (n - 1 = 2.83e-4) the electron threshold is about 21 MeV."""
    M = _model()
    dh = M.h_max / (M.n_fine - 1)
    for node in [0, 700, 2000]:
        h = node * dh                     # midpoint exactly on a table node
        n = 1.0 + oracle.eta_exact(M.atm, h)[0]
        gam_t = n / math.sqrt(n * n - 1.0)
        e_t = ME * (gam_t - 1.0)
        if node == 0:
            assert 20.9 < e_t < 21.1
        assert _yield_one(M, h, e_t * (1 - 1e-7))[0] == 0
        assert _yield_one(M, h, e_t * (1 + 1e-5))[0] > 0


def test_frank_tamm_textbook_form():
    """N = L 2 pi alpha (1 - 1/(beta n)^2)(1/l1 - 1/l2), beta from E and m_e;
    nb = ceil(N / 5) bunches of N / nb photons."""
    M = _model()
    dh = M.h_max / (M.n_fine - 1)
    rng = np.random.default_rng(1)
    for _ in range(200):
        h = rng.integers(0, 3000) * dh
        e = math.exp(rng.uniform(math.log(40.0), math.log(1e5)))
        L = rng.uniform(1, 20)
        n = 1.0 + oracle.eta_exact(M.atm, h)[0]
        gam = (e + ME) / ME
        beta = math.sqrt(1.0 - 1.0 / gam ** 2)
        N = L * 2 * math.pi * ALPHA * (1 - 1 / (beta * n) ** 2) * (1 / 300e-9 - 1 / 600e-9)
        nb, w, s2, valid = _yield_one(M, h, e, L)
        assert valid
        if N <= 0:
            assert nb == 0
            continue
        assert nb == math.ceil(N / 5.0)
        assert nb * w == pytest.approx(N, rel=1e-9)
        assert w <= 5.0 + 1e-12
        assert s2 == pytest.approx(1 - 1 / (beta * n) ** 2, rel=1e-8)


def test_frank_tamm_ultrarelativistic_sea_level():
    """beta -> 1 at sea level: about 43 photons per metre in 300-600 nm."""
    M = _model()
    nb, w, s2, _ = _yield_one(M, 0.0, 1e7, 10.0)
    n = 1.000283
    per_m = 2 * math.pi * ALPHA * (1 - 1 / n ** 2) * (1 / 300e-9 - 1 / 600e-9)
    assert nb * w / 10.0 == pytest.approx(per_m, rel=1e-6)
    assert 43.0 < per_m < 43.5


def test_no_bunch_count_limit_in_the_oracle():
    """The Frank-Tamm count has no upper limit: a 200 km step at sea-level
    density (about 8.7e6 photons, 1.7e6 bunches) and a 2000 km one (17e6
    bunches, past 2^22) both get nb = ceil(N / B) of the textbook N, valid."""
    M = _model()
    n = 1.0 + oracle.eta_exact(M.atm, 0.0)[0]
    e = 1.0e7
    gam = (e + ME) / ME
    beta = math.sqrt(1.0 - 1.0 / gam ** 2)
    for L in (2.0e5, 2.0e6):
        tr = dict(z0=np.array([0.5 * L * 1e-9]), len=np.array([L]), ekin=np.array([e]),
                  uz=np.array([-1e-9]))
        nb, w, s2, valid = M.segment_yield(tr)
        N = L * 2 * math.pi * ALPHA * (1 - 1 / (beta * n) ** 2) * (1 / 300e-9 - 1 / 600e-9)
        assert valid[0]
        assert nb[0] == math.ceil(N / 5.0)
        assert nb[0] * w[0] == pytest.approx(N, rel=1e-9)
    assert nb[0] > 2 ** 22


def test_invalid_steps_are_flagged():
    M = _model()
    tr = dict(z0=np.array([1e4, np.nan, 1e4, 1e4]), len=np.array([5.0, 5.0, -1.0, 5.0]),
              ekin=np.array([100.0, 100.0, 100.0, np.inf]), uz=np.array([-1.0] * 4))
    nb, w, s2, valid = M.segment_yield(tr)
    assert valid.tolist() == [True, False, False, False]
    assert nb[1:].tolist() == [0, 0, 0]


# --------------------------------------------------------------------------
# a3: propagation (RAYBND) -- closed forms
# --------------------------------------------------------------------------
def _dir(theta, phi):
    return (math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi),
            -math.cos(theta))


@pytest.mark.parametrize("variant", [0, 1])
def test_no_air_gives_straight_lines(variant):
    """n = 1 everywhere: the photon goes in a straight line at c."""
    atm = _atm()
    atm["n0_minus_1"] = 0.0
    M = _model(atm=atm)
    assert np.all(M.ax == 0) and np.all(M.al == 0)
    rng = np.random.default_rng(2)
    for _ in range(50):
        th = math.radians(rng.uniform(0, 69))
        ph = rng.uniform(0, 2 * math.pi)
        p = _dir(th, ph)
        xe, ye, he, te = rng.uniform(-100, 100), rng.uniform(-100, 100), \
            rng.uniform(2300, 59000), rng.uniform(0, 100)
        st, r = M.propagate_photon(xe, ye, he, te, *p, variant=variant)
        assert st == oracle.ST_GROUND
        path = (he - 2200.0) / -p[2]
        assert r[0] == pytest.approx(xe + p[0] * path, abs=1e-8)
        assert r[1] == pytest.approx(ye + p[1] * path, abs=1e-8)
        assert r[2] == pytest.approx(te + path / C, abs=1e-9)
        assert r[3:6] == pytest.approx(p, abs=1e-14)


def test_two_slab_refraction_closed_form():
    """Piecewise-constant index: straight in each slab, Snell at the interface.
    (B) must match anywhere; (T) at table nodes."""
    hb_idx = 40
    H, Z, h_obs, h_max = 201, 33, 2200.0, 60000.0
    dht = (h_max - h_obs) / (H - 1)
    hb = h_obs + hb_idx * dht
    atm = _slab_atm(0.10, 0.04, hb)
    M = _model(atm=atm, H=H, Z=Z, h_obs=h_obs, h_max=h_max)
    n1 = 1.0 + 2.83e-4 * 0.10 / 0.10
    n2 = 1.0 + 2.83e-4 * 0.04 / 0.10
    q_max = math.sin(math.radians(70.0)) ** 2

    def exact(h, sin_obs):
        s1 = sin_obs
        s2 = n1 * s1 / n2
        c1, c2 = math.sqrt(1 - s1 * s1), math.sqrt(1 - s2 * s2)
        a, b = min(h, hb) - h_obs, max(h - hb, 0.0)
        x = a * s1 / c1 + b * s2 / c2
        l_ = n1 * a / c1 + n2 * b / c2
        return x, l_

    # brute force at arbitrary points
    rng = np.random.default_rng(3)
    for _ in range(40):
        h = rng.uniform(h_obs + 10, h_max)
        so = math.sqrt(rng.uniform(0, q_max))
        x, l_ = oracle.brute_ray(atm, h_obs, h, so)
        xe, le = exact(h, so)
        assert x == pytest.approx(xe, rel=1e-9, abs=1e-9)
        assert l_ == pytest.approx(le, rel=1e-12)
    # table variant at nodes (heights on the grid, sin^2 on the grid)
    # (the node at the interface itself is left out: the fine n table
    # interpolates across the density jump there)
    for j in [1, hb_idx - 7, hb_idx + 3, H - 1]:
        for k in [0, 5, 17, Z - 1]:
            h = h_obs + j * dht
            so = math.sqrt(k * q_max / (Z - 1))
            # emission direction that refracts to sin_obs at the ground
            s_em = so * n1 / (n1 if h < hb else n2)
            p = (s_em, 0.0, -math.sqrt(1 - s_em * s_em))
            st, r = M.propagate_photon(0.0, 0.0, h, 0.0, *p, variant=0)
            assert st == oracle.ST_GROUND
            xe, le = exact(h, so)
            assert r[0] == pytest.approx(xe, rel=1e-9, abs=1e-8)
            assert r[2] * C == pytest.approx(le, rel=1e-11)


def test_vertical_optical_path_from_thickness():
    """theta = 0: the optical excess is (n0 - 1)/rho(0) times the air column
    between the two heights, sum over layers of b_i (e^{-lo/c_i} - e^{-hi/c_i})."""
    atm = _atm()
    M = _model(H=300, Z=16)
    dht = (M.h_max - M.h_obs) / (M.H - 1)
    rho0 = atm["b"][0] / atm["c"][0]

    def column(lo, hi):
        s = 0.0
        for i in range(5):
            a_, b_ = max(lo, atm["h_bound"][i]), min(hi, atm["h_bound"][i + 1])
            if b_ > a_:
                s += atm["b"][i] * (math.exp(-a_ / atm["c"][i]) - math.exp(-b_ / atm["c"][i]))
        return s

    for j in [1, 5, 31, 150, 299]:
        h = M.h_obs + j * dht
        ref = atm["n0_minus_1"] / rho0 * column(M.h_obs, h)
        assert M.al[j, 0] == pytest.approx(ref, rel=1e-11)
        # horizontal column: int (n_obs/n - 1) dh to second order in eta
        eo = oracle.eta_exact(atm, M.h_obs)[0]
        k1 = atm["n0_minus_1"] / rho0
        i1 = k1 * column(M.h_obs, h)                       # int eta
        i2 = 0.0                                           # int eta^2
        for i in range(5):
            a_, b_ = max(M.h_obs, atm["h_bound"][i]), min(h, atm["h_bound"][i + 1])
            if b_ > a_:
                r_ = atm["b"][i] / atm["c"][i]
                i2 += k1 ** 2 * r_ ** 2 * atm["c"][i] / 2 * \
                    (math.exp(-2 * a_ / atm["c"][i]) - math.exp(-2 * b_ / atm["c"][i]))
        dH = h - M.h_obs
        # (1+eo)/(1+e) - 1 = (eo - e)(1 - e + e^2 ...)
        approx = eo * dH - i1 - eo * i1 + i2
        assert M.ax[j, 0] == pytest.approx(approx, rel=2e-6, abs=1e-9)


def test_snell_invariant_table_variant():
    M = _model()
    rng = np.random.default_rng(4)
    for _ in range(100):
        th = math.radians(rng.uniform(0.1, 60))
        p = _dir(th, rng.uniform(0, 6.28))
        he = rng.uniform(2300, 59000)
        st, r = M.propagate_photon(0.0, 0.0, he, 0.0, *p, variant=0)
        assert st == oracle.ST_GROUND
        n_e = 1 + oracle.eta_lookup(M.eta_tab, M.h_max, he)[0]
        n_o = 1 + oracle.eta_lookup(M.eta_tab, M.h_max, M.h_obs)[0]
        s_obs = math.hypot(r[3], r[4])
        assert n_o * s_obs == pytest.approx(n_e * math.sin(th), rel=1e-14)
        # direction stays a unit vector and points down
        assert r[3] ** 2 + r[4] ** 2 + r[5] ** 2 == pytest.approx(1.0, abs=1e-14)
        assert r[5] < 0


def test_table_matches_brute_force_between_nodes():
    """(T) against (B) at random (h, theta): interpolation error of the
    normalised tables stays below 2 mm / 10 ps at 1000 x 64 up to 70 deg."""
    M = _model(H=1000, Z=64)
    rng = np.random.default_rng(5)
    worst_x = worst_t = 0.0
    for _ in range(300):
        th = math.radians(rng.uniform(0, 68))
        p = _dir(th, rng.uniform(0, 6.28))
        he = rng.uniform(2300, 59000)
        sT, rT = M.propagate_photon(0.0, 0.0, he, 0.0, *p, variant=0)
        sB, rB = M.propagate_photon(0.0, 0.0, he, 0.0, *p, variant=1)
        assert sT == sB == oracle.ST_GROUND
        worst_x = max(worst_x, abs(rT[0] - rB[0]), abs(rT[1] - rB[1]))
        worst_t = max(worst_t, abs(rT[2] - rB[2]))
    assert worst_x < 2e-3
    assert worst_t < 1e-2


def test_rare_conditions():
    M = _model()
    st, _ = M.propagate_photon(0, 0, 5000.0, 0, 0.1, 0.0, 0.3, variant=0)
    assert st == oracle.ST_UPWARD
    st, _ = M.propagate_photon(0, 0, 2100.0, 0, 0.0, 0.0, -1.0, variant=0)
    assert st == oracle.ST_BELOW_OBS
    st, _ = M.propagate_photon(0, 0, 60001.0, 0, 0.0, 0.0, -1.0, variant=0)
    assert st == oracle.ST_ABOVE_MAX
    p = _dir(math.radians(71.0), 0.3)
    st, _ = M.propagate_photon(0, 0, 5000.0, 0, *p, variant=0)
    assert st == oracle.ST_ANGLE
    # vertical photon: no horizontal offset at all
    st, r = M.propagate_photon(3.0, -4.0, 9000.0, 0, 0.0, 0.0, -1.0, variant=0)
    assert st == oracle.ST_GROUND and r[0] == 3.0 and r[1] == -4.0


# --------------------------------------------------------------------------
# a2 + a4: whole bunches
# --------------------------------------------------------------------------
def test_bunch_conservation_and_spectrum():
    sc = workloads.plain_fp64(n=400)
    M = oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], H=300, Z=32,
                     t_ref=sc["t_ref"])
    out = M.bunches(sc["tracks"], seed=7)
    nb, w, s2, valid = M.segment_yield(sc["tracks"])
    assert len(out["status"]) == nb.sum()
    # every bunch has exactly one status
    assert np.all((out["status"] >= 0) & (out["status"] <= 4))
    # photons per step: sum over bunches of w equals N
    per_seg = np.bincount(out["seg"], weights=out["w"], minlength=len(nb))
    assert np.allclose(per_seg, nb * w, rtol=1e-12)
    # emission points lie on the step, in the right sub-step
    tr = sc["tracks"]
    seg = out["seg"]
    f = (out["he"] - tr["z0"][seg]) / (tr["len"][seg] * tr["uz"][seg])
    assert np.all(f >= out["j"] / nb[seg] - 1e-9) and np.all(f <= (out["j"] + 1) / nb[seg] + 1e-9)
    # photon directions make the Cherenkov angle with the step
    cosang = out["px"] * tr["ux"][seg] + out["py"] * tr["uy"][seg] + out["pz"] * tr["uz"][seg]
    assert np.allclose(cosang ** 2, 1 - s2[seg], atol=1e-12)
    # 1/lambda^2 spectrum on [300, 600] nm: CDF F = (1/300 - 1/l)/(1/300 - 1/600)
    from scipy import stats
    F = lambda l: (1 / 300.0 - 1 / l) / (1 / 300.0 - 1 / 600.0)
    assert stats.kstest(out["lam"], F).pvalue > 1e-3


def test_azimuthal_symmetry_of_vertical_track():
    """A vertical step: photons spread uniformly in azimuth around it."""
    M = _model()
    n = 64
    tr = dict(x0=np.full(n, 5.0), y0=np.full(n, -7.0), z0=np.full(n, 9000.0),
              t0=np.zeros(n), len=np.full(n, 10.0), ekin=np.full(n, 500.0),
              ux=np.zeros(n), uy=np.zeros(n), uz=np.full(n, -1.0))
    out = M.bunches(tr, seed=11)
    g = out["status"] == oracle.ST_GROUND
    dx, dy = out["X"][g] - 5.0, out["Y"][g] + 7.0
    r = np.hypot(dx, dy)
    phi = np.arctan2(dy, dx)
    from scipy import stats
    assert stats.kstest((phi + math.pi) / (2 * math.pi), "uniform").pvalue > 1e-3
    # ring radius from the emission height: same for equal heights
    he = out["he"][g]
    order = np.argsort(he)
    assert np.all(np.diff(r[order]) > -1e-6)
    assert np.mean(dx) == pytest.approx(0.0, abs=4 * r.mean() / math.sqrt(g.sum()))


def test_sphere_hits_are_geometric():
    """Every recorded hit lies within R of the centre along the arrival line;
    a bunch aimed at the centre hits."""
    sc = workloads.plain_fp64(n=1000)
    M = oracle.Model(sc["atm"], sc["h_obs"], np.array([[0.0, 0.0, 3.0, 12.0],
                                                       [30.0, 0.0, 0.0, 6.0]]),
                     H=300, Z=32, t_ref=sc["t_ref"])
    out = M.bunches(sc["tracks"], seed=3)
    rec = oracle.hit_records(out)
    assert len(rec["tel"]) > 0
    tel = M.telescopes[rec["tel"]]
    # in-plane offsets within R/cos(theta) of the centre
    cz = np.sqrt(1 - rec["cx"] ** 2 - rec["cy"] ** 2)
    assert np.all(np.hypot(rec["x"], rec["y"]) <= tel[:, 3] / cz + 1e-9)
    g = out["status"] == oracle.ST_GROUND
    # misses really miss: distance from the line to every centre exceeds R
    miss = g & (out["nhit"] == 0)
    for k, (tx, ty, tz, tr) in enumerate(M.telescopes):
        d = np.stack([tx - out["X"][miss], ty - out["Y"][miss], np.full(miss.sum(), tz)], 1)
        D = np.stack([out["cx"][miss], out["cy"][miss], out["cz"][miss]], 1)
        dist = np.linalg.norm(np.cross(d, D), axis=1)
        assert np.all(dist > tr)


# --------------------------------------------------------------------------
# The differentiable read-out (smoothed density, mean arrival time)
# --------------------------------------------------------------------------
def test_density_read_out_is_the_gaussian_sum():
    """S_k = sum_b w_b G(r_bk) with the normalised 2-D Gaussian of width sigma
    cut at 6 sigma, U_k = sum w G t, over the bunches that reach the ground."""
    sc = workloads.vertical_1tev(n=3000)
    tel = np.array([[0.0, 0.0, 0.0, 12.0], [120.0, 0.0, 0.0, 8.0], [60.0, 103.9, 0.0, 6.0]])
    M = oracle.Model(sc["atm"], sc["h_obs"], tel, H=300, Z=32, t_ref=sc["t_ref"])
    out = M.bunches(sc["tracks"], seed=5)
    for sigma in (1.0, 4.0):
        S, U = M.density_sums(sc["tracks"], 5, out["nb"], sigma)
        g = out["status"] == oracle.ST_GROUND
        for k, (x, y, _, _) in enumerate(tel):
            r2 = (out["X"][g] - x) ** 2 + (out["Y"][g] - y) ** 2
            G = np.exp(-r2 / (2 * sigma ** 2)) / (2 * math.pi * sigma ** 2) * (r2 < 36 * sigma ** 2)
            assert S[k] == pytest.approx(np.sum(out["w"][g] * G), rel=1e-12, abs=1e-300)
            assert U[k] == pytest.approx(np.sum(out["w"][g] * G * out["t"][g]), rel=1e-12,
                                         abs=1e-300)
        assert S.sum() > 0


# --------------------------------------------------------------------------
# a4/a5: the record at the plane through the sphere centre, in closed form
# --------------------------------------------------------------------------
@pytest.mark.parametrize("rho2", [0.5, 1.0])
def test_record_plane_closed_form(rho2):
    """Two slabs of constant index (n1 below hb, n2 above; rho2 = 1 makes
    them one uniform medium, a straight line at c/n): a photon emitted at
    x_e, h_e > hb along p runs straight at zenith theta2 down to hb, is
    refracted there (n2 sin theta2 = n1 sin theta1) and runs straight at
    theta1 through the horizontal plane z_p = h_obs + tz of a sphere centre.
    There, relative to the centre (at the origin),
        x = x_e + h_x [(h_e - hb) tan theta2 + (hb - z_p) tan theta1],
        t = t_e + [n2 (h_e - hb) / cos theta2 + n1 (hb - z_p) / cos theta1] / c,
    with (h_x, h_y) the horizontal unit vector of p, and (c_x, c_y) =
    sin theta1 (h_x, h_y).  Each record field is checked against this to
    rounding.  With n1 - 1 = 0.5 %, a record time taken at c instead of c/n1
    along the line, or a step back along the line of the wrong sign, is off
    by 0.1 - 1 ns."""
    hb, h_obs, tz, n0m1 = 3000.0, 2200.0, 40.0, 0.005
    atm = _slab_atm(1.0, rho2, hb, n0m1=n0m1)
    n1 = 1.0 + n0m1
    n2 = 1.0 + n0m1 * rho2
    ns = 48
    rng = np.random.default_rng(7)
    th = np.radians(rng.uniform(5.0, 25.0, ns))
    ph = rng.uniform(0.0, 2 * math.pi, ns)
    tr = dict(x0=rng.uniform(-50, 50, ns), y0=rng.uniform(-50, 50, ns),
              z0=rng.uniform(4000.0, 6000.0, ns), t0=rng.uniform(0.0, 100.0, ns),
              len=np.full(ns, 4.0), ekin=np.full(ns, 1000.0),
              ux=np.sin(th) * np.cos(ph), uy=np.sin(th) * np.sin(ph), uz=-np.cos(th))
    tel = np.array([[0.0, 0.0, tz, 3000.0]])     # every downward bunch crosses it
    for variant in (1, 0):
        M = oracle.Model(atm, h_obs, tel, H=401, Z=64, h_max=43000.0, theta_max_deg=70.0,
                         n_fine=20001)
        out = M.bunches(tr, seed=5, variant=variant)
        g = out["status"] == oracle.ST_GROUND
        assert g.sum() > 100 and np.all(out["nhit"][g] == 1)
        rec = oracle.hit_records(out)
        b = rec["bunch"]
        assert len(b) == g.sum()
        xe, ye, he, te = out["xe"][b], out["ye"][b], out["he"][b], out["te"][b]
        px, py, pz = out["px"][b], out["py"][b], out["pz"][b]
        s2 = np.hypot(px, py)
        hx, hy = px / s2, py / s2
        c2 = -pz
        s1 = n2 / n1 * s2
        c1 = np.sqrt(1.0 - s1 * s1)
        zp = h_obs + tz
        assert np.all(he > hb)
        D = (he - hb) * s2 / c2 + (hb - zp) * s1 / c1
        L = n2 * (he - hb) / c2 + n1 * (hb - zp) / c1
        ex, ey, et = xe + hx * D, ye + hy * D, te + L / C
        # (B) integrates the slabs exactly; (T) interpolates its tables
        tol_x, tol_t = (1e-9, 1e-9) if variant == 1 else (1e-5, 1e-4)
        np.testing.assert_allclose(rec["x"], ex, rtol=0, atol=tol_x)
        np.testing.assert_allclose(rec["y"], ey, rtol=0, atol=tol_x)
        np.testing.assert_allclose(rec["t"], et, rtol=0, atol=tol_t)
        np.testing.assert_allclose(rec["cx"], s1 * hx, rtol=0, atol=1e-12)
        np.testing.assert_allclose(rec["cy"], s1 * hy, rtol=0, atol=1e-12)
        np.testing.assert_allclose(rec["zem"], he, rtol=0, atol=0)
        # the record time precedes the ground time by the stretch of line
        # between the plane and the ground, run at c / n1
        tg = out["t"][b]
        np.testing.assert_allclose(tg - rec["t"], n1 * tz / c1 / C, rtol=0, atol=1e-9)
