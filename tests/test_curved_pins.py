"""Pins of the oracle's curved atmosphere: spherical shells around the
Earth's centre C = (0, 0, -R_E) in the core frame, Bouguer's invariant
n r sin(zeta) along the ray, the observation sphere r_o = R_E + h_obs.

Checked against what the geometry fixes, not against the oracle's own
formulas: with no refraction (n = 1) the photon goes straight, and its
arrival is the line's intersection with the observation sphere (closed
form); for a huge radius the curved propagation (tables on their own zenith
axis and normalisation, and the ray integrals) is the flat one; every
arrival lies on the observation sphere, keeps Bouguer's invariant and stays
in the plane through C, the emission point and the direction; the curved
tables interpolated against the curved ray integrals; the step's index is
taken at the radial height of its midpoint.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

R_EARTH = 6.371e6
C_LIGHT = 0.299792458


def _model(sc, earth_radius=R_EARTH, atm=None, H=200, Z=32, theta_max_deg=80.0, **kw):
    return oracle.Model(atm or sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"],
                        H=H, Z=Z, theta_max_deg=theta_max_deg, t_ref=sc["t_ref"],
                        earth_radius=earth_radius, **kw)


@pytest.fixture(scope="module")
def sc():
    return workloads.inclined_20tev(n=2000)


def _random_photons(rng, n, max_off=40000.0, max_zen=75.0):
    """Emission points up to max_off from the core, heights 3-40 km, downward
    directions up to max_zen from the core's vertical."""
    out = []
    for _ in range(n):
        r = max_off * math.sqrt(rng.random())
        a = rng.uniform(0, 2 * math.pi)
        z = rng.uniform(3000.0, 40000.0)
        th = math.radians(rng.uniform(0.0, max_zen))
        ph = rng.uniform(0, 2 * math.pi)
        p = (math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), -math.cos(th))
        out.append(((r * math.cos(a), r * math.sin(a), z), p))
    return out


def _straight_arrival(x, p, R, h_obs):
    """Intersection of x + s p with |y - C| = R + h_obs, C = (0, 0, -R)."""
    d = np.array([x[0], x[1], x[2] + R])
    p = np.asarray(p)
    ro = R + h_obs
    b = float(d @ p)
    c = float(d @ d) - ro * ro
    disc = b * b - c
    if disc < 0:
        return None
    s = (-b - math.sqrt(disc)) if -b - math.sqrt(disc) > 0 else None
    if s is None:
        return None
    # the same root without cancellation: s = c / (-b + sqrt(disc))
    s = c / (-b + math.sqrt(disc))
    return np.asarray(x) + s * p, s


def test_no_refraction_is_the_straight_line(sc):
    atm0 = dict(sc["atm"], n0_minus_1=0.0)
    M = _model(sc, atm=atm0)
    assert np.abs(M.ax).max() < 1e-12 and np.abs(M.al).max() < 1e-9
    rng = np.random.default_rng(1)
    n_ok = 0
    for x, p in _random_photons(rng, 300):
        ref = _straight_arrival(x, p, R_EARTH, sc["h_obs"])
        for variant in (0, 1):
            st, r = M.propagate_photon(x[0], x[1], x[2], 0.0, *p, variant=variant)
            if ref is None:
                assert st != oracle.ST_GROUND
                continue
            if st != oracle.ST_GROUND:
                assert st == oracle.ST_ANGLE        # beyond the tables' 80 degrees
                continue
            (A, s) = ref
            assert r[0] == pytest.approx(A[0], abs=1e-6)
            assert r[1] == pytest.approx(A[1], abs=1e-6)
            assert r[6] == pytest.approx(A[2] - sc["h_obs"], abs=1e-6)
            assert r[2] == pytest.approx(s / C_LIGHT, rel=1e-12)
            np.testing.assert_allclose(r[3:6], p, atol=1e-12)
            n_ok += 1
    assert n_ok > 300


def test_huge_radius_is_the_flat_atmosphere(sc):
    """R_E = 1e15 m: the ray integrals (B) agree with the flat ones to the
    curvature left at that radius (~x^2 / R); the tables (T), on their own
    zenith axis and normalisation, to the interpolation error of the two
    table schemes at 200 x 32."""
    R = 1e15
    Mf = oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"], H=200,
                      Z=32, theta_max_deg=80.0, t_ref=sc["t_ref"])
    Mc = _model(sc, earth_radius=R, H=200, Z=32)
    rng = np.random.default_rng(2)
    n = 0
    for x, p in _random_photons(rng, 200, max_off=10000.0, max_zen=70.0):
        for variant, tx, tt in ((1, 1e-5, 1e-4), (0, 5e-3, 2e-2)):
            sf, rf = Mf.propagate_photon(x[0], x[1], x[2], 0.0, *p, variant=variant)
            sc_, rc = Mc.propagate_photon(x[0], x[1], x[2], 0.0, *p, variant=variant)
            assert sf == sc_
            if sf != oracle.ST_GROUND:
                continue
            n += 1
            np.testing.assert_allclose(rc[[0, 1]], rf[[0, 1]], atol=tx)
            assert rc[2] == pytest.approx(rf[2], abs=tt)
            np.testing.assert_allclose(rc[3:6], rf[3:6], atol=1e-8)
            # the observation sphere sits (X^2 + Y^2) / 2R below the tangent plane
            assert rc[6] == pytest.approx(-(rc[0] ** 2 + rc[1] ** 2) / (2 * R), abs=1e-6)
    assert n > 300


def test_arrival_on_the_sphere_with_bouguer_invariant(sc):
    M = _model(sc)
    rng = np.random.default_rng(3)
    ro = R_EARTH + sc["h_obs"]
    eta_o = oracle.eta_lookup(M.eta_tab, M.h_max, sc["h_obs"])[0]
    n = 0
    for x, p in _random_photons(rng, 300, max_off=60000.0):
        st, r = M.propagate_photon(x[0], x[1], x[2], 0.0, *p, variant=0)
        if st != oracle.ST_GROUND:
            continue
        n += 1
        A = np.array([r[0], r[1], sc["h_obs"] + r[6] + R_EARTH])   # from the centre
        assert np.linalg.norm(A) == pytest.approx(ro, abs=1e-6)
        d = np.asarray(r[3:6])
        assert np.linalg.norm(d) == pytest.approx(1.0, abs=1e-13)
        # Bouguer: n r sin(zeta) at the emission point and the arrival
        E = np.array([x[0], x[1], x[2] + R_EARTH])
        he = np.linalg.norm(E) - R_EARTH
        eta_e = oracle.eta_lookup(M.eta_tab, M.h_max, he)[0]
        inv_e = (1 + eta_e) * np.linalg.norm(np.cross(E, p))
        inv_o = (1 + eta_o) * np.linalg.norm(np.cross(A, d))
        assert inv_o == pytest.approx(inv_e, rel=1e-12)
        assert r[7] == pytest.approx(-float(A @ d) / ro, abs=1e-12)
        # the ray stays in the plane of the centre, the emission point and p
        nrm = np.cross(E, p)
        assert abs(float(A @ nrm)) <= 1e-9 * np.linalg.norm(A) * np.linalg.norm(nrm)
        assert abs(float(d @ nrm)) <= 1e-12 * np.linalg.norm(nrm)
        assert r[8] == pytest.approx(he, abs=1e-7)
    assert n > 250


def test_curved_tables_match_the_ray_integrals(sc):
    """(T) against (B) at random emission points (offsets to 60 km) and
    directions up to 78 degrees: 2 mm and 10 ps, as for the flat tables,
    away from the table rows that straddle a layer boundary (the density
    jumps there, the integrated corrections have a kink that linear
    interpolation between rows cannot follow; within 1 cm and 20 ps)."""
    M = _model(sc, H=1000, Z=64)
    rng = np.random.default_rng(4)
    dht = (M.h_max - M.h_obs) / (M.H - 1)
    bounds = np.asarray(sc["atm"]["h_bound"][1:5])
    worst_x = worst_t = edge_x = edge_t = 0.0
    n = 0
    for x, p in _random_photons(rng, 250, max_off=60000.0, max_zen=78.0):
        sT, rT = M.propagate_photon(x[0], x[1], x[2], 0.0, *p, variant=0)
        sB, rB = M.propagate_photon(x[0], x[1], x[2], 0.0, *p, variant=1)
        assert sT == sB
        if sT != oracle.ST_GROUND:
            continue
        n += 1
        ex = max(abs(rT[0] - rB[0]), abs(rT[1] - rB[1]), abs(rT[6] - rB[6]))
        et = abs(rT[2] - rB[2])
        j = int((rT[8] - M.h_obs) / dht)
        lo, hi = M.h_obs + j * dht, M.h_obs + (j + 1) * dht
        if np.any((bounds > lo) & (bounds < hi)):
            edge_x, edge_t = max(edge_x, ex), max(edge_t, et)
        else:
            worst_x, worst_t = max(worst_x, ex), max(worst_t, et)
    assert n > 200
    assert worst_x < 2e-3
    assert worst_t < 1e-2
    assert edge_x < 1e-2 and edge_t < 2e-2


def test_curvature_moves_far_arrivals(sc):
    """Sanity of scale: 30 km from the core the curved arrival differs from
    the flat one by metres (the ground there is ~70 m below the tangent
    plane), near the core by far less."""
    Mf = oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"], H=200,
                      Z=32, theta_max_deg=80.0, t_ref=sc["t_ref"])
    Mc = _model(sc)
    p = (math.sin(math.radians(60)), 0.0, -math.cos(math.radians(60)))
    _, rf = Mf.propagate_photon(30000.0, 0.0, 15000.0, 0.0, *p)
    _, rc = Mc.propagate_photon(30000.0, 0.0, 15000.0, 0.0, *p)
    assert abs(rc[0] - rf[0]) > 10.0
    _, rf = Mf.propagate_photon(0.0, 0.0, 3000.0, 0.0, 0.0, 0.0, -1.0)
    _, rc = Mc.propagate_photon(0.0, 0.0, 3000.0, 0.0, 0.0, 0.0, -1.0)
    assert abs(rc[2] - rf[2]) < 1e-6 and abs(rc[0]) < 1e-9


def test_step_index_at_the_radial_midpoint_height(sc):
    """A step far from the core emits as a flat-atmosphere step whose
    midpoint sits at its radial height."""
    Mc = _model(sc)
    Mf = oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"], H=50,
                      Z=16, theta_max_deg=80.0, t_ref=sc["t_ref"])
    n = 40
    rng = np.random.default_rng(5)
    x0 = rng.uniform(-50000, 50000, n)
    y0 = rng.uniform(-50000, 50000, n)
    z0 = rng.uniform(5000, 20000, n)
    ln = rng.uniform(1, 20, n)
    th = np.radians(rng.uniform(0, 70, n))
    ux, uy, uz = np.sin(th), np.zeros(n), -np.cos(th)
    tr = dict(x0=x0, y0=y0, z0=z0, t0=np.zeros(n), len=ln, ekin=np.full(n, 200.0),
              ux=ux, uy=uy, uz=uz, shower=np.zeros(n, np.uint32))
    nb_c, w_c, _, _ = Mc.segment_yield(tr)
    xm, ym, zm = x0 + 0.5 * ln * ux, y0 + 0.5 * ln * uy, z0 + 0.5 * ln * uz
    h_rad = np.sqrt(xm ** 2 + ym ** 2 + (zm + R_EARTH) ** 2) - R_EARTH
    assert np.max(h_rad - zm) > 100.0
    trf = dict(tr, z0=z0 + (h_rad - zm))
    nb_f, w_f, _, _ = Mf.segment_yield(trf)
    np.testing.assert_allclose(nb_c * w_c, nb_f * w_f, rtol=1e-9)
