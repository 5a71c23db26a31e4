"""Pins of the oracle's longitudinal production profile (CERLDE).

The profile puts each step's photons into atmospheric-depth bins in
proportion to the part of its path inside each bin.  It is checked against
what fixes it without retyping it: photon conservation, the depth of a
horizontal step, a split whose edge height is chosen first (so the expected
fractions are known before the oracle runs), the slant-depth scaling, and
the oracle's own bunches: stratified sub-steps put every bunch in its
sub-step's bin except where a bin edge cuts a sub-step, so the bunch
histogram differs from the profile by at most one bunch weight per step
and crossed edge.
"""
import math

import numpy as np
import pytest

import oracle
import workloads


def _model(sc):
    return oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"],
                        H=200, Z=32, theta_max_deg=sc["theta_max_deg"], t_ref=sc["t_ref"])


def _T(sc, h):
    return float(oracle.thickness(sc["atm"], h)[0])


def _one_step(z0, uz, ux=0.0, length=20.0, ekin=500.0):
    return dict(x0=np.array([0.0]), y0=np.array([0.0]), z0=np.array([z0]),
                t0=np.array([0.0]), len=np.array([length]), ekin=np.array([ekin]),
                ux=np.array([ux]), uy=np.array([0.0]), uz=np.array([uz]),
                shower=np.zeros(1, np.uint32))


def _photons(M, tracks):
    nb, w, _, _ = M.segment_yield(tracks)
    return nb, nb * w


@pytest.fixture(scope="module")
def vertical():
    sc = workloads.vertical_1tev(n=1500)
    return sc, _model(sc)


def test_profile_conserves_photons(vertical):
    sc, M = vertical
    P = M.profile(sc["tracks"], 10.0, 200)
    _, N = _photons(M, sc["tracks"])
    assert P.shape == (1, 200)
    assert P.sum() == pytest.approx(N.sum(), rel=1e-12)
    assert np.all(P >= 0.0)


def test_horizontal_step_fills_one_bin(vertical):
    sc, M = vertical
    tr = _one_step(8000.0, 0.0, ux=1.0)
    _, N = _photons(M, tr)
    assert N[0] > 0
    P = M.profile(tr, 7.0, 300)[0]
    k = int(_T(sc, 8000.0) // 7.0)
    assert P[k] == pytest.approx(N[0], rel=1e-15)
    assert np.count_nonzero(P) == 1


@pytest.mark.parametrize("cos_axis", [1.0, 0.5])
@pytest.mark.parametrize("uz", [-1.0, 1.0])
def test_split_at_a_chosen_edge(vertical, cos_axis, uz):
    """A 20 m vertical step between 6980 and 7000 m; the bin width is chosen
    so that edge m lies at 6987.3 m: 12.7/20 of the photons sit above it
    (bin m - 1), 7.3/20 below (bin m)."""
    sc, M = vertical
    m = 400
    edge = _T(sc, 6987.3) / cos_axis
    dX = edge / m
    z0 = 7000.0 if uz < 0 else 6980.0
    tr = _one_step(z0, uz)
    _, N = _photons(M, tr)
    P = M.profile(tr, dX, m + 10, axis_cos=[cos_axis])[0]
    assert P[m - 1] == pytest.approx(N[0] * 12.7 / 20.0, rel=1e-9)
    assert P[m] == pytest.approx(N[0] * 7.3 / 20.0, rel=1e-9)
    assert P.sum() == pytest.approx(N[0], rel=1e-12)


def test_slant_depth_is_vertical_depth_scaled(vertical):
    sc, M = vertical
    c = math.cos(math.radians(35.0))
    A = M.profile(sc["tracks"], 10.0, 150, axis_cos=[c])
    B = M.profile(sc["tracks"], 10.0 * c, 150)
    np.testing.assert_allclose(A, B, rtol=1e-9, atol=1e-9 * A.max())


@pytest.mark.parametrize("n_bins", [200, 50])
def test_profile_matches_bunch_histogram(vertical, n_bins):
    """Histogram of the oracle's own bunches by the depth of their emission
    height, against the profile; 50 bins of 10 g/cm^2 cut the shower so the
    deeper photons must be dropped on both sides."""
    sc, M = vertical
    dX = 10.0
    tr = sc["tracks"]
    P = M.profile(tr, dX, n_bins)[0]
    o = M.bunches(tr, 77)
    depth = oracle.thickness(sc["atm"], o["he"])
    kb = np.floor(depth / dX)
    inside = (kb >= 0) & (kb < n_bins)
    H = np.bincount(kb[inside].astype(np.int64), weights=o["w"][inside], minlength=n_bins)
    # bound: one bunch weight per step and crossed edge, on both sides of it
    nb, w, _, _ = M.segment_yield(tr)
    bound = np.zeros(n_bins + 1)
    z1 = tr["z0"] + tr["len"] * tr["uz"]
    for i in np.nonzero(nb > 0)[0]:
        Xa = _T(sc, max(tr["z0"][i], z1[i])) / dX
        Xb = _T(sc, min(tr["z0"][i], z1[i])) / dX
        for e in range(int(math.floor(Xa)) + 1, int(math.floor(Xb)) + 1):
            for k in (e - 1, e):
                if 0 <= k < n_bins:
                    bound[k] += w[i]
    diff = np.abs(P - H)
    assert np.all(diff <= bound[:n_bins] + 1e-9 * max(P.max(), 1.0))
    # the profile is not trivially inside a loose bound: most bins are far
    # larger than their bound
    big = P > 10 * bound[:n_bins]
    assert big.sum() >= 10
    if n_bins == 50:
        _, N = _photons(M, tr)
        assert P.sum() < 0.9 * N.sum()


def test_per_shower_profiles_partition():
    sc = workloads.batched_256(total=4000, n_showers=6)
    M = _model(sc)
    cz = np.cos(sc["axis_zenith_rad"])
    P = M.profile(sc["tracks"], 20.0, 80, axis_cos=cz)
    assert P.shape == (6, 80)
    sh = sc["tracks"]["shower"]
    for s in (0, 3, 5):
        sel = {k: v[sh == s] for k, v in sc["tracks"].items()}
        sel["shower"] = np.zeros(int((sh == s).sum()), np.uint32)
        Ms = oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"],
                          H=200, Z=32, theta_max_deg=sc["theta_max_deg"],
                          t_ref=sc["t_ref"][s:s + 1])
        Q = Ms.profile(sel, 20.0, 80, axis_cos=cz[s:s + 1])[0]
        np.testing.assert_allclose(P[s], Q, rtol=1e-12, atol=0)


def test_bad_arguments_are_refused(vertical):
    sc, M = vertical
    with pytest.raises(ValueError):
        M.profile(sc["tracks"], 0.0, 10)
    with pytest.raises(ValueError):
        M.profile(sc["tracks"], 10.0, 0)
