"""Pins of the oracle's beyond-table fallback: bunches whose observation-
level zenith exceeds the refraction tables' range, up to the fallback limit,
are propagated by the ray integrals themselves instead of being dropped.

Checked against a table that does cover them (the tables are pinned to the
ray integrals elsewhere, to 2 mm and 10 ps), against the drop rule at the
limit, and for doing nothing when off.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

SEED = 3


@pytest.fixture(scope="module")
def inclined():
    return workloads.inclined_20tev(n=3000)


def _model(sc, theta_max, fb):
    return oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"], H=400,
                        Z=64, theta_max_deg=theta_max, t_ref=sc["t_ref"], fallback_deg=fb)


def _zenith_deg(o):
    return np.degrees(np.arccos(np.clip(-o["cz"], -1, 1)))


def test_fallback_off_changes_nothing(inclined):
    sc = inclined
    a = _model(sc, 61.0, 0.0).bunches(sc["tracks"], SEED)
    b = _model(sc, 61.0, 50.0).bunches(sc["tracks"], SEED)      # below the table limit
    for k in ("status", "X", "Y", "t", "nhit"):
        assert np.array_equal(a[k], b[k]), k
    assert (a["status"] == oracle.ST_ANGLE).sum() > 1000


def test_fallback_matches_a_table_that_covers_the_range(inclined):
    sc = inclined
    wide = _model(sc, 75.0, 0.0).bunches(sc["tracks"], SEED)
    narrow = _model(sc, 61.0, 0.0).bunches(sc["tracks"], SEED)
    fb = _model(sc, 61.0, 80.0).bunches(sc["tracks"], SEED)
    beyond = narrow["status"] == oracle.ST_ANGLE
    assert beyond.sum() > 1000
    assert np.all(fb["status"] == oracle.ST_GROUND)
    assert np.array_equal(wide["status"], fb["status"])
    # the rescued bunches: the ray integrals against the 75-degree table
    g = beyond
    assert np.all(_zenith_deg(fb)[g] > 60.9)
    np.testing.assert_allclose(fb["X"][g], wide["X"][g], rtol=0, atol=2e-3)
    np.testing.assert_allclose(fb["Y"][g], wide["Y"][g], rtol=0, atol=2e-3)
    np.testing.assert_allclose(fb["t"][g], wide["t"][g], rtol=0, atol=1e-2)
    # the others keep the 61-degree table's values exactly
    k = ~beyond
    for q in ("X", "Y", "t", "cx", "cy"):
        assert np.array_equal(fb[q][k], narrow[q][k]), q
    # crossings: the wide table's, off the 5 cm shell of each sphere
    assert abs(int((fb["nhit"] > 0).sum()) - int((wide["nhit"] > 0).sum())) <= 2


def test_bunches_past_the_fallback_limit_are_dropped(inclined):
    sc = inclined
    wide = _model(sc, 75.0, 0.0).bunches(sc["tracks"], SEED)
    fb = _model(sc, 58.0, 61.0).bunches(sc["tracks"], SEED)
    zen = _zenith_deg(wide)
    ok = wide["status"] == oracle.ST_GROUND
    clear = ok & (np.abs(zen - 61.0) > 1e-6) & (np.abs(zen - 58.0) > 1e-6)
    assert np.all(fb["status"][clear & (zen > 61.0)] == oracle.ST_ANGLE)
    assert np.all(fb["status"][clear & (zen < 61.0)] == oracle.ST_GROUND)
    assert (clear & (zen > 58.0) & (zen < 61.0)).sum() > 1000
