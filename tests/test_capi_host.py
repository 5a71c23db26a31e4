"""The C-ABI library on a machine without a GPU: it builds, loads, exports
every symbol include/cher.h declares, rejects bad arguments before touching
CUDA, and its host table builder agrees with the oracle's tables."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2006_14927_gb300 as P
import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    P.build()
    return P.lib()


def test_exports_every_declared_symbol(L):
    hdr = open(os.path.join(ROOT, "include", "cher.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    declared = set(re.findall(r"\b(cher_[a-z0-9_]+)\s*\(", hdr))
    assert "cher_generate_propagate" in declared and len(declared) >= 13
    for name in declared:
        assert hasattr(L, name), name
    assert declared == set(P.SIGNATURES)


def test_status_strings(L):
    for code in range(8):
        assert L.cher_status_string(code)
    assert L.cher_status_string(99) == b"unknown status"


def test_create_rejects_bad_arguments_without_cuda(L):
    h = ctypes.c_void_p()
    A = P._binding.atmosphere_struct(workloads.us_standard_atmosphere())
    T = (P._binding.Telescope * 1)(P._binding.Telescope(0, 0, 0, 12.0))
    assert L.cher_create(None, 2200.0, T, 1, None, ctypes.byref(h)) == 1
    assert L.cher_create(ctypes.byref(A), 2200.0, T, 0, None, ctypes.byref(h)) == 1
    bad = (P._binding.Telescope * 1)(P._binding.Telescope(0, 0, 0, -1.0))
    assert L.cher_create(ctypes.byref(A), 2200.0, bad, 1, None, ctypes.byref(h)) == 1
    assert L.cher_build_refraction_tables(None, 10, 10, 70.0, 6e4) == 1
    assert L.cher_generate_propagate(None, None, 0, 1, None, None) == 1
    assert L.cher_destroy(None) == 0


@pytest.mark.parametrize("H,Z,zen,hmax", [(1000, 64, 70.0, 60000.0), (257, 33, 75.0, 75000.0)])
def test_host_tables_match_oracle(H, Z, zen, hmax):
    atm = workloads.us_standard_atmosphere()
    eta, ax, al = P.build_tables_host(atm, 2200.0, 10000, H, Z, zen, hmax)
    M = oracle.Model(atm, 2200.0, np.array([[0, 0, 0, 12.0]]), H=H, Z=Z, theta_max_deg=zen,
                     h_max=hmax)
    # the fine n table decides bunch counts: it must be bit-identical
    assert np.array_equal(eta, M.eta_tab)
    # refraction tables: two independent integrations of the same integrals
    assert np.max(np.abs(ax - M.ax)) < 1e-9
    assert np.max(np.abs(al - M.al)) < 1e-9


@pytest.mark.parametrize("H,Z,zen", [(200, 32, 80.0), (60, 16, 60.0)])
def test_host_curved_tables_match_oracle(H, Z, zen):
    """The library's curved tables (12-point Gauss-Legendre per interval)
    against the oracle's (adaptive Simpson): the same three normalised
    corrections on the same sec-uniform zenith nodes."""
    atm = workloads.us_standard_atmosphere()
    ax, al, ag = P.build_curved_tables_host(atm, 6.371e6, 2200.0, H, Z, zen, 60000.0)
    M = oracle.Model(atm, 2200.0, np.array([[0, 0, 0, 12.0]]), H=H, Z=Z, theta_max_deg=zen,
                     h_max=60000.0, earth_radius=6.371e6)
    for mine, theirs in ((ax, M.ax), (al, M.al), (ag, M.ag)):
        assert np.max(np.abs(mine - theirs)) < 1e-8 * max(1.0, np.abs(theirs).max())


def test_host_tables_reject_bad_ranges():
    atm = workloads.us_standard_atmosphere()
    with pytest.raises(P.CherError):
        P.build_tables_host(atm, 2200.0, 10000, 1, 64, 70.0, 60000.0)
    with pytest.raises(P.CherError):
        P.build_tables_host(atm, 2200.0, 10000, 100, 64, 89.0, 60000.0)
    with pytest.raises(P.CherError):
        P.build_tables_host(atm, 2200.0, 10000, 100, 64, 70.0, 1000.0)


def test_adjoint_sensitivity_tables_match_finite_differences():
    """d(ax, al)/d(b_i, c_i) of the host builder against central differences
    of the table builder itself (the tables are smooth in the parameters)."""
    atm = workloads.us_standard_atmosphere()
    args = (2200.0, 10000, 120, 12, 70.0, 60000.0)
    dax, dal = P.build_sensitivity_host(atm, *args)
    for q, (key, i) in enumerate([("b", k) for k in range(5)] + [("c", k) for k in range(5)]):
        eps = 1e-6
        a1 = {k: (list(v) if isinstance(v, list) else v) for k, v in atm.items()}
        a2 = {k: (list(v) if isinstance(v, list) else v) for k, v in atm.items()}
        a1[key][i] *= 1 + eps
        a2[key][i] *= 1 - eps
        _, x1, l1 = P.build_tables_host(a1, *args)
        _, x2, l2 = P.build_tables_host(a2, *args)
        h = atm[key][i] * eps
        fx, fl = (x1 - x2) / (2 * h), (l1 - l2) / (2 * h)
        sx = max(np.abs(fx).max(), 1e-30)
        sl = max(np.abs(fl).max(), 1e-30)
        assert np.abs(fx - dax[q]).max() <= 1e-5 * sx + 1e-14, (key, i)
        assert np.abs(fl - dal[q]).max() <= 1e-5 * sl + 1e-14, (key, i)


def test_round_to_float_rejects_bad_arguments(L):
    assert L.cher_round_to_float(None, None, 5, None) == 1
    assert L.cher_round_to_float(None, None, -1, None) == 1
    assert L.cher_round_to_float(None, None, 0, None) == 0
    assert L.cher_split_to_float(None, None, None, 5, None) == 1
    assert L.cher_split_to_float(None, None, None, 0, None) == 0


def test_dispersion_setter_rejects_a_missing_context(L):
    assert L.cher_set_dispersion(None, None, 0) == 1
