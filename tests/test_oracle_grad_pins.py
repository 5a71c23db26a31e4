"""Pins of the oracle's reference gradient (forward-mode dual numbers over
the read-out S_k = sum w G, U_k = sum w G t, L = sum gD S + gT U / S) to
finite differences of the oracle's own read-out, which the read-out pins
and the propagation pins fix.

The dual numbers carry the derivatives through every statement, so they
must agree with central differences to the differences' own truncation and
rounding (~1e-8 here); a dropped tangent, a wrong chain term or a sign
error fails by orders of magnitude more.  The values they carry must be the
oracle's read-out bit for bit, and n depends on the atmosphere only through
b_i and c_i, so dL/da_i is exactly zero.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

SEED = 0xAD701


@pytest.fixture(scope="module")
def case():
    oracle.build()
    sc = workloads.adjoint_300gev()
    sub = {k: v[:2500] for k, v in sc["tracks"].items()}
    M = _model(sc, sc["atm"])
    nb, _, _, _ = M.segment_yield(sub)
    rng = np.random.default_rng(99)
    n_tel = len(sc["telescopes"])
    gD = rng.normal(0.0, 1.0, n_tel)
    gT = rng.normal(0.0, 0.05, n_tel)
    S, U, ga, gs = M.density_grad(sub, SEED, nb, 1.0, gD, gT)
    return sc, sub, M, nb, gD, gT, S, U, ga, gs


def _model(sc, atm):
    return oracle.Model(atm, sc["h_obs"], sc["telescopes"], h_max=sc["h_max"],
                        n_fine=sc["n_fine"], H=sc["H"], Z=sc["Z"],
                        theta_max_deg=sc["theta_max_deg"], t_ref=sc["t_ref"])


def _loss(S, U, gD, gT):
    T = np.where(S > 0, U / np.where(S > 0, S, 1.0), 0.0)
    return float(np.sum(gD * S) + np.sum(gT * T))


def test_values_are_the_readout(case):
    sc, sub, M, nb, gD, gT, S, U, ga, gs = case
    S0, U0 = M.density_sums(sub, SEED, nb, 1.0)
    assert S0.sum() > 0
    assert np.array_equal(S, S0) and np.array_equal(U, U0)


def test_atmosphere_gradient_against_central_differences(case):
    sc, sub, M, nb, gD, gT, S, U, ga, gs = case
    assert np.all(ga[0:5] == 0.0)
    scale = np.abs(ga[5:]).max()
    assert scale > 0
    for key, i in [("b", k) for k in range(4)] + [("c", k) for k in range(4)]:
        rel = 1e-6
        vals = []
        for sgn in (+1, -1):
            a = {k: (list(v) if isinstance(v, (list, tuple, np.ndarray)) else v)
                 for k, v in sc["atm"].items()}
            a[key][i] *= 1.0 + sgn * rel
            Sp, Up = _model(sc, a).density_sums(sub, SEED, nb, 1.0)
            vals.append(_loss(Sp, Up, gD, gT))
        fd = (vals[0] - vals[1]) / (2 * rel * sc["atm"][key][i])
        g = ga[5 + i] if key == "b" else ga[10 + i]
        assert abs(g - fd) <= 1e-6 * max(abs(fd), 1e-3 * scale), (key, i, g, fd)


def test_step_gradient_against_central_differences(case):
    """Positions by 1e-4 m, u_z by 1e-7; u_x, u_y by 1e-6 of the transverse magnitude
    (the azimuth basis (-u_y, u_x) / rho turns by eps / rho and swings ground
    points ~100 m from the step through a 1 m Gaussian, so the quotient's
    truncation error is ~1e4 (eps / rho)^2)."""
    sc, sub, M, nb, gD, gT, S, U, ga, gs = case
    L0 = _loss(S, U, gD, gT)
    mag = np.abs(gs).sum(axis=0)
    steps = np.argsort(-mag)[:5]
    names = ["x0", "y0", "z0", "ux", "uy", "uz"]
    for i in steps:
        one = {k: v[i:i + 1].copy() for k, v in sub.items()}
        Si, Ui = M.density_sums(one, SEED, nb[i:i + 1], 1.0, track_base=int(i))
        rho = math.hypot(one["ux"][0], one["uy"][0])
        for m, name in enumerate(names):
            eps = 1e-4 if m < 3 else (1e-6 * min(rho, 0.01) if m < 5 else 1e-7)
            vals = []
            for sgn in (+1, -1):
                pert = {k: v.copy() for k, v in one.items()}
                pert[name] = pert[name] + sgn * eps
                Sp, Up = M.density_sums(pert, SEED, nb[i:i + 1], 1.0, track_base=int(i))
                vals.append(_loss(S - Si + Sp, U - Ui + Up, gD, gT))
            fd = (vals[0] - vals[1]) / (2 * eps)
            g = gs[m, i]
            ref = max(abs(fd), 1e-4 * np.abs(gs[m, steps]).max())
            assert abs(g - fd) <= 1e-5 * ref + 1e-12 * abs(L0), (i, name, g, fd)


def test_shifting_every_step_is_the_sum_of_the_step_gradients(case):
    """Moving every step by dx moves every ground point by dx: the
    derivative of that shift is the sum of dL/dx0 over the steps (and the
    same for y0)."""
    sc, sub, M, nb, gD, gT, S, U, ga, gs = case
    for m, name in ((0, "x0"), (1, "y0")):
        eps = 1e-4
        vals = []
        for sgn in (+1, -1):
            pert = {k: v.copy() for k, v in sub.items()}
            pert[name] = pert[name] + sgn * eps
            Sp, Up = M.density_sums(pert, SEED, nb, 1.0)
            vals.append(_loss(Sp, Up, gD, gT))
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(gs[m].sum() - fd) <= 1e-6 * np.abs(gs[m]).sum(), (name, gs[m].sum(), fd)
