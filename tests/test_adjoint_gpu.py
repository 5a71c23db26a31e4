"""The adjoint (cher_adjoint, its torch.autograd binding) against finite
differences.

Reference gradient: central differences of the FP64 oracle's read-out
(orc_density) with the bunch counts frozen: relative step 1e-6 for the
atmosphere parameters (the oracle rebuilds its tables for each), 1e-4 m for
the step positions, 1e-6 for u_z and 1e-6 times the transverse magnitude
for u_x, u_y (the azimuth basis turns by step / magnitude).  Also: the read-out itself against
the oracle, translation invariance, a_i gradients exactly zero, and central
differences of the library's own FP64 read-out.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2006_14927_gb300 as P
import workloads
from parity import FP32, FP64, context, host_tracks, oracle_model

pytestmark = pytest.mark.gpu

SEED = 0xAD701
SIGMA = 1.0


@pytest.fixture(scope="module")
def case():
    P.build()
    sc = workloads.adjoint_300gev()
    rng = np.random.default_rng(99)
    n_tel = len(sc["telescopes"])
    gD = rng.normal(0.0, 1.0, n_tel)
    gT = rng.normal(0.0, 0.05, n_tel)
    M = oracle_model(sc)
    return sc, gD, gT, M


def _loss(S, U, gD, gT):
    T = np.where(S > 0, U / np.where(S > 0, S, 1.0), 0.0)
    return float(np.sum(gD * S) + np.sum(gT * T))


def _gpu(sc, prec):
    ctx = context(sc)
    tr = host_tracks(sc, prec)
    dev = P.device_tracks(tr, prec, t_ref=sc["t_ref"])
    nb, _ = ctx.segment_yield(dev, prec)
    return ctx, tr, dev, nb


def _perturbed_atm(atm, key, i, rel):
    a = {k: (list(v) if isinstance(v, list) else v) for k, v in atm.items()}
    a[key][i] *= 1.0 + rel
    return a


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_readout_matches_oracle(case, prec):
    sc, gD, gT, M = case
    ctx, tr, dev, nb = _gpu(sc, prec)
    D, T = ctx.density(dev, SEED, prec, SIGMA, nb)
    S_o, U_o = M.density_sums(tr, SEED, nb.cpu().numpy(), SIGMA)
    T_o = np.where(S_o > 0, U_o / np.where(S_o > 0, S_o, 1), 0)
    D, T = D.cpu().numpy(), T.cpu().numpy()
    assert S_o.sum() > 0
    rtol = 1e-9 if prec == FP64 else 2e-3
    np.testing.assert_allclose(D, S_o, rtol=rtol, atol=rtol * S_o.max())
    np.testing.assert_allclose(T, T_o, rtol=0, atol=(1e-7 if prec == FP64 else 0.02))
    ctx.close()


def _oracle_fd_atm(sc, M, tr, nb, gD, gT, key, i, rel=1e-6):
    vals = []
    for sgn in (+1, -1):
        a = _perturbed_atm(sc["atm"], key, i, sgn * rel)
        Mp = oracle.Model(a, sc["h_obs"], sc["telescopes"], h_max=sc["h_max"],
                          n_fine=sc["n_fine"], H=sc["H"], Z=sc["Z"],
                          theta_max_deg=sc["theta_max_deg"], t_ref=sc["t_ref"])
        S, U = Mp.density_sums(tr, SEED, nb, SIGMA)
        vals.append(_loss(S, U, gD, gT))
    return (vals[0] - vals[1]) / (2 * rel * sc["atm"][key][i])


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_atmosphere_gradient_vs_oracle_finite_differences(case, prec):
    sc, gD, gT, M = case
    ctx, tr, dev, nb = _gpu(sc, prec)
    ga, _ = ctx.adjoint(dev, SEED, prec, gD, gT, SIGMA, nb)
    ga = ga.cpu().numpy()
    # n does not depend on a_i: exactly zero
    assert np.all(ga[0:5] == 0.0)
    nbh = nb.cpu().numpy()
    fd = {}
    for q, (key, i) in enumerate([("b", k) for k in range(4)] + [("c", k) for k in range(4)]):
        fd[(key, i)] = _oracle_fd_atm(sc, M, tr, nbh, gD, gT, key, i)
    scale = max(abs(v) for v in fd.values())
    tol = 1e-4 if prec == FP64 else 1e-3
    for (key, i), v in fd.items():
        g = ga[5 + i] if key == "b" else ga[10 + i]
        assert abs(g - v) <= tol * max(abs(v), 1e-3 * scale), (key, i, g, v)
    ctx.close()


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_step_gradients_vs_oracle_finite_differences(case, prec):
    sc, gD, gT, M = case
    ctx, tr, dev, nb = _gpu(sc, prec)
    _, gt = ctx.adjoint(dev, SEED, prec, gD, gT, SIGMA, nb)
    gt = gt.cpu().numpy()
    nbh = nb.cpu().numpy()
    S0, U0 = M.density_sums(tr, SEED, nbh, SIGMA)
    L0 = _loss(S0, U0, gD, gT)
    mag = np.abs(gt).sum(axis=0)
    steps = np.argsort(-mag)[:12]              # the steps that contribute most
    assert mag[steps[0]] > 0
    names = ["x0", "y0", "z0", "ux", "uy", "uz"]
    checked = 0
    for i in steps:
        one = {k: v[i:i + 1].copy() for k, v in tr.items()}
        Si, Ui = M.density_sums(one, SEED, nbh[i:i + 1], SIGMA, track_base=int(i))
        # direction steps relative to the transverse magnitude: the azimuth
        # basis (u_y, -u_x)/rho turns by eps/rho, so eps must stay << rho
        rho = math.hypot(one["ux"][0], one["uy"][0])
        for m, name in enumerate(names):
            eps = 1e-4 if m < 3 else (1e-6 * min(1.0, rho) if m < 5 else 1e-6)
            vals = []
            for sgn in (+1, -1):
                pert = {k: v.copy() for k, v in one.items()}
                pert[name] = pert[name] + sgn * eps
                Sp, Up = M.density_sums(pert, SEED, nbh[i:i + 1], SIGMA, track_base=int(i))
                vals.append(_loss(S0 - Si + Sp, U0 - Ui + Up, gD, gT))
            fd = (vals[0] - vals[1]) / (2 * eps)
            g = gt[m, i]
            tol = 1e-4 if prec == FP64 else 2e-3
            ref = max(abs(fd), 1e-3 * np.abs(gt[m, steps]).max())
            assert abs(g - fd) <= tol * ref + 1e-9 * abs(L0), (i, name, g, fd)
            checked += 1
    assert checked == 72
    ctx.close()


def test_translation_invariance(case):
    """Shifting every step by dx moves every ground point by dx: the sum of
    dL/dx0 over the steps is the derivative of that shift."""
    sc, gD, gT, M = case
    ctx, tr, dev, nb = _gpu(sc, FP64)
    _, gt = ctx.adjoint(dev, SEED, FP64, gD, gT, SIGMA, nb)
    gt = gt.cpu().numpy()
    nbh = nb.cpu().numpy()
    for m, key in ((0, "x0"), (1, "y0")):
        eps = 1e-4
        vals = []
        for sgn in (+1, -1):
            pert = dict(tr)
            pert[key] = tr[key] + sgn * eps
            S, U = M.density_sums(pert, SEED, nbh, SIGMA)
            vals.append(_loss(S, U, gD, gT))
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert gt[m].sum() == pytest.approx(fd, rel=1e-5, abs=1e-9)
    ctx.close()


def test_own_fp64_readout_finite_differences(case):
    """Central differences of the library's own FP64 read-out (tables rebuilt
    through cher_set_atmosphere) for two parameters."""
    sc, gD, gT, M = case
    ctx, tr, dev, nb = _gpu(sc, FP64)
    ga, _ = ctx.adjoint(dev, SEED, FP64, gD, gT, SIGMA, nb)
    ga = ga.cpu().numpy()
    for key, i in (("b", 1), ("c", 0)):
        vals = []
        for sgn in (+1, -1):
            ctx.set_atmosphere(_perturbed_atm(sc["atm"], key, i, sgn * 1e-6))
            D, T = ctx.density(dev, SEED, FP64, SIGMA, nb)
            D, T = D.cpu().numpy(), T.cpu().numpy()
            vals.append(float(np.sum(gD * D) + np.sum(gT * T)))
        fd = (vals[0] - vals[1]) / (2e-6 * sc["atm"][key][i])
        g = ga[5 + i] if key == "b" else ga[10 + i]
        assert g == pytest.approx(fd, rel=1e-4)
    ctx.set_atmosphere(sc["atm"])
    ctx.close()


def test_autograd_function(case):
    import torch
    from paper_2006_14927_gb300.autograd import telescope_readout
    sc, gD, gT, M = case
    ctx, tr, dev, nb = _gpu(sc, FP64)
    atm = sc["atm"]
    params = torch.tensor(atm["a"] + atm["b"] + atm["c"], dtype=torch.float64,
                          requires_grad=True)
    tracks = dict(dev)
    for k in ("x0", "y0", "z0", "ux", "uy", "uz"):
        tracks[k] = dev[k].clone().requires_grad_(True)
    D, T = telescope_readout(ctx, tracks, params, atm, SEED, FP64, SIGMA, nb)
    L = (torch.as_tensor(gD, device=D.device) * D).sum() + \
        (torch.as_tensor(gT, device=T.device) * T).sum()
    L.backward()
    ga, gt = ctx.adjoint(dev, SEED, FP64, gD, gT, SIGMA, nb)
    # (FP64 atomics accumulate in a different order from call to call)
    np.testing.assert_allclose(params.grad.numpy(), ga.cpu().numpy(), rtol=1e-9, atol=0)
    for m, k in enumerate(("x0", "y0", "z0", "ux", "uy", "uz")):
        g = gt[m].cpu().numpy()
        np.testing.assert_allclose(tracks[k].grad.cpu().numpy(), g, rtol=1e-9,
                                   atol=1e-12 * np.abs(g).max())
    ctx.close()


# the largest deviations from the oracle's dual-number gradient, per
# precision (read by a script that runs this file; pytest checks the bounds)
MEASURED = {}
# bounds on those deviations, relative to the largest gradient of each kind:
# the FP64 recomputation is the oracle's arithmetic to rounding (measured
# ~1e-13); the FP32 recomputation keeps FP32 directions and ground points,
# whose rounding (~1e-7 rad over ~6 km, ~1e-3 m against a 1 m Gaussian)
# leaves ~1e-5 of the largest gradient (measured 1.2e-5 for the atmosphere,
# 4.4e-5 for the steps), inside the 1e-4 the adjoint is held to.  Finite
# differences cannot check either that tightly (their own error is ~1e-4 at
# steps that keep the azimuth basis and table cells smooth).
DUAL_TOL = {FP64: dict(atm=1e-10, steps=1e-10), FP32: dict(atm=1e-4, steps=1e-4)}


@pytest.fixture(scope="module")
def dual_reference(case):
    """The oracle's forward-mode dual-number gradient of the whole workload
    (FP64, the table variant), for each precision's own track values."""
    sc, gD, gT, M = case
    ref = {}
    for prec in (FP64, FP32):
        ctx, tr, dev, nb = _gpu(sc, prec)
        nbh = nb.cpu().numpy()
        ref[prec] = (M.density_grad(tr, SEED, nbh, SIGMA, gD, gT), nbh)
        ctx.close()
    return ref


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_adjoint_vs_oracle_dual_gradient(case, dual_reference, prec):
    """Every gradient of the adjoint against the oracle's dual numbers: the
    15 atmosphere entries, and all six gradients of every step, each kind
    relative to its largest entry."""
    sc, gD, gT, M = case
    (S_o, U_o, ga_o, gs_o), nbh = dual_reference[prec]
    ctx, tr, dev, nb = _gpu(sc, prec)
    assert np.array_equal(nb.cpu().numpy(), nbh)
    ga, gt = ctx.adjoint(dev, SEED, prec, gD, gT, SIGMA, nb)
    ga, gt = ga.cpu().numpy(), gt.cpu().numpy()
    ctx.close()
    assert np.all(ga[0:5] == 0.0) and np.all(ga_o[0:5] == 0.0)
    e_atm = float(np.max(np.abs(ga - ga_o)) / np.max(np.abs(ga_o)))
    e_steps = [float(np.max(np.abs(gt[m] - gs_o[m])) / np.max(np.abs(gs_o[m])))
               for m in range(6)]
    MEASURED[prec] = dict(atm=e_atm, steps=e_steps,
                          atm_each=((ga - ga_o) / np.where(ga_o != 0, np.abs(ga_o), 1)).tolist())
    tol = DUAL_TOL[prec]
    assert e_atm <= tol["atm"], e_atm
    assert max(e_steps) <= tol["steps"], e_steps
