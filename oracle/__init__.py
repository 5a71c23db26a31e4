"""FP64 CPU oracle for Cherenkov bunch generation and propagation.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports this package and shares no code with it.

The arithmetic lives in ``cher_oracle.c`` (plain C, FP64, no fused
multiply-add); this module compiles it with gcc and marshals numpy arrays
through ctypes.  Every function cites the paper section it follows in the C
source.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cher_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

ST_GROUND, ST_UPWARD, ST_BELOW_OBS, ST_ABOVE_MAX, ST_ANGLE, ST_ABSORBED = 0, 1, 2, 3, 4, 5
MAX_HITS = 4


def build(force: bool = False) -> str:
    """Compile cher_oracle.c into liboracle.so (gcc, -O2, no FMA contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-std=c11", _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class _Atm(ctypes.Structure):
    _fields_ = [("h_bound", ctypes.c_double * 6), ("a", ctypes.c_double * 5),
                ("b", ctypes.c_double * 5), ("c", ctypes.c_double * 5),
                ("n0_minus_1", ctypes.c_double)]


_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)


class _Cfg(ctypes.Structure):
    _fields_ = [("atm", _Atm), ("h_obs", ctypes.c_double), ("h_max", ctypes.c_double),
                ("n_fine", ctypes.c_int), ("eta_tab", _dp),
                ("H", ctypes.c_int), ("Z", ctypes.c_int), ("theta_max", ctypes.c_double),
                ("ax", _dp), ("al", _dp),
                ("bunch_size", ctypes.c_double), ("lambda1_nm", ctypes.c_double),
                ("lambda2_nm", ctypes.c_double),
                ("n_tel", ctypes.c_int), ("tel", _dp),
                ("t_ref", _dp), ("n_showers", ctypes.c_int), ("bf_tol", ctypes.c_double),
                ("philox_key", ctypes.c_uint32 * 2),
                ("trans_nl", ctypes.c_int), ("trans_nh", ctypes.c_int),
                ("trans_l0", ctypes.c_double), ("trans_l1", ctypes.c_double),
                ("trans_h0", ctypes.c_double), ("trans_h1", ctypes.c_double),
                ("trans_tau", _dp), ("fb_sin2_max", ctypes.c_double),
                ("disp_k", ctypes.c_int), ("disp_kappa", _dp), ("ax_hi", _dp), ("al_hi", _dp),
                ("earth_radius", ctypes.c_double), ("ag", _dp), ("ag_hi", _dp)]


class _Tracks(ctypes.Structure):
    _fields_ = [("x0", _dp), ("y0", _dp), ("z0", _dp), ("t0", _dp), ("len", _dp),
                ("ekin", _dp), ("ux", _dp), ("uy", _dp), ("uz", _dp),
                ("shower", _u32p), ("n", ctypes.c_int64), ("track_base", ctypes.c_int64)]


class _Out(ctypes.Structure):
    _fields_ = [("status", _i32p), ("xe", _dp), ("ye", _dp), ("he", _dp), ("te", _dp),
                ("px", _dp), ("py", _dp), ("pz", _dp), ("X", _dp), ("Y", _dp), ("t", _dp),
                ("cx", _dp), ("cy", _dp), ("cz", _dp), ("lam", _dp), ("w", _dp),
                ("nhit", _i32p), ("hit_tel", _i32p), ("hit_x", _dp), ("hit_y", _dp),
                ("hit_t", _dp), ("tr_margin", _dp), ("Zg", _dp)]


_lib = None


class _Shower(ctypes.Structure):
    _fields_ = [("e0_mev", ctypes.c_double), ("zenith", ctypes.c_double),
                ("azimuth", ctypes.c_double), ("core_x", ctypes.c_double),
                ("core_y", ctypes.c_double), ("first", ctypes.c_int64), ("n", ctypes.c_int64)]


def generate_steps(showers, h_obs: float, seed: int, n_cdf: int = 1024) -> dict:
    """Steps of parameterised showers (orc_generate_steps).  `showers`: a
    sequence of dicts with e0_mev, zenith, azimuth, core_x, core_y, n; the
    steps of shower s follow those of shower s - 1.  Returns the step arrays
    (float64, shower uint32) and t_ref per shower."""
    arr = (_Shower * len(showers))()
    first = 0
    for k, s in enumerate(showers):
        arr[k] = _Shower(float(s["e0_mev"]), float(s["zenith"]), float(s["azimuth"]),
                         float(s["core_x"]), float(s["core_y"]), first, int(s["n"]))
        first += int(s["n"])
    out = {k: np.zeros(first) for k in ("x0", "y0", "z0", "t0", "len", "ekin", "ux", "uy", "uz")}
    out["shower"] = np.zeros(first, np.uint32)
    t_ref = np.zeros(len(showers))
    rc = lib().orc_generate_steps(arr, len(showers), float(h_obs), ctypes.c_uint64(seed),
                                  int(n_cdf), *[_ptr(out[k]) for k in ("x0", "y0", "z0", "t0",
                                                                     "len", "ekin", "ux", "uy",
                                                                     "uz")],
                                  _ptr(out["shower"], ctypes.c_uint32), _ptr(t_ref))
    if rc != 0:
        raise ValueError("orc_generate_steps failed")
    out["t_ref"] = t_ref
    return out


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_thickness.argtypes = [ctypes.POINTER(_Atm), ctypes.c_double]
        L.orc_thickness.restype = ctypes.c_double
        L.orc_rho.argtypes = [ctypes.POINTER(_Atm), ctypes.c_double]
        L.orc_rho.restype = ctypes.c_double
        L.orc_eta_exact.argtypes = [ctypes.POINTER(_Atm), ctypes.c_double]
        L.orc_eta_exact.restype = ctypes.c_double
        L.orc_build_eta_table.argtypes = [ctypes.POINTER(_Atm), ctypes.c_double,
                                          ctypes.c_int, _dp]
        L.orc_eta_lookup.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.orc_eta_lookup.restype = ctypes.c_double
        L.orc_segment_yield.argtypes = [ctypes.POINTER(_Cfg), ctypes.POINTER(_Tracks), _i64p,
                                        _dp, _dp, _i32p]
        L.orc_brute_ray.argtypes = [ctypes.POINTER(_Atm), ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.orc_build_refraction_tables.argtypes = [ctypes.POINTER(_Atm), ctypes.c_double,
                                                  ctypes.c_double, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_double,
                                                  ctypes.c_double, _dp, _dp]
        L.orc_propagate_photon.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int] + \
            [ctypes.c_double] * 7 + [_dp]
        L.orc_propagate_photon_k.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int] + \
            [ctypes.c_double] * 8 + [_dp]
        L.orc_brute_ray_curved.argtypes = [ctypes.POINTER(_Atm)] + [ctypes.c_double] * 5 + \
            [_dp, _dp]
        L.orc_build_curved_tables.argtypes = [ctypes.POINTER(_Atm), ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                              _dp, _dp, _dp]
        L.orc_bunches.argtypes = [ctypes.POINTER(_Cfg), ctypes.POINTER(_Tracks),
                                  ctypes.c_uint64, _i64p, ctypes.c_int,
                                  ctypes.POINTER(_Out)]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_density.argtypes = [ctypes.POINTER(_Cfg), ctypes.POINTER(_Tracks), ctypes.c_uint64,
                                  _i32p, ctypes.c_double, _dp, _dp]
        L.orc_density_grad.argtypes = [ctypes.POINTER(_Cfg), ctypes.POINTER(_Tracks),
                                       ctypes.c_uint64, _i32p, ctypes.c_double, _dp, _dp,
                                       ctypes.c_double, _dp, _dp, _dp, _dp]
        L.orc_profile.argtypes = [ctypes.POINTER(_Cfg), ctypes.POINTER(_Tracks), _dp,
                                  ctypes.c_double, ctypes.c_int, _dp]
        L.orc_generate_steps.argtypes = [ctypes.POINTER(_Shower), ctypes.c_int, ctypes.c_double,
                                         ctypes.c_uint64, ctypes.c_int] + [_dp] * 9 + \
            [_u32p, _dp]
        L.orc_philox_fill.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                      ctypes.c_int64, _u32p]
        _lib = L
    return _lib


def _ptr(a, ctype=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Atmosphere
# --------------------------------------------------------------------------
def _atm(atm: dict) -> _Atm:
    A = _Atm()
    A.h_bound[:] = list(map(float, atm["h_bound"]))
    A.a[:] = list(map(float, atm["a"]))
    A.b[:] = list(map(float, atm["b"]))
    A.c[:] = list(map(float, atm["c"]))
    A.n0_minus_1 = float(atm["n0_minus_1"])
    return A


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: ctr (4 x u32), key (2 x u32) -> 4 x u32."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                            _ptr(o, ctypes.c_uint32))
    return o


def philox_stream(seed: int, track: int, j0: int, n: int):
    """n Philox blocks (4 words each) for counters (track, j0 + m, 0)."""
    o = np.zeros((n, 4), dtype=np.uint32)
    lib().orc_philox_fill(ctypes.c_uint64(seed), ctypes.c_uint64(track),
                          ctypes.c_uint32(j0), int(n), _ptr(o, ctypes.c_uint32))
    return o


def eta_lookup(tab, h_max, h):
    """Fine-table lookup of eta = n - 1 (clamped to [0, h_max])."""
    t = _f64(tab)
    return np.array([lib().orc_eta_lookup(_ptr(t), len(t), float(h_max), float(x))
                     for x in np.atleast_1d(h)])


def thickness(atm, h):
    A = _atm(atm)
    return np.array([lib().orc_thickness(ctypes.byref(A), float(x))
                     for x in np.atleast_1d(h)])


def rho(atm, h):
    A = _atm(atm)
    return np.array([lib().orc_rho(ctypes.byref(A), float(x)) for x in np.atleast_1d(h)])


def eta_exact(atm, h):
    A = _atm(atm)
    return np.array([lib().orc_eta_exact(ctypes.byref(A), float(x))
                     for x in np.atleast_1d(h)])


def eta_table(atm, h_max, n_fine):
    A = _atm(atm)
    t = np.zeros(n_fine)
    if lib().orc_build_eta_table(ctypes.byref(A), float(h_max), int(n_fine), _ptr(t)) != 0:
        raise ValueError("bad eta table arguments")
    return t


def refraction_tables(atm, h_obs, h_max, H, Z, theta_max_rad, tol=1e-13):
    A = _atm(atm)
    ax = np.zeros((H, Z))
    al = np.zeros((H, Z))
    rc = lib().orc_build_refraction_tables(ctypes.byref(A), float(h_obs), float(h_max),
                                           int(H), int(Z), float(theta_max_rad),
                                           float(tol), _ptr(ax), _ptr(al))
    if rc != 0:
        raise ValueError("bad refraction table arguments")
    return ax, al


def curved_tables(atm, earth_radius, h_obs, h_max, H, Z, theta_max_rad, tol=1e-13):
    """Refraction tables of a curved atmosphere (corrections of the central
    angle and of the two parts of the optical path to the straight line of
    the same arrival zenith), on a zenith axis uniform in sec: ax, al, ag."""
    A = _atm(atm)
    ax = np.zeros((H, Z))
    al = np.zeros((H, Z))
    ag = np.zeros((H, Z))
    rc = lib().orc_build_curved_tables(ctypes.byref(A), float(earth_radius), float(h_obs),
                                       float(h_max), int(H), int(Z), float(theta_max_rad),
                                       float(tol), _ptr(ax), _ptr(al), _ptr(ag))
    if rc != 0:
        raise ValueError("bad curved table arguments")
    return ax, al, ag


def brute_ray_curved(atm, earth_radius, h_obs, h_e, sin_obs, tol=1e-12):
    """(B), curved: central angle phi and optical path l from h_obs to h_e."""
    A = _atm(atm)
    phi = ctypes.c_double()
    l_ = ctypes.c_double()
    rc = lib().orc_brute_ray_curved(ctypes.byref(A), float(earth_radius), float(h_obs),
                                    float(h_e), float(sin_obs), float(tol), ctypes.byref(phi),
                                    ctypes.byref(l_))
    if rc != 0:
        raise ValueError("bad ray")
    return phi.value, l_.value


def brute_ray(atm, h_obs, h_e, sin_obs, tol=1e-12):
    """(B): horizontal displacement x and optical path l from h_obs to h_e."""
    A = _atm(atm)
    x = ctypes.c_double()
    l_ = ctypes.c_double()
    rc = lib().orc_brute_ray(ctypes.byref(A), float(h_obs), float(h_e), float(sin_obs),
                             float(tol), ctypes.byref(x), ctypes.byref(l_))
    if rc != 0:
        raise ValueError("bad ray")
    return x.value, l_.value


# --------------------------------------------------------------------------
# A configured model: atmosphere + tables + telescopes + band
# --------------------------------------------------------------------------
@dataclass
class Model:
    atm: dict
    h_obs: float
    telescopes: np.ndarray               # (n_tel, 4): x, y, z, r
    h_max: float = 60000.0
    n_fine: int = 10000
    H: int = 1000
    Z: int = 64
    theta_max_deg: float = 70.0
    bunch_size: float = 5.0
    lambda1_nm: float = 300.0
    lambda2_nm: float = 600.0
    t_ref: np.ndarray | None = None
    # atmospheric transmission: dict(tau=(n_lambda, n_height) vertical optical
    # depths, lambda_nm=(first, last node), height_m=(first, last node)) or None
    transmission: dict | None = None
    # beyond-table fallback: bunches up to this observation-level zenith
    # (deg) past the tables' range take the ray integrals (0: off)
    fallback_deg: float = 0.0
    # wavelength-dependent index: kappa at k (2..9) nodes uniform in 1/lambda
    # from 1/lambda1 (node 0) to 1/lambda2, n(h, lambda) - 1 = eta(h) kappa,
    # positive and not increasing along the nodes; None: constant index
    dispersion: np.ndarray | None = None
    # curved atmosphere: the Earth's radius in m (0: flat layers); positions
    # are then Cartesian in the core frame and heights radial
    earth_radius: float = 0.0
    table_tol: float = 1e-13
    bf_tol: float = 1e-12
    eta_tab: np.ndarray = field(init=False, repr=False)
    ax: np.ndarray = field(init=False, repr=False)
    ag: np.ndarray | None = field(init=False, repr=False, default=None)
    al: np.ndarray = field(init=False, repr=False)

    def __post_init__(self):
        self.telescopes = _f64(np.asarray(self.telescopes).reshape(-1, 4))
        self.eta_tab = eta_table(self.atm, self.h_max, self.n_fine)

        def tables(atm):
            if self.earth_radius > 0.0:
                return curved_tables(atm, self.earth_radius, self.h_obs, self.h_max, self.H,
                                     self.Z, self.theta_max_rad, self.table_tol)
            return refraction_tables(atm, self.h_obs, self.h_max, self.H, self.Z,
                                     self.theta_max_rad, self.table_tol) + (None,)

        if self.dispersion is not None:
            kap = _f64(np.asarray(self.dispersion, float).ravel())
            if not (2 <= kap.size <= 9) or not np.all(kap > 0) or np.any(np.diff(kap) > 0):
                raise ValueError("dispersion: 2..9 positive, non-increasing kappa nodes")
            self.dispersion = kap
            # the tables of the band's two ends: n - 1 scaled by kappa
            lo = dict(self.atm, n0_minus_1=float(self.atm["n0_minus_1"]) * kap[-1])
            hi = dict(self.atm, n0_minus_1=float(self.atm["n0_minus_1"]) * kap[0])
            self.ax, self.al, self.ag = tables(lo)
            self.ax_hi, self.al_hi, self.ag_hi = tables(hi)
        else:
            self.ax, self.al, self.ag = tables(self.atm)
        if self.t_ref is not None:
            self.t_ref = _f64(np.atleast_1d(self.t_ref))

    @property
    def theta_max_rad(self) -> float:
        return float(self.theta_max_deg) * 3.14159265358979323846 / 180.0

    def _cfg(self) -> _Cfg:
        C = _Cfg()
        C.atm = _atm(self.atm)
        C.h_obs = self.h_obs
        C.h_max = self.h_max
        C.n_fine = self.n_fine
        C.eta_tab = _ptr(self.eta_tab)
        C.H, C.Z = self.H, self.Z
        C.theta_max = self.theta_max_rad
        C.ax, C.al = _ptr(self.ax), _ptr(self.al)
        C.bunch_size = self.bunch_size
        C.lambda1_nm, C.lambda2_nm = self.lambda1_nm, self.lambda2_nm
        C.n_tel = self.telescopes.shape[0]
        C.tel = _ptr(self.telescopes)
        if self.t_ref is not None:
            C.t_ref = _ptr(self.t_ref)
            C.n_showers = self.t_ref.shape[0]
        else:
            C.t_ref = None
            C.n_showers = 0
        C.bf_tol = self.bf_tol
        C.earth_radius = float(self.earth_radius)
        C.ag = _ptr(self.ag)
        if self.dispersion is not None:
            C.ag_hi = _ptr(self.ag_hi)
        if self.dispersion is not None:
            C.disp_k = int(self.dispersion.size)
            C.disp_kappa = _ptr(self.dispersion)
            C.ax_hi, C.al_hi = _ptr(self.ax_hi), _ptr(self.al_hi)
        if self.fallback_deg > 0.0:
            sf = math.sin(self.fallback_deg * 3.14159265358979323846 / 180.0)
            C.fb_sin2_max = sf * sf
        if self.transmission is not None:
            tr = self.transmission
            self._tau = _f64(np.asarray(tr["tau"], float))
            if self._tau.ndim != 2 or min(self._tau.shape) < 2:
                raise ValueError("transmission table needs at least 2 x 2 nodes")
            C.trans_nl, C.trans_nh = self._tau.shape
            C.trans_l0, C.trans_l1 = (float(v) for v in tr["lambda_nm"])
            C.trans_h0, C.trans_h1 = (float(v) for v in tr["height_m"])
            C.trans_tau = _ptr(self._tau)
        else:
            C.trans_tau = None
        return C

    # ---- a1: per-step yield ------------------------------------------------
    def segment_yield(self, tracks: dict):
        T, keep = self._tracks(tracks)
        n = T.n
        nb = np.zeros(n, np.int64)
        w = np.zeros(n)
        s2 = np.zeros(n)
        valid = np.zeros(n, np.int32)
        C = self._cfg()
        lib().orc_segment_yield(ctypes.byref(C), ctypes.byref(T), _ptr(nb, ctypes.c_int64),
                                _ptr(w), _ptr(s2), _ptr(valid, ctypes.c_int32))
        del keep
        return nb, w, s2, valid.astype(bool)

    def _tracks(self, tracks: dict, track_base: int = 0):
        """ctypes view of a track dict; the second value keeps the arrays alive."""
        n = len(tracks["z0"])
        arr = {}
        for k in ("x0", "y0", "z0", "t0", "len", "ekin", "ux", "uy", "uz"):
            v = tracks.get(k)
            arr[k] = _f64(v) if v is not None else np.zeros(n)
        T = _Tracks()
        for k, v in arr.items():
            setattr(T, k, _ptr(v))
        shower = tracks.get("shower")
        if shower is not None:
            shower = np.ascontiguousarray(shower, dtype=np.uint32)
            arr["shower"] = shower
            T.shower = _ptr(shower, ctypes.c_uint32)
        else:
            T.shower = None
        T.n = n
        T.track_base = int(track_base)
        return T, arr

    # ---- a2..a5: every bunch ----------------------------------------------
    def bunches(self, tracks: dict, seed: int, variant: int = 0, track_base: int = 0):
        nb, _, _, _ = self.segment_yield(tracks)
        off = np.zeros(len(nb) + 1, np.int64)
        np.cumsum(nb, out=off[1:])
        nbt = int(off[-1])
        T, keep = self._tracks(tracks, track_base)
        out = {k: np.zeros(nbt) for k in ("xe", "ye", "he", "te", "px", "py", "pz", "X", "Y",
                                          "t", "cx", "cy", "cz", "lam", "w")}
        out["status"] = np.zeros(nbt, np.int32)
        out["nhit"] = np.zeros(nbt, np.int32)
        out["hit_tel"] = np.full((nbt, MAX_HITS), -1, np.int32)
        for k in ("hit_x", "hit_y", "hit_t"):
            out[k] = np.zeros((nbt, MAX_HITS))
        out["tr_margin"] = np.full(nbt, np.nan)
        out["Zg"] = np.zeros(nbt)
        O = _Out()
        for k, v in out.items():
            setattr(O, k, _ptr(v, ctypes.c_int32 if v.dtype == np.int32 else ctypes.c_double))
        C = self._cfg()
        rc = lib().orc_bunches(ctypes.byref(C), ctypes.byref(T), ctypes.c_uint64(seed),
                               _ptr(off, ctypes.c_int64), int(variant), ctypes.byref(O))
        if rc != 0:
            raise ValueError("orc_bunches failed")
        seg = np.repeat(np.arange(len(nb), dtype=np.int64), nb)
        out["seg"] = seg
        out["j"] = np.arange(nbt, dtype=np.int64) - off[seg]
        out["nb"] = nb
        out["off"] = off
        return out

    # ---- differentiable read-out: smoothed density and mean time ----------
    def density_sums(self, tracks: dict, seed: int, nb_frozen, sigma: float = 1.0,
                     track_base: int = 0):
        """S_k = sum w G, U_k = sum w G t over the telescopes (frozen nb)."""
        T, keep = self._tracks(tracks, track_base)
        nb = np.ascontiguousarray(nb_frozen, dtype=np.int32)
        S = np.zeros(self.telescopes.shape[0])
        U = np.zeros(self.telescopes.shape[0])
        C = self._cfg()
        rc = lib().orc_density(ctypes.byref(C), ctypes.byref(T), ctypes.c_uint64(seed),
                               _ptr(nb, ctypes.c_int32), float(sigma), _ptr(S), _ptr(U))
        if rc != 0:
            raise ValueError("orc_density failed")
        del keep
        return S, U

    def density_grad(self, tracks: dict, seed: int, nb_frozen, sigma: float, gD, gT,
                     track_base: int = 0):
        """The read-out S, U and the gradients of L = sum gD S + gT U / S by
        forward-mode dual numbers (flat layers, constant index, table
        variant): grad_atm (15: a, b, c) and grad_steps (6, n: x0, y0, z0,
        ux, uy, uz)."""
        T, keep = self._tracks(tracks, track_base)
        nb = np.ascontiguousarray(nb_frozen, dtype=np.int32)
        n_tel = self.telescopes.shape[0]
        S, U = np.zeros(n_tel), np.zeros(n_tel)
        gD = _f64(np.asarray(gD, float).reshape(n_tel))
        gT = _f64(np.asarray(gT, float).reshape(n_tel))
        ga = np.zeros(15)
        gs = np.zeros((6, len(nb)))
        C = self._cfg()
        rc = lib().orc_density_grad(ctypes.byref(C), ctypes.byref(T), ctypes.c_uint64(seed),
                                    _ptr(nb, ctypes.c_int32), float(sigma), _ptr(gD), _ptr(gT),
                                    float(self.table_tol), _ptr(S), _ptr(U), _ptr(ga), _ptr(gs))
        if rc != 0:
            raise ValueError("orc_density_grad failed")
        del keep
        return S, U, ga, gs

    # ---- longitudinal production profile (CERLDE) --------------------------
    def profile(self, tracks: dict, bin_gcm2: float, n_bins: int, axis_cos=None):
        """Photons produced per depth bin and shower: (n_showers, n_bins)."""
        T, keep = self._tracks(tracks)
        C = self._cfg()
        ns = max(C.n_showers, 1)
        prof = np.zeros((ns, int(n_bins)))
        ac = None
        if axis_cos is not None:
            ac = _f64(np.atleast_1d(axis_cos))
            if ac.shape[0] < ns:
                raise ValueError("axis_cos needs one entry per shower")
        rc = lib().orc_profile(ctypes.byref(C), ctypes.byref(T),
                               _ptr(ac) if ac is not None else None, float(bin_gcm2),
                               int(n_bins), _ptr(prof))
        if rc != 0:
            raise ValueError("orc_profile failed")
        del keep
        return prof

    def propagate_photon(self, xe, ye, he, te, px, py, pz, variant=0, kappa=None):
        """One bunch to the ground; kappa scales n - 1 at its wavelength.
        r: X, Y, t, cx, cy, cz, arrival z - h_obs, cosine to the local
        vertical, emission height."""
        r = np.zeros(9)
        C = self._cfg()
        if kappa is None:
            st = lib().orc_propagate_photon(ctypes.byref(C), int(variant), xe, ye, he, te,
                                            px, py, pz, _ptr(r))
        else:
            st = lib().orc_propagate_photon_k(ctypes.byref(C), int(variant), float(kappa), xe,
                                              ye, he, te, px, py, pz, _ptr(r))
        return st, r


def hit_records(out: dict, track_base: int = 0):
    """Flatten the per-bunch hit lists into records sorted by (tel, key)."""
    nh = np.minimum(out["nhit"], MAX_HITS)
    if np.any(out["nhit"] > MAX_HITS):
        raise RuntimeError("a bunch crossed more telescopes than the oracle records")
    b = np.repeat(np.arange(len(nh)), nh)
    slot = np.concatenate([np.arange(m) for m in nh]) if len(nh) else np.zeros(0, int)
    slot = slot.astype(np.int64)
    tel = out["hit_tel"][b, slot]
    key = ((out["seg"][b] + track_base).astype(np.uint64) << np.uint64(32)) | \
        out["j"][b].astype(np.uint64)
    rec = dict(tel=tel.astype(np.int64), key=key, bunch=b,
               x=out["hit_x"][b, slot], y=out["hit_y"][b, slot], t=out["hit_t"][b, slot],
               cx=out["cx"][b], cy=out["cy"][b], zem=out["he"][b], w=out["w"][b],
               lam=out["lam"][b])
    order = np.lexsort((rec["key"], rec["tel"]))
    return {k: v[order] for k, v in rec.items()}


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """OpenMP threads of the oracle's parallel loops (timing only)."""
    lib().orc_set_num_threads(int(n))
