"""ctypes binding of libcher.so: argument marshalling only.

Every step of the photon-bunch path runs in the library's CUDA kernels (or,
for the one-off table build, in its C++ host code).  PyTorch supplies device
memory and streams.  If the library has not been built, importing works but
every call raises: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# CHER_DEBUG=1 selects the bounds-checked build (libcher_debug.so)
LIB_PATH = os.path.join(_HERE, "libcher_debug.so" if os.environ.get("CHER_DEBUG", "") == "1"
                        else "libcher.so")

CHER_FP64 = 0
CHER_FP32_BULK = 1
NSTATS = 16
STAT_NAMES = ["steps", "emitting", "invalid", "bunches", "upward", "below_obs", "above_max",
              "angle", "ground", "hits", "overflow", "absorbed", "fallback", "fb_lost", "debug"]
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error",
                4: "tables not built", 5: "out of range", 6: "overflow", 7: "timeout"}


class CherError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)} (status {code})")
        self.code = code


class Atmosphere(ctypes.Structure):
    _fields_ = [("h_bound", ctypes.c_double * 6), ("a", ctypes.c_double * 5),
                ("b", ctypes.c_double * 5), ("c", ctypes.c_double * 5),
                ("n0_minus_1", ctypes.c_double)]


class Telescope(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double), ("y", ctypes.c_double), ("z", ctypes.c_double),
                ("r", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("bunch_size", ctypes.c_double), ("lambda_min_nm", ctypes.c_double),
                ("lambda_max_nm", ctypes.c_double), ("n_fine", ctypes.c_int32)]


class Tracks(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_void_p), ("y0", ctypes.c_void_p), ("z0", ctypes.c_void_p),
                ("t0", ctypes.c_void_p), ("len", ctypes.c_void_p), ("ekin", ctypes.c_void_p),
                ("ux", ctypes.c_void_p), ("uy", ctypes.c_void_p), ("uz", ctypes.c_void_p),
                ("shower", ctypes.c_void_p), ("t_ref", ctypes.c_void_p),
                ("n_showers", ctypes.c_int32), ("n", ctypes.c_int64),
                ("track_base", ctypes.c_int64)]


class Output(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("tim", ctypes.c_void_p), ("key", ctypes.c_void_p),
                ("cap_per_tel", ctypes.c_int64), ("count", ctypes.c_void_p),
                ("stats", ctypes.c_void_p)]


class Profile(ctypes.Structure):
    _fields_ = [("profile", ctypes.c_void_p), ("n_bins", ctypes.c_int32),
                ("bin_gcm2", ctypes.c_double), ("axis_cos", ctypes.c_void_p)]


class Shower(ctypes.Structure):
    _fields_ = [("e0_mev", ctypes.c_double), ("zenith", ctypes.c_double),
                ("azimuth", ctypes.c_double), ("core_x", ctypes.c_double),
                ("core_y", ctypes.c_double), ("n_steps", ctypes.c_int64)]


class StepBuffers(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("x0", "y0", "z0", "t0", "len", "ekin", "ux", "uy",
                                               "uz", "shower", "t_ref")]


class Transmission(ctypes.Structure):
    _fields_ = [("n_lambda", ctypes.c_int32), ("n_height", ctypes.c_int32),
                ("lambda_min_nm", ctypes.c_double), ("lambda_max_nm", ctypes.c_double),
                ("h_min", ctypes.c_double), ("h_max", ctypes.c_double),
                ("tau", ctypes.POINTER(ctypes.c_double))]


class Trace(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("tim", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("nhit", ctypes.c_void_p), ("first_hit", ctypes.c_void_p),
                ("n_bunches", ctypes.c_int64)]


_S = ctypes.c_int
_P = ctypes.c_void_p
_lib = None

# name -> (restype, argtypes): every symbol of include/cher.h
SIGNATURES = {
    "cher_status_string": (ctypes.c_char_p, [_S]),
    "cher_create": (_S, [ctypes.POINTER(Atmosphere), ctypes.c_double, ctypes.POINTER(Telescope),
                         ctypes.c_int32, ctypes.POINTER(Options), ctypes.POINTER(_P)]),
    "cher_build_refraction_tables": (_S, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                          ctypes.c_double]),
    "cher_destroy": (_S, [_P]),
    "cher_generate_propagate": (_S, [_P, ctypes.POINTER(Tracks), ctypes.c_uint64, _S,
                                     ctypes.POINTER(Output), _P]),
    "cher_generate_propagate_ex": (_S, [_P, ctypes.POINTER(Tracks), ctypes.c_uint64, _S,
                                        ctypes.POINTER(Output), ctypes.POINTER(Profile), _P]),
    "cher_round_to_float": (_S, [_P, _P, ctypes.c_int64, _P]),
    "cher_split_to_float": (_S, [_P, _P, _P, ctypes.c_int64, _P]),
    "cher_set_transmission": (_S, [_P, ctypes.POINTER(Transmission)]),
    "cher_set_fallback": (_S, [_P, ctypes.c_double, ctypes.c_int64]),
    "cher_set_dispersion": (_S, [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int32]),
    "cher_set_curved": (_S, [_P, ctypes.c_double]),
    "cher_pack_records": (_S, [_P, ctypes.POINTER(Output), ctypes.c_int, ctypes.c_int64,
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p]),
    "cher_generate_steps": (_S, [_P, ctypes.POINTER(Shower), ctypes.c_int32, ctypes.c_uint64, _S,
                                 ctypes.POINTER(StepBuffers), _P]),
    "cher_generate_propagate_noalloc": (_S, [_P, ctypes.POINTER(Tracks), ctypes.c_uint64, _S,
                                             ctypes.POINTER(Output), _P]),
    "cher_graph_create": (_S, [_P, ctypes.POINTER(Tracks), ctypes.c_uint64, _S,
                               ctypes.POINTER(Output), ctypes.POINTER(_P)]),
    "cher_graph_launch": (_S, [_P, _P]),
    "cher_graph_destroy": (_S, [_P]),
    "cher_sync_status": (_S, [_P, ctypes.POINTER(Output), ctypes.POINTER(ctypes.c_ulonglong), _P]),
    "cher_set_launch": (_S, [_P, ctypes.c_int32, ctypes.c_int32]),
    "cher_get_launch": (_S, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "cher_segment_yield": (_S, [_P, ctypes.POINTER(Tracks), _S, _P, _P, _P]),
    "cher_trace_bunches": (_S, [_P, ctypes.POINTER(Tracks), ctypes.c_uint64, _S, _P,
                                ctypes.POINTER(Trace), _P]),
    "cher_get_tables": (_S, [_P, _P, _P, _P]),
    "cher_build_curved_tables_host": (_S, [ctypes.POINTER(Atmosphere), ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "cher_build_tables_host": (_S, [ctypes.POINTER(Atmosphere), ctypes.c_double, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                    ctypes.c_double, _P, _P, _P]),
    "cher_autotune": (_S, [_P, ctypes.POINTER(Tracks), ctypes.c_uint64, _S,
                           ctypes.POINTER(Output), ctypes.c_char_p, _P]),
    "cher_density": (_S, [_P, ctypes.POINTER(Tracks), ctypes.c_uint64, _S, ctypes.c_double, _P,
                          _P, _P, _P]),
    "cher_adjoint": (_S, [_P, ctypes.POINTER(Tracks), ctypes.c_uint64, _S, ctypes.c_double, _P,
                          _P, _P, _P, _P, _P]),
    "cher_set_atmosphere": (_S, [_P, ctypes.POINTER(Atmosphere)]),
    "cher_build_sensitivity_host": (_S, [ctypes.POINTER(Atmosphere), ctypes.c_double,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_double, ctypes.c_double, _P, _P]),
}


def lib():
    """Load libcher.so; raise if it has not been built (no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2006_14927_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code: int, what: str):
    if code != 0:
        raise CherError(code, what)


def atmosphere_struct(atm: dict) -> Atmosphere:
    A = Atmosphere()
    A.h_bound[:] = [float(v) for v in atm["h_bound"]]
    A.a[:] = [float(v) for v in atm["a"]]
    A.b[:] = [float(v) for v in atm["b"]]
    A.c[:] = [float(v) for v in atm["c"]]
    A.n0_minus_1 = float(atm["n0_minus_1"])
    return A


def build_tables_host(atm: dict, h_obs: float, n_fine: int, n_heights: int, n_zenith: int,
                      zenith_max_deg: float, h_max: float):
    """The library's host table builder on its own (no CUDA call)."""
    eta = np.zeros(n_fine)
    ax = np.zeros((n_heights, n_zenith))
    al = np.zeros((n_heights, n_zenith))
    A = atmosphere_struct(atm)
    _check(lib().cher_build_tables_host(ctypes.byref(A), float(h_obs), int(n_fine),
                                        int(n_heights), int(n_zenith), float(zenith_max_deg),
                                        float(h_max), eta.ctypes.data, ax.ctypes.data,
                                        al.ctypes.data), "cher_build_tables_host")
    return eta, ax, al


def build_curved_tables_host(atm: dict, earth_radius_m: float, h_obs: float, n_heights: int,
                             n_zenith: int, zenith_max_deg: float, h_max: float):
    """The curved atmosphere's host tables (no CUDA call): ax, al, ag."""
    out = [np.zeros((n_heights, n_zenith)) for _ in range(3)]
    A = atmosphere_struct(atm)
    _check(lib().cher_build_curved_tables_host(ctypes.byref(A), float(earth_radius_m),
                                               float(h_obs), int(n_heights), int(n_zenith),
                                               float(zenith_max_deg), float(h_max),
                                               *[o.ctypes.data for o in out]),
           "cher_build_curved_tables_host")
    return tuple(out)


def build_sensitivity_host(atm: dict, h_obs: float, n_fine: int, n_heights: int,
                           n_zenith: int, zenith_max_deg: float, h_max: float):
    """The adjoint's refraction-table sensitivities (host, no CUDA call):
    d ax / d p and d al / d p for p = b_0..b_4, c_0..c_4, each (10, H, Z)."""
    dax = np.zeros((10, n_heights, n_zenith))
    dal = np.zeros((10, n_heights, n_zenith))
    A = atmosphere_struct(atm)
    _check(lib().cher_build_sensitivity_host(ctypes.byref(A), float(h_obs), int(n_fine),
                                             int(n_heights), int(n_zenith),
                                             float(zenith_max_deg), float(h_max),
                                             dax.ctypes.data, dal.ctypes.data),
           "cher_build_sensitivity_host")
    return dax, dal


def _torch():
    import torch
    return torch


def device_tracks(tracks: dict, precision: int, device="cuda", t_ref=None, pin=False):
    """Copy a track dict (numpy or torch) to device tensors of the ABI's dtypes."""
    torch = _torch()
    ddir = torch.float32 if precision == CHER_FP32_BULK else torch.float64
    out = {}
    for k in ("x0", "y0", "z0", "t0", "len", "ekin"):
        out[k] = torch.as_tensor(tracks[k]).to(device=device, dtype=torch.float64).contiguous()
    for k in ("ux", "uy", "uz"):
        out[k] = torch.as_tensor(tracks[k]).to(device=device, dtype=ddir).contiguous()
    if tracks.get("shower") is not None:
        sh = np.asarray(tracks["shower"]).astype(np.uint32).view(np.int32) \
            if not hasattr(tracks["shower"], "device") else tracks["shower"]
        out["shower"] = torch.as_tensor(sh).to(device=device, dtype=torch.int32).contiguous()
    if t_ref is not None:
        out["t_ref"] = torch.as_tensor(np.atleast_1d(t_ref) if not hasattr(t_ref, "device")
                                       else t_ref).to(device=device,
                                                      dtype=torch.float64).contiguous()
    return out


def _stream_ptr(stream):
    if stream is None:
        return _torch().cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


@dataclass
class HitBuffers:
    """Per-telescope record buffers (device tensors) plus counters."""
    pos: object      # (n_tel, cap, 4): x, y, cx, cy
    tim: object      # (n_tel, cap, 4): t, z_emit, photons, lambda_nm
    key: object      # (n_tel, cap) int64 holding the u64 key bits
    count: object    # (n_tel,) int64 holding u64 counts
    stats: object    # (16,) int64
    cap: int
    precision: int

    def struct(self) -> Output:
        o = Output()
        o.pos = self.pos.data_ptr()
        o.tim = self.tim.data_ptr()
        o.key = self.key.data_ptr()
        o.cap_per_tel = self.cap
        o.count = self.count.data_ptr()
        o.stats = self.stats.data_ptr()
        return o

    def records(self):
        """Host numpy records of every telescope, sorted by (telescope, key)."""
        cnt = np.minimum(self.count.cpu().numpy(), self.cap)
        pos, tim, key = self.pos.cpu().numpy(), self.tim.cpu().numpy(), self.key.cpu().numpy()
        tel = np.concatenate([np.full(c, k, np.int64) for k, c in enumerate(cnt)]) \
            if len(cnt) else np.zeros(0, np.int64)
        sel = (tel, np.concatenate([np.arange(c) for c in cnt]).astype(np.int64))
        rec = dict(tel=tel, key=key[sel].view(np.uint64), x=pos[sel][:, 0], y=pos[sel][:, 1],
                   cx=pos[sel][:, 2], cy=pos[sel][:, 3], t=tim[sel][:, 0], zem=tim[sel][:, 1],
                   w=tim[sel][:, 2], lam=tim[sel][:, 3])
        order = np.lexsort((rec["key"], rec["tel"]))
        return {k: v[order] for k, v in rec.items()}


class Context:
    """A cher_ctx: atmosphere, observation level, telescopes and tables."""

    def __init__(self, atm: dict, h_obs: float, telescopes, bunch_size=5.0,
                 lambda_min_nm=300.0, lambda_max_nm=600.0, n_fine=10000):
        tel = np.asarray(telescopes, dtype=np.float64).reshape(-1, 4)
        self.n_tel = tel.shape[0]
        T = (Telescope * self.n_tel)(*[Telescope(*map(float, r)) for r in tel])
        O = Options(float(bunch_size), float(lambda_min_nm), float(lambda_max_nm), int(n_fine))
        A = atmosphere_struct(atm)
        h = ctypes.c_void_p()
        _check(lib().cher_create(ctypes.byref(A), float(h_obs), T, self.n_tel, ctypes.byref(O),
                                 ctypes.byref(h)), "cher_create")
        self._h = h
        self.h_obs = float(h_obs)
        self.n_fine = int(n_fine)
        self.H = self.Z = 0

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().cher_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_refraction_tables(self, n_heights=1000, n_zenith=64, zenith_max_deg=70.0,
                                h_max=60000.0):
        _check(lib().cher_build_refraction_tables(self._h, int(n_heights), int(n_zenith),
                                                  float(zenith_max_deg), float(h_max)),
               "cher_build_refraction_tables")
        self.H, self.Z = int(n_heights), int(n_zenith)

    def set_launch(self, block_threads, ctas_per_sm):
        """Steps per tile (128, 256 or 512) and persistent CTAs per SM (0: one
        CTA per tile); a new context starts at 128 / 8."""
        _check(lib().cher_set_launch(self._h, int(block_threads), int(ctas_per_sm)),
               "cher_set_launch")

    def get_launch(self):
        b, c = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().cher_get_launch(self._h, ctypes.byref(b), ctypes.byref(c)),
               "cher_get_launch")
        return b.value, c.value

    def get_tables(self):
        eta = np.zeros(self.n_fine)
        ax = np.zeros((self.H, self.Z))
        al = np.zeros((self.H, self.Z))
        _check(lib().cher_get_tables(self._h, eta.ctypes.data, ax.ctypes.data, al.ctypes.data),
               "cher_get_tables")
        return eta, ax, al

    @staticmethod
    def tracks_struct(dev: dict, track_base: int = 0) -> Tracks:
        t = Tracks()
        for k in ("x0", "y0", "z0", "t0", "len", "ekin", "ux", "uy", "uz"):
            setattr(t, k, dev[k].data_ptr())
        t.shower = dev["shower"].data_ptr() if "shower" in dev else None
        if "t_ref" in dev:
            t.t_ref = dev["t_ref"].data_ptr()
            t.n_showers = int(dev["t_ref"].numel())
        else:
            t.t_ref = None
            t.n_showers = 0
        t.n = int(dev["x0"].numel())
        t.track_base = int(track_base)
        return t

    def alloc_hits(self, cap_per_tel: int, precision: int, device="cuda") -> HitBuffers:
        torch = _torch()
        dt = torch.float32 if precision == CHER_FP32_BULK else torch.float64
        n = self.n_tel
        return HitBuffers(pos=torch.zeros((n, cap_per_tel, 4), dtype=dt, device=device),
                          tim=torch.zeros((n, cap_per_tel, 4), dtype=dt, device=device),
                          key=torch.zeros((n, cap_per_tel), dtype=torch.int64, device=device),
                          count=torch.zeros(n, dtype=torch.int64, device=device),
                          stats=torch.zeros(NSTATS, dtype=torch.int64, device=device),
                          cap=int(cap_per_tel), precision=precision)

    def generate_propagate(self, dev_tracks: dict, seed: int, precision: int,
                           out: HitBuffers, stream=None, track_base: int = 0,
                           profile=None, bin_gcm2: float = 10.0, axis_cos=None):
        """The hot path; with `profile` (a device float64 tensor of shape
        (max(n_showers, 1), n_bins), added to) also the longitudinal
        production profile in the same launch."""
        t = self.tracks_struct(dev_tracks, track_base)
        o = out.struct()
        if profile is None:
            _check(lib().cher_generate_propagate(self._h, ctypes.byref(t), ctypes.c_uint64(seed),
                                                 int(precision), ctypes.byref(o),
                                                 ctypes.c_void_p(_stream_ptr(stream))),
                   "cher_generate_propagate")
            return
        torch = _torch()
        if profile.dtype != torch.float64 or not profile.is_contiguous() or profile.dim() != 2:
            raise ValueError("profile must be a contiguous 2-D float64 device tensor")
        rows = max(int(dev_tracks["t_ref"].numel()) if dev_tracks.get("t_ref") is not None
                   else 0, 1)
        if profile.shape[0] < rows:
            raise ValueError("profile needs one row per shower")
        if axis_cos is not None:
            axis_cos = torch.as_tensor(axis_cos, dtype=torch.float64,
                                       device=profile.device).contiguous()
            if axis_cos.numel() < rows:
                raise ValueError("axis_cos needs one entry per shower")
        pr = Profile(profile.data_ptr(), int(profile.shape[1]), float(bin_gcm2),
                     axis_cos.data_ptr() if axis_cos is not None else None)
        _check(lib().cher_generate_propagate_ex(self._h, ctypes.byref(t), ctypes.c_uint64(seed),
                                                int(precision), ctypes.byref(o), ctypes.byref(pr),
                                                ctypes.c_void_p(_stream_ptr(stream))),
               "cher_generate_propagate_ex")

    def sync_status(self, out: HitBuffers, stream=None):
        st = (ctypes.c_ulonglong * NSTATS)()
        o = out.struct()
        code = lib().cher_sync_status(self._h, ctypes.byref(o), st,
                                      ctypes.c_void_p(_stream_ptr(stream)))
        if code not in (0, 6):
            raise CherError(code, "cher_sync_status")
        return code, np.array(st[:], dtype=np.uint64)

    def segment_yield(self, dev_tracks: dict, precision: int, stream=None):
        torch = _torch()
        n = int(dev_tracks["x0"].numel())
        dev = dev_tracks["x0"].device
        nb = torch.zeros(n, dtype=torch.int32, device=dev)
        w = torch.zeros(n, dtype=torch.float64, device=dev)
        t = self.tracks_struct(dev_tracks)
        _check(lib().cher_segment_yield(self._h, ctypes.byref(t), int(precision), nb.data_ptr(),
                                        w.data_ptr(), ctypes.c_void_p(_stream_ptr(stream))),
               "cher_segment_yield")
        return nb, w

    def trace_bunches(self, dev_tracks: dict, seed: int, precision: int, bunch_off,
                      stream=None, track_base: int = 0):
        torch = _torch()
        nbt = int(bunch_off[-1].item())
        dev = dev_tracks["x0"].device
        dt = torch.float32 if precision == CHER_FP32_BULK else torch.float64
        pos = torch.zeros((nbt, 4), dtype=dt, device=dev)
        tim = torch.zeros((nbt, 4), dtype=dt, device=dev)
        status = torch.full((nbt,), -1, dtype=torch.int32, device=dev)
        nhit = torch.zeros(nbt, dtype=torch.int32, device=dev)
        first = torch.zeros(nbt, dtype=torch.int32, device=dev)
        tr = Trace(pos.data_ptr(), tim.data_ptr(), status.data_ptr(), nhit.data_ptr(),
                   first.data_ptr(), nbt)
        t = self.tracks_struct(dev_tracks, track_base)
        _check(lib().cher_trace_bunches(self._h, ctypes.byref(t), ctypes.c_uint64(seed),
                                        int(precision), bunch_off.data_ptr(), ctypes.byref(tr),
                                        ctypes.c_void_p(_stream_ptr(stream))),
               "cher_trace_bunches")
        return dict(pos=pos, tim=tim, status=status, nhit=nhit, first_hit=first)

    def graph(self, dev_tracks: dict, seed: int, precision: int, out: HitBuffers,
              track_base: int = 0) -> "Graph":
        """Capture one generate_propagate call into a CUDA graph."""
        t = self.tracks_struct(dev_tracks, track_base)
        o = out.struct()
        h = ctypes.c_void_p()
        _check(lib().cher_graph_create(self._h, ctypes.byref(t), ctypes.c_uint64(seed),
                                       int(precision), ctypes.byref(o), ctypes.byref(h)),
               "cher_graph_create")
        return Graph(h, (dev_tracks, out))

    def generate_steps(self, showers, seed: int, precision: int, device="cuda", stream=None,
                       out=None):
        """Device step arrays of parameterised showers (cher_generate_steps):
        `showers` is a sequence of dicts with e0_mev, zenith, azimuth,
        core_x, core_y, n.  Returns the dict generate_propagate takes; `out`,
        a dict returned by an earlier call with the same total step count,
        shower count and precision, is written again instead of allocating."""
        torch = _torch()
        arr = (Shower * len(showers))()
        for k, s in enumerate(showers):
            arr[k] = Shower(float(s["e0_mev"]), float(s["zenith"]), float(s["azimuth"]),
                            float(s["core_x"]), float(s["core_y"]), int(s["n"]))
        n = sum(max(int(s["n"]), 0) for s in showers)    # (a negative count: EINVAL below)
        ddt = torch.float32 if precision == CHER_FP32_BULK else torch.float64
        if out is not None:
            # every array the kernel writes: size, dtype, contiguity, device
            want = {k: (n, torch.float64) for k in ("x0", "y0", "z0", "t0", "len", "ekin")}
            want.update({k: (n, ddt) for k in ("ux", "uy", "uz")})
            want["shower"] = (n, torch.int32)
            want["t_ref"] = (len(showers), torch.float64)
            cur = torch.device("cuda", torch.cuda.current_device())
            for k, (cnt, dt) in want.items():
                v = out.get(k) if isinstance(out, dict) else None
                if (v is None or not isinstance(v, torch.Tensor) or v.numel() != cnt
                        or v.dtype != dt or not v.is_contiguous() or v.device != cur):
                    raise ValueError(f"generate_steps: out[{k!r}] must be a contiguous {dt} "
                                     f"tensor of {cnt} elements on {cur}")
        else:
            out = {k: torch.empty(n, dtype=torch.float64, device=device)
                   for k in ("x0", "y0", "z0", "t0", "len", "ekin")}
            for k in ("ux", "uy", "uz"):
                out[k] = torch.empty(n, dtype=ddt, device=device)
            out["shower"] = torch.empty(n, dtype=torch.int32, device=device)
            out["t_ref"] = torch.empty(len(showers), dtype=torch.float64, device=device)
        B = StepBuffers(*[out[k].data_ptr() for k in ("x0", "y0", "z0", "t0", "len", "ekin", "ux",
                                                     "uy", "uz", "shower", "t_ref")])
        _check(lib().cher_generate_steps(self._h, arr, len(showers), ctypes.c_uint64(seed),
                                         int(precision), ctypes.byref(B),
                                         ctypes.c_void_p(_stream_ptr(stream))),
               "cher_generate_steps")
        return out

    def set_fallback(self, zenith_max_deg: float, queue_records: int = 0):
        """Propagate bunches past the tables' zenith range, up to this
        zenith, by the ray integrals (0: off); queue_records bunches per call
        (0: max(2^20, 4 x steps))."""
        _check(lib().cher_set_fallback(self._h, float(zenith_max_deg), int(queue_records)),
               "cher_set_fallback")

    def set_transmission(self, table: dict | None):
        """Atmospheric transmission: dict(tau=(n_lambda, n_height) vertical
        optical depths, lambda_nm=(first, last node), height_m=(first, last
        node)), or None to remove it."""
        if table is None:
            _check(lib().cher_set_transmission(self._h, None), "cher_set_transmission")
            return
        tau = np.ascontiguousarray(np.asarray(table["tau"], dtype=np.float64))
        if tau.ndim != 2:
            raise ValueError("tau must be 2-D")
        T = Transmission(int(tau.shape[0]), int(tau.shape[1]), float(table["lambda_nm"][0]),
                         float(table["lambda_nm"][1]), float(table["height_m"][0]),
                         float(table["height_m"][1]),
                         tau.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        _check(lib().cher_set_transmission(self._h, ctypes.byref(T)), "cher_set_transmission")

    def set_dispersion(self, kappa):
        """Wavelength-dependent index: kappa at 2..9 nodes uniform in
        1/lambda from the band's short end, n(h, lambda) - 1 = (n(h) - 1)
        kappa; None turns it off."""
        if kappa is None:
            _check(lib().cher_set_dispersion(self._h, None, 0), "cher_set_dispersion")
            return
        k = np.ascontiguousarray(np.asarray(kappa, dtype=np.float64).ravel())
        _check(lib().cher_set_dispersion(self._h, k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         int(k.size)), "cher_set_dispersion")

    def pack_records(self, out: "HitBuffers", dst: dict | None = None, stream=None):
        """Every telescope's records packed contiguously on the device:
        dict(pos, tim, key, offset) with offset[k] the first record of
        telescope k and offset[n_tel] the total.  `dst` (the same keys,
        preallocated) is reused when given; records past its room are not
        copied (offset[n_tel] still tells the total)."""
        torch = _torch()
        dev = out.pos.device
        if dst is None:
            total = int(torch.clamp(out.count, max=out.cap).sum().item())
            dt = out.pos.dtype
            dst = dict(pos=torch.empty((total, 4), dtype=dt, device=dev),
                       tim=torch.empty((total, 4), dtype=dt, device=dev),
                       key=torch.empty(total, dtype=torch.int64, device=dev),
                       offset=torch.empty(self.n_tel + 1, dtype=torch.int64, device=dev))
        o = out.struct()
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        _check(lib().cher_pack_records(self._h, ctypes.byref(o), int(out.precision),
                                       int(dst["key"].shape[0]), dst["pos"].data_ptr(),
                                       dst["tim"].data_ptr(), dst["key"].data_ptr(),
                                       dst["offset"].data_ptr(), ctypes.c_void_p(st.cuda_stream)),
               "cher_pack_records")
        return dst

    def set_curved(self, earth_radius_m: float):
        """Curved atmosphere with this Earth radius (m); 0 for flat layers."""
        _check(lib().cher_set_curved(self._h, float(earth_radius_m)), "cher_set_curved")

    def set_atmosphere(self, atm: dict):
        A = atmosphere_struct(atm)
        _check(lib().cher_set_atmosphere(self._h, ctypes.byref(A)), "cher_set_atmosphere")

    def density(self, dev_tracks: dict, seed: int, precision: int, sigma: float = 1.0,
                nb_frozen=None, stream=None, track_base: int = 0):
        """Smoothed photon density D_k and mean arrival time Tbar_k (device f64)."""
        torch = _torch()
        dev = dev_tracks["x0"].device
        D = torch.zeros(self.n_tel, dtype=torch.float64, device=dev)
        T = torch.zeros(self.n_tel, dtype=torch.float64, device=dev)
        t = self.tracks_struct(dev_tracks, track_base)
        _check(lib().cher_density(self._h, ctypes.byref(t), ctypes.c_uint64(seed), int(precision),
                                  float(sigma),
                                  nb_frozen.data_ptr() if nb_frozen is not None else None,
                                  D.data_ptr(), T.data_ptr(),
                                  ctypes.c_void_p(_stream_ptr(stream))), "cher_density")
        return D, T

    def adjoint(self, dev_tracks: dict, seed: int, precision: int, dL_dD, dL_dT,
                sigma: float = 1.0, nb_frozen=None, stream=None, track_base: int = 0):
        """Gradients of sum dL_dD D + dL_dT Tbar: (15,) atmosphere, (6, n) steps."""
        torch = _torch()
        dev = dev_tracks["x0"].device
        n = int(dev_tracks["x0"].numel())
        ga = torch.zeros(15, dtype=torch.float64, device=dev)
        gt = torch.zeros((6, n), dtype=torch.float64, device=dev)
        gD = torch.as_tensor(dL_dD, dtype=torch.float64, device=dev).contiguous()
        gT = torch.as_tensor(dL_dT, dtype=torch.float64, device=dev).contiguous()
        t = self.tracks_struct(dev_tracks, track_base)
        _check(lib().cher_adjoint(self._h, ctypes.byref(t), ctypes.c_uint64(seed), int(precision),
                                  float(sigma),
                                  nb_frozen.data_ptr() if nb_frozen is not None else None,
                                  gD.data_ptr(), gT.data_ptr(), ga.data_ptr(), gt.data_ptr(),
                                  ctypes.c_void_p(_stream_ptr(stream))), "cher_adjoint")
        return ga, gt

    def autotune(self, dev_tracks: dict, seed: int, precision: int, out: HitBuffers,
                 cache_path: str | None = None, stream=None):
        t = self.tracks_struct(dev_tracks)
        o = out.struct()
        _check(lib().cher_autotune(self._h, ctypes.byref(t), ctypes.c_uint64(seed),
                                   int(precision), ctypes.byref(o),
                                   cache_path.encode() if cache_path else None,
                                   ctypes.c_void_p(_stream_ptr(stream))), "cher_autotune")
        return self.get_launch()


def round_to_float(x):
    """The FP32 path's double -> float rounding applied to a device float64
    tensor (cher_round_to_float)."""
    torch = _torch()
    x = x.contiguous()
    if x.dtype != torch.float64 or not x.is_cuda:
        raise ValueError("a CUDA float64 tensor is needed")
    y = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    _check(lib().cher_round_to_float(x.data_ptr(), y.data_ptr(), x.numel(),
                                     ctypes.c_void_p(_stream_ptr(None))), "cher_round_to_float")
    return y


def split_to_float(x):
    """The FP32 path's float pair (hi, lo) of a device float64 tensor
    (cher_split_to_float)."""
    torch = _torch()
    x = x.contiguous()
    if x.dtype != torch.float64 or not x.is_cuda:
        raise ValueError("a CUDA float64 tensor is needed")
    hi = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    lo = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    _check(lib().cher_split_to_float(x.data_ptr(), hi.data_ptr(), lo.data_ptr(), x.numel(),
                                     ctypes.c_void_p(_stream_ptr(None))), "cher_split_to_float")
    return hi, lo


class Graph:
    """An executable CUDA graph of one generate_propagate call."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep            # the buffers the graph points into

    def launch(self, stream=None):
        _check(lib().cher_graph_launch(self._h, ctypes.c_void_p(_stream_ptr(stream))),
               "cher_graph_launch")

    def close(self):
        if self._h is not None and self._h.value:
            lib().cher_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
