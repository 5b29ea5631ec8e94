"""FP64 CPU oracle for the track x antenna radio-emission step (paper §2 flow).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this package; the product library never does.  The
arithmetic lives in ``c8r_oracle.c`` (plain C, single thread, FP64, built with
``-O2`` and no fast-math); this module only compiles it and marshals numpy arrays.

Units here are SI: metres, seconds.  Input dictionaries hold the twelve track
fields ``x0 y0 z0 x1 y1 z1 t0 t1 bx by bz q`` (times in seconds); ``tracks_from_ns``
converts the synthetic generator's nanosecond times.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "c8r_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

UNIFORM, EXPONENTIAL, EXPONENTIAL_SPHERICAL, EXPONENTIAL_RAY, RAY_LINEAR_N2 = 0, 1, 2, 3, 4
ENDPOINT, ZHS = 0, 1
MODE_NORMAL, MODE_FORCE_MIDPOINT, MODE_ZHS_EDGE_SAMPLED, MODE_ABS = 0, 1, 2, 3
DEPOSIT_BIN, DEPOSIT_LINEAR = 0, 1
FIELDS = ("x0", "y0", "z0", "x1", "y1", "z1", "t0", "t1", "bx", "by", "bz", "q")
C_LIGHT = 299792458.0


class _Tracks(ctypes.Structure):
    _fields_ = [(f, ctypes.POINTER(ctypes.c_double)) for f in FIELDS]


class _Medium(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_double), ("N0", ctypes.c_double), ("H", ctypes.c_double),
                ("R_E", ctypes.c_double), ("dn2dz", ctypes.c_double)]


def _medium_struct(medium):
    """medium dict: kind "uniform" (n), "exponential" (N0, H),
    "exponential_spherical" (N0, H, R_E), "exponential_ray" (N0, H; curved rays)
    or the pin-only "ray_linear_n2" (n at z = 0, dn2dz: n(z)^2 = n^2 + dn2dz z)."""
    kind = medium["kind"]
    k = {UNIFORM: UNIFORM, "uniform": UNIFORM, EXPONENTIAL: EXPONENTIAL, "exponential": EXPONENTIAL,
         EXPONENTIAL_SPHERICAL: EXPONENTIAL_SPHERICAL, "exponential_spherical": EXPONENTIAL_SPHERICAL,
         EXPONENTIAL_RAY: EXPONENTIAL_RAY, "exponential_ray": EXPONENTIAL_RAY,
         RAY_LINEAR_N2: RAY_LINEAR_N2, "ray_linear_n2": RAY_LINEAR_N2}[kind]
    return _Medium(k, float(medium.get("n", 1.0)), float(medium.get("N0", 0.0)), float(medium.get("H", 1.0)),
                   float(medium.get("R_E", 0.0)), float(medium.get("dn2dz", 0.0)))


class _Antennas(ctypes.Structure):
    _fields_ = [
        ("xyz", ctypes.POINTER(ctypes.c_double)),
        ("t_ref", ctypes.POINTER(ctypes.c_double)),
        ("n_ant", ctypes.c_int),
        ("n_bins", ctypes.c_int),
        ("dt", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math) into oracle/_build/."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _LIB_PATH + f".{os.getpid()}.tmp"
            subprocess.check_call(
                ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
                 "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        lib.oracle_forward.restype = ctypes.c_int64
        lib.oracle_forward.argtypes = [P(_Tracks), ctypes.c_int64, P(_Antennas), P(_Medium), ctypes.c_int,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int, P(ctypes.c_double)]
        lib.oracle_arrivals.restype = None
        lib.oracle_arrivals.argtypes = [P(_Tracks), ctypes.c_int64, P(_Antennas), P(_Medium), ctypes.c_int,
                                        ctypes.c_double, P(ctypes.c_int32), P(ctypes.c_double)]
        lib.oracle_backward.restype = None
        lib.oracle_backward.argtypes = [P(_Tracks), ctypes.c_int64, P(_Antennas), P(_Medium), ctypes.c_double,
                                        ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                                        P(ctypes.c_double)]
        lib.oracle_backward_zhs.restype = None
        lib.oracle_backward_zhs.argtypes = [P(_Tracks), ctypes.c_int64, P(_Antennas), P(_Medium), ctypes.c_int,
                                            P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                                            P(ctypes.c_double)]
        lib.oracle_propagate.restype = None
        lib.oracle_propagate.argtypes = [P(_Medium), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double)]
        lib.oracle_filter.restype = ctypes.c_int64
        lib.oracle_filter.argtypes = [P(_Tracks), ctypes.c_int64, P(ctypes.c_uint8)]
        _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class _Pack:
    """Holds contiguous float64 copies alive while a C call runs."""

    def __init__(self, tracks, ant_xyz, t_ref, n_bins, dt, medium):
        self.arrs = {f: np.ascontiguousarray(tracks[f], dtype=np.float64) for f in FIELDS}
        n = {len(v) for v in self.arrs.values()}
        if len(n) != 1:
            raise ValueError("track fields differ in length")
        self.n = n.pop()
        self.T = _Tracks(*[_dptr(self.arrs[f]) for f in FIELDS])
        self.xyz = np.ascontiguousarray(ant_xyz, dtype=np.float64).reshape(-1, 3)
        self.t_ref = np.ascontiguousarray(t_ref, dtype=np.float64).reshape(-1)
        if len(self.t_ref) != len(self.xyz):
            raise ValueError("antenna position / start time counts differ")
        self.A = _Antennas(_dptr(self.xyz), _dptr(self.t_ref), len(self.xyz), int(n_bins), float(dt))
        self.M = _medium_struct(medium)


def tracks_from_ns(tracks: dict) -> dict:
    """Copy of a track dict with t0/t1 converted from ns to s (float64)."""
    out = {f: np.asarray(tracks[f], dtype=np.float64) for f in FIELDS}
    out["t0"] = out["t0"] * 1e-9
    out["t1"] = out["t1"] * 1e-9
    return out


def forward(tracks, ant_xyz, t_ref, n_bins, dt, medium, formalism=ENDPOINT, eps_C=1e-3, mode=MODE_NORMAL,
            deposit=DEPOSIT_BIN):
    """Traces [n_ant, 3, n_bins] (V/m for Endpoint, V s/m for ZHS) and the kept-track count.
    deposit: DEPOSIT_BIN (each deposit in its arrival bin) or DEPOSIT_LINEAR
    (spread over one bin width centred on the arrival)."""
    lib = _load()
    p = _Pack(tracks, ant_xyz, t_ref, n_bins, dt, medium)
    out = np.zeros((len(p.xyz), 3, int(n_bins)), dtype=np.float64)
    kept = lib.oracle_forward(ctypes.byref(p.T), p.n, ctypes.byref(p.A), ctypes.byref(p.M), int(formalism),
                              float(eps_C), int(mode), int(deposit), _dptr(out))
    return out, int(kept)


def arrivals(tracks, ant_xyz, t_ref, n_bins, dt, medium, formalism=ENDPOINT, eps_C=1e-3):
    """(branch [n, n_ant] int32, u [n, n_ant, 2] float64 arrival positions in bins)."""
    lib = _load()
    p = _Pack(tracks, ant_xyz, t_ref, n_bins, dt, medium)
    br = np.zeros((p.n, len(p.xyz)), dtype=np.int32)
    u = np.zeros((p.n, len(p.xyz), 2), dtype=np.float64)
    lib.oracle_arrivals(ctypes.byref(p.T), p.n, ctypes.byref(p.A), ctypes.byref(p.M), int(formalism),
                        float(eps_C), br.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dptr(u))
    return br, u


def backward(tracks, ant_xyz, t_ref, n_bins, dt, medium, grad_traces, eps_C=1e-3, formalism=ENDPOINT,
             deposit=DEPOSIT_BIN):
    """Adjoint of forward(): (track_grad [n, 11], ant_grad [n_ant, 3], dN0).
    Not defined for the spherical-Earth atmosphere."""
    lib = _load()
    p = _Pack(tracks, ant_xyz, t_ref, n_bins, dt, medium)
    if p.M.kind in (EXPONENTIAL_SPHERICAL, EXPONENTIAL_RAY, RAY_LINEAR_N2):
        raise ValueError("the adjoint is not defined for the spherical-Earth atmosphere or curved rays")
    G = np.ascontiguousarray(grad_traces, dtype=np.float64)
    if G.shape != (len(p.xyz), 3, int(n_bins)):
        raise ValueError("grad_traces shape")
    tg = np.zeros((p.n, 11), dtype=np.float64)
    ag = np.zeros((len(p.xyz), 3), dtype=np.float64)
    dn = np.zeros(1, dtype=np.float64)
    if formalism == ZHS:
        lib.oracle_backward_zhs(ctypes.byref(p.T), p.n, ctypes.byref(p.A), ctypes.byref(p.M), int(deposit), _dptr(G),
                                _dptr(tg), _dptr(ag), _dptr(dn))
    else:
        lib.oracle_backward(ctypes.byref(p.T), p.n, ctypes.byref(p.A), ctypes.byref(p.M), float(eps_C),
                            int(deposit), _dptr(G), _dptr(tg), _dptr(ag), _dptr(dn))
    return tg, ag, float(dn[0])


def _propagate(medium, x_e, x_a):
    lib = _load()
    M = _medium_struct(medium)
    xe = np.ascontiguousarray(x_e, dtype=np.float64)
    xa = np.ascontiguousarray(x_a, dtype=np.float64)
    out = np.zeros(7)
    lib.oracle_propagate(ctypes.byref(M), _dptr(xe), _dptr(xa), _dptr(out))
    return out


def propagate(medium, x_e, x_a):
    """(R, n_src, n_avg, delay_s) of the path x_e -> x_a."""
    return tuple(float(v) for v in _propagate(medium, x_e, x_a)[:4])


def emission_direction(medium, x_e, x_a):
    """Unit direction of the path at x_e (the straight direction, or the ray's
    tangent for curved rays)."""
    return _propagate(medium, x_e, x_a)[4:7].copy()


def keep_mask(tracks):
    lib = _load()
    arrs = {f: np.ascontiguousarray(tracks[f], dtype=np.float64) for f in FIELDS}
    n = len(arrs["x0"])
    T = _Tracks(*[_dptr(arrs[f]) for f in FIELDS])
    keep = np.zeros(n, dtype=np.uint8)
    lib.oracle_filter(ctypes.byref(T), n, keep.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return keep.astype(bool)
