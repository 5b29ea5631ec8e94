"""Python binding of libc8r (argument marshalling only).

The functions named ``c8r_*`` mirror the C ABI in ``include/c8r.h`` one to one:
they convert torch tensors into device pointers and a stream handle, call the
library, and raise :class:`C8RError` with the library's message when a call
returns a negative status.  Every step of the hot path runs in libc8r's CUDA
kernels; there is no other implementation behind this module, and importing it
fails loudly when the compiled library is missing.

Above the one-to-one layer sit two conveniences named after the paper's objects
(§2, §4): :class:`RadioProcess` (medium + antenna collection + formalism, receives
tracks, holds the traces) and :class:`RadioTraces`, a ``torch.autograd.Function``
whose backward is the library's hand-written adjoint of the process's formalism
(Endpoint or ZHS).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libc8r.so")

C8R_OK = 0
C8R_EINVAL, C8R_ENOMEM, C8R_ECUDA, C8R_ECANCELLED, C8R_ETOOBIG, C8R_ESTATE = -1, -2, -3, -4, -5, -6
C8R_UNIFORM, C8R_EXPONENTIAL, C8R_EXPONENTIAL_SPHERICAL, C8R_EXPONENTIAL_RAY = 0, 1, 2, 3
C8R_ENDPOINT, C8R_ZHS = 0, 1
C8R_FP64, C8R_MIXED = 0, 1
C8R_F32, C8R_F64 = 0, 1
C8R_DEPOSIT_BIN, C8R_DEPOSIT_LINEAR = 0, 1
C8R_FORM_AUTO, C8R_FORM_SPLIT, C8R_FORM_DIRECT = 0, 1, 2

TRACK_FIELDS = ("x0", "y0", "z0", "x1", "y1", "z1", "t0", "t1", "bx", "by", "bz", "q")
GRAD_FIELDS = TRACK_FIELDS[:-1]


class C8RError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libc8r error {code}: {msg}")
        self.code = code


class c8r_tracks(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32)] + [(f, ctypes.c_void_p) for f in TRACK_FIELDS]


class c8r_track_grads(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32)] + [(f, ctypes.c_void_p) for f in GRAD_FIELDS]


class c8r_stats_t(ctypes.Structure):
    _fields_ = [("tracks_pushed", ctypes.c_int64), ("tracks_kept", ctypes.c_int64), ("pairs", ctypes.c_int64),
                ("arrival_form", ctypes.c_int64)]


class c8r_batch_desc(ctypes.Structure):
    _fields_ = [
        ("n_showers", ctypes.c_int32),
        ("n_tracks", ctypes.POINTER(ctypes.c_int64)),
        ("track_offset", ctypes.POINTER(ctypes.c_int64)),
        ("n_ant", ctypes.POINTER(ctypes.c_int32)),
        ("ant_offset", ctypes.POINTER(ctypes.c_int32)),
        ("pos_xyz", ctypes.POINTER(ctypes.c_double)),
        ("t_start_ns", ctypes.POINTER(ctypes.c_double)),
        ("n_bins", ctypes.c_int32),
        ("dt_ns", ctypes.c_double),
        ("formalism", ctypes.c_int32),
    ]


_lib = None

# (name, restype, argtypes) of every exported entry point
_P = ctypes.c_void_p
_SIGNATURES = [
    ("c8r_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int]),
    ("c8r_destroy", None, [_P]),
    ("c8r_last_error", ctypes.c_char_p, [_P]),
    ("c8r_set_medium", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
    ("c8r_set_medium_spherical", ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    ("c8r_set_antennas", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int]),
    ("c8r_set_cherenkov_threshold", ctypes.c_int, [_P, ctypes.c_double]),
    ("c8r_set_deposit", ctypes.c_int, [_P, ctypes.c_int]),
    ("c8r_set_launch_shape", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int64]),
    ("c8r_set_arrival_form", ctypes.c_int, [_P, ctypes.c_int]),
    ("c8r_push_tracks", ctypes.c_int, [_P, ctypes.POINTER(c8r_tracks), ctypes.c_int64, _P]),
    ("c8r_fetch_traces", ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, _P]),
    ("c8r_reset", ctypes.c_int, [_P, _P]),
    ("c8r_backward", ctypes.c_int, [_P, ctypes.POINTER(c8r_tracks), ctypes.c_int64, _P,
                                    ctypes.POINTER(c8r_track_grads), _P, _P, _P]),
    ("c8r_stats", ctypes.c_int, [_P, ctypes.POINTER(c8r_stats_t)]),
    ("c8r_profile", ctypes.c_int, [_P, ctypes.c_int]),
    ("c8r_profile_read", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    ("c8r_arrivals", ctypes.c_int, [_P, ctypes.POINTER(c8r_tracks), ctypes.c_int64, _P, _P, _P, _P]),
    ("c8r_batch_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(c8r_batch_desc),
                                        ctypes.c_int, ctypes.c_double, ctypes.c_double]),
    ("c8r_batch_destroy", None, [_P]),
    ("c8r_batch_last_error", ctypes.c_char_p, [_P]),
    ("c8r_batch_run", ctypes.c_int, [_P, ctypes.POINTER(c8r_tracks), _P, ctypes.c_int, _P]),
    ("c8r_batch_set_cancel", ctypes.c_int, [_P, ctypes.c_int]),
    ("c8r_batch_sync", ctypes.c_int, [_P, _P]),
    ("c8r_measure_peaks", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    ("c8r_generate_tracks", ctypes.c_int, [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                           ctypes.POINTER(c8r_tracks), _P]),
    ("c8r_traces_noalloc", ctypes.c_int, [ctypes.POINTER(c8r_tracks), ctypes.c_int64, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_int32, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_double, _P, _P]),
    ("c8r_set_wait_limit", ctypes.c_int, [ctypes.c_int64]),
    ("c8r_inject_alloc_failures", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32]),
]


def load(path: str | None = None):
    """Load libc8r (built by ``paper_2309_03717_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libc8r is not built ({p} missing); run paper_2309_03717_gb300.build.build() first")
    lib = ctypes.CDLL(p)
    for name, res, args in _SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_names():
    return [s[0] for s in _SIGNATURES]


def _check(ctx, rc):
    if rc < 0:
        msg = load().c8r_last_error(ctx)
        raise C8RError(rc, msg.decode() if msg else "")
    return rc


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def tracks_struct(tracks: dict) -> c8r_tracks:
    """c8r_tracks over a dict of 12 contiguous CUDA tensors of one dtype (float32/float64)."""
    ts = [tracks[f] for f in TRACK_FIELDS]
    dt = ts[0].dtype
    n = ts[0].numel()
    for t in ts:
        if t.dtype != dt or t.numel() != n or not t.is_cuda or not t.is_contiguous():
            raise ValueError("track fields must be contiguous CUDA tensors of one dtype and length")
    if dt not in (torch.float32, torch.float64):
        raise ValueError("track dtype must be float32 or float64")
    s = c8r_tracks()
    s.dtype = C8R_F64 if dt == torch.float64 else C8R_F32
    for f, t in zip(TRACK_FIELDS, ts):
        setattr(s, f, t.data_ptr())
    return s


# ---------------------------------------------------------------------------
# one-to-one layer
# ---------------------------------------------------------------------------
def c8r_create(device: int = 0):
    lib = load()
    h = ctypes.c_void_p()
    rc = lib.c8r_create(ctypes.byref(h), int(device))
    if rc < 0:
        raise C8RError(rc, lib.c8r_last_error(None).decode())
    return h


def c8r_destroy(ctx):
    load().c8r_destroy(ctx)


def c8r_last_error(ctx):
    m = load().c8r_last_error(ctx)
    return m.decode() if m else ""


def c8r_set_medium(ctx, kind, n_or_N0, scale_height_m=1.0):
    return _check(ctx, load().c8r_set_medium(ctx, int(kind), float(n_or_N0), float(scale_height_m)))


def c8r_set_medium_spherical(ctx, N0, scale_height_m, earth_radius_m):
    return _check(ctx, load().c8r_set_medium_spherical(ctx, float(N0), float(scale_height_m), float(earth_radius_m)))


def c8r_set_antennas(ctx, pos_xyz, t_start_ns, n_bins, dt_ns, formalism, precision):
    pos = np.ascontiguousarray(pos_xyz, dtype=np.float64).reshape(-1, 3)
    ts = np.ascontiguousarray(t_start_ns, dtype=np.float64).reshape(-1)
    if len(ts) != len(pos):
        raise ValueError("pos_xyz and t_start_ns differ in length")
    dp = ctypes.POINTER(ctypes.c_double)
    return _check(ctx, load().c8r_set_antennas(ctx, len(pos), pos.ctypes.data_as(dp), ts.ctypes.data_as(dp),
                                               int(n_bins), float(dt_ns), int(formalism), int(precision)))


def c8r_set_cherenkov_threshold(ctx, eps_C):
    return _check(ctx, load().c8r_set_cherenkov_threshold(ctx, float(eps_C)))


def c8r_set_deposit(ctx, deposit):
    return _check(ctx, load().c8r_set_deposit(ctx, int(deposit)))


def c8r_set_launch_shape(ctx, a_tile=0, waves=0, chunk_tracks=0):
    return _check(ctx, load().c8r_set_launch_shape(ctx, int(a_tile), int(waves), int(chunk_tracks)))


def c8r_set_arrival_form(ctx, form):
    return _check(ctx, load().c8r_set_arrival_form(ctx, int(form)))


def c8r_push_tracks(ctx, tracks: dict, stream=None):
    s = tracks_struct(tracks)
    n = tracks["x0"].numel()
    return _check(ctx, load().c8r_push_tracks(ctx, ctypes.byref(s), n, _stream(stream)))


def c8r_fetch_traces(ctx, dst: torch.Tensor, reset=False, stream=None):
    if not dst.is_contiguous():
        raise ValueError("dst must be contiguous")
    return _check(ctx, load().c8r_fetch_traces(ctx, _ptr(dst), 1 if dst.is_cuda else 0, 1 if reset else 0,
                                               _stream(stream)))


def c8r_reset(ctx, stream=None):
    return _check(ctx, load().c8r_reset(ctx, _stream(stream)))


def c8r_stats(ctx):
    st = c8r_stats_t()
    _check(ctx, load().c8r_stats(ctx, ctypes.byref(st)))
    return {"tracks_pushed": st.tracks_pushed, "tracks_kept": st.tracks_kept, "pairs": st.pairs,
            "arrival_form": {C8R_FORM_SPLIT: "split", C8R_FORM_DIRECT: "direct"}.get(st.arrival_form, "?")}


def c8r_profile(ctx, enable=True):
    return _check(ctx, load().c8r_profile(ctx, 1 if enable else 0))


def c8r_profile_read(ctx):
    pm, im = ctypes.c_double(), ctypes.c_double()
    pl, il = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, load().c8r_profile_read(ctx, ctypes.byref(pm), ctypes.byref(pl), ctypes.byref(im), ctypes.byref(il)))
    return {"pair_ms": pm.value, "pair_launches": pl.value, "ingest_ms": im.value, "ingest_launches": il.value}


def c8r_arrivals(ctx, tracks: dict, n_ant: int, stream=None):
    """(branch [n, n_ant] int32, bin [n, n_ant, 2] int32, frac [n, n_ant, 2] float32) on the device."""
    s = tracks_struct(tracks)
    n = tracks["x0"].numel()
    dev = tracks["x0"].device
    br = torch.empty((n, n_ant), dtype=torch.int32, device=dev)
    b = torch.empty((n, n_ant, 2), dtype=torch.int32, device=dev)
    fr = torch.empty((n, n_ant, 2), dtype=torch.float32, device=dev)
    _check(ctx, load().c8r_arrivals(ctx, ctypes.byref(s), n, _ptr(br), _ptr(b), _ptr(fr), _stream(stream)))
    return br, b, fr


def c8r_backward(ctx, tracks: dict, grad_traces: torch.Tensor, track_grads: dict, ant_grad: torch.Tensor,
                 dN0: torch.Tensor, stream=None):
    s = tracks_struct(tracks)
    n = tracks["x0"].numel()
    g = c8r_track_grads()
    dt = track_grads["x0"].dtype
    g.dtype = C8R_F64 if dt == torch.float64 else C8R_F32
    for f in GRAD_FIELDS:
        t = track_grads[f]
        if t.dtype != dt or t.numel() != n or not t.is_cuda or not t.is_contiguous():
            raise ValueError("gradient arrays must be contiguous CUDA tensors matching the tracks")
        setattr(g, f, t.data_ptr())
    if ant_grad.dtype != torch.float64 or dN0.dtype != torch.float64:
        raise ValueError("ant_grad and dN0 are float64")
    return _check(ctx, load().c8r_backward(ctx, ctypes.byref(s), n, _ptr(grad_traces.contiguous()),
                                           ctypes.byref(g), _ptr(ant_grad), _ptr(dN0), _stream(stream)))


def c8r_measure_peaks(device: int = 0):
    out = (ctypes.c_double * 6)()
    rc = load().c8r_measure_peaks(int(device), out)
    if rc < 0:
        raise C8RError(rc, "peaks microbenchmark failed")
    keys = ("ffma_per_s", "dfma_per_s", "rsqrt_per_s", "shared_atomic_f32_per_s", "shared_atomic_f64_per_s",
            "global_red_f32x4_per_s")
    return dict(zip(keys, list(out)))


def c8r_generate_tracks(seed: int, first: int, n: int, zenith_deg: float = 0.0, stream=None, device=None):
    """Tracks first .. first+n-1 of the counter-based synthetic shower `seed`,
    generated on the device: a dict of FP32 CUDA tensors (the host twin is
    synth.make_tracks_counter)."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    out = {f: torch.empty(int(n), dtype=torch.float32, device=dev) for f in TRACK_FIELDS}
    s = c8r_tracks(C8R_F32, *[_ptr(out[f]) for f in TRACK_FIELDS])  # same layout as c8r_tracks_out
    rc = load().c8r_generate_tracks(int(seed), int(first), int(n), float(zenith_deg), ctypes.byref(s), _stream(stream))
    if rc < 0:
        raise C8RError(rc, "c8r_generate_tracks failed")
    return out


def c8r_set_wait_limit(polls: int):
    """Polls of every bounded wait on a staged track tile (< 0: the default;
    0: give up at once).  Process-wide test knob."""
    return _check(None, load().c8r_set_wait_limit(int(polls)))


def c8r_inject_alloc_failures(skip: int, n: int):
    """Of the library's next device allocations let ``skip`` through and make
    the following ``n`` fail (ENOMEM).  Process-wide test knob."""
    rc = load().c8r_inject_alloc_failures(int(skip), int(n))
    if rc < 0:
        raise C8RError(rc, "skip and n must be >= 0")
    return rc


# ---------------------------------------------------------------------------
# paper-level convenience objects
# ---------------------------------------------------------------------------
_MEDIUM = {"uniform": C8R_UNIFORM, "exponential": C8R_EXPONENTIAL, "exponential_spherical": C8R_EXPONENTIAL_SPHERICAL,
           "exponential_ray": C8R_EXPONENTIAL_RAY}
_FORMALISM = {"endpoint": C8R_ENDPOINT, "coreas": C8R_ENDPOINT, "zhs": C8R_ZHS}
_PRECISION = {"fp64": C8R_FP64, "mixed": C8R_MIXED}
_DEPOSIT = {"bin": C8R_DEPOSIT_BIN, "linear": C8R_DEPOSIT_LINEAR}
_FORM = {"auto": C8R_FORM_AUTO, "split": C8R_FORM_SPLIT, "direct": C8R_FORM_DIRECT}


class RadioProcess:
    """One radio process (§2): a medium for the straight-line propagator, an
    antenna collection and one formalism.  ``push`` hands it tracks; ``traces``
    returns the accumulated [n_ant, 3, n_bins] traces (float64 for precision
    'fp64', float32 for 'mixed').  ``deposit`` is 'bin' (each deposit in its
    arrival bin) or 'linear' (spread over one bin width centred on the arrival)."""

    def __init__(self, medium: dict, ant_xyz, t_start_ns, n_bins: int, dt_ns: float, formalism="endpoint",
                 precision="mixed", device: int | None = None, eps_C: float | None = None, deposit="bin"):
        if device is None:
            device = torch.cuda.current_device()
        self.device = torch.device("cuda", device)
        self.ctx = c8r_create(device)
        self.ant_xyz = np.array(ant_xyz, dtype=np.float64).reshape(-1, 3)
        self.t_start_ns = np.array(t_start_ns, dtype=np.float64).reshape(-1)
        self.n_ant = int(self.ant_xyz.shape[0])
        self.n_bins = int(n_bins)
        self.dt_ns = float(dt_ns)
        self.precision = precision
        self.formalism = formalism
        self.medium = dict(medium)
        self._apply_medium()
        c8r_set_antennas(self.ctx, self.ant_xyz, self.t_start_ns, n_bins, dt_ns, _FORMALISM[formalism],
                         _PRECISION[precision])
        if eps_C is not None:
            c8r_set_cherenkov_threshold(self.ctx, eps_C)
        c8r_set_deposit(self.ctx, _DEPOSIT[deposit])
        self.deposit = deposit

    def _apply_medium(self):
        m = self.medium
        kind = _MEDIUM[m["kind"]]
        if kind == C8R_UNIFORM:
            c8r_set_medium(self.ctx, kind, m["n"], 1.0)
        elif kind == C8R_EXPONENTIAL_SPHERICAL:
            c8r_set_medium_spherical(self.ctx, m["N0"], m["H"], m["R_E"])
        else:
            c8r_set_medium(self.ctx, kind, m["N0"], m["H"])

    @property
    def refractivity(self) -> float:
        """N0 of an exponential medium, n - 1 of a uniform one."""
        m = self.medium
        return float(m["n"]) - 1.0 if m["kind"] == "uniform" else float(m["N0"])

    def set_refractivity(self, value: float):
        """Set N0 (exponential media) or n - 1 (uniform medium); traces are kept."""
        value = float(value)
        if value == self.refractivity:
            return
        if self.medium["kind"] == "uniform":
            self.medium["n"] = 1.0 + value
        else:
            self.medium["N0"] = value
        self._apply_medium()

    def set_antenna_positions(self, ant_xyz):
        """Move the antennas (same count; each keeps its trace start time).  The
        accumulated traces are discarded."""
        pos = np.array(ant_xyz, dtype=np.float64).reshape(-1, 3)
        if pos.shape != self.ant_xyz.shape:
            raise ValueError("antenna count differs from the process's")
        if np.array_equal(pos, self.ant_xyz):
            return
        c8r_set_antennas(self.ctx, pos, self.t_start_ns, self.n_bins, self.dt_ns, _FORMALISM[self.formalism],
                         _PRECISION[self.precision])
        self.ant_xyz = pos

    @property
    def trace_dtype(self):
        return torch.float64 if self.precision == "fp64" else torch.float32

    def set_launch_shape(self, a_tile=0, waves=0, chunk_tracks=0):
        c8r_set_launch_shape(self.ctx, a_tile, waves, chunk_tracks)

    def set_arrival_form(self, form="auto"):
        """Pin ("split", "direct") or free ("auto") the form of the FP32 arrival
        of the mixed one-bin Endpoint kernels; the bins are the same either way."""
        c8r_set_arrival_form(self.ctx, _FORM[form])

    def push(self, tracks: dict, stream=None):
        c8r_push_tracks(self.ctx, tracks, stream)

    def traces(self, reset=False, stream=None, out=None):
        if out is None:
            out = torch.empty((self.n_ant, 3, self.n_bins), dtype=self.trace_dtype, device=self.device)
        c8r_fetch_traces(self.ctx, out, reset=reset, stream=stream)
        return out

    def reset(self, stream=None):
        c8r_reset(self.ctx, stream)

    def stats(self):
        return c8r_stats(self.ctx)

    def arrivals(self, tracks: dict, stream=None):
        return c8r_arrivals(self.ctx, tracks, self.n_ant, stream)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            c8r_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RadioTraces(torch.autograd.Function):
    """traces = RadioTraces.apply(process, N0, *track_tensors, ant_xyz_tensor)

    A function of all its tensor inputs: forward first configures ``process``
    with the values of N0 (a 0-d tensor: the refractivity N0 of an exponential
    medium, n - 1 of a uniform one) and of the antenna positions [n_ant, 3] (the
    library is reconfigured only when they changed), then pushes the tracks
    (reset first) and returns the traces.  Backward runs the library's adjoint
    of the process's formalism (Endpoint or ZHS) and returns gradients for N0,
    the twelve track tensors (zero for q) and the antenna positions."""

    @staticmethod
    def forward(ctx, process: RadioProcess, N0, *args):
        tracks = dict(zip(TRACK_FIELDS, args[:12]))
        ant = args[12]
        process.set_refractivity(float(N0.detach().cpu()))
        process.set_antenna_positions(ant.detach().cpu().numpy())
        process.reset()
        process.push(tracks)
        out = process.traces()
        ctx.process = process
        ctx.save_for_backward(*args[:12], ant, N0)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        saved = ctx.saved_tensors
        tracks = dict(zip(TRACK_FIELDS, saved[:12]))
        ant = saved[12]
        N0 = saved[13]
        process = ctx.process
        gdt = torch.float64 if process.precision == "fp64" else torch.float32
        n = tracks["x0"].numel()
        tg = {f: torch.zeros(n, dtype=gdt, device=process.device) for f in GRAD_FIELDS}
        ag = torch.zeros((process.n_ant, 3), dtype=torch.float64, device=process.device)
        dn = torch.zeros(1, dtype=torch.float64, device=process.device)
        g = grad_out.to(process.trace_dtype).contiguous()
        c8r_backward(process.ctx, tracks, g, tg, ag, dn)
        grads = [tg[f].to(tracks[f].dtype) for f in GRAD_FIELDS] + [torch.zeros_like(tracks["q"])]
        return (None, dn.reshape(()).to(N0.dtype), *grads, ag.to(ant.dtype))


class Batch:
    """Many showers of uneven size in persistent launches (c8r_batch_*; one per
    form of the Endpoint FP32 arrival that its showers take).

    showers: list of dicts with ``n_tracks``, ``ant_xyz`` [A, 3] and ``t_start_ns``
    [A]; their tracks are concatenated in order, and so are the output traces
    [sum A, 3, n_bins] (float32)."""

    def __init__(self, showers, medium: dict, n_bins: int, dt_ns: float, formalism="endpoint", device=None):
        lib = load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = torch.device("cuda", device)
        n_tracks = np.array([int(s["n_tracks"]) for s in showers], dtype=np.int64)
        n_ant = np.array([len(s["ant_xyz"]) for s in showers], dtype=np.int32)
        self.track_offset = np.concatenate([[0], np.cumsum(n_tracks)[:-1]]).astype(np.int64)
        self.ant_offset = np.concatenate([[0], np.cumsum(n_ant)[:-1]]).astype(np.int32)
        pos = np.ascontiguousarray(np.concatenate([np.asarray(s["ant_xyz"], np.float64) for s in showers]))
        ts = np.ascontiguousarray(np.concatenate([np.asarray(s["t_start_ns"], np.float64) for s in showers]))
        self._keep = (n_tracks, n_ant, pos, ts)
        d = c8r_batch_desc()
        d.n_showers = len(showers)
        d.n_tracks = n_tracks.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        d.track_offset = self.track_offset.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        d.n_ant = n_ant.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.ant_offset = self.ant_offset.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.pos_xyz = pos.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.t_start_ns = ts.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.n_bins = int(n_bins)
        d.dt_ns = float(dt_ns)
        d.formalism = _FORMALISM[formalism]
        kind = _MEDIUM[medium["kind"]]
        a = medium["n"] if kind == C8R_UNIFORM else medium["N0"]
        H = 1.0 if kind == C8R_UNIFORM else medium["H"]
        h = ctypes.c_void_p()
        rc = lib.c8r_batch_create(ctypes.byref(h), int(device), ctypes.byref(d), kind, float(a), float(H))
        self.h = h
        if rc < 0:
            msg = lib.c8r_batch_last_error(h).decode() if h.value else "batch creation failed"
            self.close()
            raise C8RError(rc, msg)
        self.n_ant_total = int(n_ant.sum())
        self.n_bins = int(n_bins)

    def _check(self, rc):
        if rc < 0:
            raise C8RError(rc, load().c8r_batch_last_error(self.h).decode())
        return rc

    def run(self, tracks: dict, out: torch.Tensor, use_graph=True, stream=None):
        s = tracks_struct(tracks)
        if out.dtype != torch.float32 or not out.is_cuda or not out.is_contiguous():
            raise ValueError("out must be a contiguous float32 CUDA tensor")
        return self._check(load().c8r_batch_run(self.h, ctypes.byref(s), _ptr(out), 1 if use_graph else 0,
                                                _stream(stream)))

    def set_cancel(self, value: bool):
        return self._check(load().c8r_batch_set_cancel(self.h, 1 if value else 0))

    def sync(self, stream=None):
        return self._check(load().c8r_batch_sync(self.h, _stream(stream)))

    def new_output(self):
        return torch.zeros((self.n_ant_total, 3, self.n_bins), dtype=torch.float32, device=self.device)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().c8r_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
