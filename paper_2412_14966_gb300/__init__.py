"""GB300-native primary-vertex finding and fitting (arXiv:2412.14966, Sec. 3).

Thin Python binding of ``libpvgb300.so`` (the C ABI of ``include/pv.h``).
Every step of the method runs in the library's CUDA kernels; this module only
marshals arguments (torch tensors for device memory and streams, numpy for
host buffers).  It never computes a result itself and has no CPU fallback: if
the library is missing it raises ``LibraryMissing``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpvgb300.so")

TRACK_FIELDS = ("x", "y", "z", "tx", "ty", "cxx", "cxtx", "ctxtx", "cyy", "cyty", "ctyty")

# include/pv.h constants
PV_OK, PV_ERR_ARG, PV_ERR_CUDA, PV_ERR_CAPACITY, PV_ERR_NOMEM = 0, 1, 2, 3, 4
PV_ERR_TIMEOUT, PV_ERR_BUSY, PV_ERR_NOTFOUND = 5, 6, 7
ST_CONVERGED, ST_MAXITER, ST_SINGULAR, ST_REJ_BEAM, ST_REJ_NTRK, ST_ACCEPTED = 1, 2, 4, 8, 16, 32
ST_DUPLICATE = 64
EV_SEED_OVERFLOW, EV_BAD_OFFSETS = 1, 4
ONE = 4096
MAX_SEEDS = 64
ACCUM_FP32, ACCUM_KAHAN, ACCUM_FP64 = 0, 1, 2
PATH_FUSED, PATH_PLAIN = 0, 1
SPLIT_ZORDER, SPLIT_RECURSIVE = 0, 1
PROFILE_CUBIC, PROFILE_TEMPLATE = 0, 1

EXPORTED = (
    "pv_config_default", "pv_init", "pv_destroy", "pv_find_batch", "pv_fit_batch",
    "pv_extrapolate_batch", "pv_histogram_batch", "pv_num_bins", "pv_run_host", "pv_submit",
    "pv_poll", "pv_request_latency_ns", "pv_strerror", "pv_last_cuda_error", "pv_launch_count",
    "pv_find_fit_static", "pv_autotune", "pv_launch_config", "pv_set_launch_config",
    "pv_fit_multi", "pv_check_report", "pv_device_bytes", "pv_serve_start", "pv_serve_status",
)


class LibraryMissing(RuntimeError):
    pass


class PVError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        msg = f"{where}: {_strerror(code)} ({code})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


class pv_config(C.Structure):
    _fields_ = [
        ("z_min", C.c_float), ("z_max", C.c_float), ("dz", C.c_float), ("z_gas", C.c_float),
        ("sigma_max_pp", C.c_float), ("sigma_max_gas", C.c_float),
        ("min_integral_pp", C.c_float), ("min_integral_gas", C.c_float),
        ("bin_threshold", C.c_uint32), ("dip_num", C.c_int32), ("dip_den", C.c_int32),
        ("min_assoc_pp", C.c_int32), ("min_assoc_gas", C.c_int32),
        ("min_pv_tracks_pp", C.c_int32), ("min_pv_tracks_gas", C.c_int32),
        ("chi2_max", C.c_float), ("dchi2_tol", C.c_float), ("dz_tol", C.c_float),
        ("max_iter", C.c_int32), ("max_r_beam", C.c_float),
        ("accum_mode", C.c_int32), ("path", C.c_int32),
        ("use_graph", C.c_int32), ("reserved", C.c_int32),
        ("pool_bytes", C.c_uint64), ("max_spin_ns", C.c_uint64),
        ("mv_chi2_cut", C.c_float), ("mv_dz_tol", C.c_float), ("mv_w_assoc", C.c_float),
        ("mv_dup_sep2", C.c_float), ("split_mode", C.c_int32), ("profile_mode", C.c_int32),
    ]


class pv_beamline(C.Structure):
    _fields_ = [("x_b", C.c_float), ("y_b", C.c_float), ("tx_b", C.c_float), ("ty_b", C.c_float)]


_FP = C.c_void_p


class pv_tracks(C.Structure):
    _fields_ = [(k, _FP) for k in TRACK_FIELDS] + [
        ("event_offsets", _FP), ("n_tracks", C.c_int64), ("n_events", C.c_int32)]


VERTEX_FLOAT = ("x", "y", "z", "cov", "chi2", "ndof")
VERTEX_INT = ("n_tracks", "n_iter", "status", "bin_lo", "bin_hi", "bin_max")


class pv_vertices(C.Structure):
    _fields_ = [(k, _FP) for k in VERTEX_FLOAT + VERTEX_INT] + [
        ("n_per_event", _FP), ("event_status", _FP), ("track_vertex", _FP),
        ("capacity", C.c_int32)]


_LIB = None


def load():
    """Load libpvgb300.so (build it first with ``paper_2412_14966_gb300.build``)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise LibraryMissing(f"{LIB_PATH} not built; run `python -m paper_2412_14966_gb300.build`")
    L = C.CDLL(LIB_PATH)
    P = C.POINTER
    L.pv_config_default.argtypes = [P(pv_config)]
    L.pv_config_default.restype = None
    L.pv_init.argtypes = [P(pv_config), P(pv_beamline), C.c_int, P(C.c_void_p)]
    L.pv_destroy.argtypes = [C.c_void_p]
    L.pv_find_batch.argtypes = [C.c_void_p, P(pv_tracks), P(pv_vertices), C.c_void_p]
    L.pv_fit_batch.argtypes = [C.c_void_p, P(pv_tracks), P(pv_vertices), P(pv_vertices),
                               C.c_void_p]
    L.pv_fit_multi.argtypes = [C.c_void_p, P(pv_tracks), P(pv_vertices), P(pv_vertices),
                               C.c_void_p]
    L.pv_extrapolate_batch.argtypes = [C.c_void_p, P(pv_tracks), C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]
    L.pv_histogram_batch.argtypes = [C.c_void_p, P(pv_tracks), C.c_void_p, C.c_void_p]
    L.pv_num_bins.argtypes = [C.c_void_p]
    L.pv_check_report.argtypes = [P(C.c_uint32), P(C.c_uint32)]
    L.pv_run_host.argtypes = [C.c_void_p, P(pv_tracks), P(pv_vertices), C.c_void_p]
    L.pv_submit.argtypes = [C.c_void_p, P(pv_tracks), P(pv_vertices), P(C.c_uint64)]
    L.pv_poll.argtypes = [C.c_void_p, C.c_uint64, P(C.c_int)]
    L.pv_request_latency_ns.argtypes = [C.c_void_p, C.c_uint64, P(C.c_uint64)]
    L.pv_strerror.argtypes = [C.c_int]
    L.pv_strerror.restype = C.c_char_p
    L.pv_last_cuda_error.argtypes = [C.c_void_p]
    L.pv_last_cuda_error.restype = C.c_char_p
    L.pv_launch_count.argtypes = [C.c_void_p]
    L.pv_launch_count.restype = C.c_uint64
    L.pv_device_bytes.argtypes = [C.c_void_p]
    L.pv_device_bytes.restype = C.c_uint64
    L.pv_serve_start.argtypes = [C.c_void_p]
    L.pv_serve_status.argtypes = [C.c_void_p, P(C.c_int), P(C.c_int)]
    L.pv_find_fit_static.argtypes = [C.c_void_p, P(pv_tracks), P(pv_vertices), C.c_void_p]
    L.pv_autotune.argtypes = [C.c_void_p, P(pv_tracks), P(pv_vertices), C.c_void_p]
    L.pv_set_launch_config.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
    L.pv_launch_config.argtypes = [C.c_void_p, P(pv_tracks), P(C.c_int), P(C.c_int), P(C.c_int),
                                   P(C.c_int)]
    _LIB = L
    return L


def _strerror(code: int) -> str:
    try:
        return load().pv_strerror(code).decode()
    except LibraryMissing:
        return "error"


def default_config(**overrides) -> pv_config:
    cfg = pv_config()
    load().pv_config_default(C.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Tracks:
    """SoA tracks + CSR event offsets (torch CUDA tensors or numpy arrays)."""

    def __init__(self, cols: dict, offsets):
        self.cols = cols
        self.offsets = offsets
        self.n_tracks = int(cols["x"].shape[0])
        self.n_events = int(offsets.shape[0]) - 1

    @classmethod
    def from_batch(cls, batch, device="cuda"):
        """Copy a ``synthetic.EventBatch`` (host numpy) to the device."""
        import torch
        cols = {k: torch.from_numpy(np.ascontiguousarray(batch.tracks[k], np.float32)).to(device)
                for k in TRACK_FIELDS}
        offs = torch.from_numpy(np.ascontiguousarray(batch.offsets, np.int64)).to(device)
        return cls(cols, offs)

    @classmethod
    def from_host(cls, batch, pinned=True):
        """Host (optionally pinned) copies of a batch, for ``Context.run_host``."""
        import torch
        cols = {}
        for k in TRACK_FIELDS:
            t = torch.from_numpy(np.ascontiguousarray(batch.tracks[k], np.float32))
            cols[k] = t.pin_memory() if pinned else t
        offs = torch.from_numpy(np.ascontiguousarray(batch.offsets, np.int64))
        return cls(cols, offs.pin_memory() if pinned else offs)

    def struct(self) -> pv_tracks:
        s = pv_tracks()
        for k in TRACK_FIELDS:
            setattr(s, k, _ptr(self.cols[k]))
        s.event_offsets = _ptr(self.offsets)
        s.n_tracks = self.n_tracks
        s.n_events = self.n_events
        return s

    def nbytes(self) -> int:
        return 44 * self.n_tracks + 8 * (self.n_events + 1)


class Vertices:
    """Per-event seeds or vertices (row-major [event][capacity])."""

    def __init__(self, arrays: dict, capacity: int):
        self.a = arrays
        self.capacity = capacity

    @classmethod
    def empty(cls, n_events: int, n_tracks: int, capacity: int = MAX_SEEDS, device="cuda",
              fit: bool = True, bins: bool = True, host: bool = False, pinned: bool = False):
        import torch
        kw = dict(device="cpu" if host else device)
        shape = (max(n_events, 0), capacity)
        mk = (lambda *s, dt: torch.empty(*s, dtype=dt, **kw).pin_memory()) if (host and pinned) else \
             (lambda *s, dt: torch.empty(*s, dtype=dt, **kw))
        a = {k: mk(*shape, dt=torch.float32) for k in ("x", "y", "z")}
        if fit:
            a["cov"] = mk(*shape, 6, dt=torch.float32)
            a["chi2"] = mk(*shape, dt=torch.float32)
            a["ndof"] = mk(*shape, dt=torch.float32)
            for k in ("n_tracks", "n_iter", "status"):
                a[k] = mk(*shape, dt=torch.int32)
        if bins:
            for k in ("bin_lo", "bin_hi", "bin_max"):
                a[k] = mk(*shape, dt=torch.int32)
        a["n_per_event"] = mk(max(n_events, 0), dt=torch.int32)
        a["event_status"] = mk(max(n_events, 0), dt=torch.int32)
        a["track_vertex"] = mk(max(n_tracks, 1), dt=torch.int32)
        return cls(a, capacity)

    def struct(self) -> pv_vertices:
        s = pv_vertices()
        for k in VERTEX_FLOAT + VERTEX_INT + ("n_per_event", "event_status", "track_vertex"):
            setattr(s, k, _ptr(self.a.get(k)))
        s.capacity = self.capacity
        return s

    def __getitem__(self, k):
        return self.a[k]

    def numpy(self) -> dict:
        return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in self.a.items()}


def check_report() -> tuple:
    """``pv_check_report``: (checked build?, out-of-bounds count, first code)."""
    n, first = C.c_uint32(0), C.c_uint32(0)
    rc = load().pv_check_report(C.byref(n), C.byref(first))
    return rc == PV_OK, int(n.value), int(first.value)


class Context:
    """A library context on one CUDA device (``pv_init`` / ``pv_destroy``)."""

    def __init__(self, device: int = 0, beamline=(0.0, 0.0, 0.0, 0.0), **config):
        self.lib = load()
        self.cfg = default_config(**config)
        self.beam = pv_beamline(*[float(v) for v in beamline])
        h = C.c_void_p()
        rc = self.lib.pv_init(C.byref(self.cfg), C.byref(self.beam), int(device), C.byref(h))
        if rc != PV_OK:
            raise PVError(rc, "pv_init")
        self.h = h
        self.device = device
        self.nbins = self.lib.pv_num_bins(self.h)

    def _check(self, rc: int, where: str):
        if rc != PV_OK:
            detail = self.lib.pv_last_cuda_error(self.h).decode() if rc == PV_ERR_CUDA else ""
            raise PVError(rc, where, detail)

    def close(self):
        if getattr(self, "h", None):
            self._check(self.lib.pv_destroy(self.h), "pv_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self) -> int:
        return int(self.lib.pv_launch_count(self.h))

    def device_bytes(self) -> int:
        """``pv_device_bytes``: device memory the context holds."""
        return int(self.lib.pv_device_bytes(self.h))

    # -- device entry points --------------------------------------------------
    def find_batch(self, tracks: Tracks, out: Vertices | None = None, stream=None) -> Vertices:
        out = out or Vertices.empty(tracks.n_events, tracks.n_tracks, fit=False)
        t, o = tracks.struct(), out.struct()
        self._check(self.lib.pv_find_batch(self.h, C.byref(t), C.byref(o), _stream_handle(stream)),
                    "pv_find_batch")
        return out

    def fit_batch(self, tracks: Tracks, seeds: Vertices | None = None, out: Vertices | None = None,
                  stream=None) -> Vertices:
        out = out or Vertices.empty(tracks.n_events, tracks.n_tracks)
        t, o = tracks.struct(), out.struct()
        s = seeds.struct() if seeds is not None else None
        self._check(self.lib.pv_fit_batch(self.h, C.byref(t), C.byref(s) if s is not None else None,
                                          C.byref(o), _stream_handle(stream)), "pv_fit_batch")
        return out

    def fit_multi(self, tracks: Tracks, seeds: Vertices | None = None, out: Vertices | None = None,
                  stream=None) -> Vertices:
        """``pv_fit_multi``: the multi-vertex fit of every seed (seeds = None:
        find them first)."""
        out = out or Vertices.empty(tracks.n_events, tracks.n_tracks)
        t, o = tracks.struct(), out.struct()
        s = seeds.struct() if seeds is not None else None
        self._check(self.lib.pv_fit_multi(self.h, C.byref(t), C.byref(s) if s is not None else None,
                                          C.byref(o), _stream_handle(stream)), "pv_fit_multi")
        return out

    def extrapolate_batch(self, tracks: Tracks, stream=None):
        import torch
        n = max(tracks.n_tracks, 1)
        zp = torch.empty(n, dtype=torch.float32, device="cuda")
        sg = torch.empty(n, dtype=torch.float32, device="cuda")
        cb = torch.empty(n, dtype=torch.int32, device="cuda")
        t = tracks.struct()
        self._check(self.lib.pv_extrapolate_batch(self.h, C.byref(t), _ptr(zp), _ptr(sg), _ptr(cb),
                                                  _stream_handle(stream)), "pv_extrapolate_batch")
        return zp[:tracks.n_tracks], sg[:tracks.n_tracks], cb[:tracks.n_tracks]

    def histogram_batch(self, tracks: Tracks, stream=None):
        import torch
        h = torch.empty((max(tracks.n_events, 1), self.nbins), dtype=torch.int32, device="cuda")
        t = tracks.struct()
        self._check(self.lib.pv_histogram_batch(self.h, C.byref(t), _ptr(h), _stream_handle(stream)),
                    "pv_histogram_batch")
        return h[:tracks.n_events]

    def find_fit_static(self, tracks: Tracks, out: Vertices | None = None,
                        stream=None) -> Vertices:
        """``pv_find_fit_static``: the fused find + fit with the library's
        static device scratch instead of allocated memory, for callers that
        cannot allocate device memory while they run.  A batch needs 31 bytes
        per track plus 32 per entry of the four size-class vertex work lists
        within 8 MiB (about 165,000 tracks of 160-track events at capacity 64;
        larger batches get PV_ERR_CAPACITY); overlapping calls race (they
        share the scratch)."""
        out = out or Vertices.empty(tracks.n_events, tracks.n_tracks)
        t, o = tracks.struct(), out.struct()
        self._check(self.lib.pv_find_fit_static(self.h, C.byref(t), C.byref(o),
                                                _stream_handle(stream)), "pv_find_fit_static")
        return out

    def autotune(self, tracks: Tracks, out: Vertices | None = None, stream=None) -> tuple:
        """``pv_autotune`` on a sample batch; returns the chosen launch shape."""
        out = out or Vertices.empty(tracks.n_events, tracks.n_tracks)
        t, o = tracks.struct(), out.struct()
        self._check(self.lib.pv_autotune(self.h, C.byref(t), C.byref(o), _stream_handle(stream)),
                    "pv_autotune")
        return self.launch_config(tracks)

    def set_launch_config(self, bucket: int, find_threads: int, fit_threads: int):
        """``pv_set_launch_config``: block sizes of one event-size bucket."""
        self._check(self.lib.pv_set_launch_config(self.h, bucket, find_threads, fit_threads),
                    "pv_set_launch_config")

    def launch_config(self, tracks: Tracks) -> tuple:
        """(find threads, fit threads, find grid, fit grid) the fused path would use."""
        t = tracks.struct()
        v = [C.c_int() for _ in range(4)]
        self._check(self.lib.pv_launch_config(self.h, C.byref(t), *[C.byref(x) for x in v]),
                    "pv_launch_config")
        return tuple(x.value for x in v)

    # -- host entry point -----------------------------------------------------
    def run_host(self, tracks: Tracks, out: Vertices, stream=None) -> Vertices:
        t, o = tracks.struct(), out.struct()
        self._check(self.lib.pv_run_host(self.h, C.byref(t), C.byref(o), _stream_handle(stream)),
                    "pv_run_host")
        return out

    # -- serving ----------------------------------------------------------------
    def submit(self, tracks: Tracks, out: Vertices) -> int:
        t, o = tracks.struct(), out.struct()
        ticket = C.c_uint64()
        self._check(self.lib.pv_submit(self.h, C.byref(t), C.byref(o), C.byref(ticket)), "pv_submit")
        return int(ticket.value)

    def submit_nowait(self, tracks: Tracks, out: Vertices):
        """Like submit, but returns (code, ticket) instead of raising on BUSY."""
        t, o = tracks.struct(), out.struct()
        ticket = C.c_uint64()
        rc = self.lib.pv_submit(self.h, C.byref(t), C.byref(o), C.byref(ticket))
        if rc not in (PV_OK, PV_ERR_BUSY):
            self._check(rc, "pv_submit")
        return rc, int(ticket.value)

    def poll(self, ticket: int) -> bool:
        done = C.c_int()
        self._check(self.lib.pv_poll(self.h, C.c_uint64(ticket), C.byref(done)), "pv_poll")
        return bool(done.value)

    def serve_start(self):
        """``pv_serve_start``: start the serving kernel now."""
        self._check(self.lib.pv_serve_start(self.h), "pv_serve_start")

    def serve_status(self) -> tuple:
        """``pv_serve_status``: (running, last exit code)."""
        r, x = C.c_int(0), C.c_int(0)
        self._check(self.lib.pv_serve_status(self.h, C.byref(r), C.byref(x)), "pv_serve_status")
        return bool(r.value), int(x.value)

    def latency_ns(self, ticket: int) -> int:
        ns = C.c_uint64()
        self._check(self.lib.pv_request_latency_ns(self.h, C.c_uint64(ticket), C.byref(ns)),
                    "pv_request_latency_ns")
        return int(ns.value)
