"""CPU oracle for primary-vertex finding and fitting (arXiv:2412.14966, Sec. 3).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may import this package.  The product path (the CUDA
library and its binding) never imports it and shares no code with it.

The arithmetic lives in ``pv_oracle.c`` (plain C, built with gcc,
``-ffp-contract=off``); this module compiles it on first use and marshals numpy
arrays through ctypes.  ``default_params()`` holds the paper's constants,
each with the passage it comes from.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pv_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

ONE = 4096  # histogram weight of one track (reading R3 in pv_oracle.c)

CONVERGED, MAXITER, SINGULAR, REJ_BEAM, REJ_NTRK, ACCEPTED = 1, 2, 4, 8, 16, 32
DUPLICATE = 64   # multi-vertex fit: rejected as a duplicate (reading R15)
EV_SEED_OVERFLOW = 1

TRACK_FIELDS = ("x", "y", "z", "tx", "ty", "cxx", "cxtx", "ctxtx", "cyy", "cyty", "ctyty")


class Params(C.Structure):
    _fields_ = [
        ("z_min", C.c_float), ("z_max", C.c_float), ("dz", C.c_float),
        ("z_gas", C.c_float),
        ("sigma_max_pp", C.c_float), ("sigma_max_gas", C.c_float),
        ("min_integral_pp", C.c_float), ("min_integral_gas", C.c_float),
        ("bin_threshold", C.c_uint32),
        ("dip_num", C.c_int32), ("dip_den", C.c_int32),
        ("min_assoc_pp", C.c_int32), ("min_assoc_gas", C.c_int32),
        ("min_pv_tracks_pp", C.c_int32), ("min_pv_tracks_gas", C.c_int32),
        ("chi2_max", C.c_double), ("dchi2_tol", C.c_double), ("dz_tol", C.c_double),
        ("max_iter", C.c_int32),
        ("max_r_beam", C.c_double),
        ("max_seeds", C.c_int32),
        ("x_b", C.c_float), ("y_b", C.c_float), ("tx_b", C.c_float), ("ty_b", C.c_float),
        ("split_mode", C.c_int32), ("profile_mode", C.c_int32),
    ]


class MvParams(C.Structure):
    """Settings of the GPU-flavour multi-vertex fit (readings R12-R15)."""
    _fields_ = [("chi2_cut", C.c_double), ("dz_tol", C.c_double), ("w_assoc", C.c_double),
                ("dup_sep2", C.c_double), ("max_iter", C.c_int32)]


def default_mv_params(**kw) -> MvParams:
    m = MvParams(
        chi2_cut=4.0,        # Sec. 3.5, weight figure: chi2_max = 4 (R12)
        dz_tol=0.5e-3,       # Sec. 3.5: GPU rule |dz| < 0.5 um (R13)
        w_assoc=0.5,         # R14: the weight of a track at chi2 = chi2_cut alone
        dup_sep2=25.0,       # Sec. 3.5: dz^2 / (sum of z variances) below 25 (R15)
        max_iter=10,         # Sec. 3.5: at most ten iterations
    )
    for k, v in kw.items():
        setattr(m, k, v)
    return m


def default_params(**kw) -> Params:
    """The paper's settings (units: mm)."""
    p = Params(
        z_min=-550.0, z_max=300.0, dz=0.25,          # Sec. 3.2: range [-550, 300] mm, 0.25 mm bins
        z_gas=-300.0,                                # Table smog-pp: p-gas region below -300 mm
        sigma_max_pp=1.5, sigma_max_gas=10.0,        # Sec. 3.2: maximal sigma_poca
        min_integral_pp=2.5, min_integral_gas=1.75,  # Table smog-pp: min. cluster integral
        bin_threshold=205,                           # not given in the paper (R4): 0.05 track
        dip_num=4, dip_den=5,                        # not given in the paper (R5): dip < 80%
        min_assoc_pp=3, min_assoc_gas=2,             # Sec. 3.4: association thresholds
        min_pv_tracks_pp=4, min_pv_tracks_gas=3,     # Table smog-pp: min. tracks in the PV
        chi2_max=12.0,                               # Sec. 3.5, Eq. tukey
        dchi2_tol=0.01, dz_tol=1e-3, max_iter=10,    # Sec. 3.5: x86 convergence rule
        max_r_beam=0.3,                              # Sec. 3.5: 0.3 mm from the beamline
        max_seeds=64,
        x_b=0.0, y_b=0.0, tx_b=0.0, ty_b=0.0,
        split_mode=0,                                # Sec. 3.3: GPU (z order); 1 = x86 (R16)
        profile_mode=0,                              # Sec. 3.2: GPU (cubic CDF); 1 = x86 templates (R17)
    )
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def tight_params(**kw) -> Params:
    """Fit run to (near) full convergence; used to compare fixed points.  The
    paper's stopping rule looks at dchi2 and dz only, so the tolerances are
    made small enough that x and y have settled too."""
    base = dict(dchi2_tol=1e-12, dz_tol=1e-10, max_iter=400)
    base.update(kw)
    return default_params(**base)


def build(force: bool = False) -> str:
    """Compile pv_oracle.c into liboracle.so next to it (gcc, no contraction)."""
    with _LOCK:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _LIB
    if _LIB is None:
        path = build()
        L = C.CDLL(path)
        P = C.POINTER
        fp, dp, ip, i64p, up = (P(C.c_float), P(C.c_double), P(C.c_int32),
                                P(C.c_int64), P(C.c_uint32))
        pp = P(Params)
        arr11 = C.c_void_p * 11
        L.oc_num_bins.argtypes = [pp]
        L.oc_num_bins.restype = C.c_int
        L.oc_gas_bin.argtypes = [pp]
        L.oc_gas_bin.restype = C.c_int
        L.oc_prepare_tracks_f32.argtypes = [arr11, C.c_int64, pp, fp, fp, ip, ip, ip, ip]
        L.oc_prepare_tracks_f64.argtypes = [arr11, C.c_int64, pp, dp, dp]
        L.oc_track_profile.argtypes = [C.c_float, C.c_float, pp, ip, up, C.c_int]
        L.oc_track_profile.restype = C.c_int
        L.oc_find_batch.argtypes = [arr11, i64p, C.c_int32, pp, fp, fp, fp, ip, ip, ip, ip, ip, ip,
                                    C.c_void_p]
        L.oc_fit_batch.argtypes = [arr11, i64p, C.c_int32, pp, fp, fp, fp, ip, ip,
                                   dp, dp, dp, dp, dp, dp, ip, ip, ip]
        L.oc_fit_tracks.argtypes = [arr11, C.c_int64, C.c_float, C.c_float, C.c_float, pp,
                                    dp, dp, dp, dp, ip, ip, ip]
        L.oc_template_classes.restype = C.c_int
        L.oc_template_table.argtypes = [pp, dp, dp, ip, ip, ip, C.c_int]
        L.oc_template_table.restype = C.c_int
        L.oc_seeds_from_hist.argtypes = [up, pp, ip, ip, ip, fp, C.c_int]
        L.oc_seeds_from_hist.restype = C.c_int
        L.oc_associate_bins.argtypes = [ip, C.c_int64, ip, ip, ip, C.c_int, pp, ip, ip]
        L.oc_associate_bins.restype = C.c_int
        L.oc_find_batch_f64.argtypes = [arr11, i64p, C.c_int32, pp, dp, ip, ip]
        L.oc_profile_error.argtypes = [arr11, C.c_int64, pp, dp]
        L.oc_mv_fit_batch.argtypes = [arr11, i64p, C.c_int32, pp, P(MvParams), fp, fp, fp, ip,
                                      dp, dp, dp, dp, dp, dp, ip, ip, ip, ip]
        _LIB = L
    return _LIB


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _tracks_arg(tracks: dict):
    cols = [np.ascontiguousarray(tracks[k], dtype=np.float32) for k in TRACK_FIELDS]
    arr = (C.c_void_p * 11)(*[c.ctypes.data for c in cols])
    return arr, cols


def num_bins(p: Params) -> int:
    return lib().oc_num_bins(C.byref(p))


def gas_bin(p: Params) -> int:
    return lib().oc_gas_bin(C.byref(p))


def prepare_f32(tracks: dict, p: Params) -> dict:
    """Step (a) in the pinned binary32 sequence: z_poca, sigma_poca, center bin,
    profile window [j0, j1] and the fill flag of every track."""
    arr, keep = _tracks_arg(tracks)
    n = len(keep[0])
    out = {k: np.zeros(n, np.float32) for k in ("zpoca", "sigma")}
    out.update({k: np.zeros(n, np.int32) for k in ("center", "j0", "j1", "filled")})
    lib().oc_prepare_tracks_f32(arr, n, C.byref(p), _ptr(out["zpoca"], C.c_float),
                                _ptr(out["sigma"], C.c_float), _ptr(out["center"], C.c_int32),
                                _ptr(out["j0"], C.c_int32), _ptr(out["j1"], C.c_int32),
                                _ptr(out["filled"], C.c_int32))
    return out


def prepare_f64(tracks: dict, p: Params) -> dict:
    """Step (a) in binary64 (for error reports only)."""
    arr, keep = _tracks_arg(tracks)
    n = len(keep[0])
    zp = np.zeros(n, np.float64)
    sg = np.zeros(n, np.float64)
    lib().oc_prepare_tracks_f64(arr, n, C.byref(p), _ptr(zp, C.c_double), _ptr(sg, C.c_double))
    return {"zpoca": zp, "sigma": sg}


def find_batch_f64(batch, p: Params) -> dict:
    """Steps (a)-(d1) replayed in binary64 (z_poca, sigma_poca, window and
    cubic CDF in binary64, the same integer histogram rules, peak search and
    association): every event's surviving seeds, their maximum bin and their z
    before any rounding to binary32.  For error reports only."""
    arr, keep = _tracks_arg(batch.tracks)
    E = batch.n_events
    cap = p.max_seeds
    z = np.zeros((E, cap), np.float64)
    b = np.zeros((E, cap), np.int32)
    n = np.zeros(E, np.int32)
    offs = np.ascontiguousarray(batch.offsets, np.int64)
    lib().oc_find_batch_f64(arr, _ptr(offs, C.c_int64), E, C.byref(p), _ptr(z, C.c_double),
                            _ptr(b, C.c_int32), _ptr(n, C.c_int32))
    return {"z": z, "bin": b, "n": n}


def profile_error(tracks: dict, p: Params) -> dict:
    """Per-bin error of the binary32 integer profile (reading R3, or R17 for
    profile_mode 1) against the Gaussian bin integral of the binary64 z_poca
    and sigma_poca, over the bins within 5 sigma of every filled track, in
    track units: largest and RMS, and the largest truncation of a window (its
    weight sum against the Gaussian mass in range).  For error reports only."""
    arr, keep = _tracks_arg(tracks)
    n = len(keep[0])
    out = np.zeros(4, np.float64)
    lib().oc_profile_error(arr, n, C.byref(p), _ptr(out, C.c_double))
    return {"max": float(out[0]), "rms": float(np.sqrt(out[1] / max(out[2], 1.0))),
            "bins": int(out[2]), "truncation_max": float(out[3])}


def track_profile(zpoca: float, sigma: float, p: Params):
    """(first_bin, integer weights) of one track's histogram contribution."""
    cap = num_bins(p) + 8
    w = np.zeros(cap, np.uint32)
    first = C.c_int32(0)
    n = lib().oc_track_profile(float(zpoca), float(sigma), C.byref(p), C.byref(first),
                               _ptr(w, C.c_uint32), cap)
    if n < 0:
        raise ValueError("profile window larger than the histogram")
    return int(first.value), w[:n].copy()


def template_table(p: Params) -> dict:
    """The x86 flavour's template profiles (reading R17): per class its sigma,
    the lowest sigma_poca it takes, its half-width H and its quantised
    cumulative values Q[0 .. 2H+1] at the bin edges around the centre bin."""
    L = lib()
    K = L.oc_template_classes()
    sig = np.zeros(K, np.float64); bound = np.zeros(K, np.float64)
    half = np.zeros(K, np.int32); first = np.zeros(K, np.int32)
    total = L.oc_template_table(C.byref(p), None, None, None, None, None, 0)
    q = np.zeros(total, np.int32)
    L.oc_template_table(C.byref(p), _ptr(sig, C.c_double), _ptr(bound, C.c_double),
                        _ptr(half, C.c_int32), _ptr(first, C.c_int32), _ptr(q, C.c_int32), total)
    return {"sigma": sig, "bound": bound, "half": half,
            "q": [q[first[k]:first[k] + 2 * half[k] + 2].copy() for k in range(K)]}


def seeds_from_hist(hist: np.ndarray, p: Params, cap: int = 4096) -> dict:
    """Step (c) on one histogram: z-ordered seed clusters [lo, hi], their
    maximum bin and z_seed."""
    h = np.ascontiguousarray(hist, dtype=np.uint32)
    assert h.shape[0] == num_bins(p)
    lo = np.zeros(cap, np.int32); hi = np.zeros(cap, np.int32)
    b = np.zeros(cap, np.int32); z = np.zeros(cap, np.float32)
    n = lib().oc_seeds_from_hist(_ptr(h, C.c_uint32), C.byref(p), _ptr(lo, C.c_int32),
                                 _ptr(hi, C.c_int32), _ptr(b, C.c_int32), _ptr(z, C.c_float), cap)
    m = min(n, cap)
    return {"n": n, "lo": lo[:m], "hi": hi[:m], "bin": b[:m], "z": z[:m]}


def associate_bins(center: np.ndarray, lo, hi, binmax, p: Params) -> dict:
    """Step (d1): association of tracks (given their center bins, -1 = not
    filled) to seed clusters with the removal loop."""
    c = np.ascontiguousarray(center, dtype=np.int32)
    lo = np.ascontiguousarray(lo, dtype=np.int32)
    hi = np.ascontiguousarray(hi, dtype=np.int32)
    bm = np.ascontiguousarray(binmax, dtype=np.int32)
    K = len(lo)
    keep = np.zeros(max(K, 1), np.int32)
    cl = np.zeros(max(len(c), 1), np.int32)
    n = lib().oc_associate_bins(_ptr(c, C.c_int32), len(c), _ptr(lo, C.c_int32),
                                _ptr(hi, C.c_int32), _ptr(bm, C.c_int32), K, C.byref(p),
                                _ptr(keep, C.c_int32), _ptr(cl, C.c_int32))
    return {"n": n, "keep": keep[:K].astype(bool), "cluster": cl[:len(c)]}


def find_batch(batch, p: Params, want_hist: bool = False) -> dict:
    """Steps (a)-(d1) on a batch of events (``synthetic.EventBatch``)."""
    arr, keep = _tracks_arg(batch.tracks)
    E = batch.n_events
    cap = p.max_seeds
    offs = np.ascontiguousarray(batch.offsets, dtype=np.int64)
    out = {k: np.zeros((E, cap), np.float32) for k in ("x", "y", "z")}
    out.update({k: np.zeros((E, cap), np.int32) for k in ("lo", "hi", "bin")})
    out["n"] = np.zeros(E, np.int32)
    out["event_status"] = np.zeros(E, np.int32)
    out["track_cluster"] = np.zeros(max(batch.n_tracks, 1), np.int32)
    nb = num_bins(p)
    hist = np.zeros((E, nb), np.uint32) if want_hist else None
    lib().oc_find_batch(arr, _ptr(offs, C.c_int64), E, C.byref(p),
                        _ptr(out["x"], C.c_float), _ptr(out["y"], C.c_float),
                        _ptr(out["z"], C.c_float), _ptr(out["lo"], C.c_int32),
                        _ptr(out["hi"], C.c_int32), _ptr(out["bin"], C.c_int32),
                        _ptr(out["n"], C.c_int32), _ptr(out["event_status"], C.c_int32),
                        _ptr(out["track_cluster"], C.c_int32),
                        hist.ctypes.data if want_hist else None)
    out["track_cluster"] = out["track_cluster"][:batch.n_tracks]
    if want_hist:
        out["hist"] = hist
    return out


def fit_batch(batch, found: dict, p: Params) -> dict:
    """Steps (d2)-(d3): fit every seed from its assigned tracks (binary64)."""
    arr, keep = _tracks_arg(batch.tracks)
    E = batch.n_events
    cap = p.max_seeds
    offs = np.ascontiguousarray(batch.offsets, dtype=np.int64)
    out = {k: np.zeros((E, cap), np.float64) for k in ("x", "y", "z", "chi2", "ndof")}
    out["cov"] = np.zeros((E, cap, 6), np.float64)
    out.update({k: np.zeros((E, cap), np.int32) for k in ("n_tracks", "n_iter", "status")})
    sx = np.ascontiguousarray(found["x"], np.float32)
    sy = np.ascontiguousarray(found["y"], np.float32)
    sz = np.ascontiguousarray(found["z"], np.float32)
    ns = np.ascontiguousarray(found["n"], np.int32)
    tc = np.ascontiguousarray(found["track_cluster"], np.int32)
    if tc.shape[0] == 0:
        tc = np.zeros(1, np.int32)
    lib().oc_fit_batch(arr, _ptr(offs, C.c_int64), E, C.byref(p), _ptr(sx, C.c_float),
                       _ptr(sy, C.c_float), _ptr(sz, C.c_float), _ptr(ns, C.c_int32),
                       _ptr(tc, C.c_int32), _ptr(out["x"], C.c_double),
                       _ptr(out["y"], C.c_double), _ptr(out["z"], C.c_double),
                       _ptr(out["cov"], C.c_double), _ptr(out["chi2"], C.c_double),
                       _ptr(out["ndof"], C.c_double), _ptr(out["n_tracks"], C.c_int32),
                       _ptr(out["n_iter"], C.c_int32), _ptr(out["status"], C.c_int32))
    out["n"] = ns.copy()
    return out


def mv_fit_batch(batch, found: dict, p: Params, m: MvParams | None = None) -> dict:
    """GPU-flavour multi-vertex fit of every seed (Sec. 3.5, readings R12-R15),
    duplicate removal and final selection.  ``found`` holds the seeds (x, y, z,
    n) as find_batch returns them.  Adds ``track_vertex`` (R14)."""
    m = m or default_mv_params()
    arr, keep = _tracks_arg(batch.tracks)
    E = batch.n_events
    cap = p.max_seeds
    offs = np.ascontiguousarray(batch.offsets, dtype=np.int64)
    out = {k: np.zeros((E, cap), np.float64) for k in ("x", "y", "z", "chi2", "ndof")}
    out["cov"] = np.zeros((E, cap, 6), np.float64)
    out.update({k: np.zeros((E, cap), np.int32) for k in ("n_tracks", "n_iter", "status")})
    tv = np.full(max(batch.n_tracks, 1), -1, np.int32)
    sx = np.ascontiguousarray(found["x"], np.float32)
    sy = np.ascontiguousarray(found["y"], np.float32)
    sz = np.ascontiguousarray(found["z"], np.float32)
    ns = np.ascontiguousarray(found["n"], np.int32)
    lib().oc_mv_fit_batch(arr, _ptr(offs, C.c_int64), E, C.byref(p), C.byref(m),
                          _ptr(sx, C.c_float), _ptr(sy, C.c_float), _ptr(sz, C.c_float),
                          _ptr(ns, C.c_int32), _ptr(out["x"], C.c_double),
                          _ptr(out["y"], C.c_double), _ptr(out["z"], C.c_double),
                          _ptr(out["cov"], C.c_double), _ptr(out["chi2"], C.c_double),
                          _ptr(out["ndof"], C.c_double), _ptr(out["n_tracks"], C.c_int32),
                          _ptr(out["n_iter"], C.c_int32), _ptr(out["status"], C.c_int32),
                          _ptr(tv, C.c_int32))
    out["n"] = ns.copy()
    out["track_vertex"] = tv[:batch.n_tracks]
    return out


def fit_tracks(tracks: dict, seed, p: Params) -> dict:
    """Fit one vertex from the given tracks starting at ``seed`` (x, y, z)."""
    arr, keep = _tracks_arg(tracks)
    n = len(keep[0])
    x = np.zeros(3); cov = np.zeros(6)
    chi2 = C.c_double(); ndof = C.c_double()
    ntrk = C.c_int32(); nit = C.c_int32(); st = C.c_int32()
    lib().oc_fit_tracks(arr, n, float(seed[0]), float(seed[1]), float(seed[2]), C.byref(p),
                        _ptr(x, C.c_double), _ptr(cov, C.c_double), C.byref(chi2),
                        C.byref(ndof), C.byref(ntrk), C.byref(nit), C.byref(st))
    return {"x": x, "cov": cov, "chi2": chi2.value, "ndof": ndof.value,
            "n_tracks": ntrk.value, "n_iter": nit.value, "status": st.value}


def find_fit(batch, p: Params) -> tuple:
    """The whole method on a batch: (find result, fit result)."""
    f = find_batch(batch, p)
    return f, fit_batch(batch, f, p)
