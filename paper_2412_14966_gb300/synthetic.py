"""Seeded synthetic bunch-crossing events for primary-vertex finding.

This module only draws random inputs; it holds none of the vertexing arithmetic.
Both the CUDA path and the CPU oracle read its output, so it is the one module
the two sides share.

The events mimic the shape of the simulated LHCb Run 3 samples the paper
measures on (Sec. 4): a luminous region that is long in z (PVs spread over tens
of mm) and narrow in x, y (tens of um), about five visible pp interactions per
crossing (Sec. 1), VELO-like straight tracks whose state is given near the
interaction point with a covariance matrix (Sec. 2), and an optional SMOG2-like
fixed-target region upstream of the pp region (Sec. 4.2, Table "smog-pp").
Units are mm and dimensionless slopes.

Recipe (one function per workload below):
  * n_PV ~ Poisson(mu), at least 1.  PV z ~ N(0, 45 mm), PV x, y ~ N(0, 15 um)
    about a beamline at (0, 0) with zero slope.
  * tracks per PV = 1 + NegBinomial(mean m, k = 2).
  * true slopes tx, ty ~ U(-0.3, 0.3); measured slopes = true + N(0, 1e-3).
  * state z = PV z + U(-10, 10) mm; x, y = PV + t_true * (z - PV z) + N(0, s_IP)
    with s_IP = min(12 um + 25 um * 0.3 / |t|, 200 um).
  * covariance: V_xx = V_yy = s_IP^2, V_txtx = V_tyty = 1e-6, off-diagonals 0.
  * fakes: round(0.1 * n_tracks) tracks from z ~ U(-200, 200) mm,
    x, y ~ N(0, 0.5 mm), same slope and resolution model.
  * track order within an event is shuffled.
"""
from __future__ import annotations

import dataclasses

import numpy as np

TRACK_FIELDS = ("x", "y", "z", "tx", "ty", "cxx", "cxtx", "ctxtx", "cyy", "cyty", "ctyty")


@dataclasses.dataclass
class EventBatch:
    """Structure-of-arrays track container plus CSR event offsets and truth."""

    tracks: dict            # name -> float32[n_tracks], names in TRACK_FIELDS
    offsets: np.ndarray     # int64[n_events + 1]
    pv_event: np.ndarray    # int64[n_pv]   event index of each true PV
    pv_pos: np.ndarray      # float64[n_pv, 3]
    pv_ntracks: np.ndarray  # int64[n_pv]
    pv_secondary: np.ndarray  # bool[n_pv]
    pv_gas: np.ndarray      # bool[n_pv]
    track_pv: np.ndarray    # int64[n_tracks], global PV index or -1 for fakes
    name: str = ""

    @property
    def n_events(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_tracks(self) -> int:
        return int(self.offsets[-1])

    def event_sizes(self) -> np.ndarray:
        return np.diff(self.offsets)

    def subset(self, events) -> "EventBatch":
        """A new batch made of the given event indices (in the given order)."""
        events = np.asarray(events, dtype=np.int64)
        sizes = self.event_sizes()[events]
        offs = np.zeros(len(events) + 1, dtype=np.int64)
        np.cumsum(sizes, out=offs[1:])
        idx = _ranges(self.offsets[events], sizes)
        pv_sel = np.isin(self.pv_event, events)
        remap = -np.ones(self.n_events, dtype=np.int64)
        remap[events] = np.arange(len(events))
        pv_ids = np.nonzero(pv_sel)[0]
        pv_remap = -np.ones(self.pv_event.shape[0] + 1, dtype=np.int64)
        pv_remap[pv_ids] = np.arange(len(pv_ids))
        tp = self.track_pv[idx]
        tp = np.where(tp >= 0, pv_remap[tp], -1)
        return EventBatch(
            tracks={k: np.ascontiguousarray(v[idx]) for k, v in self.tracks.items()},
            offsets=offs,
            pv_event=remap[self.pv_event[pv_sel]],
            pv_pos=self.pv_pos[pv_sel],
            pv_ntracks=self.pv_ntracks[pv_sel],
            pv_secondary=self.pv_secondary[pv_sel],
            pv_gas=self.pv_gas[pv_sel],
            track_pv=tp,
            name=self.name + "[subset]",
        )

    def concat(self, other: "EventBatch") -> "EventBatch":
        n_pv = self.pv_event.shape[0]
        tp2 = np.where(other.track_pv >= 0, other.track_pv + n_pv, -1)
        return EventBatch(
            tracks={k: np.concatenate([self.tracks[k], other.tracks[k]]) for k in TRACK_FIELDS},
            offsets=np.concatenate([self.offsets, other.offsets[1:] + self.offsets[-1]]),
            pv_event=np.concatenate([self.pv_event, other.pv_event + self.n_events]),
            pv_pos=np.concatenate([self.pv_pos, other.pv_pos]),
            pv_ntracks=np.concatenate([self.pv_ntracks, other.pv_ntracks]),
            pv_secondary=np.concatenate([self.pv_secondary, other.pv_secondary]),
            pv_gas=np.concatenate([self.pv_gas, other.pv_gas]),
            track_pv=np.concatenate([self.track_pv, tp2]),
            name=self.name + "+" + other.name,
        )


def _ranges(starts: np.ndarray, sizes: np.ndarray) -> np.ndarray:
    """Concatenation of arange(s, s + n) for each (s, n)."""
    total = int(sizes.sum())
    if total == 0:
        return np.zeros(0, dtype=np.int64)
    rep_start = np.repeat(starts - np.concatenate([[0], np.cumsum(sizes)[:-1]]), sizes)
    return rep_start + np.arange(total, dtype=np.int64)


def _resolution(tx: np.ndarray, ty: np.ndarray) -> np.ndarray:
    """Transverse impact-parameter resolution model (mm) of the recipe above."""
    t = np.sqrt(tx * tx + ty * ty)
    t = np.maximum(t, 1e-6)
    return np.minimum(0.012 + 0.025 * 0.3 / t, 0.200)


def generate(
    n_events: int,
    seed: int,
    *,
    mu=5.0,
    mean_tracks: float = 20.0,
    secondary_frac: float = 0.0,
    gas_event_frac: float = 0.0,
    fake_frac: float = 0.1,
    pv_z_sigma: float = 45.0,
    pv_xy_sigma: float = 0.015,
    gas_overlay: bool = False,
    beam=(0.0, 0.0, 0.0, 0.0),
    name: str = "",
) -> EventBatch:
    """Draw ``n_events`` independent events.

    ``mu`` is either a number (Poisson mean of the PV count) or a pair
    ``(lo, hi)``: then each event draws its own mean from U(lo, hi).
    ``gas_event_frac`` of the events are fixed-target: all their PVs have
    z ~ U(-541, -341) mm and slopes uniform on the disk |t| < 0.15.
    ``secondary_frac`` of the PVs are displaced by an exponential flight of mean
    1 mm along a random direction with a positive z component.
    ``gas_overlay`` adds one p-gas PV to every event (pp + p-gas overlay).
    ``beam`` = (x_b, y_b, t_x,b, t_y,b): PVs are placed around the beamline
    x_b + t_x,b z, y_b + t_y,b z (the beamline at z = 0 and its slopes).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if isinstance(mu, tuple):
        mu_ev = rng.uniform(mu[0], mu[1], size=n_events)
    else:
        mu_ev = np.full(n_events, float(mu))
    n_pv = np.maximum(rng.poisson(mu_ev), 1).astype(np.int64)
    gas_ev = rng.uniform(size=n_events) < gas_event_frac
    if gas_overlay:
        n_pv = n_pv + 1                    # the last PV of each event is the p-gas one
    total_pv = int(n_pv.sum())
    pv_event = np.repeat(np.arange(n_events, dtype=np.int64), n_pv)
    pv_gas = gas_ev[pv_event]
    if gas_overlay:
        last = np.cumsum(n_pv) - 1
        pv_gas = pv_gas.copy()
        pv_gas[last] = True

    pv_z = rng.normal(0.0, pv_z_sigma, size=total_pv)
    pv_z_gas = rng.uniform(-541.0, -341.0, size=total_pv)
    pv_z = np.where(pv_gas, pv_z_gas, pv_z)
    pv_x = rng.normal(0.0, pv_xy_sigma, size=total_pv)
    pv_y = rng.normal(0.0, pv_xy_sigma, size=total_pv)

    pv_sec = rng.uniform(size=total_pv) < secondary_frac
    flight = rng.exponential(1.0, size=total_pv)
    cos_t = rng.uniform(0.0, 1.0, size=total_pv)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=total_pv)
    sin_t = np.sqrt(1.0 - cos_t * cos_t)
    d = np.where(pv_sec, flight, 0.0)
    pv_x = pv_x + d * sin_t * np.cos(phi)
    pv_y = pv_y + d * sin_t * np.sin(phi)
    pv_z = pv_z + d * cos_t
    if any(beam):
        pv_x = pv_x + beam[0] + beam[2] * pv_z
        pv_y = pv_y + beam[1] + beam[3] * pv_z

    p_nb = 2.0 / (2.0 + mean_tracks)
    ntrk = 1 + rng.negative_binomial(2, p_nb, size=total_pv).astype(np.int64)
    n_real = int(ntrk.sum())
    trk_pv = np.repeat(np.arange(total_pv, dtype=np.int64), ntrk)
    trk_gas = pv_gas[trk_pv]

    # slopes: pp uniform in the square, fixed-target uniform on the small disk
    tx_pp = rng.uniform(-0.3, 0.3, size=n_real)
    ty_pp = rng.uniform(-0.3, 0.3, size=n_real)
    r_g = 0.15 * np.sqrt(rng.uniform(size=n_real))
    a_g = rng.uniform(0.0, 2.0 * np.pi, size=n_real)
    tx_t = np.where(trk_gas, r_g * np.cos(a_g), tx_pp)
    ty_t = np.where(trk_gas, r_g * np.sin(a_g), ty_pp)

    # fakes per event
    ev_real = np.zeros(n_events, dtype=np.int64)
    np.add.at(ev_real, pv_event, ntrk)
    n_fake_ev = np.rint(fake_frac * ev_real).astype(np.int64)
    n_fake = int(n_fake_ev.sum())
    fake_event = np.repeat(np.arange(n_events, dtype=np.int64), n_fake_ev)
    f_z0 = rng.uniform(-200.0, 200.0, size=n_fake)
    f_x0 = rng.normal(0.0, 0.5, size=n_fake)
    f_y0 = rng.normal(0.0, 0.5, size=n_fake)
    f_tx = rng.uniform(-0.3, 0.3, size=n_fake)
    f_ty = rng.uniform(-0.3, 0.3, size=n_fake)

    # assemble origins and true slopes of all tracks (real first, then fakes)
    ox = np.concatenate([pv_x[trk_pv], f_x0])
    oy = np.concatenate([pv_y[trk_pv], f_y0])
    oz = np.concatenate([pv_z[trk_pv], f_z0])
    txt = np.concatenate([tx_t, f_tx])
    tyt = np.concatenate([ty_t, f_ty])
    ev = np.concatenate([pv_event[trk_pv], fake_event])
    label = np.concatenate([trk_pv, -np.ones(n_fake, dtype=np.int64)])
    n_all = ev.shape[0]

    s_ip = _resolution(txt, tyt)
    zs = oz + rng.uniform(-10.0, 10.0, size=n_all)
    x = ox + txt * (zs - oz) + rng.normal(0.0, 1.0, size=n_all) * s_ip
    y = oy + tyt * (zs - oz) + rng.normal(0.0, 1.0, size=n_all) * s_ip
    tx = txt + rng.normal(0.0, 1e-3, size=n_all)
    ty = tyt + rng.normal(0.0, 1e-3, size=n_all)

    # group by event, shuffled within each event
    key = rng.uniform(size=n_all)
    order = np.lexsort((key, ev))
    sizes = np.bincount(ev, minlength=n_events).astype(np.int64)
    offsets = np.zeros(n_events + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])

    v = s_ip * s_ip
    zero = np.zeros(n_all)
    slope_var = np.full(n_all, 1e-6)
    cols = {
        "x": x, "y": y, "z": zs, "tx": tx, "ty": ty,
        "cxx": v, "cxtx": zero, "ctxtx": slope_var,
        "cyy": v, "cyty": zero, "ctyty": slope_var,
    }
    tracks = {k: np.ascontiguousarray(cols[k][order].astype(np.float32)) for k in TRACK_FIELDS}
    return EventBatch(
        tracks=tracks,
        offsets=offsets,
        pv_event=pv_event,
        pv_pos=np.stack([pv_x, pv_y, pv_z], axis=1),
        pv_ntracks=ntrk,
        pv_secondary=pv_sec,
        pv_gas=pv_gas,
        track_pv=label[order],
        name=name,
    )


# --- the named workloads --------------------------------------------------

def workload_small(n_events: int = 100, seed: int = 0) -> EventBatch:
    """100 pp events, mu = 5, 1 + NB(mean 20, k = 2) tracks per PV, 10% fakes."""
    return generate(n_events, seed, mu=5.0, mean_tracks=20.0, name="pp-mu5-m20")


def workload_nominal(n_events: int = 10_000, seed: int = 1) -> EventBatch:
    """10,000 pp events, mu = 5, 1 + NB(mean 28) tracks per PV (~160/event),
    5% of PVs displaced by an exponential 1 mm flight (secondaries)."""
    return generate(n_events, seed, mu=5.0, mean_tracks=28.0, secondary_frac=0.05,
                    name="pp-mu5-m28-sec5")


def workload_mixture(n_events: int = 200_000, seed: int = 2) -> EventBatch:
    """Uneven events: per-event mu ~ U(1, 12); 20% fixed-target events."""
    return generate(n_events, seed, mu=(1.0, 12.0), mean_tracks=28.0, gas_event_frac=0.2,
                    name="mix-mu1to12-gas20")


def workload_pileup(n_events: int = 20_000, seed: int = 3) -> EventBatch:
    """High pile-up: mu = 40, ~1,200 tracks per event, overlapping PVs."""
    return generate(n_events, seed, mu=40.0, mean_tracks=28.0, name="pp-mu40-m28")


def workload_overlay(n_events: int = 2000, seed: int = 5, beam=(0.0, 0.0, 0.0, 0.0)) -> EventBatch:
    """pp events (mu = 5) each overlaid with one p-gas PV in the gas cell
    (Sec. 4, the pp + p-gas overlay sample), around the given beamline."""
    return generate(n_events, seed, mu=5.0, mean_tracks=28.0, gas_overlay=True, beam=beam,
                    name="pp-mu5-plus-gas")


# a beamline displaced and inclined like a crossing angle (unit: mm, rad)
TILTED_BEAM = (0.6, -0.35, 2.0e-4, -1.5e-4)


WORKLOADS = {
    "small": workload_small,
    "nominal": workload_nominal,
    "mixture": workload_mixture,
    "pileup": workload_pileup,
    "overlay": workload_overlay,
}


def poisson_arrivals(n: int, rate_hz: float, seed: int) -> np.ndarray:
    """Arrival times (s) of an open-loop Poisson process with the given rate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n))


def straight_tracks(origin, slopes, z_states, cov_xx=1e-4, cov_tt=1e-6) -> dict:
    """Noise-free tracks through ``origin`` (x, y, z) with the given slopes,
    their states placed at ``z_states``.  Used to build hand-made test events."""
    slopes = np.asarray(slopes, dtype=np.float64).reshape(-1, 2)
    zs = np.asarray(z_states, dtype=np.float64).reshape(-1)
    n = slopes.shape[0]
    ox, oy, oz = origin
    x = ox + slopes[:, 0] * (zs - oz)
    y = oy + slopes[:, 1] * (zs - oz)
    cols = {
        "x": x, "y": y, "z": zs, "tx": slopes[:, 0], "ty": slopes[:, 1],
        "cxx": np.full(n, cov_xx), "cxtx": np.zeros(n), "ctxtx": np.full(n, cov_tt),
        "cyy": np.full(n, cov_xx), "cyty": np.zeros(n), "ctyty": np.full(n, cov_tt),
    }
    return {k: np.ascontiguousarray(cols[k].astype(np.float32)) for k in TRACK_FIELDS}


def batch_from_events(events: list) -> EventBatch:
    """Pack a list of per-event track dicts (as from ``straight_tracks``) into a batch."""
    sizes = np.array([len(e["x"]) for e in events], dtype=np.int64)
    offs = np.zeros(len(events) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offs[1:])
    tracks = {k: np.ascontiguousarray(np.concatenate([e[k] for e in events]).astype(np.float32)
                                      if len(events) else np.zeros(0, np.float32))
              for k in TRACK_FIELDS}
    n = int(offs[-1])
    return EventBatch(tracks=tracks, offsets=offs, pv_event=np.zeros(0, np.int64),
                      pv_pos=np.zeros((0, 3)), pv_ntracks=np.zeros(0, np.int64),
                      pv_secondary=np.zeros(0, bool), pv_gas=np.zeros(0, bool),
                      track_pv=-np.ones(n, np.int64), name="hand-made")
