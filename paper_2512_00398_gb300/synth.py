"""Seeded synthetic filterbanks shaped like the single-pulse search workloads.

This module only *simulates what a receiver records*: quantised radiometer
noise, dispersed Gaussian pulses and radio-frequency interference.  It holds
none of the search arithmetic (no delay table, no dedispersion, no baseline,
no statistics, no thresholds), so the CPU oracle and the CUDA library can both
be fed from it without sharing any of the method.

Data model (the filterbank of Section II-B, "Incoherent Dedispersion"):
``uint8[nsamps][nchans]``, time-major (each spectrum of ``nchans`` bytes is
contiguous).  Channel ``c`` sits at ``f_top + c * chan_bw`` MHz with
``chan_bw < 0`` (frequency falls with channel index).

Signal model: a pulse that arrives at ``f_top`` at time ``t0`` arrives in a
channel of frequency ``f`` at ``t0 + K_DM * DM * (f**-2 - f_top**-2)`` seconds
(cold-plasma dispersion, continuous time, nothing rounded), with a Gaussian
profile of the given FWHM.  Signal and interference are added to the float
noise before rounding and clipping, so sub-count amplitudes survive.

Determinism: noise is drawn in fixed chunks of rows, chunk ``i`` from
``PCG64(SeedSequence([seed, i]))``, so the bytes do not depend on the number of
worker threads.
"""
from __future__ import annotations

import math
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

#: Cold-plasma dispersion constant in s MHz^2 pc^-1 cm^3 (signal model only).
K_DM = 4148.808

_TABLE_BITS = 16


@dataclass(frozen=True)
class Observation:
    """Shape and radiometer statistics of one synthetic filterbank."""

    nchans: int
    f_top: float          # MHz, frequency of channel 0
    chan_bw: float        # MHz, negative
    tsamp: float          # s
    nsamps: int
    mean: float = 128.0   # counts
    sigma: float = 16.0   # counts, per channel per sample

    @property
    def duration(self) -> float:
        return self.nsamps * self.tsamp

    def freqs(self) -> np.ndarray:
        return self.f_top + np.arange(self.nchans, dtype=np.float64) * self.chan_bw


@dataclass(frozen=True)
class Pulse:
    """A dispersed Gaussian pulse.

    ``t0`` is the arrival time (s) of the pulse peak at ``f_top``; ``amp`` is
    the per-channel peak amplitude in counts.
    """

    dm: float
    t0: float
    fwhm: float
    amp: float
    snr: float = float("nan")   # nominal best-boxcar S/N the amplitude was derived from


@dataclass(frozen=True)
class RFI:
    """Interference of the stress workload.

    * ``spike_period`` s: one-sample broadband (undispersed) spikes of
      ``spike_amp`` counts in every channel, once per period.
    * ``tone_frac`` of the channels (seeded choice) carry a constant
      ``tone_amp`` counts for the whole file.
    * a common drift ``drift_amp * sin(2 pi t / drift_period)`` in all channels.
    """

    spike_period: float = 1.0
    spike_amp: float = 48.0
    tone_frac: float = 0.05
    tone_amp: float = 40.0
    drift_amp: float = 10.0
    drift_period: float = 10.0
    seed: int = 0


@dataclass
class Synthetic:
    """A generated filterbank plus what was put into it."""

    obs: Observation
    data: np.ndarray                      # uint8 [nsamps][nchans]
    pulses: list = field(default_factory=list)
    rfi: RFI | None = None


def _noise_tables(mean: float, sigma: float):
    from scipy.special import ndtri

    k = np.arange(1 << _TABLE_BITS, dtype=np.float64)
    z = ndtri((k + 0.5) / float(1 << _TABLE_BITS))
    q = np.clip(np.rint(mean + sigma * z), 0, 255).astype(np.uint8)
    return q, z


def _pulse_points(obs: Observation, pulses):
    """Flat indices (t*nchans + c) and float signal of every pulse sample."""
    if not pulses:
        return np.zeros(0, np.int64), np.zeros(0, np.float64)
    freqs = obs.freqs()
    idx_parts, val_parts = [], []
    for p in pulses:
        tau = p.t0 + K_DM * p.dm * (freqs ** -2 - obs.f_top ** -2)       # s per channel
        half = 4.0 * p.fwhm
        lo = np.maximum(np.floor((tau - half) / obs.tsamp).astype(np.int64), 0)
        hi = np.minimum(np.ceil((tau + half) / obs.tsamp).astype(np.int64), obs.nsamps - 1)
        n = np.maximum(hi - lo + 1, 0)
        if n.sum() == 0:
            continue
        chan = np.repeat(np.arange(obs.nchans, dtype=np.int64), n)
        start = np.repeat(lo, n)
        offs = np.arange(n.sum(), dtype=np.int64) - np.repeat(np.cumsum(n) - n, n)
        t = start + offs
        dt = t * obs.tsamp - tau[chan]
        sig = p.amp * np.exp(-4.0 * math.log(2.0) * (dt / p.fwhm) ** 2)
        idx_parts.append(t * obs.nchans + chan)
        val_parts.append(sig)
    if not idx_parts:
        return np.zeros(0, np.int64), np.zeros(0, np.float64)
    idx = np.concatenate(idx_parts)
    val = np.concatenate(val_parts)
    uniq, inv = np.unique(idx, return_inverse=True)
    acc = np.zeros(uniq.size, np.float64)
    np.add.at(acc, inv, val)
    return uniq, acc


def filterbank(obs: Observation, seed: int, pulses=(), rfi: RFI | None = None,
               threads: int = 8) -> Synthetic:
    """Generate a seeded ``uint8[nsamps][nchans]`` filterbank."""
    q_tab, z_tab = _noise_tables(obs.mean, obs.sigma)
    out = np.empty((obs.nsamps, obs.nchans), dtype=np.uint8)
    rows = max(1, (1 << 22) // obs.nchans)
    nchunks = (obs.nsamps + rows - 1) // rows
    pidx, pval = _pulse_points(obs, list(pulses))

    tone = None
    if rfi is not None:
        rr = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, rfi.seed, 7])))
        ntone = int(round(rfi.tone_frac * obs.nchans))
        tone = np.zeros(obs.nchans, np.float64)
        tone[rr.choice(obs.nchans, size=ntone, replace=False)] = rfi.tone_amp
        spike_every = max(1, int(round(rfi.spike_period / obs.tsamp)))

    def job(i):
        r0 = i * rows
        r1 = min(obs.nsamps, r0 + rows)
        g = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, i])))
        u = g.integers(0, 1 << _TABLE_BITS, size=(r1 - r0, obs.nchans), dtype=np.uint16)
        if rfi is None:
            out[r0:r1] = q_tab[u]
            a, b = np.searchsorted(pidx, [r0 * obs.nchans, r1 * obs.nchans])
            if b > a:
                flat = pidx[a:b] - r0 * obs.nchans
                uu = u.reshape(-1)[flat]
                v = obs.mean + obs.sigma * z_tab[uu] + pval[a:b]
                out.reshape(-1)[pidx[a:b]] = np.clip(np.rint(v), 0, 255).astype(np.uint8)
            return
        t = np.arange(r0, r1, dtype=np.float64)
        v = obs.mean + obs.sigma * z_tab[u]
        v += (rfi.drift_amp * np.sin(2.0 * math.pi * t * obs.tsamp / rfi.drift_period))[:, None]
        v += tone[None, :]
        spk = (np.arange(r0, r1) % spike_every) == (spike_every // 2)
        v[spk] += rfi.spike_amp
        a, b = np.searchsorted(pidx, [r0 * obs.nchans, r1 * obs.nchans])
        if b > a:
            v.reshape(-1)[pidx[a:b] - r0 * obs.nchans] += pval[a:b]
        out[r0:r1] = np.clip(np.rint(v), 0, 255).astype(np.uint8)

    if threads > 1 and nchunks > 1:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(job, range(nchunks)))
    else:
        for i in range(nchunks):
            job(i)
    return Synthetic(obs, out, list(pulses), rfi)


# --------------------------------------------------------------------------
# Search-grid helpers (inputs to the plan, not part of the search).
# --------------------------------------------------------------------------

def dm_list_uniform(dm_lo: float, dm_hi: float, n: int) -> np.ndarray:
    """``n`` trial DMs spaced uniformly on [dm_lo, dm_hi] (float32)."""
    return np.linspace(dm_lo, dm_hi, n).astype(np.float32)


def _dm_grid(obs: Observation, dm_lo, dm_hi, tol, w_int):
    """Trial DMs whose spacing grows as intra-channel smearing allows.

    Step: dDM = tol * sqrt(tsamp^2 + t_chan(DM)^2 + w_int^2) / (K * (f_lo^-2 - f_top^-2)),
    with t_chan = 8.3 us * DM * |chan_bw| / f_GHz^3 at the band centre
    (Cordes & McLaughlin 2003).
    """
    f_lo = obs.f_top + (obs.nchans - 1) * obs.chan_bw
    f_c = 0.5 * (obs.f_top + f_lo) / 1000.0
    span = K_DM * (f_lo ** -2 - obs.f_top ** -2)
    dms = [float(dm_lo)]
    while True:
        dm = dms[-1]
        t_chan = 8.3e-6 * dm * abs(obs.chan_bw) / f_c ** 3
        step = tol * math.sqrt(obs.tsamp ** 2 + t_chan ** 2 + w_int ** 2) / span
        nxt = dm + step
        if nxt > dm_hi:
            break
        dms.append(nxt)
    return np.asarray(dms, dtype=np.float32)


def dm_list_smearing(obs: Observation, dm_lo: float, dm_hi: float, target: int,
                     w_int: float = 0.0) -> np.ndarray:
    """Smearing-driven DM grid with ``tol`` solved so the count is ~``target``."""
    lo, hi = 1e-3, 1e4
    best = None
    for _ in range(80):
        mid = math.sqrt(lo * hi)
        g = _dm_grid(obs, dm_lo, dm_hi, mid, w_int)
        if best is None or abs(len(g) - target) < abs(len(best) - target):
            best = g
        if len(g) > target:
            lo = mid
        else:
            hi = mid
        if len(g) == target:
            break
    return best


def widths_pow2(wmax: int) -> np.ndarray:
    """Boxcar ladder 1, 2, 4, ..., wmax (int32)."""
    w, out = 1, []
    while w <= wmax:
        out.append(w)
        w *= 2
    return np.asarray(out, dtype=np.int32)


def amp_for_matched_snr(snr: float, fwhm_samples: float, nchans: int, sigma: float,
                        widths=None) -> float:
    """Per-channel peak amplitude giving a nominal best-boxcar S/N of ``snr``.

    Ideal dedispersion at the true DM is assumed: the summed pulse is
    ``nchans * amp * g(t)`` over white noise of rms ``sigma * sqrt(nchans)``.
    """
    if widths is None:
        widths = widths_pow2(1 << 14)
    half = int(math.ceil(6 * fwhm_samples)) + 2
    t = np.arange(-half, half + 1, dtype=np.float64)
    g = np.exp(-4.0 * math.log(2.0) * (t / max(fwhm_samples, 1e-9)) ** 2)
    c = np.concatenate([[0.0], np.cumsum(g)])
    best = 0.0
    for w in widths:
        w = int(w)
        if w > len(g):
            break
        s = (c[w:] - c[:-w]).max()
        best = max(best, s / math.sqrt(w))
    return snr * sigma * math.sqrt(nchans) / (nchans * best)
