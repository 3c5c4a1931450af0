"""Synthetic search workloads shaped like the paper's experiments (Section V-A).

The paper's data (a 1 GB CRAFTS file, the 142 GB M5 file and the 125 FAST-FREX
files) are not available; these seeded recipes stand in for them with the same
channel counts, sampling times, band, lengths and DM ranges.  Each recipe
returns the search parameters plus a callable that produces the filterbank.

* ``tiny``    128 ch, 32 768 samples, 100 uniform trials on DM 0-400, widths 1..64.
* ``fast``    4096 ch over 1000-1500 MHz, 2^20 samples of 49.152 us, ~1500
              trials on DM 0-2000, widths 1..4096 (the single-file FAST shape).
* ``batch``   16 files of 2^17-2^20 samples, 1024/2048/4096 ch, DM 0-1000.
* ``serve``   19 beams x 4096 ch, gulps of 65 536 samples, DM 0-2000.
* ``stress``  the fast band with 2^21 samples, ~4000 trials on DM 0-5000,
              widths 1..8192, broadband spikes, narrowband tones and drift.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import synth


@dataclass
class Workload:
    name: str
    obs: synth.Observation
    dm_list: np.ndarray          # float32 [ndm]
    widths: np.ndarray           # int32 [nw]
    threshold: float
    seed: int
    pulses: list = field(default_factory=list)
    rfi: synth.RFI | None = None

    def generate(self, threads: int = 8) -> synth.Synthetic:
        return synth.filterbank(self.obs, self.seed, self.pulses, self.rfi, threads=threads)

    @property
    def ndm(self) -> int:
        return int(len(self.dm_list))

    @property
    def nw(self) -> int:
        return int(len(self.widths))


FAST_BAND = dict(nchans=4096, f_top=1500.0, chan_bw=-500.0 / 4096, tsamp=49.152e-6)


def tiny(nsamps: int = 32768, seed: int = 1) -> Workload:
    obs = synth.Observation(nchans=128, f_top=1500.0, chan_bw=-1.953125, tsamp=64e-6,
                            nsamps=nsamps, mean=128.0, sigma=16.0)
    amp = 8.0 * obs.sigma
    pulses = [synth.Pulse(50.0, 0.30, 256e-6, amp),
              synth.Pulse(120.0, 0.80, 512e-6, amp),
              synth.Pulse(300.0, 1.30, 1024e-6, amp)]
    return Workload("tiny", obs, synth.dm_list_uniform(0.0, 400.0, 100),
                    synth.widths_pow2(64), 6.0, seed, pulses)


def _random_pulses(obs, rng, n, dm_hi, fwhm_lo, fwhm_hi, snr_lo, snr_hi, t_hi):
    out = []
    for _ in range(n):
        dm = float(rng.uniform(0.0, dm_hi))
        fwhm = float(math.exp(rng.uniform(math.log(fwhm_lo), math.log(fwhm_hi))))
        snr = float(rng.uniform(snr_lo, snr_hi))
        t0 = float(rng.uniform(0.05 * t_hi, 0.95 * t_hi))
        amp = synth.amp_for_matched_snr(snr, fwhm / obs.tsamp, obs.nchans, obs.sigma)
        out.append(synth.Pulse(dm, t0, fwhm, amp, snr))
    return out


def _max_delay_s(obs, dm):
    f_lo = obs.f_top + (obs.nchans - 1) * obs.chan_bw
    return synth.K_DM * dm * (f_lo ** -2 - obs.f_top ** -2)


def fast(nsamps: int = 1 << 20, seed: int = 2, ndm_target: int = 1500,
         dm_hi: float = 2000.0, wmax: int = 4096, npulses: int = 20) -> Workload:
    obs = synth.Observation(nsamps=nsamps, mean=128.0, sigma=12.0, **FAST_BAND)
    dms = synth.dm_list_smearing(obs, 0.0, dm_hi, ndm_target)
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 99])))
    t_hi = nsamps * obs.tsamp - _max_delay_s(obs, dm_hi) - 0.05
    pulses = _random_pulses(obs, rng, npulses, dm_hi, 0.1e-3, 20e-3, 6.0, 30.0, max(t_hi, 0.1))
    return Workload("fast", obs, dms, synth.widths_pow2(wmax), 6.0, seed, pulses)


def stress(nsamps: int = 1 << 21, seed: int = 5, ndm_target: int = 4000,
           dm_hi: float = 5000.0, wmax: int = 8192, npulses: int = 50) -> Workload:
    obs = synth.Observation(nsamps=nsamps, mean=128.0, sigma=12.0, **FAST_BAND)
    dms = synth.dm_list_smearing(obs, 0.0, dm_hi, ndm_target)
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 99])))
    t_hi = nsamps * obs.tsamp - _max_delay_s(obs, dm_hi) - 0.05
    pulses = _random_pulses(obs, rng, npulses, dm_hi, 0.1e-3, 20e-3, 6.0, 30.0, max(t_hi, 0.1))
    rfi = synth.RFI(spike_period=1.0, spike_amp=3.0 * obs.sigma, tone_frac=0.05,
                    tone_amp=40.0, drift_amp=10.0, drift_period=10.0, seed=seed)
    return Workload("stress", obs, dms, synth.widths_pow2(wmax), 6.0, seed, pulses, rfi)


def batch(nfiles: int = 16, seed0: int = 100, len_lo: int = 1 << 17, len_hi: int = 1 << 20,
          dm_hi: float = 1000.0, wmax: int = 4096, trial_density: float = 0.75):
    """Files of uneven length, channel count and sampling time (DM 0-1000).

    ``trial_density`` trials per DM unit at the fast band's spacing; the grid
    of each file is the smearing-driven grid with the count scaled to it.
    """
    files = []
    for i in range(nfiles):
        s = seed0 + i
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([s, 11])))
        nsamps = int(rng.integers(len_lo // 1024, len_hi // 1024 + 1)) * 1024
        nch = int(rng.choice([1024, 2048, 4096]))
        tsamp = float(rng.choice([49.152e-6, 64e-6]))
        obs = synth.Observation(nchans=nch, f_top=1500.0, chan_bw=-500.0 / nch, tsamp=tsamp,
                                nsamps=nsamps, mean=128.0, sigma=12.0)
        dms = synth.dm_list_smearing(obs, 0.0, dm_hi, int(round(trial_density * dm_hi)))
        npul = int(rng.integers(0, 11))
        t_hi = nsamps * tsamp - _max_delay_s(obs, dm_hi) - 0.05
        pulses = _random_pulses(obs, rng, npul, dm_hi, 0.1e-3, 20e-3, 8.0, 30.0, max(t_hi, 0.1))
        files.append(Workload(f"batch{i}", obs, dms, synth.widths_pow2(wmax), 6.0, s, pulses))
    return files


def stream_tiny(nbeams: int = 3, ngulps: int = 8, gulp: int = 4096, seed0: int = 200,
                npulses: int = 4) -> list:
    """Beams for the streamed-search tests: the tiny band (128 ch, 64 us),
    ngulps * gulp samples each (one continuous series per beam), DM 0-400,
    widths 1..64, pulses of 8-12 sigma per channel at random DM and time."""
    beams = []
    for b in range(nbeams):
        s = seed0 + b
        obs = synth.Observation(nchans=128, f_top=1500.0, chan_bw=-1.953125, tsamp=64e-6,
                                nsamps=ngulps * gulp, mean=128.0, sigma=16.0)
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([s, 12])))
        t_hi = obs.nsamps * obs.tsamp - _max_delay_s(obs, 400.0) - 0.02
        pulses = []
        for _ in range(npulses):
            dm = float(rng.uniform(20.0, 380.0))
            fwhm = float(math.exp(rng.uniform(math.log(128e-6), math.log(2e-3))))
            t0 = float(rng.uniform(0.02, max(t_hi, 0.05)))
            pulses.append(synth.Pulse(dm, t0, fwhm, float(rng.uniform(8.0, 12.0)) * obs.sigma))
        beams.append(Workload(f"stream{b}", obs, synth.dm_list_uniform(0.0, 400.0, 100),
                              synth.widths_pow2(64), 6.0, s, pulses))
    return beams


def serve(nbeams: int = 19, gulp: int = 65536, seconds: float = 600.0, seed0: int = 300,
          ndm_target: int = 1500, dm_hi: float = 2000.0, wmax: int = 4096) -> list:
    """The 19-beam stream: each beam the FAST band (4096 ch, 49.152 us), DM
    0-2000 on the smearing grid (~1500 trials), widths 1..4096, whole gulps of
    `gulp` samples covering `seconds`, about one pulse per beam-minute."""
    beams = []
    for b in range(nbeams):
        s = seed0 + b
        ng = max(1, int(round(seconds / (gulp * FAST_BAND["tsamp"]))))
        obs = synth.Observation(nsamps=ng * gulp, mean=128.0, sigma=12.0, **FAST_BAND)
        dms = synth.dm_list_smearing(obs, 0.0, dm_hi, ndm_target)
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([s, 13])))
        npul = max(1, int(round(obs.duration / 60.0)))
        t_hi = obs.duration - 0.05
        pulses = _random_pulses(obs, rng, npul, dm_hi, 0.1e-3, 20e-3, 8.0, 30.0, t_hi)
        beams.append(Workload(f"beam{b}", obs, dms, synth.widths_pow2(wmax), 6.0, s, pulses))
    return beams


def recovered(pulse, clusters, w, snr_min=10.0):
    """Is an injected pulse found?  A cluster must lie within max(2, 5% of the
    trials) of the nearest trial DM, start within max(W_eff, W_rep) samples of
    the arrival at f_top minus W_rep/2, and have a width index within 1 of
    log2(W_eff).  W_eff combines the FWHM with the smearing across the band
    left by the nearest trial: |DM - DM_trial| times the band's delay (in
    samples) per DM unit, from the cold-plasma law."""
    o = w.obs
    dms = np.asarray(w.dm_list, np.float64)
    d_true = int(np.argmin(np.abs(dms - pulse.dm)))
    f_lo = o.f_top + (o.nchans - 1) * o.chan_bw
    per_dm = synth.K_DM * (f_lo ** -2 - o.f_top ** -2) / o.tsamp
    w_eff = math.hypot(pulse.fwhm / o.tsamp, abs(dms[d_true] - pulse.dm) * per_dm)
    tol_dm = max(2, int(round(0.05 * dms.size)))
    for c in clusters:
        wrep = int(w.widths[c["width_idx"]])
        t_exp = pulse.t0 / o.tsamp - wrep / 2.0
        if (abs(int(c["dm_idx"]) - d_true) <= tol_dm
                and abs(int(c["sample"]) - t_exp) <= max(w_eff, wrep)
                and abs(int(c["width_idx"]) - math.log2(max(w_eff, 1.0))) <= 1.0 + 1e-9
                and c["snr"] >= snr_min):
            return True
    return False
