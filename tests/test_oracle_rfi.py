"""Pins of the oracle's RFI mitigation (Sections II-B and III-C; the reading is
written out in oracle/hp_oracle.c): an independent numpy formulation on small
inputs, planted narrowband tones and broadband spikes found exactly, a
dispersed pulse left alone, clean noise left alone."""
import numpy as np
import pytest

import oracle
from paper_2512_00398_gb300 import synth, workloads


def _lower_median(v):
    v = np.sort(np.asarray(v).ravel())
    return int(v[(v.size - 1) // 2])


def _brute(x, tsamp, nb_k, bb_k, mode=0, baseline_s=2.0):
    nsamps, nch = x.shape
    xi = x.astype(np.int64)
    m = np.array([_lower_median(xi[:, c]) for c in range(nch)])
    s = np.array([_lower_median(np.abs(xi[:, c] - m[c])) for c in range(nch)])
    Mm, Ms = _lower_median(m), _lower_median(s)
    Dm, Ds = _lower_median(np.abs(m - Mm)), _lower_median(np.abs(s - Ms))
    cf = (np.abs(m - Mm) > nb_k * max(Dm, 1)) | (np.abs(s - Ms) > nb_k * max(Ds, 1))
    z = np.where(cf[None, :], m[None, :], xi).sum(axis=1).astype(np.int32)
    y = oracle.subtract_baseline(z, mode, oracle.baseline_window(baseline_s, tsamp))
    sg = 1.482602218505602 * _lower_median(np.abs(y))
    sf = np.array([sg > 0 and float(abs(int(v))) >= float(np.float32(bb_k)) * sg for v in y])
    out = np.where(cf[None, :] | sf[:, None], m[None, :], xi).astype(np.uint8)
    return out, cf, sf, m


@pytest.mark.parametrize("seed", range(5))
def test_rfi_bruteforce(seed):
    rng = np.random.default_rng(700 + seed)
    nsamps, nch = int(rng.integers(300, 2000)), int(rng.integers(8, 40))
    x = np.clip(rng.normal(100, 10, size=(nsamps, nch)), 0, 255)
    x[:, rng.integers(0, nch, 2)] += 60                       # hot channels
    x[:, rng.integers(0, nch)] *= 0.3                         # a quiet channel
    x[rng.integers(0, nsamps, 4), :] += 80                    # broadband spikes
    x = np.clip(np.rint(x), 0, 255).astype(np.uint8)
    nb_k, bb_k = int(rng.integers(2, 6)), float(np.float32(rng.uniform(3, 6)))
    for mode in (0, 1):
        r = oracle.rfi_clean(x, 1e-3, nb_k, bb_k, mode, 0.2)
        out, cf, sf, m = _brute(x, 1e-3, nb_k, bb_k, mode, 0.2)
        assert np.array_equal(r.chan_median, m)
        assert np.array_equal(r.chan_flag, cf)
        assert np.array_equal(r.samp_flag, sf)
        assert np.array_equal(r.cleaned, out)


def _noise(nsamps, nch, seed, sigma=12.0):
    obs = synth.Observation(nchans=nch, f_top=1500.0, chan_bw=-500.0 / nch, tsamp=64e-6,
                            nsamps=nsamps, mean=128.0, sigma=sigma)
    return obs, synth.filterbank(obs, seed).data


def test_planted_tones_and_spikes_found_exactly():
    obs, x = _noise(40000, 256, 3)
    x = x.astype(np.int32)
    tones = np.array([5, 77, 78, 200])
    spikes = np.array([1234, 20000, 33333])
    x[:, tones] += 40
    x[spikes, :] += 36
    x = np.clip(x, 0, 255).astype(np.uint8)
    r = oracle.rfi_clean(x, obs.tsamp)
    assert np.array_equal(np.flatnonzero(r.chan_flag), tones)
    assert np.array_equal(np.flatnonzero(r.samp_flag), spikes)
    # cleaned: flagged rows and columns hold the channel medians, the rest unchanged
    keep = ~r.chan_flag[None, :] & ~r.samp_flag[:, None]
    assert np.array_equal(r.cleaned[keep], x[keep])
    assert (r.cleaned[spikes][:, ~r.chan_flag] == r.chan_median[~r.chan_flag]).all()
    assert (r.cleaned[:, tones] == r.chan_median[tones]).all()


def test_clean_noise_and_dispersed_pulses_are_left_alone(tiny_workload):
    w, s = tiny_workload
    o = w.obs
    r = oracle.rfi_clean(s.data, o.tsamp)
    assert not r.chan_flag.any()
    assert r.samp_flag.sum() <= 1
    # the injected pulses (DM 50-300) are still recovered after cleaning
    res = oracle.search(r.cleaned, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    for p in s.pulses:
        assert workloads.recovered(p, res.clusters, w), p


def test_stress_rfi_flags_tones_and_spikes():
    w = workloads.stress(nsamps=1 << 18)
    s = w.generate(threads=8)
    r = oracle.rfi_clean(s.data, w.obs.tsamp)
    every = int(round(w.rfi.spike_period / w.obs.tsamp))
    spikes = np.arange(every // 2, s.data.shape[0], every)
    assert r.samp_flag[spikes].all()
    assert r.chan_flag.sum() == int(round(w.rfi.tone_frac * w.obs.nchans))


def test_channel_threshold_is_strict_and_floor_of_one():
    # constant channels: medians 100 x 8, 105 (= 5 x max(D, 1) away: kept) and
    # 106 (flagged); spreads all 0, the zero-DM series constant (no sample flags)
    x = np.full((600, 10), 100, np.uint8)
    x[:, 8] = 105
    x[:, 9] = 106
    r = oracle.rfi_clean(x, 1e-3, nb_k=5, bb_k=5.0, baseline_s=0.05)
    assert np.flatnonzero(r.chan_flag).tolist() == [9]
    assert not r.samp_flag.any() and r.sigma_z == 0.0
    # a channel whose spread alone is off is flagged too
    rng = np.random.default_rng(5)
    x = np.clip(rng.normal(100, 3, size=(4000, 12)), 0, 255).astype(np.uint8)
    x[:, 4] = np.clip(rng.normal(100, 30, size=4000), 0, 255).astype(np.uint8)
    r = oracle.rfi_clean(x, 1e-3, nb_k=5, bb_k=50.0, baseline_s=0.5)
    assert np.flatnonzero(r.chan_flag).tolist() == [4]
