"""RFI mitigation on the GPU (hp_rfi_clean, and hp_search with HP_PARAM_RFI)
against the oracle's reading of Sections II-B and III-C: channel medians,
channel and sample flags and the cleaned filterbank bit-exact; a search of an
RFI-bearing input with the stage on equals the oracle's search of the
oracle-cleaned input (tuples exact, S/N within 1e-4)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
FIELDS = ("dm_idx", "width_idx", "sample", "members", "dm_lo", "dm_hi", "t_lo", "t_hi")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_00398_gb300 as hp
    return torch, hp


def _plan(hp, obs, dms, widths, thr=6.0, **kw):
    return hp.Plan(obs.nchans, obs.f_top, obs.chan_bw, obs.tsamp, dms, widths, thr, **kw)


def _check(torch, hp, plan, x, obs, mode=0, nb_k=5, bb_k=5.0):
    fb = torch.from_numpy(x).cuda()
    out, cf, sf, med = hp.hp_rfi_clean(plan, fb)
    assert hp.hp_plan_sync_status(plan) == hp.HP_OK
    r = oracle.rfi_clean(x, obs.tsamp, nb_k, bb_k, mode, plan.get_param("baseline_s"))
    assert np.array_equal(med.cpu().numpy(), r.chan_median)
    assert np.array_equal(cf.cpu().numpy().astype(bool), r.chan_flag)
    assert np.array_equal(sf.cpu().numpy().astype(bool), r.samp_flag)
    assert np.array_equal(out.cpu().numpy(), r.cleaned)
    return r


def test_planted_tones_and_spikes(env):
    torch, hp = env
    from paper_2512_00398_gb300 import synth
    obs = synth.Observation(nchans=256, f_top=1500.0, chan_bw=-500.0 / 256, tsamp=64e-6,
                            nsamps=40000, mean=128.0, sigma=12.0)
    x = synth.filterbank(obs, 3).data.astype(np.int32)
    x[:, [5, 77, 78, 200]] += 40
    x[[1234, 20000, 33333], :] += 36
    x = np.clip(x, 0, 255).astype(np.uint8)
    p = _plan(hp, obs, np.linspace(0, 100, 8).astype(np.float32), np.array([1, 2, 4], np.int32))
    r = _check(torch, hp, p, x, obs)
    assert r.chan_flag.sum() == 4 and r.samp_flag.sum() == 3


@pytest.mark.parametrize("mode", [0, 1])
def test_stress_band_bit_exact(env, mode):
    """The FAST band with the stress RFI (spikes, tones, drift), 2^17 samples,
    both baseline modes for the zero-DM series."""
    torch, hp = env
    from paper_2512_00398_gb300 import workloads
    w = workloads.stress(nsamps=1 << 17)
    s = w.generate(threads=16)
    p = _plan(hp, w.obs, w.dm_list[:64], w.widths[:8], baseline_mode=mode)
    r = _check(torch, hp, p, s.data, w.obs, mode=mode)
    assert r.chan_flag.any() and r.samp_flag.any()


def test_ragged_channels_and_thresholds(env):
    """100 channels (not a multiple of 16), other thresholds, a quiet channel."""
    torch, hp = env
    rng = np.random.default_rng(41)
    from paper_2512_00398_gb300 import synth
    obs = synth.Observation(nchans=100, f_top=1400.0, chan_bw=-2.0, tsamp=1e-4, nsamps=30011,
                            mean=100.0, sigma=10.0)
    x = synth.filterbank(obs, 9).data.astype(np.float64)
    x[:, 17] = 100 + 0.2 * (x[:, 17] - 100)
    x[:, 63] += 25
    x[rng.integers(0, obs.nsamps, 6), :] += 30
    x = np.clip(np.rint(x), 0, 255).astype(np.uint8)
    p = _plan(hp, obs, np.array([0.0, 10.0], np.float32), np.array([1, 4], np.int32),
              rfi_nb_k=3, rfi_bb_k=4.0)
    r = _check(torch, hp, p, x, obs, nb_k=3, bb_k=4.0)
    assert r.chan_flag[[17, 63]].all()


def test_search_with_rfi_matches_oracle(env):
    """hp_search with the RFI stage on, on an RFI-bearing tiny-band input."""
    torch, hp = env
    from paper_2512_00398_gb300 import workloads
    w = workloads.tiny()
    s = w.generate()
    o = w.obs
    x = s.data.astype(np.int32)
    x[:, [3, 40]] += 50
    x[[5000, 17000, 29000], :] += 60
    x = np.clip(x, 0, 255).astype(np.uint8)
    p = _plan(hp, o, w.dm_list, w.widths, w.threshold, rfi=1)
    got = hp.search(p, torch.from_numpy(x).cuda())
    r = oracle.rfi_clean(x, o.tsamp)
    want = oracle.search(r.cleaned, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths,
                         w.threshold).clusters
    assert len(got) == len(want) and len(got) > 0
    for f in FIELDS:
        assert np.array_equal(got[f], want[f]), f
    assert np.abs(got["snr"].astype(np.float64) - want["snr"]).max() <= 1e-4
    st = hp.hp_plan_stats(p)
    assert st["stage_calls"]["rfi"] >= 0
