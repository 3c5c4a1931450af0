"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every symbol include/hp.h declares, validates arguments, and its FP64 delay
table is bit-identical to the oracle's (computed independently)."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2512_00398_gb300 as hp
from paper_2512_00398_gb300 import synth, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(hp_\w+)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = hp.lib()
    declared = _declared()
    assert "hp_search" in declared and "hp_plan_create" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(hp.EXPORTS) >= declared


def test_status_strings():
    assert hp.status_str(0) == "HP_OK"
    assert hp.status_str(-6) == "HP_ERR_NSAMPS_TOO_SHORT"
    assert hp.status_str(12345) == "HP_ERR_UNKNOWN"


@pytest.mark.parametrize("make", [workloads.tiny, lambda: workloads.fast(nsamps=1 << 17),
                                  lambda: workloads.stress(nsamps=1 << 18)])
def test_delay_table_matches_oracle(make):
    w = make()
    o = w.obs
    with hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold) as p:
        assert np.array_equal(p.delays(), oracle.delays(o.nchans, o.f_top, o.chan_bw, o.tsamp,
                                                        w.dm_list))
        assert p.max_delay == int(p.delays().max())


def test_delay_table_matches_oracle_batch_files():
    for w in workloads.batch(nfiles=4):
        o = w.obs
        with hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, 6.0) as p:
            assert np.array_equal(p.delays(), oracle.delays(o.nchans, o.f_top, o.chan_bw,
                                                            o.tsamp, w.dm_list))


BAD = [
    dict(nchans=0), dict(nchans=70000), dict(f_top=-1.0), dict(chan_bw=0.0), dict(chan_bw=1.0),
    dict(chan_bw=-30.0), dict(tsamp=0.0), dict(tsamp=float("nan")), dict(dm_list=[]),
    dict(dm_list=[5.0, 1.0]), dict(dm_list=[-1.0]), dict(dm_list=[float("inf")]), dict(widths=[]),
    dict(widths=[2, 2]), dict(widths=[0, 1]), dict(widths=list(range(1, 40))), dict(widths=[1, 32768]),
    dict(thr=0.0), dict(thr=float("nan")),
]


@pytest.mark.parametrize("bad", BAD)
def test_plan_rejects_bad_arguments(bad):
    args = dict(nchans=64, f_top=1500.0, chan_bw=-2.0, tsamp=1e-4, dm_list=[0.0, 10.0],
                widths=[1, 2, 4], thr=6.0)
    args.update(bad)
    with pytest.raises(hp.HPError) as e:
        hp.Plan(args["nchans"], args["f_top"], args["chan_bw"], args["tsamp"], args["dm_list"],
                args["widths"], args["thr"])
    assert e.value.code == hp.HP_ERR_INVALID_ARG


def test_subband_stage1_tile_shape_default():
    """The sub-band variant's stage 1 takes tile shape 12 unless one was set;
    a shape the caller set stays through switching the variant on and off."""
    w = workloads.tiny()
    o = w.obs
    with hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, 6.0) as p:
        p.set_param("subband_chans", 16)
        assert p.get_param("dedisp_config") == 12
        p.set_param("subband_chans", 0)
        assert p.get_param("dedisp_config") == 17
        p.set_param("dedisp_config", 14)
        p.set_param("subband_chans", 16)
        assert p.get_param("dedisp_config") == 14
        p.set_param("subband_chans", 0)
        assert p.get_param("dedisp_config") == 14


def test_params_roundtrip_and_validation():
    w = workloads.tiny()
    o = w.obs
    with hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, 6.0) as p:
        assert p.get_param("w_tol") == w.nw
        assert p.get_param("dedisp_config") == 17
        for name, val in [("baseline_mode", 1), ("baseline_s", 0.5), ("dm_tol", 3), ("t_gap", -2),
                          ("w_tol", 1), ("raw_capacity", 4096), ("dedisp_config", 3),
                          ("stage_timing", 1), ("timeout_s", 0.25)]:
            p.set_param(name, val)
            assert p.get_param(name) == pytest.approx(val)
        for name, val in [("baseline_mode", 2), ("baseline_s", 0), ("dm_tol", -1), ("w_tol", 0.5),
                          ("raw_capacity", 10), ("dedisp_config", hp.HP_NUM_DEDISP_CONFIGS),
                          ("timeout_s", 0)]:
            with pytest.raises(hp.HPError):
                p.set_param(name, val)
        with pytest.raises(hp.HPError):
            p.set_param(99, 1.0)


def test_workspace_sizes():
    w = workloads.fast(nsamps=1 << 20)
    o = w.obs
    with hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, 6.0) as p:
        nout = p.nout(1 << 20)
        ws = p.workspace_bytes(1 << 20)
        assert ws >= o.nchans * (1 << 20) + 4 * w.ndm * nout        # transposed input + series
        assert ws < 12e9
        with pytest.raises(hp.HPError) as e:
            p.workspace_bytes(p.max_delay + int(w.widths[-1]))
        assert e.value.code == hp.HP_ERR_NSAMPS_TOO_SHORT


def test_fuse_levels_param_and_workspace():
    """HP_PARAM_FUSE_LEVELS: off by default, 0 or 1 only; on, the workspace holds
    the second remedian level [ndm][round4(ceil(nout / 25))] int32 (256-byte
    aligned) for the median baseline with at least two levels and direct
    dedispersion, and nothing more otherwise."""
    w = workloads.fast(nsamps=1 << 20)
    o = w.obs
    with hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, 6.0) as p:
        assert p.get_param("fuse_levels") == 0
        for bad in (-1, 0.5, 2):
            with pytest.raises(hp.HPError):
                p.set_param("fuse_levels", bad)
        nout = p.nout(1 << 20)
        plain = p.workspace_bytes(1 << 20)
        p.set_param("fuse_levels", 1)
        lv2 = w.ndm * ((-(-nout // 25) + 3) // 4 * 4) * 4
        assert p.workspace_bytes(1 << 20) - plain == (lv2 + 255) // 256 * 256
        p.set_param("baseline_mode", 1)                     # moving mean: no remedian
        mean = p.workspace_bytes(1 << 20)
        p.set_param("fuse_levels", 0)
        assert p.workspace_bytes(1 << 20) == mean
        p.set_param("fuse_levels", 1)
        p.set_param("baseline_mode", 0)
        p.set_param("baseline_s", 0.0005)                  # one level (10 samples)
        one = p.workspace_bytes(1 << 20)
        p.set_param("fuse_levels", 0)
        assert p.workspace_bytes(1 << 20) == one
        p.set_param("fuse_levels", 1)
        p.set_param("baseline_s", 2.0)
        p.set_param("subband_chans", 64)                   # the sub-band variant keeps D's remedian
        sb = p.workspace_bytes(1 << 20)
        p.set_param("fuse_levels", 0)
        assert p.workspace_bytes(1 << 20) == sb


@pytest.mark.parametrize("kw", [dict(nbeams=0), dict(nbeams=hp.HP_STREAM_MAX_BEAMS + 1),
                                dict(gulp=32), dict(max_batch=-1), dict(max_batch=33),
                                dict(hbm_budget=-5), dict(cand_capacity=0),
                                dict(raw_capacity=100)])
def test_stream_rejects_bad_config(kw):
    # argument checks come before any CUDA call, so they run without a GPU
    w = workloads.tiny()
    o = w.obs
    plan = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    args = dict(nbeams=2, gulp=4096)
    args.update(kw)
    with pytest.raises(hp.HPError) as e:
        hp.Stream(plan, **args)
    assert e.value.code == hp.HP_ERR_INVALID_ARG


def test_stream_null_arguments():
    import ctypes as C
    L = hp.lib()
    assert L.hp_stream_open(None, None, None) == hp.HP_ERR_INVALID_ARG
    assert L.hp_stream_push(None, 0, None, 0) == hp.HP_ERR_INVALID_ARG
    assert L.hp_stream_end_beam(None, 0) == hp.HP_ERR_INVALID_ARG
    assert L.hp_stream_get_stats(None, None) == hp.HP_ERR_INVALID_ARG
    assert L.hp_stream_close(None) == hp.HP_OK
    h = C.c_void_p()
    assert L.hp_stream_open(C.byref(h), None, None) == hp.HP_ERR_INVALID_ARG and not h.value


def test_plan_allocator_arguments():
    w = workloads.tiny()
    o = w.obs
    plan = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    L = hp.lib()
    # an allocator needs both callables; none restores cudaMalloc
    assert L.hp_plan_set_allocator(plan.handle, hp._lib_mod.ALLOC_FN(lambda n, c: 0),
                                   hp._lib_mod.FREE_FN(), None) == hp.HP_ERR_INVALID_ARG
    assert L.hp_plan_set_allocator(None, hp._lib_mod.ALLOC_FN(), hp._lib_mod.FREE_FN(),
                                   None) == hp.HP_ERR_INVALID_ARG
    calls = []
    plan.use_allocator(lambda n: calls.append(n) or 0, lambda p, n: calls.append(-n))
    plan.use_allocator()          # nothing was allocated yet, so nothing is freed
    assert calls == []
    with pytest.raises(hp.HPError):
        plan.use_allocator(lambda n: 0, None)


def test_rfi_params():
    w = workloads.tiny()
    o = w.obs
    plan = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    assert plan.get_param("rfi") == 0 and plan.get_param("rfi_nb_k") == 5
    assert plan.get_param("rfi_bb_k") == 5.0
    plan.set_param("rfi", 1)
    plan.set_param("rfi_nb_k", 3)
    plan.set_param("rfi_bb_k", 4.5)
    assert (plan.get_param("rfi"), plan.get_param("rfi_nb_k"), plan.get_param("rfi_bb_k")) == \
        (1, 3, 4.5)
    for name, bad in (("rfi", 2), ("rfi_nb_k", -1), ("rfi_nb_k", 2.5), ("rfi_bb_k", 0.0)):
        with pytest.raises(hp.HPError):
            plan.set_param(name, bad)


@pytest.mark.parametrize("S,G", [(1, 8), (64, 1), (64, 8), (48, 5), (4096, 3), (100, 7)])
def test_subband_table_matches_oracle(S, G):
    """The plan's effective table of the sub-band variant (host code, no GPU)
    equals the oracle's, and the maximum delay and nout follow it."""
    w = workloads.fast(nsamps=1 << 17)
    o = w.obs
    with hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold) as p:
        direct = p.delays()
        p.set_param("subband_chans", S)
        p.set_param("subband_group", G)
        want = oracle.subband_delays(direct, S, G)
        assert np.array_equal(p.delays(), want)
        assert p.max_delay == int(want.max())
        assert p.nout(1 << 20) == (1 << 20) - int(want.max())
        p.set_param("subband_chans", 0)                 # back to direct dedispersion
        assert np.array_equal(p.delays(), direct) and p.max_delay == int(direct.max())


def test_subband_params_and_workspace():
    w = workloads.fast(nsamps=1 << 20)
    o = w.obs
    with hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, 6.0) as p:
        assert p.get_param("subband_chans") == 0 and p.get_param("subband_group") == 8
        direct_ws = p.workspace_bytes(1 << 20)
        for name, bad in (("subband_chans", -1), ("subband_chans", o.nchans + 1),
                          ("subband_chans", 2.5), ("subband_group", 0),
                          ("subband_group", w.ndm + 1)):
            with pytest.raises(hp.HPError):
                p.set_param(name, bad)
        p.set_param("subband_chans", 64)
        p.set_param("subband_group", 8)
        ws = p.workspace_bytes(1 << 20)
        # partial sums: 64 sub-bands x 24 nominal trials per chunk, 2 chunks at once (< 16 GiB);
        # the direct layout alone holds the second remedian level its dedispersion writes
        nb = p.nout(1 << 20) + int(p.delays()[:, ::64].max())
        groups = -(-p.nout(1 << 20) // 25)
        lv2 = w.ndm * ((groups + 3) // 4 * 4) * 4
        assert ws - (direct_ws - lv2) >= 2 * 64 * 24 * nb * 4
        assert ws < direct_ws + (16 << 30) + (1 << 30)


def test_width_sigma_param_and_arguments():
    import ctypes as C
    w = workloads.tiny()
    o = w.obs
    with hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold) as p:
        assert p.get_param("width_sigma") == 0
        for bad in (2, -1, 0.5):
            with pytest.raises(hp.HPError):
                p.set_param("width_sigma", bad)
        L = hp.lib()
        buf = C.create_string_buffer(8)
        # mode off, or on with nothing searched yet: refused before any CUDA call
        assert L.hp_width_sigmas(p.handle, buf, None, None) == hp.HP_ERR_INVALID_ARG
        p.set_param("width_sigma", 1)
        assert p.get_param("width_sigma") == 1
        assert L.hp_width_sigmas(p.handle, buf, None, None) == hp.HP_ERR_INVALID_ARG
        assert L.hp_width_sigmas(p.handle, None, None, None) == hp.HP_ERR_INVALID_ARG
        assert L.hp_width_sigmas(None, buf, None, None) == hp.HP_ERR_INVALID_ARG
        ws_on = p.workspace_bytes(o.nsamps)
        p.set_param("width_sigma", 0)
        # the radix-select counts: [ndm][nw][2 x 4096] uint32
        assert ws_on - p.workspace_bytes(o.nsamps) >= w.ndm * len(w.widths) * 2 * 4096 * 4


def test_dedisp_config_shapes():
    shapes = [hp.hp_dedisp_config(c) for c in range(hp.HP_NUM_DEDISP_CONFIGS)]
    assert shapes[12] == {"RD": 2, "NW": 7, "WD": 12, "WT": 1, "stage_bytes": 54 * 1024,
                          "stages": 4, "unroll": 2, "threads": 32 * 13}
    assert all(s["RD"] >= 1 and s["NW"] >= 1 and s["threads"] <= 1024 for s in shapes)
    # an odd word count per lane keeps the row loads conflict-free
    assert all(s["NW"] % 2 == 1 for s in shapes)
    for bad in (-1, hp.HP_NUM_DEDISP_CONFIGS):
        with pytest.raises(hp.HPError):
            hp.hp_dedisp_config(bad)


def test_decimate_param():
    w = workloads.fast(nsamps=1 << 17)       # widths up to 4096
    o = w.obs
    with hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold) as p:
        assert p.get_param("decimate") == 0
        base = p.workspace_bytes(1 << 20)
        p.set_param("decimate", 16)
        assert p.get_param("decimate") == 16
        # scrunched series for q = 2 .. 256 (widths 32 .. 4096): under the size of y
        extra = p.workspace_bytes(1 << 20) - base
        assert 0 < extra < w.ndm * (1 << 20) * 4 * 1.05
        for bad in (-1, 2.5, 2):          # 4096 / 2 > 1024 blocks per sample
            with pytest.raises(hp.HPError):
                p.set_param("decimate", bad)


def test_selftest_bounded_wait_arguments():
    lib = hp.lib()
    import ctypes as C
    out = (C.c_int32 * 4)()
    assert lib.hp_selftest_bounded_wait(0, out) == hp.HP_ERR_INVALID_ARG
    assert lib.hp_selftest_bounded_wait(-5, out) == hp.HP_ERR_INVALID_ARG
    assert lib.hp_selftest_bounded_wait(20_000_000_000, out) == hp.HP_ERR_INVALID_ARG
    assert lib.hp_selftest_bounded_wait(1000, None) == hp.HP_ERR_INVALID_ARG
