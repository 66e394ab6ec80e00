"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every symbol
declared in include/snd.h, validates arguments, and its plan tables agree with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def snd():
    lib = os.path.join(ROOT, "paper_2606_15361_gb300", "libsnd.so")
    if not os.path.exists(lib):
        import __graft_entry__
        __graft_entry__.build()
    import paper_2606_15361_gb300 as g
    return g


def test_exports_match_header(snd):
    hdr = open(os.path.join(ROOT, "include", "snd.h")).read()
    declared = set(re.findall(r"\b(snd_[a-z_0-9]+)\s*\(", hdr))
    assert declared >= {"snd_plan", "snd_execute", "snd_candidates"}
    for name in declared:
        assert hasattr(snd.lib, name), name
    assert declared == set(snd.EXPORTS)


def test_options_defaults(snd):
    o = snd.options(snd.MODE_BINARY)
    assert (o.cluster_size, o.k_leaf, o.k_internal, o.enc_theta, o.det_theta, o.sigma_min) == (4, 2, 2, 1.5, 7.0, 0.2)
    assert snd.options(snd.MODE_GRADED).enc_theta == 0.75 and snd.options(snd.MODE_GRADED).graded_cap == 255
    assert snd.options(snd.MODE_FLOAT).enc_theta == 1.5


def _plan_rc(snd, freqs, dms, B=2, mode=0, opts=None, nchan=None, ndm=None, dt=1.38e-4):
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    d = np.ascontiguousarray(dms, dtype=np.float64)
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    o = opts if opts is not None else snd.options(mode)
    rc = snd.lib.snd_plan_ex(f.ctypes.data_as(dp), f.size if nchan is None else nchan, dt, d.ctypes.data_as(dp),
                             d.size if ndm is None else ndm, B, mode, ctypes.byref(o), ctypes.byref(h))
    if rc == 0:
        snd.lib.snd_destroy(h)
    else:
        assert not h.value
    return rc


def test_plan_argument_errors(snd):
    f = synth.channel_freqs(16)
    d = np.linspace(0, 50, 8)
    E = snd.ERR
    assert _plan_rc(snd, f, d) == 0
    assert _plan_rc(snd, f, d, B=1) == E["SND_ERR_ARG"]
    assert _plan_rc(snd, f, d, nchan=0) == E["SND_ERR_ARG"]
    assert _plan_rc(snd, f, d, ndm=0) == E["SND_ERR_ARG"]
    assert _plan_rc(snd, f, d, dt=0.0) == E["SND_ERR_ARG"]
    assert _plan_rc(snd, f, d, mode=7, opts=snd.options(0)) == E["SND_ERR_ARG"]
    bad = f.copy(); bad[3] = bad[2]
    assert _plan_rc(snd, bad, d) == E["SND_ERR_FREQ_ORDER"]
    bad = f.copy(); bad[0] = np.nan
    assert _plan_rc(snd, bad, d) == E["SND_ERR_FREQ_ORDER"]
    assert _plan_rc(snd, f, np.array([1.0, -2.0])) == E["SND_ERR_DM"]
    assert _plan_rc(snd, f, np.array([1.0, np.inf])) == E["SND_ERR_DM"]
    for k, v, err in [("cluster_size", 8, "SND_ERR_UNSUPPORTED"), ("k_leaf", 0, "SND_ERR_UNSUPPORTED"),
                      ("det_theta", 0.0, "SND_ERR_ARG"), ("closing_size", 4, "SND_ERR_ARG"),
                      ("max_chunk", 0, "SND_ERR_ARG"), ("flags", 8, "SND_ERR_ARG")]:
        assert _plan_rc(snd, f, d, opts=snd.options(0, **{k: v})) == E[err], k
    assert _plan_rc(snd, f, d, mode=1, opts=snd.options(1, graded_cap=256)) == E["SND_ERR_UNSUPPORTED"]
    # unsorted grids, duplicate DMs and a single DM are accepted
    assert _plan_rc(snd, f[::-1], np.array([30.0, 0.0, 30.0, 12.5])) == 0
    assert _plan_rc(snd, f, np.array([0.0])) == 0


def test_unbound_calls_fail_cleanly(snd):
    p = snd.Plan(synth.channel_freqs(16), 1.38e-4, np.linspace(0, 10, 4), 2, snd.MODE_FLOAT, bind=False)
    ne = ctypes.c_int32()
    assert snd.lib.snd_execute(p.handle, ctypes.c_void_p(1), 10, None, None, ctypes.byref(ne)) == snd.ERR["SND_ERR_STATE"]
    n = ctypes.c_int32()
    assert snd.lib.snd_candidates(p.handle, None, 0, ctypes.byref(n)) == snd.ERR["SND_ERR_STATE"]
    assert snd.lib.snd_bind_workspace(p.handle, None, 0, None) == snd.ERR["SND_ERR_WORKSPACE"]
    assert snd.lib.snd_bind_workspace(p.handle, ctypes.c_void_p(256 * 3 + 8), p.workspace_bytes, None) == \
        snd.ERR["SND_ERR_WORKSPACE"]
    assert snd.lib.snd_workspace_size(None) == 0
    assert snd.lib.snd_error_string(-9) == b"device list capacity overflowed"


@pytest.mark.parametrize("B", [2, 4, 8])
def test_plan_stats_nc(snd, B):
    from oracle import delays, tree
    w = synth.NC1024
    p = snd.Plan(w.freqs(), synth.NC_DT, w.dms(), B, snd.MODE_BINARY, bind=False)
    s = p.stats()
    lv = tree.tree_levels(1024, 4, B)
    assert s.nlevels == len(lv) and list(s.nodes_per_level[:s.nlevels]) == [len(l) for l in lv]
    assert s.max_delay == 28324 and s.wmax == 1024
    # every DM has its own root pattern; the leaves share (Table 2 style neuron counts)
    assert s.unique_per_level[s.nlevels - 1] == 2048
    assert s.unique_per_level[0] == 49223
    assert (p.delay_table() == delays.delay_table(w.freqs(), synth.NC_DT, w.dms())).all()


def test_delay_table_matches_oracle_unsorted(snd):
    from oracle import delays
    rng = np.random.default_rng(5)
    f = rng.permutation(synth.channel_freqs(50))
    d = rng.uniform(0, 300, 33)
    p = snd.Plan(f, 2.56e-4, d, 3, snd.MODE_GRADED, bind=False)
    assert (p.delay_table() == delays.delay_table(f, 2.56e-4, d)).all()


def _mr_rc(snd, freqs, dms, s_max=64, mode=1, **kw):
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    d = np.ascontiguousarray(dms, dtype=np.float64)
    o = snd.options(mode, **kw)
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    rc = snd.lib.snd_multirate_plan(f.ctypes.data_as(dp), f.size, 1.38e-4, d.ctypes.data_as(dp), d.size, 2, mode,
                                    ctypes.byref(o), s_max, ctypes.byref(h))
    if rc == 0:
        snd.lib.snd_multirate_destroy(h)
    else:
        assert not h.value
    return rc


def test_multirate_plan_bands_match_oracle(snd):
    """Band split (Eq. scrunch) of the library equals the oracle's, for several grids and caps."""
    from oracle import delays as odelays
    from oracle import multirate as omr
    for nchan, dms, s_max in [(64, synth.dm_grid(128, 100.0), 64), (1024, synth.dm_grid(2048, 2000.0), 16),
                              (1024, synth.dm_grid(2048, 2000.0), 4), (256, np.array([3.0, 900.0, 0.0, 450.0]), 64)]:
        f = synth.channel_freqs(nchan)
        m = snd.MultiRatePlan(f, 1.38e-4, dms, 2, snd.MODE_GRADED, s_max=s_max, bind=False)
        exp = omr.bands(f, 1.38e-4, dms, s_max)
        assert m.scrunch == [s for s, _ in exp]
        assert m.band_ndm == [len(i) for _, i in exp]
        for b, (s, idx) in enumerate(exp):
            bp = m.band_plan(b)
            st = bp.stats()
            assert st.ndm == len(idx)
            # the band runs its DM subset at sample interval S*dt
            assert (bp.delay_table() == odelays.delay_table(f, s * 1.38e-4, np.asarray(dms)[idx])).all()
        assert m.workspace_bytes > 0


def test_multirate_plan_argument_errors(snd):
    f = synth.channel_freqs(64)
    d = synth.dm_grid(128, 100.0)
    E = snd.ERR
    assert _mr_rc(snd, f, d) == 0
    assert _mr_rc(snd, f, d, s_max=3) == E["SND_ERR_ARG"]
    assert _mr_rc(snd, f, d, s_max=0) == E["SND_ERR_ARG"]
    assert _mr_rc(snd, f, d, s_max=2048) == E["SND_ERR_ARG"]
    assert _mr_rc(snd, f, np.array([1.0, -2.0])) == E["SND_ERR_DM"]
    # max_chunk must be a multiple of the largest scrunch factor in use
    assert _mr_rc(snd, f, d, max_chunk=16384 + 1) == E["SND_ERR_ARG"]


def test_zfloat_flags_and_stats(snd):
    f = synth.channel_freqs(64)
    d = synth.dm_grid(128, 100.0)
    E = snd.ERR
    assert _plan_rc(snd, f, d, mode=snd.MODE_ZFLOAT) == 0
    assert _plan_rc(snd, f, d, mode=snd.MODE_ZFLOAT, opts=snd.options(snd.MODE_ZFLOAT, flags=2)) == 0
    # FP16 storage is a zfloat option; the reference kernel does not evaluate zfloat
    assert _plan_rc(snd, f, d, mode=snd.MODE_FLOAT, opts=snd.options(snd.MODE_FLOAT, flags=2)) == E["SND_ERR_ARG"]
    assert _plan_rc(snd, f, d, mode=snd.MODE_ZFLOAT,
                    opts=snd.options(snd.MODE_ZFLOAT, flags=1)) == E["SND_ERR_UNSUPPORTED"]
    assert _plan_rc(snd, f, d, mode=4, opts=snd.options(snd.MODE_FLOAT)) == E["SND_ERR_ARG"]
    p16 = snd.Plan(f, 1.38e-4, d, 2, snd.MODE_ZFLOAT, snd.options(snd.MODE_ZFLOAT, flags=2), bind=False)
    p32 = snd.Plan(f, 1.38e-4, d, 2, snd.MODE_ZFLOAT, bind=False)
    s16, s32 = p16.stats(), p32.stats()
    assert s16.tree_tile_dms == 16 and s16.tree_smem_bytes <= 2 * 52 * 1024 + 4096  # two staging buffers
    # FP16 storage halves the per-node history of Eq. hist_mem relative to FP32
    assert s16.hist_mem_bytes < s32.hist_mem_bytes
    assert p16.workspace_bytes < p32.workspace_bytes


def test_uint8_plane_option(snd):
    f = synth.channel_freqs(64)
    d = synth.dm_grid(128, 100.0)
    E = snd.ERR
    for mode in (snd.MODE_BINARY, snd.MODE_GRADED):
        assert _plan_rc(snd, f, d, mode=mode, opts=snd.options(mode, plane_dtype=1)) == 0
    assert _plan_rc(snd, f, d, mode=snd.MODE_FLOAT, opts=snd.options(snd.MODE_FLOAT, plane_dtype=1)) == E["SND_ERR_ARG"]
    assert _plan_rc(snd, f, d, mode=snd.MODE_GRADED, opts=snd.options(snd.MODE_GRADED, plane_dtype=2)) == E["SND_ERR_ARG"]
    assert ctypes.sizeof(snd.SndOptions) % 8 == 0 and snd.options(snd.MODE_BINARY).plane_dtype == 0


def test_injected_host_allocation_failures_return_nomem(snd):
    """Every host allocation point of plan, multi-rate plan and batch construction, made to
    fail in turn by the injection hook, gives SND_ERR_NOMEM and no object; once the countdown
    passes the last point the call succeeds (the hook disarms itself after firing)."""
    E = snd.ERR
    f = synth.channel_freqs(64)
    d = np.linspace(0, 80, 40)
    try:
        k = 0
        while True:
            snd.lib.snd_debug_fail_host_alloc(k)
            rc = _plan_rc(snd, f, d, mode=snd.MODE_FLOAT)
            if rc == 0:
                break
            assert rc == E["SND_ERR_NOMEM"], (k, rc)
            k += 1
        assert k >= 5  # the plan object, delays, leaf patterns, statistics, kernel tables
        snd.lib.snd_debug_fail_host_alloc(-1)  # the countdown outlived the last point: disarm
        # multi-rate plan (its band plans included)
        fp = np.ascontiguousarray(f)
        dp = ctypes.POINTER(ctypes.c_double)
        dm = np.ascontiguousarray(np.linspace(0, 600, 64))
        k = 0
        while True:
            snd.lib.snd_debug_fail_host_alloc(k)
            h = ctypes.c_void_p()
            o = snd.options(snd.MODE_GRADED, max_chunk=4096)
            rc = snd.lib.snd_multirate_plan(fp.ctypes.data_as(dp), 64, 1.38e-4, dm.ctypes.data_as(dp), dm.size, 2,
                                            snd.MODE_GRADED, ctypes.byref(o), 16, ctypes.byref(h))
            if rc == 0:
                snd.lib.snd_multirate_destroy(h)
                break
            assert rc == E["SND_ERR_NOMEM"] and not h.value, (k, rc)
            k += 1
        assert k >= 3
        snd.lib.snd_debug_fail_host_alloc(-1)
        # batch of two plans
        plans = [snd.Plan(f, 1.38e-4, d, 2, snd.MODE_FLOAT, bind=False) for _ in range(2)]
        arr = (ctypes.c_void_p * 2)(plans[0].handle.value, plans[1].handle.value)
        for k in range(2):
            snd.lib.snd_debug_fail_host_alloc(k)
            b = ctypes.c_void_p()
            assert snd.lib.snd_batch_create(arr, 2, ctypes.byref(b)) == E["SND_ERR_NOMEM"] and not b.value
        snd.lib.snd_debug_fail_host_alloc(-1)
        b = ctypes.c_void_p()
        assert snd.lib.snd_batch_create(arr, 2, ctypes.byref(b)) == 0
        snd.lib.snd_batch_destroy(b)
    finally:
        snd.lib.snd_debug_fail_host_alloc(-1)
